"""lsnif_query_rays_noalloc: the query for callers that cannot allocate
device memory while they run (a frame loop where cudaMalloc/cudaFree would
stall the device, a plug-in whose host engine owns all allocations). Its
scratch is a static device array; it must give the results of the regular
query, call after call, without allocating."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2504_21627_gb300 import inputs as I  # noqa: E402
from paper_2504_21627_gb300 import lsnif  # noqa: E402

# the tolerance of the BF16 path's tests (one BF16 step of a hidden activation)
BF16_TOL = 2.0 ** -7


def _compare(a, b, n_out_scale):
    assert torch.equal(a.hit, b.hit)
    assert torch.equal(a.mat, b.mat)
    fin = torch.isfinite(a.t)
    assert torch.equal(fin, torch.isfinite(b.t))
    assert torch.allclose(a.t[fin], b.t[fin], rtol=0, atol=BF16_TOL * n_out_scale)
    assert torch.allclose(a.normal, b.normal, rtol=0, atol=BF16_TOL)


def test_noalloc_query_matches_the_regular_query_twice_in_a_row():
    cfg = I.cfg_torus_4m()
    mesh = I.noise_torus(seed=2, nu=200, nv=80)
    params = I.random_params(cfg, seed=5, table_range=0.05, bias_range=0.1)
    with lsnif.Context(0) as ctx:
        obj = ctx.load_object(mesh, cfg, tables=params.tables, mlp=params.packed_mlp())
        cam = I.seeded_camera(2, width=256, height=256)
        rays = torch.from_numpy(I.rays_pinhole(cam)).cuda()            # 65536 rays
        ref = ctx.query_rays(rays, obj=obj, precision=lsnif.BF16_FUSED)
        ctx.check()
        scale = float(torch.nan_to_num(ref.t, posinf=0).abs().max()) + 1.0
        before_lib = ctx.device_bytes()
        before_torch = torch.cuda.memory_allocated()
        for call in range(2):
            out = ctx._alloc_hits(rays.shape[1], 0, False)
            torch.cuda.synchronize()
            torch_before_call = torch.cuda.memory_allocated()
            ctx.query_rays_noalloc(rays, out, obj=obj)
            ctx.check()
            assert torch.cuda.memory_allocated() == torch_before_call
            assert ctx.device_bytes() == before_lib, "the no-alloc query grew the library's device memory"
            _compare(out, ref, scale)
        del before_torch
        # the same on a second, differently sized batch (the scratch keeps the
        # previous call's contents; the result must not depend on them)
        small = torch.from_numpy(I.rays_pinhole(I.seeded_camera(4, width=64, height=96))).cuda()
        ref2 = ctx.query_rays(small, obj=obj, precision=lsnif.BF16_FUSED)
        out2 = ctx.query_rays_noalloc(small, ctx._alloc_hits(small.shape[1], 0, False), obj=obj)
        ctx.check()
        _compare(out2, ref2, scale)


def test_noalloc_query_rejects_batches_beyond_its_scratch():
    cfg = I.cfg_icosphere_small()
    with lsnif.Context(0) as ctx:
        obj = ctx.load_object(I.icosphere(2), cfg)
        big = torch.zeros((8, 1 << 20), device="cuda")
        out = ctx._alloc_hits(big.shape[1], 0, False)
        with pytest.raises(lsnif.LsnifError) as e:
            ctx.query_rays_noalloc(big, out, obj=obj)
        assert e.value.code == -1 and "static scratch" in str(e.value)
