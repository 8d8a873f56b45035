"""lsnif_query_rays_noalloc: the query for callers that cannot allocate
device memory while they run (a frame loop where cudaMalloc/cudaFree would
stall the device, a plug-in whose host engine owns all allocations). Its
scratch is a static device array. It runs the kernels of lsnif_query_rays at
BF16 with the context's traversal and grouping choices, so its results must
equal the regular query's bit for bit, call after call, without allocating --
whatever the previous call left in the shared array."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2504_21627_gb300 import inputs as I  # noqa: E402
from paper_2504_21627_gb300 import lsnif  # noqa: E402


def _same(a, b):
    assert torch.equal(a.hit, b.hit)
    assert torch.equal(a.mat, b.mat)
    assert torch.equal(a.t, b.t)           # +inf on misses in both
    assert torch.equal(a.normal, b.normal)
    assert torch.equal(a.albedo, b.albedo)


def test_noalloc_query_matches_the_regular_query_twice_in_a_row():
    cfg = I.cfg_torus_4m()
    mesh = I.noise_torus(seed=2, nu=200, nv=80)
    params = I.random_params(cfg, seed=5, table_range=0.05, bias_range=0.1)
    with lsnif.Context(0) as ctx:
        obj = ctx.load_object(mesh, cfg, tables=params.tables, mlp=params.packed_mlp())
        cam = I.seeded_camera(2, width=256, height=256)
        rays = torch.from_numpy(I.rays_pinhole(cam)).cuda()            # 65536 rays
        for trace_mode, group_mode in ((1, 0), (0, 1), (1, 2), (2, 1)):
            ctx.set_trace_mode(trace_mode)
            ctx.set_group_mode(group_mode)
            ref = ctx.query_rays(rays, obj=obj, precision=lsnif.BF16_FUSED)
            ctx.check()
            before_lib = ctx.device_bytes()
            for call in range(2):
                out = ctx._alloc_hits(rays.shape[1], 0, False)
                torch.cuda.synchronize()
                torch_before_call = torch.cuda.memory_allocated()
                ctx.query_rays_noalloc(rays, out, obj=obj)
                ctx.check()
                assert torch.cuda.memory_allocated() == torch_before_call
                assert ctx.device_bytes() == before_lib, "the no-alloc query grew the library's device memory"
                _same(out, ref)
            # a second, differently sized batch: the scratch keeps the previous
            # call's contents and the result must not depend on them
            small = torch.from_numpy(I.rays_pinhole(I.seeded_camera(4, width=64, height=96))).cuda()
            ref2 = ctx.query_rays(small, obj=obj, precision=lsnif.BF16_FUSED)
            out2 = ctx.query_rays_noalloc(small, ctx._alloc_hits(small.shape[1], 0, False), obj=obj)
            ctx.check()
            _same(out2, ref2)


def test_noalloc_query_with_an_object_per_ray():
    cfg = I.cfg_icosphere_small()
    with lsnif.Context(0) as ctx:
        objs = []
        for k in range(2):
            mesh = I.noise_icosphere(seed=20 + k, target_tris=2000, amplitude=0.06, n_mat=2)
            p = I.random_params(cfg, seed=30 + k, table_range=0.3, bias_range=0.1)
            objs.append(ctx.load_object(mesh, cfg, tables=p.tables, mlp=p.packed_mlp()))
        lo, hi = np.full(3, -1.1, np.float32), np.full(3, 1.1, np.float32)
        rays = torch.from_numpy(I.rays_sphere_to_box(20000, 3.0, lo, hi, seed=41)).cuda()
        per_ray = torch.from_numpy(np.asarray(objs, np.uint32)[np.arange(20000) % 2]).cuda()
        for trace_mode, group_mode in ((1, 1), (2, 2)):
            ctx.set_trace_mode(trace_mode)
            ctx.set_group_mode(group_mode)
            ref = ctx.query_rays(rays, obj_per_ray=per_ray, precision=lsnif.BF16_FUSED)
            ctx.check()
            for call in range(2):
                out = ctx.query_rays_noalloc(rays, ctx._alloc_hits(20000, 0, False), obj_per_ray=per_ray)
                ctx.check()
                _same(out, ref)


def test_noalloc_query_rejects_batches_beyond_its_scratch():
    cfg = I.cfg_icosphere_small()
    with lsnif.Context(0) as ctx:
        obj = ctx.load_object(I.icosphere(2), cfg)
        big = torch.zeros((8, 1 << 20), device="cuda")
        out = ctx._alloc_hits(big.shape[1], 0, False)
        with pytest.raises(lsnif.LsnifError) as e:
            ctx.query_rays_noalloc(big, out, obj=obj)
        assert e.value.code == -1 and "static scratch" in str(e.value)
