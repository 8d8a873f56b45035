"""Every stage on tiny meshes -- a tetrahedron, a single tilted triangle, an
axis-aligned (flat) triangle whose box is widened along its normal, and
icospheres at subdivision 0 and 1 -- against the oracle: occupancy, box and
level resolutions bit-exact, voxel counts exact away from voxel faces, and
the query's logits and decisions in
the FP32, BF16 and FP16 paths at the tolerances of the query tests (FP32:
1e-4 of the largest logit at these lattice resolutions; BF16 2^-7 and FP16
2^-9 on top, against the oracle run with the same operand rounding)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2504_21627_gb300 import inputs as I  # noqa: E402
from paper_2504_21627_gb300 import lsnif  # noqa: E402

MESHES = {
    "tetrahedron": lambda: I.tetrahedron(n_mat=2),
    "triangle": lambda: I.single_triangle((-0.8, -0.5, -0.3), (0.9, -0.2, 0.4), (0.1, 0.8, -0.6), n_mat=2),
    "flat_triangle": lambda: I.single_triangle((-0.8, -0.5, 0.2), (0.9, -0.2, 0.2), (0.1, 0.8, 0.2), n_mat=2),
    "icosphere0": lambda: I.icosphere(0),
    "icosphere1": lambda: I.icosphere(1),
}
TOL = {lsnif.FP32_PLAIN: 1e-4, lsnif.BF16_FUSED: 2.0 ** -7 + 1e-4, lsnif.FP16_FUSED: 2.0 ** -9 + 1e-4}
ORACLE = {lsnif.FP32_PLAIN: "f64", lsnif.BF16_FUSED: "bf16", lsnif.FP16_FUSED: "fp16"}


@pytest.fixture(scope="module")
def ctx():
    c = lsnif.Context(0)
    yield c
    c.close()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name", list(MESHES))
def test_tiny_mesh_all_stages(ctx, name):
    mesh = MESHES[name]()
    cfg = I.Config(V=8, H=18, L=4, F=2, log2_T=10, N_min=4, N_max=32, n_hidden=2, width=64, n_mat=mesh.n_mat)
    p = I.random_params(cfg, seed=17, table_range=0.5, bias_range=0.5)
    p.weights[-1][1][0] = 1.0   # occupancy logit biased towards hits
    orc = O.build_object(mesh, cfg, p)
    h = ctx.load_object(mesh, cfg, tables=p.tables, mlp=p.packed_mlp())
    try:
        # occupancy, box, level resolutions
        assert np.array_equal(ctx.read_params(h, lsnif.PARAM_OCCUPANCY), O.occupancy_bits(orc.occ))
        info = ctx.object_info(h)
        assert np.array_equal(np.array(info.bmin, np.float32), orc.bmin)
        assert np.array_equal(np.array(info.bmax, np.float32), orc.bmax)
        assert list(info.res[: cfg.L]) == list(orc.res)
        assert info.n_occupied == int(orc.occ.sum()) > 0
        rays = I.rays_sphere_to_box(3000, 3.0, orc.bmin, orc.bmax, seed=23)
        # traversal: voxel counts exact away from voxel faces
        k, _, _, _ = ctx.trace(_cuda(rays), h)
        seg = O.ray_segments(orc, rays)
        ok = ~seg.near
        assert np.array_equal(k.cpu().numpy()[ok], seg.k[ok])
        assert (seg.k[ok] > 0).sum() > 100
        for prec in (lsnif.FP32_PLAIN, lsnif.BF16_FUSED, lsnif.FP16_FUSED):
            out = ctx.query_rays(_cuda(rays), obj=h, precision=prec, logits=True)
            ctx.check()
            ref, _ = O.query(orc, rays, precision=ORACLE[prec], seg=seg)
            live = ref.live & ok
            lg = out.logits.cpu().numpy()
            scale = np.abs(ref.logits[live]).max()
            err = np.abs(lg[live] - ref.logits[live]).max() / scale
            assert err < TOL[prec], (name, prec, err)
            miss = ~ref.live & ok
            assert not out.hit.cpu().numpy()[miss].any()
            assert np.all(np.isinf(out.t.cpu().numpy()[miss]))
            firm = np.abs(ref.logits[live, 0]) > 4 * TOL[prec] * scale
            assert np.array_equal(out.hit.cpu().numpy().astype(bool)[live][firm], ref.hit[live][firm])
            zm = np.sort(ref.logits[live, 8:], axis=1)
            firm_m = (zm[:, -1] - zm[:, -2]) > 8 * TOL[prec] * scale
            assert np.array_equal(out.mat.cpu().numpy()[live][firm_m], ref.mat[live][firm_m])
    finally:
        ctx.unload_object(h)
