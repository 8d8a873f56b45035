"""GPU mesh objects (triangles + BVH, the hybrid pipeline's non-LSNIF objects,
Sec. 4) against the oracle's brute-force answers.

Tolerance: the GPU tests triangles in FP32 (stored v0, e1, e2), the oracle in
FP64 on the same FP32 rays. Away from triangle edges both find the same
triangle: hit flags equal, t within 1e-5 relative, normals within 1e-4,
materials equal. A ray within ~1e-5 (barycentric) of an edge may hit either
neighbour or slip through the seam; such rays are excluded and must stay
below 1% of the batch.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2504_21627_gb300 import inputs as I  # noqa: E402
from paper_2504_21627_gb300 import lsnif  # noqa: E402

OUT_BIAS = [5.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 2.0, 0.0]


@pytest.fixture(scope="module")
def ctx():
    c = lsnif.Context(0)
    yield c
    c.close()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _edge_margin(mesh, j):
    m = np.full(j.t.size, np.inf)
    h = j.tri >= 0
    m[h] = np.minimum.reduce([j.u[h], j.v[h], 1 - j.u[h] - j.v[h]])
    return m


@pytest.mark.parametrize("which", ["icosphere", "torus"])
def test_mesh_object_query_matches_brute_force(ctx, which):
    mesh = I.icosphere(3) if which == "icosphere" else I.noise_torus_tris(8, 20000, n_mat=3)
    h = ctx.load_mesh(mesh)
    info = ctx.object_info(h)
    assert info.kind == 1 and info.n_triangles == mesh.tris.shape[0] and info.bvh_nodes > 0
    rays = I.rays_sphere_to_box(20000, 3.0, mesh.verts.min(0), mesh.verts.max(0), seed=9)
    rays[6, :2000] = np.random.default_rng(1).uniform(0.0, 2.0, 2000)     # some rays start later
    rays[7, 2000:4000] = np.random.default_rng(2).uniform(0.5, 3.0, 2000)  # some end early
    out = ctx.query_rays(_cuda(rays), obj=h, precision=lsnif.FP32_PLAIN)
    ctx.check()
    torch.cuda.synchronize()
    ref, _ = O.mesh_query(O.mesh_object(mesh), rays)
    j = O.judge(mesh, rays)
    firm = ~(_edge_margin(mesh, j) < 1e-5)
    assert (~firm).mean() < 0.01
    hit = out.hit.cpu().numpy().astype(bool)
    assert np.array_equal(hit[firm], ref.hit[firm])
    both = firm & ref.hit
    assert both.sum() > 5000
    t = out.t.cpu().numpy()
    assert np.allclose(t[both], ref.t[both], rtol=1e-5)
    assert np.allclose(out.normal.cpu().numpy().T[both], ref.normal[both], atol=1e-4)
    assert np.array_equal(out.mat.cpu().numpy()[both], ref.mat[both])
    assert np.allclose(out.albedo.cpu().numpy().T[both], ref.albedo[both], atol=1e-7)
    miss = firm & ~ref.hit
    assert np.all(np.isinf(t[miss])) and np.all(out.mat.cpu().numpy()[miss] == -1)
    # every precision path answers mesh objects the same way (no network)
    for prec in (lsnif.BF16_FUSED, lsnif.FP8_FUSED):
        o2 = ctx.query_rays(_cuda(rays), obj=h, precision=prec)
        torch.cuda.synchronize()
        assert torch.equal(o2.hit, out.hit) and torch.equal(o2.t, out.t)
    ctx.unload_object(h)


def test_face_count_switch_and_lsnif_only_calls(ctx):
    small, big = I.icosphere(2), I.noise_icosphere(seed=3, target_tris=5000, n_mat=2)
    cfg = I.cfg_icosphere_small()
    hs = ctx.load_object(small, cfg, bvh_below_faces=1000)
    hb = ctx.load_object(big, cfg, bvh_below_faces=1000)
    assert ctx.object_info(hs).kind == 1 and ctx.object_info(hb).kind == 0
    rays = _cuda(I.rays_sphere_to_box(64, 3.0, (-1, -1, -1), (1, 1, 1), seed=3))
    for call in (lambda: ctx.read_params(hs, lsnif.PARAM_MLP), lambda: ctx.save_object(hs),
                 lambda: ctx.trace(rays, hs), lambda: ctx.label_rays(rays, hs)):
        with pytest.raises(lsnif.LsnifError) as e:
            call()
        assert e.value.code == -10
    ctx.unload_object(hs)
    ctx.unload_object(hb)


def test_mixed_batch_and_scene_with_mesh_objects(ctx):
    """LSNIF objects and mesh objects in one per-ray batch and in one
    instanced scene: each ray gets its own object's answer; the scene keeps
    the nearest over both kinds."""
    cfg = I.Config(V=8, H=18, L=4, F=2, log2_T=10, N_min=4, N_max=16, n_hidden=1, width=64, n_mat=3)
    cube = I.cube(n_mat=3)
    p = I.constant_params(cfg, OUT_BIAS)
    h_cube = ctx.load_object(cube, cfg, tables=p.tables, mlp=p.packed_mlp())
    sphere = I.icosphere(3)
    h_sph = ctx.load_mesh(sphere, n_mat=3)
    torus = I.noise_torus_tris(4, 6000, n_mat=3)
    h_tor = ctx.load_mesh(torus)
    # per-ray batch over the three objects
    n = 9000
    rays = np.concatenate([I.rays_sphere_to_box(n // 3, 3.0, m.verts.min(0), m.verts.max(0), seed=20 + i)
                           for i, m in enumerate([cube, sphere, torus])], axis=1)
    objs = np.repeat(np.array([h_cube, h_sph, h_tor], np.uint32), n // 3)
    for prec in (lsnif.FP32_PLAIN, lsnif.BF16_FUSED):
        out = ctx.query_rays(_cuda(rays), obj_per_ray=_cuda(objs), precision=prec)
        ctx.check()
        torch.cuda.synchronize()
        hit = out.hit.cpu().numpy().astype(bool)
        t = out.t.cpu().numpy()
        for i, m in enumerate([sphere, torus]):
            sl = slice((i + 1) * (n // 3), (i + 2) * (n // 3))
            ref, _ = O.mesh_query(O.mesh_object(m), rays[:, sl])
            firm = _edge_margin(m, O.judge(m, rays[:, sl])) >= 1e-5
            assert np.array_equal(hit[sl][firm], ref.hit[firm])
            b = firm & ref.hit
            assert np.allclose(t[sl][b], ref.t[b], rtol=1e-5)
        # the LSNIF cube's rays: the constant network's midpoint hits
        orc = O.build_object(cube, cfg, p)
        ref, seg = O.query(orc, rays[:, : n // 3])
        ok = ~seg.near
        assert np.array_equal(hit[: n // 3][ok], ref.hit[ok])
    # instanced scene: LSNIF cube + mesh sphere + mesh torus
    R = I.rotation([0.2, 0.9, 0.1], 1.1)
    insts = [O.Instance(0, np.eye(3), np.zeros(3)), O.Instance(1, R.T / 0.6, -(R.T / 0.6) @ np.array([2.0, 0.5, 0.3])),
             O.Instance(2, np.eye(3), -np.array([-1.5, 1.0, -0.5])), O.Instance(1, np.eye(3) * 2, np.array([0, 0, -3.0]))]
    insts = [O.Instance(i.obj, i.A.astype(np.float32).astype(np.float64), i.b.astype(np.float32).astype(np.float64))
             for i in insts]
    handles = [h_cube, h_sph, h_tor]
    g = np.random.default_rng(5)
    m = 20000
    eye = g.normal(size=(m, 3))
    eye = 9.0 * eye / np.linalg.norm(eye, axis=1, keepdims=True)
    tgt = g.uniform(-2.5, 2.5, size=(m, 3))
    wr = np.zeros((8, m), np.float32)
    wr[0:3] = eye.T
    wr[3:6] = (tgt - eye).T
    wr[7] = np.inf
    res, inst = ctx.query_scene(_cuda(wr), [(handles[i.obj], i.A, i.b) for i in insts], precision=lsnif.FP32_PLAIN)
    torch.cuda.synchronize()
    ref = O.scene_query([O.build_object(cube, cfg, p), O.mesh_object(sphere), O.mesh_object(torus)], insts, wr)
    got_inst = inst.cpu().numpy()
    ok = ~ref["near"]
    agree = got_inst[ok] == ref["inst"][ok]
    assert agree.mean() > 0.995, agree.mean()
    both = ok & (got_inst == ref["inst"]) & ref["hit"]
    assert both.sum() > 3000
    assert np.allclose(res.t.cpu().numpy()[both], ref["t"][both], rtol=1e-5)
    for h in handles:
        ctx.unload_object(h)


def test_gbuffer_of_mesh_objects(ctx):
    """The rasteriser reads mesh objects' triangles directly."""
    sphere = I.icosphere(3)
    h = ctx.load_mesh(sphere)
    eye = np.array([0.0, -4.0, 1.0])
    f = -eye / np.linalg.norm(eye)
    r = np.cross(f, [0, 0, 1.0])
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    eye, f, r, u = (np.asarray(x, np.float32).astype(np.float64) for x in (eye, f, r, u))
    tan = float(np.float32(0.4))
    gb = ctx.raster_gbuffer(eye, f, r, u, tan, 64, 48, [(h, np.eye(3), np.zeros(3))])
    torch.cuda.synchronize()
    ref = O.gbuffer([sphere], [O.Instance(0, np.eye(3), np.zeros(3))], eye, f, r, u, tan, 64, 48)
    got = gb.shape.cpu().numpy().reshape(-1)
    assert (got == ref["shape"]).mean() > 0.99 and (ref["shape"] >= 0).sum() > 500
    ctx.unload_object(h)
