"""GPU instanced-scene query and bounce rays against the oracle (Sec. 4
wavefront integration over the instancing of Sec. 6)."""
import math

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


def _aim(insts, n, seed, objs_box):
    """Rays from a radius-12 sphere at jittered instance box centres; 30% of
    them start past the ray origin (tmin > 0)."""
    g = np.random.default_rng(seed)
    eye = g.normal(size=(n, 3))
    eye = 12.0 * eye / np.linalg.norm(eye, axis=1, keepdims=True)
    cen = []
    for inst in insts:
        lo, hi = objs_box[inst.obj]
        cen.append(np.linalg.solve(inst.A, 0.5 * (lo + hi) - inst.b))
    cen = np.array(cen)
    tgt = cen[g.integers(0, len(insts), n)] + g.uniform(-0.6, 0.6, size=(n, 3))
    rays = np.zeros((8, n), np.float32)
    rays[0:3] = eye.T
    rays[3:6] = (tgt - eye).T
    rays[6] = np.where(g.random(n) < 0.3, g.uniform(0.0, 0.9, n), 0.0)
    rays[7] = np.inf
    return rays


def _gpu_scene(ctx, rays, insts, handles, prec):
    res, inst = ctx.query_scene(_cuda(rays), [(handles[i.obj], i.A, i.b) for i in insts], precision=prec)
    torch.cuda.synchronize()
    return dict(hit=res.hit.cpu().numpy().astype(bool), t=res.t.cpu().numpy(), normal=res.normal.cpu().numpy().T,
                mat=res.mat.cpu().numpy(), albedo=res.albedo.cpu().numpy().T, inst=inst.cpu().numpy())


def _f32(insts):
    """The transforms as the library receives them (FP32), back in FP64."""
    return [O.Instance(i.obj, i.A.astype(np.float32).astype(np.float64), i.b.astype(np.float32).astype(np.float64))
            for i in insts]


@pytest.mark.parametrize("prec", [lsnif.FP32_PLAIN, lsnif.BF16_FUSED])
def test_cube_scene_matches_oracle_and_closed_form(ctx, prec):
    cfg = I.Config(V=8, H=18, L=4, F=2, log2_T=10, N_min=4, N_max=16, n_hidden=1, width=64, n_mat=3)
    mesh = I.cube(n_mat=3)
    p = I.constant_params(cfg, OUT_BIAS)
    obj = O.build_object(mesh, cfg, p)
    h = ctx.load_object(mesh, cfg, tables=p.tables, mlp=p.packed_mlp())
    R = I.rotation([0, 0, 1], math.pi / 2)
    S = I.rotation([1, 1, 0], 0.7)
    insts = _f32([O.Instance(0, np.eye(3), np.zeros(3)),
                  O.Instance(0, R.T, -R.T @ np.array([3.0, 0.5, 0.0])),
                  O.Instance(0, S.T / 0.5, -(S.T / 0.5) @ np.array([-2.5, 1.0, 1.5]))])
    rays = _aim(insts, 20000, 3, {0: (obj.bmin.astype(np.float64), obj.bmax.astype(np.float64))})
    got = _gpu_scene(ctx, rays, insts, {0: h}, prec)
    ref = O.scene_query([obj], insts, rays)
    ok = ~ref["near"]
    assert ok.mean() > 0.9
    assert np.array_equal(got["hit"][ok], ref["hit"][ok])
    hh = ok & ref["hit"]
    assert hh.mean() > 0.5
    assert np.array_equal(got["inst"][ok], ref["inst"][ok])
    assert np.allclose(got["t"][hh], ref["t"][hh], rtol=2e-6, atol=1e-6)
    assert np.allclose(got["normal"][hh], ref["normal"][hh], atol=2e-6)
    assert np.all(got["mat"][hh] == 1)
    assert np.allclose(got["albedo"][hh], 0.5)
    miss = ok & ~ref["hit"]
    assert np.all(np.isinf(got["t"][miss])) and np.all(got["mat"][miss] == -1)
    ctx.unload_object(h)


@pytest.fixture(scope="module")
def scene(ctx):
    objs, handles, boxes = [], {}, {}
    for k, (mesh, cfg) in enumerate([(I.noise_icosphere(seed=11, target_tris=5000, amplitude=0.08, n_mat=2),
                                      I.cfg_icosphere_small()),
                                     (I.icosphere(3), I.cfg_icosphere_small())]):
        p = I.random_params(cfg, 40 + k, table_range=0.5, bias_range=0.5)
        p.weights[-1][1][0] = 2.0   # occupancy logit biased towards hits
        objs.append(O.build_object(mesh, cfg, p))
        handles[k] = ctx.load_object(mesh, cfg, tables=p.tables, mlp=p.packed_mlp())
        boxes[k] = (objs[-1].bmin.astype(np.float64), objs[-1].bmax.astype(np.float64))
    insts = _f32([O.Instance(o, A, b) for o, A, b in I.seeded_instances(6, 2, seed=21)])
    return dict(objs=objs, handles=handles, boxes=boxes, insts=insts)


ORACLE_PRECISION = {lsnif.FP32_PLAIN: "f64", lsnif.BF16_FUSED: "bf16", lsnif.FP8_FUSED: "fp8",
                    lsnif.FP16_FUSED: "fp16"}


@pytest.mark.parametrize("prec", [lsnif.FP32_PLAIN, lsnif.BF16_FUSED, lsnif.FP8_FUSED, lsnif.FP16_FUSED])
def test_instanced_scene_matches_oracle(ctx, scene, prec):
    rays = _aim(scene["insts"], 6000, 5, scene["boxes"])
    got = _gpu_scene(ctx, rays, scene["insts"], scene["handles"], prec)
    ref = O.scene_query(scene["objs"], scene["insts"], rays, ORACLE_PRECISION[prec])
    ok = ~ref["near"]
    assert ok.mean() > 0.8
    agree = got["hit"][ok] == ref["hit"][ok]
    assert agree.mean() > (0.999 if prec == lsnif.FP32_PLAIN else 0.99), agree.mean()
    both = ok & got["hit"] & ref["hit"]
    assert both.sum() > 500
    same = both & (got["inst"] == ref["inst"])
    assert same.sum() >= 0.99 * both.sum()
    diag = max(np.linalg.norm(b[1] - b[0]) for b in scene["boxes"].values())
    tol = 1e-4 if prec == lsnif.FP32_PLAIN else 2e-2
    assert np.quantile(np.abs(got["t"][same] - ref["t"][same]), 0.99) < tol * diag
    cosang = np.einsum("ij,ij->i", got["normal"][same], ref["normal"][same])
    assert np.quantile(cosang, 0.01) > (1 - 1e-6 if prec == lsnif.FP32_PLAIN else 0.99)
    assert (got["mat"][same] == ref["mat"][same]).mean() > 0.99


@pytest.mark.parametrize("prec", [lsnif.FP32_PLAIN, lsnif.BF16_FUSED, lsnif.FP8_FUSED])
def test_grouping_modes_give_identical_scene_results(ctx, scene, prec):
    """Pairs grouped by (object, point count) or by object in ray order:
    the same bits."""
    rays = _cuda(_aim(scene["insts"], 6000, 13, scene["boxes"]))
    insts = [(scene["handles"][i.obj], i.A, i.b) for i in scene["insts"]]
    got = []
    try:
        for g in (0, 1):
            ctx.set_group_mode(g)
            res, inst = ctx.query_scene(rays, insts, precision=prec)
            ctx.check()
            got.append([x.cpu() for x in (res.hit, res.t, res.normal, res.mat, inst)])
    finally:
        ctx.set_group_mode(0)
    for a, b in zip(*got):
        assert torch.equal(torch.nan_to_num(a, posinf=-1.0), torch.nan_to_num(b, posinf=-1.0))


def test_identity_instance_equals_plain_query(ctx, scene):
    h = scene["handles"][0]
    obj = scene["objs"][0]
    rays = I.rays_sphere_to_box(5000, 3.0, obj.bmin, obj.bmax, seed=6)
    for prec in (lsnif.FP32_PLAIN, lsnif.BF16_FUSED):
        res, inst = ctx.query_scene(_cuda(rays), [(h, np.eye(3), np.zeros(3))], precision=prec)
        plain = ctx.query_rays(_cuda(rays), obj=h, precision=prec)
        torch.cuda.synchronize()
        hit = plain.hit.bool()
        assert torch.equal(res.hit, plain.hit)
        assert torch.equal(res.t[hit], plain.t[hit])
        assert torch.equal(res.mat[hit], plain.mat[hit])
        assert torch.allclose(res.normal[:, hit], plain.normal[:, hit], atol=1e-6)
        assert torch.all(inst[hit] == 0) and torch.all(inst[~hit] == -1)


def test_bounce_rays_match_oracle(ctx):
    g = np.random.default_rng(7)
    n = 50000
    rays = np.zeros((8, n), np.float32)
    rays[0:3] = g.normal(size=(3, n))
    rays[3:6] = g.normal(size=(3, n))
    rays[7] = np.inf
    hit = g.random(n) < 0.8
    t = g.uniform(0.5, 2.0, n).astype(np.float32)
    normal = g.normal(size=(n, 3))
    normal[:100] = 0.0
    u = g.random((n, 2)).astype(np.float32)
    res = lsnif.QueryResult(_cuda(hit.astype(np.uint8)), _cuda(t), _cuda(normal.T.astype(np.float32)),
                            _cuda(np.zeros(n, np.int32)), _cuda(np.zeros((3, n), np.float32)), None)
    out = ctx.bounce_rays(_cuda(rays), res, _cuda(u), 1e-3).cpu().numpy()
    ref = O.bounce_rays(rays, hit, t.astype(np.float64), normal.astype(np.float32).astype(np.float64),
                        u.astype(np.float64), 1e-3)
    assert np.allclose(out[0:6], ref[0:6], atol=2e-5)
    assert np.array_equal(out[6], ref[6]) and np.all(np.isinf(out[7]))
    live = hit & (np.arange(n) >= 100)
    assert np.allclose(np.linalg.norm(out[3:6, live], axis=0), 1.0, atol=1e-5)


def test_scene_rejects_bad_instances(ctx, scene):
    rays = _cuda(np.zeros((8, 16), np.float32))
    with pytest.raises(lsnif.LsnifError):
        ctx.query_scene(rays, [(scene["handles"][0], np.zeros((3, 3)), np.zeros(3))])
    with pytest.raises(lsnif.LsnifError):
        ctx.query_scene(rays, [(12345, np.eye(3), np.zeros(3))])
