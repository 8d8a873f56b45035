"""Pins of the oracle's instanced-scene query and bounce rays (Sec. 4
wavefront integration, Sec. 6 instancing) against closed forms: a cube
object whose network outputs are constants, so the nearest hit of every ray
is the midpoint of its box interval in the nearest instance."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_21627_gb300 import inputs as I

# occupancy logit 5, local t logit 0 (midpoint), normal +x, albedo logits 0,
# material logits favour material 1
OUT_BIAS = [5.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 2.0, 0.0]


def _cube_object():
    cfg = I.Config(V=8, H=18, L=4, F=2, log2_T=10, N_min=4, N_max=16, n_hidden=1, width=64, n_mat=3)
    mesh = I.cube(n_mat=3)
    return O.build_object(mesh, cfg, I.constant_params(cfg, OUT_BIAS)), mesh, cfg


def _instances():
    R = I.rotation([0, 0, 1], math.pi / 2)
    S = I.rotation([1, 1, 0], 0.7)
    return [
        O.Instance(0, np.eye(3), np.zeros(3)),
        O.Instance(0, R.T, -R.T @ np.array([3.0, 0.5, 0.0])),
        O.Instance(0, S.T / 0.5, -(S.T / 0.5) @ np.array([-2.5, 1.0, 1.5])),   # scaled by 0.5
    ]


def _rays(n, seed, insts):
    g = np.random.default_rng(seed)
    eye = g.normal(size=(n, 3))
    eye = 12.0 * eye / np.linalg.norm(eye, axis=1, keepdims=True)
    centres = np.array([np.linalg.solve(i.A, np.full(3, 0.5) - i.b) for i in insts])
    tgt = centres[g.integers(0, len(insts), n)] + g.uniform(-0.6, 0.6, size=(n, 3))
    d = tgt - eye
    rays = np.zeros((8, n), np.float32)
    rays[0:3] = eye.T
    rays[3:6] = d.T
    rays[6] = np.where(g.random(n) < 0.3, g.uniform(0.0, 0.9, n), 0.0)   # some start past a box
    rays[7] = np.inf
    return rays


def _closed_form(rays, insts):
    """Nearest box-interval midpoint over the instances, by a plain slab test
    of the world ray mapped into each instance's frame (the cube is [0,1]^3)."""
    r = rays.astype(np.float64)
    n = r.shape[1]
    best = np.full(n, np.inf)
    who = np.full(n, -1)
    for i, inst in enumerate(insts):
        o = (inst.A @ r[0:3]).T + inst.b
        d = (inst.A @ r[3:6]).T
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (0.0 - o) / d
            tb = (1.0 - o) / d
        lo = np.nanmax(np.minimum(ta, tb), axis=1)
        hi = np.nanmin(np.maximum(ta, tb), axis=1)
        t0 = np.maximum(lo, r[6])
        ok = hi > t0
        mid = t0 + 0.5 * (hi - t0)
        take = ok & (mid < best)
        best[take] = mid[take]
        who[take] = i
    return best, who


def test_scene_query_matches_closed_form():
    obj, _, _ = _cube_object()
    insts = _instances()
    rays = _rays(3000, 3, insts)
    res = O.scene_query([obj], insts, rays)
    t, who = _closed_form(rays, insts)
    ok = ~res["near"]
    assert ok.mean() > 0.9
    assert np.array_equal(res["hit"][ok], np.isfinite(t[ok]))
    assert (res["hit"][ok]).mean() > 0.5
    h = ok & res["hit"]
    assert np.array_equal(res["inst"][h], who[h])
    assert np.allclose(res["t"][h], t[h], rtol=1e-5)
    # world normal: A^T e_x, normalised
    for i, inst in enumerate(insts):
        m = h & (res["inst"] == i)
        want = inst.A.T @ np.array([1.0, 0.0, 0.0])
        want /= np.linalg.norm(want)
        assert m.sum() > 50
        assert np.allclose(res["normal"][m], want, atol=1e-12)
    assert np.all(res["mat"][h] == 1)
    assert np.allclose(res["albedo"][h], 0.5)
    miss = ok & ~res["hit"]
    assert np.all(res["inst"][miss] == -1) and np.all(np.isinf(res["t"][miss]))
    assert np.all(res["mat"][miss] == -1)


def test_identity_instance_equals_plain_query():
    cfg = I.cfg_icosphere_small()
    mesh = I.icosphere(3)
    obj = O.build_object(mesh, cfg, I.random_params(cfg, 3, table_range=0.5, bias_range=0.5))
    rays = I.rays_sphere_to_box(800, 3.0, obj.bmin, obj.bmax, seed=8)
    res = O.scene_query([obj], [O.Instance(0, np.eye(3), np.zeros(3))], rays)
    h, _ = O.query(obj, rays)
    assert np.array_equal(res["hit"], h.hit)
    assert np.array_equal(res["t"][h.hit], h.t[h.hit])
    assert np.array_equal(res["mat"][h.hit], h.mat[h.hit])
    nrm = h.normal[h.hit] / np.linalg.norm(h.normal[h.hit], axis=1, keepdims=True)
    assert np.allclose(res["normal"][h.hit], nrm, atol=1e-15)


def test_rotation_keeps_angles_and_ties_take_the_lowest_instance():
    """A rotated instance sees the rotated ray: the angle between ray and
    normal is the object-frame angle; two coincident instances tie and the
    lower index wins."""
    cfg = I.cfg_icosphere_small()
    mesh = I.icosphere(3)
    obj = O.build_object(mesh, cfg, I.random_params(cfg, 5, table_range=0.5, bias_range=0.5))
    R = I.rotation([0.3, -0.5, 0.8], 1.1)
    inst = O.Instance(0, R.T, np.zeros(3))
    rays = I.rays_sphere_to_box(800, 3.0, obj.bmin, obj.bmax, seed=9).astype(np.float64)
    world = rays.copy()
    world[0:3] = R @ rays[0:3]
    world[3:6] = R @ rays[3:6]
    res = O.scene_query([obj], [inst, inst], world.astype(np.float32))
    h = res["hit"] & ~res["near"]
    assert h.sum() > 100
    assert np.all(res["inst"][res["hit"]] == 0)
    loc, _ = O.query(obj, O.to_object_frame(world.astype(np.float32), inst).astype(np.float32))
    d_w = world[3:6, h].T / np.linalg.norm(world[3:6, h].T, axis=1, keepdims=True)
    d_l = (R.T @ world[3:6, h]).T
    d_l /= np.linalg.norm(d_l, axis=1, keepdims=True)
    n_l = loc.normal[h] / np.linalg.norm(loc.normal[h], axis=1, keepdims=True)
    cos_w = np.einsum("ij,ij->i", d_w, res["normal"][h])
    cos_l = np.einsum("ij,ij->i", d_l, n_l)
    assert np.allclose(cos_w, cos_l, atol=1e-9)


def test_bounce_rays():
    g = np.random.default_rng(4)
    n = 20000
    rays = np.zeros((8, n))
    rays[0:3] = g.normal(size=(3, n))
    rays[3:6] = g.normal(size=(3, n))
    rays[7] = np.inf
    hit = g.random(n) < 0.8
    t = g.uniform(0.5, 2.0, n)
    normal = g.normal(size=(n, 3))
    normal /= np.linalg.norm(normal, axis=1, keepdims=True)
    normal[:50] = 0.0                              # zero normal: dead ray
    u = g.random((n, 2))
    out = O.bounce_rays(rays, hit, t, normal, u, eps=1e-3)
    live = hit & (np.arange(n) >= 50)
    assert np.all(out[3:6, ~live] == 0) and np.all(np.isinf(out[7]))
    d = rays[3:6].T
    nf = np.where((np.einsum("ij,ij->i", normal, d) > 0)[:, None], -normal, normal)
    p = rays[0:3].T + t[:, None] * d + 1e-3 * nf
    assert np.allclose(out[0:3, live].T, p[live], atol=1e-12)
    dirs = out[3:6, live].T
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1.0, atol=1e-12)
    cos = np.einsum("ij,ij->i", dirs, nf[live])
    assert np.all(cos >= -1e-12)
    # cosine-weighted hemisphere: E[cos] = 2/3, Var[cos] = 1/2 - 4/9
    sd = math.sqrt((0.5 - 4.0 / 9.0) / live.sum())
    assert abs(cos.mean() - 2.0 / 3.0) < 4 * sd
    # u0 = 0 is the normal itself
    out0 = O.bounce_rays(rays[:, :5], np.ones(5, bool), t[:5], normal[50:55], np.zeros((5, 2)), eps=0.0)
    nf0 = np.where((np.einsum("ij,ij->i", normal[50:55], d[:5]) > 0)[:, None], -normal[50:55], normal[50:55])
    assert np.allclose(out0[3:6].T, nf0, atol=1e-12)


def test_mesh_object_in_a_scene_is_exact():
    """A mesh object (a flat quad, vertex normals +z, two materials) through a
    rotated, scaled, translated instance beside an LSNIF cube: hits on the
    quad are the plane intersection in closed form, with the world normal
    A^T e_z normalised and the triangle's material; a ray hitting both keeps
    the nearer."""
    v = np.array([[-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 1, 0]], np.float32)
    quad = I.Mesh(v, np.array([[0, 1, 2], [1, 3, 2]], np.int32), np.tile(np.array([[0, 0, 1.0]], np.float32), (4, 1)),
                  np.array([0, 1], np.int32), np.array([[0.2, 0.3, 0.4], [0.6, 0.5, 0.1]], np.float32), 2)
    cube_obj, _, _ = _cube_object()
    R = I.rotation([0.3, 0.4, 1.0], 0.8)
    A = R.T / 1.5
    c = np.array([0.5, -2.0, 0.7])
    insts = [O.Instance(1, A, -A @ c), O.Instance(0, np.eye(3), np.zeros(3))]
    objs = [cube_obj, O.mesh_object(quad)]
    g = np.random.default_rng(7)
    n = 4000
    # rays from above the quad's plane towards random points of the quad
    nrm_w = R @ np.array([0.0, 0.0, 1.0])
    tgt_local = np.c_[g.uniform(-1.2, 1.2, (n, 2)), np.zeros(n)]
    tgt = (R @ (1.5 * tgt_local).T).T + c
    eye = tgt + 4.0 * nrm_w + g.normal(size=(n, 3))
    rays = np.zeros((8, n), np.float32)
    rays[0:3] = eye.T
    rays[3:6] = (tgt - eye).T
    rays[7] = np.inf
    res = O.scene_query(objs, insts, rays)
    r = rays.astype(np.float64)
    local = O.to_object_frame(r, insts[0]).astype(np.float32).astype(np.float64)
    t_plane = -local[2] / local[5]
    p = local[0:3] + t_plane * local[3:6]
    on_quad = (np.abs(p[0]) < 1 - 1e-6) & (np.abs(p[1]) < 1 - 1e-6) & (np.abs(p[0] + p[1]) > 1e-6)
    only_quad = on_quad & (res["inst"] != 1)
    assert only_quad.sum() > 1000
    assert np.all(res["inst"][only_quad] == 0) and np.all(res["hit"][only_quad])
    assert np.allclose(res["t"][only_quad], t_plane[only_quad], rtol=1e-12)
    want_n = A.T @ np.array([0, 0, 1.0])
    assert np.allclose(res["normal"][only_quad], want_n / np.linalg.norm(want_n), atol=1e-12)
    tri = np.where(p[0] + p[1] < 0, 0, 1)
    assert np.array_equal(res["mat"][only_quad], tri[only_quad])
    assert np.allclose(res["albedo"][only_quad], quad.albedo[tri[only_quad]])
    assert np.all(~res["hit"][~on_quad & (res["inst"] != 1)])
