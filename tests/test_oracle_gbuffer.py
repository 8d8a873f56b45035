"""Pins of the oracle's primary-ray G-buffer (Sec. 4, Fig. 4a: shape index,
primitive index, barycentric UV and camera distance per pixel) against
closed forms: the pinhole projection (the inverse of the pixel rays), a
face-on view of the unit cube, 2-D point-in-triangle tests of projected
triangles, plane distances, occlusion order and instance transforms."""
import math

import numpy as np

from oracle import oracle as O
from paper_2504_21627_gb300 import inputs as I


def _cam(eye, target, up0=(0.0, 0.0, 1.0)):
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, up0)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    return eye, f, r, u


def _project(p, eye, f, r, u, tan, W, H):
    """Continuous screen position of world points (pixel centres at +0.5)."""
    q = p - eye
    xc, yc, zc = q @ r, q @ u, q @ f
    sx = (xc / zc / (tan * W / H) + 1.0) * W / 2.0
    sy = (1.0 - yc / zc / tan) * H / 2.0
    return sx, sy, zc


def test_pixel_rays_invert_the_projection():
    eye, f, r, u = _cam([3.0, -2.0, 1.5], [0.1, 0.2, -0.1])
    W, H, tan = 37, 23, math.tan(math.radians(30.0))
    o, d = O.pixel_rays(eye, f, r, u, tan, W, H)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    sx, sy, zc = _project(o + 2.5 * d, eye, f, r, u, tan, W, H)
    py, px = np.divmod(np.arange(W * H), W)
    assert np.all(zc > 0)
    assert np.allclose(sx, px + 0.5, atol=1e-9) and np.allclose(sy, py + 0.5, atol=1e-9)


def test_face_on_cube():
    """Camera on the cube's axis at z = -2 looking at +z: a pixel hits the
    face z = 0 iff the ray's point there lies in [0,1]^2; triangle 0 (v0,
    v2, v1) holds x + y <= 1 with (u, v) = (y, x), triangle 1 (v1, v2, v3)
    the rest with (u, v) = (1 - x, x + y - 1); distance 2 / d_z."""
    W = H = 64
    eye, f, r, u = np.array([0.5, 0.5, -2.0]), np.array([0.0, 0.0, 1.0]), np.array([-1.0, 0.0, 0.0]), \
        np.array([0.0, 1.0, 0.0])
    tan = 0.4
    g = O.gbuffer([I.cube()], [O.Instance(0, np.eye(3), np.zeros(3))], eye, f, r, u, tan, W, H)
    _, d = O.pixel_rays(eye, f, r, u, tan, W, H)
    t = 2.0 / d[:, 2]
    p = eye[None, :] + t[:, None] * d
    x, y = p[:, 0], p[:, 1]
    inside = (x >= 0) & (x <= 1) & (y >= 0) & (y <= 1)
    margin = np.minimum.reduce([x, 1 - x, y, 1 - y, np.abs(x + y - 1)])
    firm = margin > 1e-9
    assert inside.sum() > 300 and (~inside).sum() > 300
    assert np.array_equal(g["shape"][firm], np.where(inside[firm], 0, -1))
    hit = firm & inside
    lower = x + y < 1
    assert np.array_equal(g["prim"][hit], np.where(lower[hit], 0, 1))
    assert np.allclose(g["dist"][hit], t[hit], rtol=1e-13)
    want_u = np.where(lower, y, 1 - x)
    want_v = np.where(lower, x, x + y - 1)
    assert np.allclose(g["u"][hit], want_u[hit], atol=1e-12) and np.allclose(g["v"][hit], want_v[hit], atol=1e-12)
    miss = firm & ~inside
    assert np.all(np.isinf(g["dist"][miss])) and np.all(g["prim"][miss] == -1)
    # pixels on the diagonal: either triangle is a correct answer
    diag = inside & (np.abs(x + y - 1) <= 1e-9) & (np.minimum.reduce([x, 1 - x, y, 1 - y]) > 1e-9)
    assert diag.sum() > 0 and np.all(np.isin(g["prim"][diag], [0, 1]))


def test_single_triangles_cover_their_projection():
    """A triangle in front of the camera covers exactly the pixel centres
    inside its 2-D projection (edge functions of the projected vertices);
    the distance is the ray's distance to the triangle's plane; (u, v)
    rebuild the hit point."""
    rng = np.random.default_rng(5)
    W, H, tan = 48, 40, math.tan(math.radians(25.0))
    for trial in range(6):
        eye, f, r, u = _cam(rng.normal(size=3) * 3 + np.array([0, 0, 4.0]), rng.normal(size=3) * 0.2)
        verts = (eye + 5.0 * f + rng.normal(size=(3, 3)) * 1.2).astype(np.float32)
        mesh = I.single_triangle(*verts)
        g = O.gbuffer([mesh], [O.Instance(0, np.eye(3), np.zeros(3))], eye, f, r, u, tan, W, H)
        a, b, c = verts.astype(np.float64)
        sx, sy, zc = _project(np.stack([a, b, c]), eye, f, r, u, tan, W, H)
        assert np.all(zc > 0)
        py, px = np.divmod(np.arange(W * H), W)
        qx, qy = px + 0.5, py + 0.5
        e = []
        for i, j in ((0, 1), (1, 2), (2, 0)):
            ex, ey = sx[j] - sx[i], sy[j] - sy[i]
            e.append((ex * (qy - sy[i]) - ey * (qx - sx[i])) / math.hypot(ex, ey))
        e = np.stack(e)
        inside = np.all(e > 0, axis=0) | np.all(e < 0, axis=0)
        firm = np.min(np.abs(e), axis=0) > 1e-6
        assert np.array_equal(g["shape"][firm] == 0, inside[firm]), trial
        hit = firm & inside
        assert hit.sum() > 0
        o, d = O.pixel_rays(eye, f, r, u, tan, W, H)
        n = np.cross(b - a, c - a)
        t = ((a - o) @ n) / (d @ n)
        assert np.allclose(g["dist"][hit], t[hit], rtol=1e-10)
        p = (1 - g["u"] - g["v"])[:, None] * a + g["u"][:, None] * b + g["v"][:, None] * c
        assert np.allclose(p[hit], (o + g["dist"][:, None] * d)[hit], atol=1e-9)
        assert np.all(g["prim"][hit] == 0)


def _quad(z, half=1.0):
    v = np.array([[-half, -half, z], [half, -half, z], [-half, half, z], [half, half, z]], np.float32)
    t = np.array([[0, 1, 2], [1, 3, 2]], np.int32)
    return I.Mesh(v, t, np.tile(np.array([[0, 0, 1.0]], np.float32), (4, 1)), np.zeros(2, np.int32),
                  np.full((1, 3), 0.5, np.float32), 1)


def test_occlusion_and_instance_ties():
    """Three instances of one quad: instance 0 far (z = 0 plane shifted to z
    = 2 by its transform), instances 1 and 2 coincident and nearer (z = 1)
    but narrower. Where they overlap the nearest wins, and of the two
    coincident instances the lower index."""
    quad = _quad(0.0)
    far = O.Instance(0, np.eye(3), np.array([0.0, 0.0, -2.0]))            # p_obj = p - (0,0,2): plane z = 2
    s = 2.0                                                                # object = 2 x world: half width 0.5
    near = O.Instance(0, np.eye(3) * s, np.array([0.0, 0.0, -s * 1.0]))   # plane z = 1
    eye, f, r, u = np.array([0.0, 0.0, -3.0]), np.array([0.0, 0.0, 1.0]), np.array([-1.0, 0.0, 0.0]), \
        np.array([0.0, 1.0, 0.0])
    W = H = 40
    tan = 0.3
    g = O.gbuffer([quad], [far, near, near], eye, f, r, u, tan, W, H)
    _, d = O.pixel_rays(eye, f, r, u, tan, W, H)
    t1, t2 = 4.0 / d[:, 2], 5.0 / d[:, 2]
    p1 = eye + t1[:, None] * d
    p2 = eye + t2[:, None] * d
    in_near = (np.abs(p1[:, 0]) < 0.5 - 1e-9) & (np.abs(p1[:, 1]) < 0.5 - 1e-9)
    in_far = (np.abs(p2[:, 0]) < 1.0 - 1e-9) & (np.abs(p2[:, 1]) < 1.0 - 1e-9)
    assert in_near.sum() > 20 and (in_far & ~in_near).sum() > 20
    assert np.all(g["shape"][in_near] == 1)
    assert np.allclose(g["dist"][in_near], t1[in_near], rtol=1e-13)
    only_far = in_far & ~in_near & ~((np.abs(np.abs(p1[:, 0]) - 0.5) < 1e-9) | (np.abs(np.abs(p1[:, 1]) - 0.5) < 1e-9))
    assert np.all(g["shape"][only_far] == 0)
    assert np.allclose(g["dist"][only_far], t2[only_far], rtol=1e-13)


def test_instance_equals_the_pretransformed_mesh():
    mesh = I.icosphere(2)
    A = I.rotation([0.3, 0.8, -0.2], 0.9) / 1.7
    b = np.array([0.4, -0.3, 0.9])
    inv = np.linalg.inv(A)
    world = I.Mesh(((mesh.verts.astype(np.float64) - b) @ inv.T).astype(np.float32), mesh.tris, mesh.vnormals,
                   mesh.tri_mat, mesh.albedo, mesh.n_mat)
    eye, f, r, u = _cam([4.0, 3.0, 2.0], [0.0, 0.0, 0.0])
    W, H, tan = 56, 42, math.tan(math.radians(22.0))
    gi = O.gbuffer([mesh], [O.Instance(0, A, b)], eye, f, r, u, tan, W, H)
    gw = O.gbuffer([world], [O.Instance(0, np.eye(3), np.zeros(3))], eye, f, r, u, tan, W, H)
    hit = gi["shape"] >= 0
    assert 200 < hit.sum() < W * H
    # the world mesh is rounded to FP32: compare away from triangle edges
    firm = hit & (np.minimum.reduce([gi["u"], gi["v"], 1 - gi["u"] - gi["v"]]) > 1e-4)
    assert firm.sum() > 0.8 * hit.sum()
    assert ((gw["shape"] >= 0) == hit).mean() > 0.99
    assert np.array_equal(gw["prim"][firm], gi["prim"][firm])
    assert np.allclose(gw["dist"][firm], gi["dist"][firm], rtol=1e-6)
    assert np.allclose(gw["u"][firm], gi["u"][firm], atol=1e-5) and np.allclose(gw["v"][firm], gi["v"][firm], atol=1e-5)


def test_normals_and_unclipped_triangle_solution():
    """A flat quad whose vertex normals are +z, seen through a rotated and
    scaled instance: every hit's world normal is A^T e_z normalised (R e_z
    for A = R^T / s); and the unclipped ray-triangle solution of the winning
    triangle reproduces each hit's (t, u, v)."""
    quad = _quad(0.0)
    R = I.rotation([0.2, 1.0, 0.3], 0.6)
    inst = O.Instance(0, R.T / 1.5, np.array([0.1, -0.2, 0.3]))
    eye, f, r, u = _cam([0.5, -1.0, -4.0], [0.0, 0.0, 0.0])
    W, H, tan = 40, 30, 0.35
    g = O.gbuffer([quad], [inst], eye, f, r, u, tan, W, H)
    hit = g["shape"] == 0
    assert hit.sum() > 100
    assert np.allclose(g["normal"][hit], R[:, 2][None, :], atol=1e-12)
    assert np.all(g["normal"][~hit] == 0)
    o, d = O.pixel_rays(eye, f, r, u, tan, W, H)
    t, uu, vv = O.ray_triangle(quad, inst, g["prim"][hit], o[hit], d[hit])
    assert np.allclose(t, g["dist"][hit], rtol=1e-12)
    assert np.allclose(uu, g["u"][hit], atol=1e-12) and np.allclose(vv, g["v"][hit], atol=1e-12)
