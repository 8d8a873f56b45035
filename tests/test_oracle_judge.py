"""Pins for the oracle's geometric judge and training-ray sampler (Sec. 5.2)."""
import numpy as np

from oracle import oracle as O
from paper_2504_21627_gb300 import inputs as I


def test_single_triangle_closed_form():
    m = I.single_triangle((0, 0, 1), (2, 0, 1), (0, 2, 1))
    rays = np.concatenate([
        I.pack_rays(np.array([[0.5, 0.25, 5.0]]), np.array([[0, 0, -1.0]])),   # hits at t = 4
        I.pack_rays(np.array([[1.5, 1.5, 5.0]]), np.array([[0, 0, -1.0]])),    # outside (u+v>1)
        I.pack_rays(np.array([[0.5, 0.25, 5.0]]), np.array([[1.0, 0, 0]])),    # parallel: det 0
        I.pack_rays(np.array([[0.5, 0.25, 5.0]]), np.array([[0, 0, -1.0]]), tmax=3.0),  # beyond tmax
        I.pack_rays(np.array([[1.0, 1.0, 5.0]]), np.array([[0, 0, -1.0]])),    # on the edge u+v=1
    ], axis=1)
    j = O.judge(m, rays)
    assert j.t[0] == 4.0 and j.tri[0] == 0
    # barycentrics against a linear solve
    A = np.array([[2.0, 0.0], [0.0, 2.0]])
    u, v = np.linalg.solve(A, np.array([0.5, 0.25]))
    assert abs(j.u[0] - u) < 1e-15 and abs(j.v[0] - v) < 1e-15
    assert j.tri[1] == -1 and j.tri[2] == -1 and j.tri[3] == -1
    assert j.tri[4] == 0 and j.t[4] == 4.0


def test_icosphere_hits_between_inscribed_and_unit_sphere():
    m = I.icosphere(3)
    v = m.verts.astype(np.float64)
    nrm = np.cross(v[m.tris[:, 1]] - v[m.tris[:, 0]], v[m.tris[:, 2]] - v[m.tris[:, 0]])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r_in = np.min(np.abs(np.sum(nrm * v[m.tris[:, 0]], axis=1)))
    g = np.random.default_rng(0)
    o = g.normal(size=(300, 3))
    o = 3.0 * o / np.linalg.norm(o, axis=1, keepdims=True)
    d = -o / 3.0
    j = O.judge(m, I.pack_rays(o, d))
    assert np.all(j.tri >= 0)
    assert np.all(j.t >= 3.0 - 1.0 - 1e-6) and np.all(j.t <= 3.0 - r_in + 1e-6)
    # nearest hit: from the centre outward there is exactly one hit at radius in [r_in, 1]
    j2 = O.judge(m, I.pack_rays(np.zeros((300, 3)), d))
    assert np.all((j2.t >= r_in - 1e-6) & (j2.t <= 1.0 + 1e-6))
    # shading normal ~ radial direction
    sn = O.shading_normal(m, j)
    hitp = o + j.t[:, None] * d
    radial = hitp / np.linalg.norm(hitp, axis=1, keepdims=True)
    assert np.all(np.sum(sn * radial, axis=1) > 0.99)


def test_training_rays_outside_half():
    m = I.icosphere(2)
    lo, hi = O.bbox(m.verts)
    u = I.uniforms(20000, O.N_UNIFORMS, seed=1)
    rays, surf = O.training_rays(m, lo, hi, u, n_outside=20000)
    assert not surf.any()
    c = 0.5 * (lo.astype(np.float64) + hi)
    R = 1.05 * 0.5 * np.linalg.norm(hi.astype(np.float64) - lo)
    o = rays[0:3].T.astype(np.float64)
    d = rays[3:6].T.astype(np.float64)
    assert np.allclose(np.linalg.norm(o - c, axis=1), R, rtol=1e-6)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
    inward = (c - o) / np.linalg.norm(c - o, axis=1, keepdims=True)
    cos = np.sum(d * inward, axis=1)
    assert np.all(cos >= -1e-6)
    # cosine-weighted hemisphere: E[cos] = 2/3, E[cos^2] = 1/2
    assert abs(cos.mean() - 2.0 / 3.0) < 0.01 and abs((cos ** 2).mean() - 0.5) < 0.01
    # origins uniform on the sphere: E[z] = 0, E[z^2] = R^2 / 3
    z = (o - c)[:, 2]
    assert abs(z.mean()) < 0.02 * R and abs((z ** 2).mean() - R * R / 3) < 0.02 * R * R


def test_orthonormal_basis():
    g = np.random.default_rng(2)
    n = g.normal(size=(1000, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n[0] = [0, 0, -1.0]
    n[1] = [0, 0, 1.0]
    t, b = O.onb(n)
    for x, y in ((t, b), (t, n), (b, n)):
        assert np.allclose(np.sum(x * y, axis=1), 0.0, atol=1e-12)
    for x in (t, b):
        assert np.allclose(np.linalg.norm(x, axis=1), 1.0, atol=1e-12)
    # right-handed: t x b = n
    assert np.allclose(np.cross(t, b), n, atol=1e-12)


def test_training_rays_surface_half_and_labels():
    m = I.icosphere(2)
    lo, hi = O.bbox(m.verts)
    n = 2000
    u = I.uniforms(n, O.N_UNIFORMS, seed=3)
    rays, surf = O.training_rays(m, lo, hi, u, n_outside=n // 2)
    assert not surf[: n // 2].any() and surf[n // 2:].mean() > 0.9
    diag = np.linalg.norm(hi.astype(np.float64) - lo)
    o = rays[0:3].T.astype(np.float64)
    d = rays[3:6].T.astype(np.float64)
    # surface-ray origins sit 1e-4 x diagonal off the unit-radius-ish surface
    r = np.linalg.norm(o[surf], axis=1)
    assert np.all(r > 0.9) and np.all(r < 1.0 + 2e-4 * diag)
    # labels: outside rays hit the sphere with the probability of the cosine
    # lobe inside its silhouette cone; surface rays leave a convex object and
    # never hit it again
    lab0 = O.labels(m, rays, np.tile([0.0, 1.0], (n, 1)))
    occ = lab0.occ > 0
    Rs = 1.05 * 0.5 * diag
    p_hit = (1.0 / Rs) ** 2            # sin^2 of the half-angle of the unit sphere seen from Rs
    assert abs(occ[: n // 2].mean() - p_hit) < 0.06
    assert occ[surf].mean() < 0.01
    assert np.allclose(np.linalg.norm(lab0.normal[occ], axis=1), 1.0, atol=1e-9)
    assert set(np.unique(lab0.mat[occ])) <= {0, 1}
    assert np.all(np.isfinite(d))
    # surface rays leave on the outward side of their facet; facets of this
    # icosphere tilt less than 20 degrees from the radial direction
    radial = o[surf] / np.linalg.norm(o[surf], axis=1, keepdims=True)
    assert np.all(np.sum(d[surf] * radial, axis=1) > -np.sin(np.radians(20)))
