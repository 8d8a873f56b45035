"""Pins for the oracle's traversal: the ordered occupied-voxel segments and
their boundary points (Fig. 2, Sec. 3.1), checked against closed forms and an
independent dense ray-marching enumeration."""
import numpy as np

from oracle import oracle as O
from paper_2504_21627_gb300 import inputs as I


def _obj(V, occ, H=18):
    cfg = I.Config(V=V, H=H, L=1, F=1, log2_T=4, N_min=2, N_max=2, n_hidden=1, width=8, n_mat=1)
    return O.OracleObject(cfg, np.zeros(3, np.float32), np.ones(3, np.float32),
                          occ.astype(np.uint8), np.array([2], np.int32),
                          np.zeros((1, 16, 1)), [])


def _rays(o, d, tmin=0.0, tmax=np.inf):
    return I.pack_rays(np.atleast_2d(np.asarray(o, np.float64)),
                       np.atleast_2d(np.asarray(d, np.float64)), tmin, tmax)


def test_axis_aligned_ray_full_grid_closed_form():
    V = 16
    obj = _obj(V, np.ones(V ** 3))
    y, z = (5 + 0.5) / V, (9 + 0.5) / V
    seg = O.ray_segments(obj, _rays((-1.0, y, z), (1.0, 0, 0)))
    assert seg.k[0] == 9 and not seg.near[0]
    assert seg.t01[0, 0] == 1.0 and seg.t01[0, 1] == 2.0
    for s in range(9):
        p_in, p_out = seg.pts[0, 2 * s], seg.pts[0, 2 * s + 1]
        assert p_in[0] == s / V and p_out[0] == (s + 1) / V
        assert abs(p_in[1] - y) < 1e-15 and abs(p_in[2] - z) < 1e-15
        assert seg.vox[0, s] == (9 * V + 5) * V + s
    # reversed direction walks from the far side
    seg = O.ray_segments(obj, _rays((2.0, y, z), (-1.0, 0, 0)))
    assert seg.k[0] == 9 and seg.pts[0, 0, 0] == 1.0 and seg.pts[0, 1, 0] == (V - 1) / V


def test_misses_and_degenerate_rays():
    V = 8
    obj = _obj(V, np.ones(V ** 3))
    rays = np.concatenate([
        _rays((-1, 2, 0.5), (1, 0, 0)),          # passes beside the cube
        _rays((-1, 0.5, 0.5), (-1, 0, 0)),       # points away
        _rays((0.5, 0.5, 0.5), (0, 0, 0)),       # zero direction
        _rays((np.nan, 0.5, 0.5), (1, 0, 0)),    # NaN origin
        _rays((-1, 0.5, 0.5), (1, 0, 0), tmin=5.0),  # tmin beyond the cube
    ], axis=1)
    seg = O.ray_segments(obj, rays)
    assert np.all(seg.k == 0)
    assert np.all(np.isnan(seg.t01))
    assert np.all(seg.pts == 0) and np.all(seg.vox == -1)
    empty = _obj(V, np.zeros(V ** 3))
    seg = O.ray_segments(empty, _rays((-1, 0.5, 0.5), (1, 0.1, 0.2)))
    assert seg.k[0] == 0 and not np.isnan(seg.t01[0, 0])


def test_origin_inside_and_tmin_clip_give_interior_first_point():
    V = 8
    obj = _obj(V, np.ones(V ** 3))
    o = np.array([0.3, 0.41, 0.52])
    d = np.array([0.6, 0.3, 0.2])
    seg = O.ray_segments(obj, _rays(o, d))
    assert seg.t01[0, 0] == 0.0
    assert np.allclose(seg.pts[0, 0], o.astype(np.float32), atol=1e-7)
    # the first voxel is the one containing the origin
    ix = np.floor(o.astype(np.float32) * V).astype(int)
    assert seg.vox[0, 0] == (ix[2] * V + ix[1]) * V + ix[0]
    seg2 = O.ray_segments(obj, _rays((-1, 0.41, 0.52), (1, 0, 0), tmin=1.3))
    assert abs(seg2.t01[0, 0] - 1.3) < 1e-7 and abs(seg2.pts[0, 0, 0] - 0.3) < 1e-6


def test_points_lie_on_the_faces_of_their_voxels():
    V = 16
    g = np.random.default_rng(3)
    occ = (g.random(V ** 3) < 0.35)
    obj = _obj(V, occ)
    rays = I.rays_sphere_to_box(400, 2.0, (0, 0, 0), (1, 1, 1), seed=4)
    seg = O.ray_segments(obj, rays)
    assert seg.k.max() == 9 and (seg.k > 0).mean() > 0.9
    for i in range(rays.shape[1]):
        for s in range(seg.k[i]):
            vid = seg.vox[i, s]
            ix = np.array([vid % V, (vid // V) % V, vid // (V * V)])
            assert occ[vid]
            for p in (seg.pts[i, 2 * s], seg.pts[i, 2 * s + 1]):
                assert np.all(p >= ix / V - 1e-12) and np.all(p <= (ix + 1) / V + 1e-12)
                on_face = np.isclose(p * V, np.round(p * V), rtol=0, atol=0) & (
                    (np.round(p * V) == ix) | (np.round(p * V) == ix + 1))
                assert on_face.any(), "a boundary point is not snapped to a face"
        # slots past 2k are zero
        assert np.all(seg.pts[i, 2 * seg.k[i]:] == 0)


def _march(o, d, t0, t1, V, occ, steps=200000):
    """Independent enumeration: sample the segment densely and list the
    distinct voxels visited, in order."""
    ts = t0 + (np.arange(steps) + 0.5) / steps * (t1 - t0)
    p = o[None, :] + ts[:, None] * d[None, :]
    ix = np.clip(np.floor(p * V).astype(np.int64), 0, V - 1)
    ids = (ix[:, 2] * V + ix[:, 1]) * V + ix[:, 0]
    keep = np.ones(steps, bool)
    keep[1:] = ids[1:] != ids[:-1]
    seq = ids[keep]
    return [int(v) for v in seq if occ[v]]


def test_brute_force_matches_dense_marching():
    V = 10
    g = np.random.default_rng(7)
    occ = (g.random(V ** 3) < 0.25)
    obj = _obj(V, occ)
    rays = I.rays_sphere_to_box(120, 2.5, (0, 0, 0), (1, 1, 1), seed=8)
    seg = O.ray_segments(obj, rays)
    checked = 0
    for i in range(rays.shape[1]):
        if seg.near[i] or np.isnan(seg.t01[i, 0]):
            continue
        o = rays[0:3, i].astype(np.float64)
        d = rays[3:6, i].astype(np.float64)
        seq = _march(o, d, seg.t01[i, 0], seg.t01[i, 1], V, occ)[:9]
        assert seq == [int(v) for v in seg.vox[i, :seg.k[i]]], i
        checked += 1
    assert checked > 100


def test_near_face_flag():
    V = 8
    obj = _obj(V, np.ones(V ** 3))
    # exactly along a voxel edge line y = 2/8, z = 3/8
    seg = O.ray_segments(obj, _rays((-1, 2 / V, 3 / V), (1, 0, 0)))
    assert seg.near[0]
    # parallel to a face, 1e-7 away from it
    seg = O.ray_segments(obj, _rays((-1, 2 / V + 1e-7, 3.5 / V), (1, 0, 0)))
    assert seg.near[0]
    # through voxel centres: robust
    seg = O.ray_segments(obj, _rays((-1, 2.5 / V, 3.5 / V), (1, 0, 0)))
    assert not seg.near[0]
    # a flagged voxel beyond the kept prefix does not flag the ray
    seg = O.ray_segments(obj, _rays((-1, 2.5 / V, 3.5 / V), (1, 0, 0), tmin=0))
    assert not seg.near[0]
