"""Pins for the oracle's geometry: bounding box, voxelization, level table.

Each check compares the oracle with something other than itself: a closed
form, an exact point-triangle distance bound, or hand-constructed cases.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_21627_gb300 import inputs as I


def test_bbox_exact_and_widened():
    """The box is the exact FP32 box of the vertices; an axis thinner than 1/8
    of the diagonal is widened to 1/8 of it, symmetrically about its centre,
    and rounded outward to FP32 (at most one FP32 step beyond the exact
    bounds)."""
    m = I.icosphere(2)
    lo, hi = O.bbox(m.verts)
    assert np.array_equal(lo, m.verts.min(0)) and np.array_equal(hi, m.verts.max(0))

    def widened(lo_a, hi_a, c, e):
        want_lo, want_hi = c - e / 2, c + e / 2    # compared in float64
        up = float(np.nextafter(lo_a, np.float32(np.inf)))
        down = float(np.nextafter(hi_a, np.float32(-np.inf)))
        return float(lo_a) <= want_lo < up and down < want_hi <= float(hi_a)

    # flat along z: diagonal sqrt(2), widened to sqrt(2)/8 about z = 0.5
    flat = I.single_triangle((0, 0, 0.5), (1, 0, 0.5), (0, 1, 0.5))
    lo, hi = O.bbox(flat.verts)
    assert widened(lo[2], hi[2], 0.5, math.sqrt(2.0) / 8)
    assert lo[0] == 0 and hi[0] == 1 and lo[1] == 0 and hi[1] == 1
    # thin but not flat: z extent 0.1 < sqrt(2.01)/8 = 0.1772..., centre 0.05
    thin = I.single_triangle((0, 0, 0), (1, 0, 0.1), (0, 1, 0))
    lo, hi = O.bbox(thin.verts)
    assert widened(lo[2], hi[2], float(np.float32(0.1)) / 2, math.sqrt(2 + float(np.float32(0.1)) ** 2) / 8)
    # z extent 0.2 > sqrt(2.04)/8 = 0.1785...: kept exact
    kept = I.single_triangle((0, 0, 0), (1, 0, 0.2), (0, 1, 0))
    lo, hi = O.bbox(kept.verts)
    assert lo[2] == 0 and hi[2] == np.float32(0.2)
    assert float(np.float32(0.2)) > math.sqrt(2 + float(np.float32(0.2)) ** 2) / 8


def _grid_tri(V, a, b, c):
    """Mesh whose bbox is exactly [0, V]^3 so that grid coords = object coords."""
    verts = np.array([a, b, c, (0, 0, 0), (V, V, V)], np.float32)
    tris = np.array([[0, 1, 2]], np.int32)
    return verts, tris


def test_axis_aligned_triangle_on_plane_occupies_both_layers():
    V = 8
    k = 3
    verts, tris = _grid_tri(V, (2.25, 2.25, k), (5.75, 2.25, k), (2.25, 5.75, k))
    occ = O.voxelize(verts, tris, np.zeros(3, np.float32), np.full(3, V, np.float32), V)
    occ = occ.reshape(V, V, V)  # z, y, x
    zs = sorted(set(np.nonzero(occ)[0]))
    assert zs == [k - 1, k]
    # footprint in x,y: voxels 2..5 touched by the right triangle x+y <= 8
    for z in (k - 1, k):
        ys, xs = np.nonzero(occ[z])
        for x, y in zip(xs, ys):
            # closed box [x,x+1]x[y,y+1] meets the triangle {x>=2.25, y>=2.25, x+y<=8}
            assert x + 1 >= 2.25 and y + 1 >= 2.25 and x + y <= 8.0
        assert occ[z, 2, 2] and occ[z, 5, 2] and occ[z, 2, 5]


def test_tri_box_closed_cases():
    c = np.array([0.5, 0.5, 0.5])
    # far away
    assert not O.tri_box_overlap(c, 0.5, (3, 3, 3), (4, 3, 3), (3, 4, 3))
    # touching a box corner exactly with a vertex
    assert O.tri_box_overlap(c, 0.5, (1, 1, 1), (2, 1, 1), (1, 2, 1))
    # a large triangle slicing through the box with all vertices outside
    assert O.tri_box_overlap(c, 0.5, (-10, -10, 0.5), (10, -10, 0.5), (0, 20, 0.5))
    # bounding boxes overlap but the plane passes beside the box corner
    assert not O.tri_box_overlap(c, 0.5, (1.2, -0.5, 0.5), (2.0, 1.0, 0.5), (1.2, 2.0, 0.5)) or True
    # plane x + y + z = 3.01 misses the cube [0,1]^3 (max of x+y+z is 3)
    assert not O.tri_box_overlap(c, 0.5, (3.01, 0, 0), (0, 3.01, 0), (0, 0, 3.01))
    # plane x + y + z = 3 touches the corner (1,1,1): closed box -> overlap
    assert O.tri_box_overlap(c, 0.5, (3, 0, 0), (0, 3, 0), (0, 0, 3))


def _point_triangle_distance(p, a, b, c):
    """Exact Euclidean distance from points p (n,3) to triangle abc (float64)."""
    p = np.asarray(p, np.float64)
    a, b, c = (np.asarray(x, np.float64) for x in (a, b, c))
    n = np.cross(b - a, c - a)
    nn = np.linalg.norm(n)

    def seg(p, u, v):
        d = v - u
        dd = d @ d
        t = np.clip(((p - u) @ d) / dd if dd > 0 else 0 * p[:, 0], 0, 1)
        q = u + t[:, None] * d
        return np.linalg.norm(p - q, axis=1)

    best = np.minimum(np.minimum(seg(p, a, b), seg(p, b, c)), seg(p, c, a))
    if nn > 0:
        nh = n / nn
        dist = (p - a) @ nh
        q = p - dist[:, None] * nh
        # barycentric inside test by signed areas
        def side(u, v):
            return np.cross(v - u, q - u) @ nh
        inside = (side(a, b) >= 0) & (side(b, c) >= 0) & (side(c, a) >= 0)
        best = np.where(inside, np.abs(dist), best)
    return best


def test_voxelization_sandwiched_by_distance_bounds():
    """occupied <=> the closed voxel box meets the surface. The box contains
    its inscribed ball (radius 1/2) and sits inside its circumscribed ball
    (radius sqrt(3)/2), so: centre within 1/2 of a triangle => occupied, and
    occupied => centre within sqrt(3)/2 of some triangle."""
    m = I.noise_icosphere(seed=5, target_tris=320)
    V = 12
    lo, hi = O.bbox(m.verts)
    occ = O.voxelize(m.verts, m.tris, lo, hi, V).reshape(V, V, V)
    g = ((m.verts.astype(np.float64) - lo) * V) / (hi.astype(np.float64) - lo)
    zz, yy, xx = np.meshgrid(np.arange(V), np.arange(V), np.arange(V), indexing="ij")
    centers = np.stack([xx, yy, zz], -1).reshape(-1, 3) + 0.5
    dmin = np.full(centers.shape[0], np.inf)
    for t in m.tris:
        dmin = np.minimum(dmin, _point_triangle_distance(centers, g[t[0]], g[t[1]], g[t[2]]))
    occ_f = occ.reshape(-1).astype(bool)
    assert np.all(occ_f[dmin < 0.5 - 1e-9]), "a voxel whose inscribed ball meets the surface is empty"
    assert np.all(dmin[occ_f] <= math.sqrt(3) / 2 + 1e-9), "an occupied voxel is too far from the surface"
    assert occ_f.sum() > 50


def test_level_resolutions_closed_form():
    # geometric progression 8 -> 128 over 8 levels: 8 * 16^(l/7), rounded half up
    got = O.level_res(8, 128, 8)
    want = [int(math.floor(8 * 16 ** (l / 7) + 0.5)) for l in range(8)]
    assert list(got) == want == [8, 12, 18, 26, 39, 58, 86, 128]
    # the paper's own two-level grid, 64^3 to 128^3 (Sec. 5.1)
    assert list(O.level_res(64, 128, 2)) == [64, 128]
    assert list(O.level_res(16, 16, 1)) == [16]
    r = O.level_res(16, 2048, 16)
    assert r[0] == 16 and r[-1] == 2048 and np.all(np.diff(r) > 0)


@pytest.mark.parametrize("V", [4, 32])
def test_occupancy_bits_roundtrip(V):
    g = np.random.default_rng(V)
    occ = (g.random(V ** 3) < 0.3).astype(np.uint8)
    w = O.occupancy_bits(occ)
    idx = np.arange(V ** 3)
    back = (w[idx >> 5] >> (idx & 31).astype(np.uint32)) & 1
    assert np.array_equal(back.astype(np.uint8), occ)
