"""The traversal's occupancy distance field (host, no GPU) against brute
force: for every voxel, the Chebyshev distance to the nearest occupied
voxel, capped; 0 exactly on occupied voxels. The traversal crosses the empty
cube of radius D - 1 around a voxel in one step, so a distance that is too
large would skip occupied voxels and one that is too small only costs
steps; both directions are checked exactly."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_21627_gb300 import inputs as I
from paper_2504_21627_gb300 import lsnif


def _brute(occ, V, cap):
    pts = np.argwhere(occ.reshape(V, V, V))          # (z, y, x)
    zz, yy, xx = np.meshgrid(np.arange(V), np.arange(V), np.arange(V), indexing="ij")
    grid = np.stack([zz, yy, xx], -1).reshape(-1, 3)
    if len(pts) == 0:
        return np.full(V ** 3, cap, np.uint8)
    d = np.full(V ** 3, cap, np.int64)
    for p in pts:
        d = np.minimum(d, np.abs(grid - p).max(axis=1))
    return np.minimum(d, cap).astype(np.uint8)


def _words(occ):
    bits = np.zeros(((occ.size + 31) // 32) * 32, np.uint8)
    bits[:occ.size] = occ
    return np.packbits(bits.reshape(-1, 32)[:, ::-1], axis=1).view(">u4").astype(np.uint32).reshape(-1)


@pytest.mark.parametrize("V,density,cap", [(8, 0.02, 32), (16, 0.005, 32), (16, 0.0, 5), (12, 0.3, 3), (16, 0.003, 2)])
def test_distance_field_matches_brute_force(V, density, cap):
    g = np.random.default_rng(V * 7 + cap)
    occ = (g.random(V ** 3) < density).astype(np.uint8)
    got = lsnif.occupancy_distance_host(_words(occ), V, cap)
    assert np.array_equal(got, _brute(occ, V, cap))
    assert np.all((got == 0) == (occ == 1))


def test_distance_field_of_a_voxelised_mesh():
    mesh = I.icosphere(2)
    V = 24
    lo, hi = O.bbox(mesh.verts)
    occ = O.voxelize(mesh.verts, mesh.tris, lo, hi, V)
    got = lsnif.occupancy_distance_host(_words(occ), V, 32)
    assert np.array_equal(got, _brute(occ, V, 32))
    assert got.max() > 3        # the hollow inside is far from the shell
