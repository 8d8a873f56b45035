"""The mesh objects' BVH builder, on the host (no GPU): structural
invariants that make a depth-first traversal exact -- every triangle in
exactly one leaf, every leaf box holding its triangles, every internal box
holding its children -- and a brute-force check that nearest hits found by
walking the built tree equal those of a loop over all triangles."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_21627_gb300 import inputs as I
from paper_2504_21627_gb300 import lsnif


def _check_tree(verts, tris):
    nodes, order, depth = lsnif.bvh_build_host(verts, tris)
    nt = tris.shape[0]
    assert len(nodes) <= 2 * nt - 1 and depth < 64
    assert np.array_equal(np.sort(order), np.arange(nt))
    seen = np.zeros(nt, np.int32)
    stack = [(0, 0)]
    v = verts.astype(np.float32)
    while stack:
        i, d = stack.pop()
        nd = nodes[i]
        if nd["n"] > 0:
            assert nd["n"] <= 4
            ids = order[nd["a"]:nd["a"] + nd["n"]]
            seen[ids] += 1
            pts = v[tris[ids]].reshape(-1, 3)
            assert np.all(pts >= nd["lo"]) and np.all(pts <= nd["hi"])
        else:
            a = nd["a"]
            for c in (a, a + 1):
                assert np.all(nodes[c]["lo"] >= nd["lo"]) and np.all(nodes[c]["hi"] <= nd["hi"])
                stack.append((c, d + 1))
    assert np.all(seen == 1)
    return nodes, order


def _walk(nodes, order, verts, tris, o, d):
    """Nearest hit by a depth-first walk of the built tree (boxes by an FP64
    slab test with a small tolerance, triangles by the oracle's judge)."""
    best_t, best = np.inf, -1
    stack = [0]
    while stack:
        nd = nodes[stack.pop()]
        with np.errstate(divide="ignore", invalid="ignore"):
            t0 = (nd["lo"].astype(np.float64) - o) / d
            t1 = (nd["hi"].astype(np.float64) - o) / d
        tn = np.nanmax(np.minimum(t0, t1))
        tf = np.nanmin(np.maximum(t0, t1))
        if not (tn <= tf * (1 + 1e-9) + 1e-12 and tf >= 0 and tn <= best_t):
            continue
        if nd["n"] > 0:
            ids = order[nd["a"]:nd["a"] + nd["n"]]
            sub = I.Mesh(verts, tris[ids], verts, np.zeros(len(ids), np.int32), np.zeros((1, 3), np.float32), 1)
            ray = np.concatenate([o, d, [0.0, np.inf]]).astype(np.float32)[:, None]
            j = O.judge(sub, ray)
            if j.tri[0] >= 0 and (j.t[0] < best_t or (j.t[0] == best_t and ids[j.tri[0]] < best)):
                best_t, best = j.t[0], ids[j.tri[0]]
        else:
            stack += [nd["a"], nd["a"] + 1]
    return best_t, best


@pytest.mark.parametrize("mesh", [I.icosphere(3), I.noise_torus_tris(3, 4000), I.cube(), I.single_triangle(
    [0, 0, 0], [1, 0, 0], [0, 1, 0])], ids=["icosphere", "torus", "cube", "triangle"])
def test_bvh_structure(mesh):
    _check_tree(mesh.verts, mesh.tris)


def test_bvh_degenerate_inputs():
    # many triangles with one centroid (stacked copies): split by index
    tri = np.array([[0, 1, 2]] * 50, np.int32)
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    _check_tree(v, tri)
    with pytest.raises(lsnif.LsnifError):
        lsnif.bvh_build_host(v, np.array([[0, 1, 5]], np.int32))


def test_walking_the_tree_finds_the_brute_force_hit():
    mesh = I.noise_torus_tris(5, 3000)
    nodes, order = _check_tree(mesh.verts, mesh.tris)
    rays = I.rays_sphere_to_box(300, 3.0, mesh.verts.min(0), mesh.verts.max(0), seed=4)
    j = O.judge(mesh, rays)
    assert (j.tri >= 0).sum() > 100
    for i in range(rays.shape[1]):
        o, d = rays[0:3, i].astype(np.float64), rays[3:6, i].astype(np.float64)
        t, tri = _walk(nodes, order, mesh.verts, mesh.tris, o, d)
        assert tri == j.tri[i], i
        if tri >= 0:
            assert t == j.t[i]
