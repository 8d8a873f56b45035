"""GPU primary-ray G-buffer (lsnif_raster_gbuffer) against the oracle's
brute-force FP64 casting (Sec. 4, Fig. 4a).

Tolerances: the GPU maps triangles to world space and tests the pixel ray in
FP32; the oracle maps the ray to the object frame in FP64. Away from edges
and depth ties both pick the same triangle: shape and primitive identical,
distance within 1e-5 relative. The FP32 hit point carries an error of a few
ulps of the world coordinates and of the distance, so (u, v) are compared
through the point they define: |du e1 + dv e2| (object frame) within 1e-5
of the distance, mapped by the instance's scale; normals within 1e-3. A
pixel whose ray passes within rounding of an edge, or where two surfaces are
equally near, may get either answer: there the GPU's triangle must be a
valid one -- its unclipped barycentrics inside up to 1e-4 and its distance
within 1e-4 relative of the oracle's nearest -- and such pixels stay below
1% of the image.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2504_21627_gb300 import inputs as I  # noqa: E402
from paper_2504_21627_gb300 import lsnif  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = lsnif.Context(0)
    yield c
    c.close()


def _cam(eye, target, up0=(0.0, 0.0, 1.0)):
    """Camera vectors rounded to FP32 (what the library receives), as FP64."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, up0)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    return tuple(np.asarray(x, np.float32).astype(np.float64) for x in (eye, f, r, u))


def _f32(insts):
    return [O.Instance(i.obj, i.A.astype(np.float32).astype(np.float64), i.b.astype(np.float32).astype(np.float64))
            for i in insts]


@pytest.fixture(scope="module")
def scene(ctx):
    meshes = [I.icosphere(3), I.cube(n_mat=2), I.noise_icosphere(seed=12, target_tris=5000, amplitude=0.08, n_mat=2)]
    cfgs = [I.cfg_icosphere_small(), I.Config(V=16, H=18, L=4, F=2, log2_T=10, N_min=4, N_max=16, n_hidden=1,
                                              width=64, n_mat=2), I.cfg_icosphere_small()]
    handles = [ctx.load_object(m, c, keep_mesh=True) for m, c in zip(meshes, cfgs)]
    insts = _f32([O.Instance(o, A, b) for o, A, b in I.seeded_instances(7, 3, seed=31, spread=5.0)])
    return dict(meshes=meshes, handles=handles, insts=insts)


def _gpu(ctx, scene, cam, W, H, insts=None):
    insts = scene["insts"] if insts is None else insts
    eye, f, r, u = cam
    tan = float(np.float32(math.tan(math.radians(24.0))))
    g = ctx.raster_gbuffer(eye, f, r, u, tan, W, H, [(scene["handles"][i.obj], i.A, i.b) for i in insts])
    ctx.check()
    torch.cuda.synchronize()
    got = {k: getattr(g, k).cpu().numpy().reshape(-1) for k in ("hit", "shape", "prim", "u", "v", "dist")}
    got["normal"] = g.normal.cpu().numpy().reshape(3, -1).T
    ref = O.gbuffer(scene["meshes"], insts, eye, f, r, u, tan, W, H)
    return got, ref, tan


def _check(scene, got, ref, cam, tan, W, H, insts, min_hit=0.2):
    assert np.array_equal(got["hit"], (got["shape"] >= 0).astype(np.uint8))
    same = (got["shape"] == ref["shape"]) & (got["prim"] == ref["prim"])
    hit = same & (ref["shape"] >= 0)
    assert hit.sum() > min_hit * W * H
    assert np.allclose(got["dist"][hit], ref["dist"][hit], rtol=1e-5)
    for k, inst in enumerate(insts):
        m = hit & (ref["shape"] == k)
        if not m.any():
            continue
        mesh = scene["meshes"][inst.obj]
        v3 = mesh.verts.astype(np.float64)
        tri = mesh.tris[ref["prim"][m]]
        e1, e2 = v3[tri[:, 1]] - v3[tri[:, 0]], v3[tri[:, 2]] - v3[tri[:, 0]]
        du = (got["u"][m] - ref["u"][m])[:, None]
        dv = (got["v"][m] - ref["v"][m])[:, None]
        err = np.linalg.norm(du * e1 + dv * e2, axis=1)
        assert np.all(err <= 1e-5 * ref["dist"][m] * np.linalg.norm(inst.A, 2) + 1e-6), (k, err.max())
    assert np.allclose(got["normal"][hit], ref["normal"][hit], atol=1e-3)
    bg = same & (ref["shape"] < 0)
    assert np.all(np.isinf(got["dist"][bg])) and np.all(got["prim"][bg] == -1) and np.all(got["normal"][bg] == 0)
    diff = ~same
    assert diff.mean() < 0.01, diff.mean()
    if diff.any():
        o, d = O.pixel_rays(*cam, tan, W, H)
        for i in np.flatnonzero(diff):
            if got["shape"][i] >= 0:
                inst = insts[got["shape"][i]]
                t, u, v = O.ray_triangle(scene["meshes"][inst.obj], inst, np.array([got["prim"][i]]), o[i:i + 1],
                                         d[i:i + 1])
                assert min(u[0], v[0], 1 - u[0] - v[0]) > -1e-4, i
                if ref["shape"][i] >= 0:
                    assert abs(t[0] - ref["dist"][i]) <= 1e-4 * ref["dist"][i], i
            else:
                # the GPU saw background: the oracle's hit lies on an edge
                r_ = ref
                assert min(r_["u"][i], r_["v"][i], 1 - r_["u"][i] - r_["v"][i]) < 1e-4, i


@pytest.mark.parametrize("W,H", [(160, 120), (97, 61)])
def test_gbuffer_matches_oracle(ctx, scene, W, H):
    cam = _cam([6.0, -4.5, 3.0], [0.0, 0.0, 0.0])
    got, ref, tan = _gpu(ctx, scene, cam, W, H)
    _check(scene, got, ref, cam, tan, W, H, scene["insts"])


def test_gbuffer_close_camera_and_straddling_triangles(ctx, scene):
    """A camera inside the cloud of instances: triangles behind it, beside it
    and crossing its plane (swept over the whole image)."""
    cam = _cam([0.3, 0.2, 0.4], [3.0, 2.0, -1.0])
    got, ref, tan = _gpu(ctx, scene, cam, 128, 96)
    _check(scene, got, ref, cam, tan, 128, 96, scene["insts"])


def test_gbuffer_coincident_instances_tie_to_the_lower(ctx, scene):
    insts = [scene["insts"][0], scene["insts"][0], scene["insts"][1]]
    centre = np.linalg.solve(insts[0].A, -insts[0].b)       # the icosphere's centre in world space
    cam = _cam(centre + np.array([2.5, 2.0, 1.5]), centre)
    got, ref, tan = _gpu(ctx, scene, cam, 96, 72, insts)
    assert (got["shape"] == 0).sum() > 0.1 * 96 * 72
    assert not np.any(got["shape"] == 1)
    _check(scene, got, ref, cam, tan, 96, 72, insts, min_hit=0.1)


def test_gbuffer_rejects_bad_input(ctx, scene):
    cam = _cam([9.0, -7.0, 5.0], [0.0, 0.0, 0.0])
    h0 = scene["handles"][0]
    with pytest.raises(lsnif.LsnifError):
        ctx.raster_gbuffer(cam[0], cam[1], cam[1], cam[3], 0.4, 8, 8, [(h0, np.eye(3), np.zeros(3))])
    with pytest.raises(lsnif.LsnifError):
        ctx.raster_gbuffer(*cam, 0.4, 8, 8, [(h0, np.zeros((3, 3)), np.zeros(3))])
    nomesh = ctx.load_object(I.icosphere(1), I.cfg_icosphere_small())
    with pytest.raises(lsnif.LsnifError) as e:
        ctx.raster_gbuffer(*cam, 0.4, 8, 8, [(nomesh, np.eye(3), np.zeros(3))])
    assert e.value.code == -10
    ctx.unload_object(nomesh)
