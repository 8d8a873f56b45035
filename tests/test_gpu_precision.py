"""The half-precision bounds of the query against the FP64 oracle, on trained
networks (Sec. 5: inference in half precision). Random-weight networks put
many decisions at the boundary, so the bounds are stated on networks trained
by the library's own training step: the icosphere object of the training
tests, a noise torus at the full benchmark configuration (V 128, 16
levels, 2^19 entries, 4 x 64) and an object of the path-tracing stress
configuration's network shape (16 levels x 4 features, 4 x 128; 2^19
entries per level instead of 2^21, to bound the oracle's FP64 copy), which
runs on the streamed FP16 kernel. Every output is compared with the oracle's
FP64 query on the same FP32 master parameters:

  visibility mismatch <= 0.1% of the rays, hit distance within 1e-3 of the
  box diagonal (read at the 99th percentile of the rays both call a hit),
  material equal on >= 99.9% of those rays.

Near-face rays (several voxel orders are correct) are counted and left out.
FP8 E4M3 is printed, not asserted: it serves the stress configuration only
where these bounds hold."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2504_21627_gb300 import inputs as I  # noqa: E402
from paper_2504_21627_gb300 import lsnif  # noqa: E402

VIS_MAX, T_P99_MAX, MAT_MIN = 1e-3, 1e-3, 0.999


def _train(ctx, mesh, cfg, steps, batch, n_pool, seed):
    h = ctx.load_object(mesh, cfg, keep_mesh=True)
    u = torch.rand((n_pool, lsnif.TRAIN_UNIFORMS), device="cuda", generator=torch.Generator("cuda").manual_seed(seed))
    pool, _ = ctx.make_training_rays(h, u, n_outside=n_pool // 2)
    lab = ctx.label_rays(pool, h)
    keep = lab["k"] > 0
    pool = pool[:, keep].contiguous()
    lab = {k: v[keep].contiguous() for k, v in lab.items()}
    gen = torch.Generator("cuda").manual_seed(seed + 1)
    first = last = None
    for s in range(steps):
        idx = torch.randint(0, pool.shape[1], (batch,), device="cuda", generator=gen)
        st = ctx.train_step(pool[:, idx].contiguous(), {k: v[idx].contiguous() for k, v in lab.items()}, h,
                            lr=0.01, stats=(s == 0 or s == steps - 1))
        if st is not None:
            first, last = (st.total, None) if first is None else (first, st.total)
    assert last < 0.1 * first, (first, last)
    return h


@pytest.fixture(scope="module")
def ctx():
    c = lsnif.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def trained(ctx):
    out = {}
    cfg = I.cfg_icosphere_small()
    mesh = I.noise_icosphere(seed=6, target_tris=1280, amplitude=0.08, n_mat=2)
    h = _train(ctx, mesh, cfg, 800, 1 << 14, 1 << 18, 3)
    lo, hi = O.bbox(mesh.verts)
    out["icosphere"] = (h, mesh, cfg, I.rays_sphere_to_box(4000, 2.5, lo, hi, seed=77))
    cfg = I.cfg_torus_4m()
    mesh = I.noise_torus(seed=1)
    h = _train(ctx, mesh, cfg, 2000, 1 << 16, 1 << 21, 5)
    lo, hi = O.bbox(mesh.verts)
    rays = np.concatenate([I.rays_sphere_to_box(6000, 2.5, lo, hi, seed=78),
                           I.rays_pinhole(I.seeded_camera(2, width=96, height=96))], axis=1)
    out["torus"] = (h, mesh, cfg, np.ascontiguousarray(rays))
    cfg = I.cfg_stress_object(log2_T=19)
    mesh = I.noise_torus_tris(8, 50000, amplitude=0.05, n_mat=4)
    h = _train(ctx, mesh, cfg, 1500, 1 << 16, 1 << 20, 7)
    lo, hi = O.bbox(mesh.verts)
    out["stress"] = (h, mesh, cfg, I.rays_sphere_to_box(8000, 2.5, lo, hi, seed=79))
    return out


_ref_cache = {}


def _reference(ctx, trained, name):
    if name not in _ref_cache:
        h, mesh, cfg, rays = trained[name]
        p = I.Params(ctx.read_params(h, lsnif.PARAM_TABLES), I.unpack_mlp(cfg, ctx.read_params(h, lsnif.PARAM_MLP)))
        orc = O.build_object(mesh, cfg, p)
        ref, seg = O.query(orc, rays, precision="f64")
        diag = float(np.linalg.norm(orc.bmax.astype(np.float64) - orc.bmin))
        _ref_cache[name] = (ref, seg, diag)
    return _ref_cache[name]


def _errors(ctx, trained, name, prec):
    h, _, _, rays = trained[name]
    ref, seg, diag = _reference(ctx, trained, name)
    out = ctx.query_rays(torch.from_numpy(rays).cuda(), obj=h, precision=prec)
    ctx.check()
    hit = out.hit.cpu().numpy().astype(bool)
    t = out.t.cpu().numpy().astype(np.float64)
    mat = out.mat.cpu().numpy()
    ok = ~seg.near
    both = ok & hit & ref.hit
    dt = np.abs(t[both] - ref.t[both]) / diag
    return dict(vis=float((hit[ok] != ref.hit[ok]).mean()), p50=float(np.median(dt)),
                p99=float(np.quantile(dt, 0.99)), mat=float((mat[both] == ref.mat[both]).mean()),
                n=int(ok.sum()), near=int(seg.near.sum()), hits=int(both.sum()))


def _show(name, label, e):
    print(f"{name} {label} vs FP64 oracle: visibility mismatch {e['vis']:.4%}, hit-t error p50 {e['p50']:.2e} "
          f"p99 {e['p99']:.2e} of the diagonal, material {e['mat']:.4%} ({e['hits']} hits of {e['n']} rays, "
          f"{e['near']} near-face left out)")


@pytest.mark.parametrize("name,prec,label", [
    ("icosphere", lsnif.BF16_FUSED, "BF16"), ("icosphere", lsnif.FP16_FUSED, "FP16"),
    ("torus", lsnif.BF16_FUSED, "BF16"), ("torus", lsnif.FP16_FUSED, "FP16"),
    ("stress", lsnif.FP16_FUSED, "FP16 (streamed weights)")])
def test_half_precision_meets_the_bounds_against_the_fp64_oracle(ctx, trained, name, prec, label):
    e = _errors(ctx, trained, name, prec)
    _show(name, label, e)
    assert e["hits"] > 500
    assert e["vis"] <= VIS_MAX, e
    assert e["p99"] <= T_P99_MAX, e
    assert e["mat"] >= MAT_MIN, e


@pytest.mark.parametrize("name", ["icosphere", "torus", "stress"])
def test_fp32_and_fp8_against_the_fp64_oracle(ctx, trained, name):
    e32 = _errors(ctx, trained, name, lsnif.FP32_PLAIN)
    _show(name, "FP32", e32)
    # the FP32 path carries only FP32 rounding: far inside the half-precision bounds
    assert e32["vis"] <= VIS_MAX and e32["p99"] <= 1e-4 and e32["mat"] >= MAT_MIN, e32
    _show(name, "FP8 (not accepted; printed)", _errors(ctx, trained, name, lsnif.FP8_FUSED))
