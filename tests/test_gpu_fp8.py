"""GPU parity of the FP8 (E4M3) fused query against the oracle's FP8
network (same power-of-two scales, same E4M3 rounding of inputs, weights and
hidden activations, FP64 sums), and its error against the FP64 oracle.

Two kinds of rays:
  exact-point rays: axis-parallel rays with dyadic origins through an object
  whose box is [0, 1]^3, so every sample point is exact in FP32 and equals
  the oracle's. GPU and oracle then differ only where an FP32 value (feature
  interpolation, accumulator) and its FP64 counterpart round to neighbouring
  E4M3 values, which needs the value within ~2^-20 of a rounding midpoint:
  at least 95% of live rays agree to 1e-5 of the batch's largest |logit|,
  every ray to 2^-2 of it (a wrong layout, scale or operand gives errors of
  order one on most rays).
  general rays: the FP32 trace moves points by a few ulps (up to ~2e-5 of
  the box at grazing angles); at fine levels that is enough to move a
  scaled feature across an E4M3 rounding midpoint, i.e. by one E4M3 step
  (up to 2^-3 of it). Such flips touch many rays but move logits little:
  the 95th percentile of the logit error stays below 2^-4 of the largest
  |logit|, every error below 2^-2, and decisions whose logit margin exceeds
  2^-3 of it agree on at least 99% of live rays.
"""
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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _make(ctx, mesh, cfg, seed, table_range):
    p = I.random_params(cfg, seed, table_range=table_range, bias_range=0.1)
    orc = O.build_object(mesh, cfg, p)
    h = ctx.load_object(mesh, cfg, tables=p.tables, mlp=p.packed_mlp())
    return dict(h=h, orc=orc, p=p, cfg=cfg)


@pytest.fixture(scope="module")
def torus(ctx):
    """F = 2, 4 x 64 network (the torus workload's shape)."""
    return _make(ctx, I.noise_torus(seed=2), I.cfg_torus_4m(), seed=5, table_range=0.05)


@pytest.fixture(scope="module")
def stress(ctx):
    """The stress configuration's network shape: L = 16, F = 4, 4 x 128
    (table 2^18 per level instead of 2^21 to keep the oracle's copy small;
    the kernel does not depend on T)."""
    cfg = I.cfg_stress_object(log2_T=18)
    return _make(ctx, I.noise_icosphere(seed=205, target_tris=60000, amplitude=0.08, n_mat=4), cfg, seed=7,
                 table_range=0.05)


def _camera_sample(n, seed):
    cam = I.seeded_camera(2)
    g = np.random.default_rng(seed)
    return np.ascontiguousarray(I.rays_pinhole(cam)[:, g.choice(2048 * 2048, n, replace=False)])


def _exact_rays(n, seed, V):
    """Axis-parallel rays (both directions on each axis) with dyadic origins
    strictly inside a voxel column, half of them in the wall columns of a
    box-shaped object (long runs of occupied voxels, so duplicate boundary
    points and the H cap occur), some starting inside the box (dyadic
    tmin)."""
    g = np.random.default_rng(seed)
    axis = g.integers(0, 3, n)
    sign = np.where(g.random(n) < 0.5, 1.0, -1.0)
    cols = np.where(g.random((n, 2)) < 0.5, g.choice([0, V - 1], size=(n, 2)), g.integers(0, V, (n, 2)))
    off = g.choice([1, 3, 5, 7], size=(n, 2)) / 8.0
    rays = np.zeros((8, n), np.float32)
    for i in range(n):
        a = axis[i]
        o = np.zeros(3)
        others = [b for b in range(3) if b != a]
        o[others[0]] = (cols[i, 0] + off[i, 0]) / V
        o[others[1]] = (cols[i, 1] + off[i, 1]) / V
        o[a] = -0.5 if sign[i] > 0 else 1.5
        rays[0:3, i] = o
        rays[3 + a, i] = sign[i]
    rays[6] = np.where(g.random(n) < 0.2, 0.5 + g.integers(0, 256, n) / 512.0, 0.0)
    rays[7] = np.inf
    return rays


def _logit_err(out, ref, seg):
    live = ref.live & ~seg.near
    assert live.sum() > 200
    lg = out.logits.cpu().numpy()
    scale = np.abs(ref.logits[live]).max()
    return live, lg, np.abs(lg[live] - ref.logits[live]).max(axis=1) / scale, scale


def _miss_record(out, ref, seg):
    miss = ~ref.live & ~seg.near
    hit = out.hit.cpu().numpy().astype(bool)
    assert not hit[miss].any() and np.all(np.isinf(out.t.cpu().numpy()[miss]))
    assert np.all(out.mat.cpu().numpy()[miss] == -1) and np.all(np.isnan(out.logits.cpu().numpy()[miss]))


@pytest.fixture(scope="module", params=[(2, 64), (4, 128)], ids=["F2-64", "F4-128"])
def box(ctx, request):
    """A box-shaped object, [0, 1]^3 exactly, with a random network of the
    torus shape (F = 2, 4 x 64) or of the stress shape (F = 4, 4 x 128)."""
    F, width = request.param
    cfg = I.Config(V=128, H=18, L=16, F=F, log2_T=16, N_min=16, N_max=2048, n_hidden=4, width=width, n_mat=4)
    o = _make(ctx, I.cube(n_mat=4), cfg, seed=20 + F, table_range=0.05)
    assert np.array_equal(o["orc"].bmin, [0, 0, 0]) and np.array_equal(o["orc"].bmax, [1, 1, 1])
    return o


def test_fp8_exact_points_match_oracle_fp8(ctx, box):
    rays = _exact_rays(3000, 31, box["cfg"].V)
    out = ctx.query_rays(_cuda(rays), obj=box["h"], precision=lsnif.FP8_FUSED, logits=True)
    ctx.check()
    # the GPU's sample points are the oracle's, exactly
    k, _, pts, _ = ctx.trace(_cuda(rays), box["h"])
    torch.cuda.synchronize()
    ref, seg = O.query(box["orc"], rays, precision="fp8")
    assert np.array_equal(k.cpu().numpy(), seg.k)
    assert np.array_equal(pts.cpu().numpy().astype(np.float64), seg.pts)
    assert (seg.k == box["cfg"].H // 2).sum() > 300          # capped runs with duplicate points
    live, lg, err, scale = _logit_err(out, ref, seg)
    assert (err < 1e-5).mean() >= 0.95, (err < 1e-5).mean()
    assert err.max() < 2.0 ** -2, err.max()
    _miss_record(out, ref, seg)


def _general_compare(ctx, o, rays):
    out = ctx.query_rays(_cuda(rays), obj=o["h"], precision=lsnif.FP8_FUSED, logits=True)
    ctx.check()
    torch.cuda.synchronize()
    ref, seg = O.query(o["orc"], rays, precision="fp8")
    live, lg, err, scale = _logit_err(out, ref, seg)
    assert np.quantile(err, 0.95) < 2.0 ** -4, np.quantile(err, 0.95)
    assert err.max() < 2.0 ** -2, err.max()
    hit = out.hit.cpu().numpy().astype(bool)[live]
    firm = np.abs(ref.logits[live, 0]) > 2.0 ** -3 * scale
    assert (hit[firm] == ref.hit[live][firm]).mean() >= 0.99
    zm = np.sort(ref.logits[live, 8:], axis=1)
    firm_m = (zm[:, -1] - zm[:, -2]) > 2.0 ** -3 * scale
    assert (out.mat.cpu().numpy()[live][firm_m] == ref.mat[live][firm_m]).mean() >= 0.99
    _miss_record(out, ref, seg)
    return out, ref, seg


def test_fp8_torus_matches_oracle_fp8(ctx, torus):
    _general_compare(ctx, torus, _camera_sample(1024, 11))


def test_fp8_stress_shape_matches_oracle_fp8(ctx, stress):
    o = stress["orc"]
    rays = I.rays_sphere_to_box(1500, 3.0, o.bmin, o.bmax, seed=12)
    out, ref, seg = _general_compare(ctx, stress, rays)
    # error against the FP64 network (random weights: many decisions sit
    # near zero, so this is a statement, not the acceptance bound)
    f64, _ = O.query(o, rays, precision="f64")
    live = f64.live & ~seg.near
    hit = out.hit.cpu().numpy().astype(bool)
    vis = (hit[live] != f64.hit[live]).mean()
    both = live & hit & f64.hit
    diag = float(np.linalg.norm(o.bmax.astype(np.float64) - o.bmin))
    t_err = np.abs(out.t.cpu().numpy()[both] - f64.t[both]) / diag
    mat = (out.mat.cpu().numpy()[both] == f64.mat[both]).mean()
    print(f"FP8 vs FP64 oracle (random network): visibility mismatch {vis:.4%}, hit-t error p50 "
          f"{np.median(t_err):.2e} p99 {np.quantile(t_err, 0.99):.2e} of the diagonal, material agreement {mat:.4%}")


def test_fp8_full_size_launch(ctx, torus):
    """2048 x 2048 primary rays in one launch (the benchmark's launch
    configuration): a seeded sample against the oracle's FP8 network and
    the properties of every ray."""
    rays = I.rays_pinhole(I.seeded_camera(2))
    out = ctx.query_rays(_cuda(rays), obj=torus["h"], precision=lsnif.FP8_FUSED)
    ctx.check()
    torch.cuda.synchronize()
    g = np.random.default_rng(13)
    idx = np.sort(g.choice(rays.shape[1], 384, replace=False))
    ref, seg = O.query(torus["orc"], np.ascontiguousarray(rays[:, idx]), precision="fp8")
    t = out.t.cpu().numpy()
    hit = out.hit.cpu().numpy().astype(bool)
    live = ref.live & ~seg.near
    scale = np.abs(ref.logits[live]).max()
    firm = live & (np.abs(ref.logits[:, 0]) > 2.0 ** -3 * scale)
    assert (hit[idx][firm] == ref.hit[firm]).mean() >= 0.99
    assert np.array_equal(np.isinf(t[idx])[~seg.near & ~ref.live], np.ones((~seg.near & ~ref.live).sum(), bool))
    mat = out.mat.cpu().numpy()
    assert np.all(np.isfinite(t[hit])) and np.all(t[hit] >= 0)
    assert np.all((mat == -1) == np.isinf(t))
    assert np.all((mat >= -1) & (mat < torus["cfg"].n_mat))


def test_fp8_follows_parameter_updates(ctx, torus):
    """The FP8 network is rebuilt after the parameters change."""
    rays = _camera_sample(512, 14)
    h = torus["h"]
    before = ctx.query_rays(_cuda(rays), obj=h, precision=lsnif.FP8_FUSED, logits=True).logits.cpu()
    mlp = ctx.read_params(h, lsnif.PARAM_MLP)
    scaled = mlp.copy()
    scaled[-torus["cfg"].n_out:] += 0.75      # output biases
    ctx.write_params(h, lsnif.PARAM_MLP, scaled)
    try:
        after = ctx.query_rays(_cuda(rays), obj=h, precision=lsnif.FP8_FUSED, logits=True).logits.cpu()
        live = ~torch.isnan(before[:, 0])
        assert live.sum() > 100
        assert torch.allclose(after[live] - before[live], torch.full_like(after[live], 0.75), atol=1e-5)
    finally:
        ctx.write_params(h, lsnif.PARAM_MLP, mlp)


def test_fp8_submit_graph_and_query_agree(ctx, torus):
    """The serving loop, graph replay and the direct call run the same
    kernel: identical results."""
    rays = _cuda(_camera_sample(3000, 15))
    direct = ctx.query_rays(rays, obj=torus["h"], precision=lsnif.FP8_FUSED, logits=True)
    res = ctx._alloc_hits(rays.shape[1], torus["cfg"].n_out, True)
    ticket = ctx.submit(rays, res, obj=torus["h"], precision=lsnif.FP8_FUSED)
    ctx.poll(ticket, timeout_us=30_000_000)
    ctx.set_graph_mode(True)
    try:
        g1 = ctx.query_rays(rays, obj=torus["h"], precision=lsnif.FP8_FUSED, logits=True)
        g2 = ctx.query_rays(rays, obj=torus["h"], precision=lsnif.FP8_FUSED, logits=True)
    finally:
        ctx.set_graph_mode(False)
    torch.cuda.synchronize()
    for other in (res, g1, g2):
        assert torch.equal(other.hit, direct.hit)
        assert torch.equal(other.mat, direct.mat)
        assert torch.equal(torch.nan_to_num(other.t, posinf=-1.0), torch.nan_to_num(direct.t, posinf=-1.0))
        assert torch.equal(torch.nan_to_num(other.logits, nan=-1e30), torch.nan_to_num(direct.logits, nan=-1e30))


def test_fp8_variants_give_identical_results(ctx, stress):
    o = stress["orc"]
    rays = _cuda(I.rays_sphere_to_box(20000, 3.0, o.bmin, o.bmax, seed=16))
    got = []
    try:
        for v in range(len(lsnif.Context.variants8())):
            ctx.set_variant8(v)
            out = ctx.query_rays(rays, obj=stress["h"], precision=lsnif.FP8_FUSED, logits=True)
            ctx.check()
            got.append((out.hit.cpu(), out.t.cpu(), out.mat.cpu(), torch.nan_to_num(out.logits.cpu(), nan=-1e30)))
    finally:
        ctx.set_variant8(0)
    assert len(got) >= 2
    for other in got[1:]:
        for a, b in zip(got[0], other):
            assert torch.equal(torch.nan_to_num(a, posinf=-1.0), torch.nan_to_num(b, posinf=-1.0))


def test_fp8_unsupported_shape_is_refused(ctx):
    cfg = I.Config(V=8, H=8, L=2, F=4, log2_T=8, N_min=4, N_max=8, n_hidden=1, width=32, n_mat=2)
    h = ctx.load_object(I.icosphere(1), cfg)
    r = _cuda(I.rays_sphere_to_box(10, 3.0, (-1, -1, -1), (1, 1, 1), seed=1))
    with pytest.raises(lsnif.LsnifError) as e:
        ctx.query_rays(r, obj=h, precision=lsnif.FP8_FUSED)
    assert e.value.code == -10
    ctx.unload_object(h)
