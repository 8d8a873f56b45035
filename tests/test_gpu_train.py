"""GPU training path against the oracle: balanced training rays (Sec. 5.2),
ground-truth labels by ray casting, one step's loss and gradients, the Adam
update, and what the trained network gains over the method without it."""
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


@pytest.fixture(scope="module")
def sphere(ctx):
    cfg = I.cfg_icosphere_small()
    mesh = I.noise_icosphere(seed=4, target_tris=1280, amplitude=0.08, n_mat=2)
    p = I.random_params(cfg, 9, table_range=0.3, bias_range=0.1)
    orc = O.build_object(mesh, cfg, p)
    h = ctx.load_object(mesh, cfg, tables=p.tables, mlp=p.packed_mlp(), keep_mesh=True)
    return dict(h=h, orc=orc, p=p, mesh=mesh, cfg=cfg)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_training_rays_match_oracle(ctx, sphere):
    n = 4096
    u = I.uniforms(n, lsnif.TRAIN_UNIFORMS, seed=12)
    rays, surf = ctx.make_training_rays(sphere["h"], _cuda(u), n_outside=n // 2)
    torch.cuda.synchronize()
    rays, surf = rays.cpu().numpy(), surf.cpu().numpy().astype(bool)
    ref, rsurf = O.training_rays(sphere["mesh"], sphere["orc"].bmin, sphere["orc"].bmax, u, n // 2)
    assert not surf[: n // 2].any()
    out = slice(0, n // 2)
    assert np.allclose(rays[:, out], ref[:, out], atol=2e-5)
    agree = surf == rsurf
    assert agree.mean() > 0.995, agree.mean()
    both = surf & rsurf
    diag = np.linalg.norm(sphere["orc"].bmax.astype(np.float64) - sphere["orc"].bmin)
    assert np.allclose(rays[0:3, both], ref[0:3, both], atol=1e-4 * diag)
    assert np.allclose(rays[3:6, both], ref[3:6, both], atol=1e-3)
    assert surf[n // 2:].mean() > 0.5


def test_labels_match_the_judge(ctx, sphere):
    n = 4096
    u = I.uniforms(n, lsnif.TRAIN_UNIFORMS, seed=13)
    rays, _ = O.training_rays(sphere["mesh"], sphere["orc"].bmin, sphere["orc"].bmax, u, n // 2)
    lab = ctx.label_rays(_cuda(rays), sphere["h"])
    torch.cuda.synchronize()
    lab = {k: v.cpu().numpy() for k, v in lab.items()}
    seg = O.ray_segments(sphere["orc"], rays)
    j = O.judge(sphere["mesh"], rays)
    ref = O.labels(sphere["mesh"], rays, np.nan_to_num(seg.t01))
    occ_agree = (lab["occ"] > 0) == (ref.occ > 0)
    assert occ_agree.mean() > 0.998
    same = (lab["tri"] == j.tri) & (j.tri >= 0)
    assert same.sum() >= 0.99 * (j.tri >= 0).sum()
    assert np.allclose(lab["t_hit"][same], j.t[same], rtol=1e-5, atol=1e-6)
    assert np.allclose(lab["normal"][same], ref.normal[same], atol=1e-4)
    assert np.array_equal(lab["mat"][same], ref.mat[same])
    assert np.allclose(lab["albedo"][same], ref.albedo[same], atol=1e-6)
    assert np.allclose(lab["t_local"][same], ref.t_local[same], atol=1e-4)
    ok = ~seg.near
    assert np.array_equal(lab["k"][ok], seg.k[ok])


def _batch(sphere, n, seed, margin=3e-4):
    """Seeded rays with their oracle labels. Left out: rays the network never
    sees, near-face rays (point lists not unique), and rays whose gradient is
    not unique between FP32 and FP64 -- a hidden pre-activation within
    `margin` times its layer's RMS of the ReLU kink (about three times the
    FP32 pre-activation error at this lattice resolution), or a hit distance
    within 1e-3 of the MAE term's sign change. One such ray flips its whole
    contribution to the summed gradient."""
    orc = sphere["orc"]
    rays = I.rays_sphere_to_box(n, 2.2, orc.bmin, orc.bmax, seed=seed)
    seg = O.ray_segments(orc, rays)
    keep = (seg.k > 0) & ~seg.near
    rays = np.ascontiguousarray(rays[:, keep])
    seg = O.ray_segments(orc, rays)
    lab = O.labels(sphere["mesh"], rays, seg.t01)
    Z, cache = O.mlp_forward(O.features(orc, seg), orc.weights, orc.cfg.activation, keep=True)
    ok = np.ones(rays.shape[1], bool)
    for _, z in cache[:-1]:
        ok &= np.all(np.abs(z) > margin * np.sqrt(np.mean(z * z)), axis=1)
    ok &= np.abs(O.sigmoid(Z[:, 1]) - lab.t_local) > 1e-3
    assert ok.mean() > 0.8, ok.mean()
    rays = np.ascontiguousarray(rays[:, ok])
    seg = O.ray_segments(orc, rays)
    lab = O.labels(sphere["mesh"], rays, seg.t01)
    return rays, seg, lab


def _lab_cuda(lab):
    return dict(occ=_cuda(lab.occ.astype(np.float32)), t_local=_cuda(lab.t_local.astype(np.float32)),
                normal=_cuda(lab.normal.astype(np.float32)), albedo=_cuda(lab.albedo.astype(np.float32)),
                mat=_cuda(lab.mat.astype(np.int32)))


# The network's products: tensor cores (two-term BF16 operands, FP32
# accumulation: each product carries a relative error of about 2^-16, far
# inside the 1e-4 bound) or the FP32 SIMT reference.
PRODUCTS = [lsnif.TRAIN_TENSOR_CORES, lsnif.TRAIN_FP32_SIMT]


@pytest.mark.parametrize("products", PRODUCTS)
def test_gradients_match_oracle(ctx, sphere, products):
    rays, seg, lab = _batch(sphere, 3000, seed=17)
    st = ctx.train_step(_cuda(rays), _lab_cuda(lab), sphere["h"], apply_update=False, products=products)
    g_mlp = ctx.read_params(sphere["h"], lsnif.PARAM_GRAD_MLP)
    g_tab = ctx.read_params(sphere["h"], lsnif.PARAM_GRAD_TABLES)
    terms, grads, gt = O.forward_backward(sphere["orc"], rays, lab, seg)
    assert abs(st.total - terms["total"]) < 1e-4 * abs(terms["total"])
    for name in ("occ", "t", "normal", "albedo", "mat"):
        assert abs(getattr(st, name) - terms[name]) < 1e-4 * abs(terms["total"]), name
    ref_mlp = np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in grads])
    err = np.abs(g_mlp - ref_mlp).max() / np.abs(ref_mlp).max()
    err_t = np.abs(g_tab - gt).max() / np.abs(gt).max()
    print(f"products {products}: network gradient error {err:.2e}, table gradient error {err_t:.2e} of the largest")
    assert err < 1e-4, f"network gradient error {err:.3g}"
    assert err_t < 1e-4, f"table gradient error {err_t:.3g}"
    # no update was applied
    assert np.array_equal(ctx.read_params(sphere["h"], lsnif.PARAM_TABLES), sphere["p"].tables)


@pytest.mark.parametrize("products", PRODUCTS)
def test_adam_step_matches_oracle(ctx, sphere, products):
    rays, seg, lab = _batch(sphere, 3000, seed=19)
    h = ctx.load_object(sphere["mesh"], sphere["cfg"], tables=sphere["p"].tables, mlp=sphere["p"].packed_mlp())
    ctx.train_step(_cuda(rays), _lab_cuda(lab), h, lr=0.01, apply_update=True, products=products)
    new_mlp = ctx.read_params(h, lsnif.PARAM_MLP).astype(np.float64)
    new_tab = ctx.read_params(h, lsnif.PARAM_TABLES).astype(np.float64)
    _, grads, gt = O.forward_backward(sphere["orc"], rays, lab, seg)
    g = np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in grads])
    p0 = sphere["p"].packed_mlp().astype(np.float64)
    st = O.adam_init([p0, sphere["orc"].tables])
    want_mlp, want_tab = O.adam_step([p0, sphere["orc"].tables], [g, gt], st, lr=0.01)
    for got, want, grad in ((new_mlp, want_mlp, g), (new_tab, want_tab, gt)):
        firm = np.abs(grad) > 1e-2 * np.abs(grad).max()
        assert np.allclose(got[firm], want[firm], atol=2e-5)
        # every entry moves by at most the learning rate on the first step
        base = p0 if got is new_mlp else sphere["orc"].tables
        assert np.all(np.abs(got - base) <= 0.01 * (1 + 1e-5))
    ctx.unload_object(h)


def test_training_learns_and_beats_voxel_only(ctx):
    """Train an object from its seeded initialisation on GPU-generated rays
    and labels, then compare with the method without the network: a ray hits
    at the entry of its first occupied voxel."""
    cfg = I.cfg_icosphere_small()
    mesh = I.noise_icosphere(seed=6, target_tris=1280, amplitude=0.08, n_mat=2)
    h = ctx.load_object(mesh, cfg, keep_mesh=True)
    n_pool, B, steps = 1 << 18, 1 << 14, 800
    u = torch.rand((n_pool, lsnif.TRAIN_UNIFORMS), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    pool, _ = ctx.make_training_rays(h, u, n_outside=n_pool // 2)
    lab = ctx.label_rays(pool, h)
    keep = lab["k"] > 0
    pool = pool[:, keep].contiguous()
    lab = {k: v[keep].contiguous() for k, v in lab.items()}
    n = pool.shape[1]
    losses = []
    gen = torch.Generator("cuda").manual_seed(5)
    for s in range(steps):
        idx = torch.randint(0, n, (B,), device="cuda", generator=gen)
        st = ctx.train_step(pool[:, idx].contiguous(), {k: v[idx].contiguous() for k, v in lab.items()}, h,
                            lr=0.01, stats=(s % 100 == 0 or s == steps - 1))
        if st is not None:
            losses.append(st.total)
    assert losses[-1] < 0.5 * losses[0], losses
    # held-out evaluation against the FP64 judge
    orc_occ = O.voxelize(mesh.verts, mesh.tris, *O.bbox(mesh.verts), cfg.V)
    lo, hi = O.bbox(mesh.verts)
    test = I.rays_sphere_to_box(4000, 2.5, lo, hi, seed=77)
    j = O.judge(mesh, test)
    out = ctx.query_rays(_cuda(test), obj=h, precision=lsnif.BF16_FUSED)
    k, t01, pts, vox = ctx.trace(_cuda(test), h)
    torch.cuda.synchronize()
    hit = out.hit.cpu().numpy().astype(bool)
    t = out.t.cpu().numpy()
    k = k.cpu().numpy()
    pts = pts.cpu().numpy()
    truth = j.tri >= 0
    vox_hit = k > 0
    # voxel-only hit distance: entry point of the first occupied voxel
    o = test[0:3].T.astype(np.float64)
    d = test[3:6].T.astype(np.float64)
    ext = hi.astype(np.float64) - lo
    p_world = lo + pts[:, 0, :] * ext
    t_vox = np.einsum("ij,ij->i", p_world - o, d) / np.einsum("ij,ij->i", d, d)
    both_net = truth & hit
    both_vox = truth & vox_hit
    err_net = np.median(np.abs(t[both_net] - j.t[both_net]))
    err_vox = np.median(np.abs(t_vox[both_vox] - j.t[both_vox]))
    acc_net = (hit == truth).mean()
    acc_vox = (vox_hit == truth).mean()
    print(f"hit-t median error: network {err_net:.4g}, voxel-only {err_vox:.4g}; "
          f"visibility accuracy: network {acc_net:.4f}, voxel-only {acc_vox:.4f}; losses {losses}")
    assert err_net < err_vox
    assert acc_net > acc_vox
    # reduced precision on the trained network, against its FP32 evaluation
    ref = ctx.query_rays(_cuda(test), obj=h, precision=lsnif.FP32_PLAIN)
    torch.cuda.synchronize()
    r_hit, r_t, r_mat = ref.hit.cpu().numpy().astype(bool), ref.t.cpu().numpy(), ref.mat.cpu().numpy()
    diag = float(np.linalg.norm(ext))
    for name, prec in (("BF16", lsnif.BF16_FUSED), ("FP16", lsnif.FP16_FUSED), ("FP8", lsnif.FP8_FUSED)):
        q = ctx.query_rays(_cuda(test), obj=h, precision=prec)
        torch.cuda.synchronize()
        q_hit, q_t, q_mat = q.hit.cpu().numpy().astype(bool), q.t.cpu().numpy(), q.mat.cpu().numpy()
        both = q_hit & r_hit
        vis = (q_hit != r_hit).mean()
        dt = np.abs(q_t[both] - r_t[both]) / diag
        mat_ok = (q_mat[both] == r_mat[both]).mean()
        print(f"{name} vs FP32 on the trained network: visibility mismatch {vis:.4%}, hit-t error p50 "
              f"{np.median(dt):.2e} p90 {np.quantile(dt, 0.9):.2e} p99 {np.quantile(dt, 0.99):.2e} of the "
              f"diagonal, material agreement {mat_ok:.4%}")
        if prec == lsnif.FP16_FUSED:
            # the half-precision bounds, met at the 99th percentile of the hit distance
            assert vis <= 0.001 and mat_ok >= 0.999 and np.quantile(dt, 0.99) <= 1e-3
    del orc_occ
    ctx.unload_object(h)
