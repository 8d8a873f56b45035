"""Pins for the oracle's network, decode, losses, backward pass, Adam and
storage model (Sec. 5.1-5.3)."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_21627_gb300 import inputs as I

torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_mlp_matches_torch_addmm_chain():
    cfg = I.cfg_icosphere_small()
    p = I.random_params(cfg, 3, bias_range=0.1)
    g = np.random.default_rng(0)
    X = g.normal(size=(64, cfg.n_in))
    got = O.mlp_forward(X, [(W.astype(np.float64), b.astype(np.float64)) for W, b in p.weights])
    h = torch.from_numpy(X)
    for i, (W, b) in enumerate(p.weights):
        h = torch.addmm(torch.from_numpy(b.astype(np.float64)), h, torch.from_numpy(W.astype(np.float64)).T)
        if i < len(p.weights) - 1:
            h = torch.relu(h)
    assert np.allclose(got, h.numpy(), rtol=1e-13, atol=1e-13)
    # leaky variant
    got = O.mlp_forward(X, [(W.astype(np.float64), b.astype(np.float64)) for W, b in p.weights], act=1)
    h = torch.from_numpy(X)
    for i, (W, b) in enumerate(p.weights):
        h = torch.addmm(torch.from_numpy(b.astype(np.float64)), h, torch.from_numpy(W.astype(np.float64)).T)
        if i < len(p.weights) - 1:
            h = torch.nn.functional.leaky_relu(h, 0.01)
    assert np.allclose(got, h.numpy(), rtol=1e-13, atol=1e-13)


def test_decode_closed_form():
    Z = np.array([[2.0, 0.0, 3.0, 0.0, 4.0, 0.0, 100.0, -100.0, 0.1, 0.7, 0.7, -1.0],
                  [-1e-9, math.log(3.0), 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, 5.0, 1.0, 2.0, 3.0],
                  [0.5, -50.0, 1.0, 1.0, 1.0, 0, 0, 0, 0, 0, 0, 0]])
    t01 = np.array([[1.0, 3.0], [2.0, 6.0], [0.0, 1.0]])
    d = O.decode(Z, t01, tmin=np.array([0.0, 0.0, 0.5]), tmax=np.array([np.inf, np.inf, np.inf]))
    assert list(d["hit"]) == [True, False, False]      # z0 <= 0 -> miss; row 3: t < tmin
    assert d["t"][0] == 2.0                            # 1 + 0.5 * 2
    assert abs(d["t"][1] - (2.0 + 0.75 * 4.0)) < 1e-15  # sigmoid(ln 3) = 3/4
    assert np.allclose(d["normal"][0], [0.6, 0.0, 0.8], atol=1e-15)
    assert np.array_equal(d["normal"][1], [0, 0, 0])   # zero stays zero
    assert list(d["mat"]) == [1, 0, 0]                  # tie 0.7/0.7 -> lowest
    assert abs(d["albedo"][0, 1] - 1.0) < 1e-15 and d["albedo"][0, 2] < 1e-40
    assert np.allclose(d["albedo"][1], 1.0 / (1.0 + math.exp(-1.0)), atol=1e-15)


def _labels(n, n_mat, g):
    nrm = g.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return O.Labels(occ=(g.random(n) < 0.6).astype(np.float64), t_local=g.random(n), normal=nrm,
                    albedo=g.random((n, 3)), mat=g.integers(0, n_mat, n).astype(np.int32))


def _torch_loss(Z, lab):
    z = torch.from_numpy(Z).requires_grad_(True)
    y = torch.from_numpy(lab.occ)
    l_occ = torch.nn.functional.binary_cross_entropy_with_logits(z[:, 0], y, reduction="none")
    l_t = (torch.sigmoid(z[:, 1]) - torch.from_numpy(lab.t_local)).abs()
    n = torch.from_numpy(lab.normal)
    zn = z[:, 2:5]
    l_n = 1.0 - (zn * n).sum(1) / zn.norm(dim=1).clamp_min(O.NORMAL_EPS)
    sa = torch.sigmoid(z[:, 5:8])
    l_a = ((sa - torch.from_numpy(lab.albedo)) ** 2 / (sa.detach() ** 2 + O.REL_L2_EPS)).mean(1)
    l_m = torch.nn.functional.cross_entropy(z[:, 8:], torch.from_numpy(lab.mat).long(), reduction="none")
    tot = (l_occ + y * (l_t + l_n + l_a + l_m)).mean()
    tot.backward()
    return tot.item(), z.grad.numpy()


def test_loss_and_logit_gradient_match_torch_autograd():
    g = np.random.default_rng(1)
    n, n_mat = 257, 4
    Z = g.normal(size=(n, 8 + n_mat)) * 2
    lab = _labels(n, n_mat, g)
    terms, dZ = O.loss_terms(Z, lab)
    tot, gref = _torch_loss(Z, lab)
    assert abs(terms["total"] - tot) < 1e-12
    assert np.allclose(dZ, gref, rtol=1e-10, atol=1e-14)
    assert abs(sum(terms[k] for k in ("occ", "t", "normal", "albedo", "mat")) - terms["total"]) < 1e-12


def test_bce_closed_form():
    lab = O.Labels(np.array([1.0, 0.0]), np.zeros(2), np.tile([0, 0, 1.0], (2, 1)), np.zeros((2, 3)),
                   np.zeros(2, np.int32))
    Z = np.zeros((2, 9))
    Z[:, 4] = 1.0  # normal = label -> zero cosine loss
    terms, _ = O.loss_terms(Z, lab)
    assert abs(terms["occ"] - math.log(2.0)) < 1e-15          # BCE(0.5)
    assert abs(terms["t"] - 0.5 * 0.5) < 1e-15                 # |0.5 - 0| on the occluded ray
    assert abs(terms["normal"]) < 1e-15
    assert abs(terms["mat"] - 0.5 * math.log(1.0)) < 1e-15     # single material


def _tiny_object(seed=0, act=0):
    cfg = I.Config(V=4, H=6, L=2, F=2, log2_T=6, N_min=3, N_max=7, n_hidden=2, width=8, n_mat=2,
                   activation=act)
    m = I.icosphere(1, seed=seed)
    p = I.random_params(cfg, seed, table_range=0.5, bias_range=0.2)
    return cfg, m, O.build_object(m, cfg, p)


@pytest.mark.parametrize("act", [0, 1])
def test_backward_matches_torch_autograd_end_to_end(act):
    cfg, m, obj = _tiny_object(1, act)
    rays = I.rays_sphere_to_box(64, 3.0, obj.bmin, obj.bmax, seed=2)
    seg = O.ray_segments(obj, rays)
    keep = seg.k > 0
    rays = rays[:, keep]
    seg = O.ray_segments(obj, rays)
    lab = O.labels(m, rays, seg.t01)
    terms, grads, gt = O.forward_backward(obj, rays, lab, seg)
    # the same model in torch autograd, with the encoding as a dense linear map
    Tt = torch.from_numpy(obj.tables.copy()).requires_grad_(True)
    n = rays.shape[1]
    live = np.arange(cfg.H)[None, :] < 2 * seg.k[:, None]
    _, idx, w = O.encode(seg.pts[live], obj.res, cfg.F, cfg.log2_T, obj.tables, debug=True)
    feats = torch.zeros(n, cfg.H, cfg.L, cfg.F, dtype=torch.float64)
    lv = torch.from_numpy(np.argwhere(live))
    vals = []
    for l in range(cfg.L):
        corner = Tt[l][torch.from_numpy(idx[:, l, :].astype(np.int64))]        # (P, 8, F)
        vals.append((corner * torch.from_numpy(w[:, l, :])[..., None]).sum(1))
    vals = torch.stack(vals, 1)                                               # (P, L, F)
    feats = feats.index_put((lv[:, 0], lv[:, 1]), vals)
    h = feats.reshape(n, -1)
    Ws = [(torch.from_numpy(W.copy()).requires_grad_(True), torch.from_numpy(b.copy()).requires_grad_(True))
          for W, b in obj.weights]
    for i, (W, b) in enumerate(Ws):
        h = h @ W.T + b
        if i < len(Ws) - 1:
            h = torch.relu(h) if act == 0 else torch.nn.functional.leaky_relu(h, 0.01)
    Z = h.detach().numpy()
    tot, gZ = _torch_loss(Z, lab)
    h.backward(torch.from_numpy(gZ))
    assert abs(terms["total"] - tot) < 1e-12
    for (gW, gb), (W, b) in zip(grads, Ws):
        assert np.allclose(gW, W.grad.numpy(), rtol=1e-9, atol=1e-13)
        assert np.allclose(gb, b.grad.numpy(), rtol=1e-9, atol=1e-13)
    assert np.allclose(gt, Tt.grad.numpy(), rtol=1e-9, atol=1e-13)


def test_backward_matches_finite_differences(monkeypatch):
    # The albedo term divides by a stopped-gradient sigmoid^2 (Noise2Noise's
    # relative L2), which a finite difference of the loss value would
    # differentiate through; a huge constant makes that term vanish here. Its
    # gradient is pinned by the autograd test above, which detaches it.
    monkeypatch.setattr(O, "REL_L2_EPS", 1e12)
    cfg, m, obj = _tiny_object(3, act=1)
    rays = I.rays_sphere_to_box(48, 3.0, obj.bmin, obj.bmax, seed=5)
    seg = O.ray_segments(obj, rays)
    rays = rays[:, seg.k > 0]
    seg = O.ray_segments(obj, rays)
    lab = O.labels(m, rays, seg.t01)
    _, grads, gt = O.forward_backward(obj, rays, lab, seg)
    g = np.random.default_rng(7)
    h = 1e-6

    def loss():
        return O.forward_backward(obj, rays, lab, seg)[0]["total"]

    checked = 0
    nz = np.argwhere(np.abs(gt) > 1e-6)
    for l, e, f in nz[g.choice(len(nz), 6, replace=False)]:
        old = obj.tables[l, e, f]
        obj.tables[l, e, f] = old + h
        lp = loss()
        obj.tables[l, e, f] = old - h
        lm = loss()
        obj.tables[l, e, f] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gt[l, e, f]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8
        checked += 1
    for li in range(len(obj.weights)):
        W = obj.weights[li][0]
        for _ in range(3):
            i, j = g.integers(0, W.shape[0]), g.integers(0, W.shape[1])
            old = W[i, j]
            W[i, j] = old + h
            lp = loss()
            W[i, j] = old - h
            lm = loss()
            W[i, j] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[li][0][i, j]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8
            checked += 1
    assert checked >= 15


def test_adam_first_step_closed_form():
    g = np.random.default_rng(0)
    p0 = g.normal(size=100)
    gr = g.normal(size=100)
    st = O.adam_init([p0])
    (p1,) = O.adam_step([p0], [gr], st, lr=0.01)
    # after one step m_hat = g and v_hat = g^2
    assert np.allclose(p1, p0 - 0.01 * gr / (np.abs(gr) + 1e-8), rtol=0, atol=1e-15)
    # matches torch.optim.Adam over a few steps
    tp = torch.from_numpy(p0.copy()).requires_grad_(True)
    opt = torch.optim.Adam([tp], lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    st = O.adam_init([p0])
    p = p0.copy()
    for s in range(5):
        grad = g.normal(size=100)
        tp.grad = torch.from_numpy(grad.copy())
        opt.step()
        (p,) = O.adam_step([p], [grad], st, lr=0.01)
    assert np.allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def _golden_footprint():
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_footprint.txt")):
        s = line.split("#")[0].split()
        if len(s) == 3:
            out[s[0]] = float(s[1]) * (1024 if s[2] == "KB" else 1024 * 1024)
    return out


def test_storage_model_against_printed_numbers():
    gf = _golden_footprint()
    # Sec. 5.1: V=32, 2 levels x 2^17 x 3 features, MLP 108 -> 128 -> 128 -> 9
    # (input = H*L*F = 18*2*3; output 8 + N_mat with one material), FP16 storage
    dims = [(108, 128), (128, 128), (128, 9)]
    fp = O.footprint_bytes(V=32, L=2, T=2 ** 17, F=3, layer_dims=dims)
    assert fp["voxels"] == gf["voxels_32"]
    assert fp["encoder"] == gf["encoder"]
    assert round(fp["network"] / 1024) == 62                         # "about 62 KB"
    assert round(fp["total"] / 2 ** 20, 2) == 1.56
    assert O.footprint_bytes(64, 2, 2 ** 17, 3, dims)["voxels"] == gf["voxels_64"]
    for e in (8, 11, 14, 17):
        enc = O.footprint_bytes(32, 2, 2 ** e, 3, dims)["encoder"]
        assert enc == gf[f"hash_2^{e}"]
    per_obj = round(fp["total"] / 2 ** 20, 2)
    for key, count in (("scene_statues", 4), ("scene_junkshop", 9), ("scene_classroom", 15)):
        assert round(count * per_obj * 2 ** 20) == round(gf[key])


def test_rays_without_points_take_no_part_in_the_loss():
    cfg, m, obj = _tiny_object(4)
    rays = I.rays_sphere_to_box(80, 3.0, 2.5 * obj.bmin, 2.5 * obj.bmax, seed=9)   # some miss the object
    seg = O.ray_segments(obj, rays)
    assert (seg.k == 0).any() and (seg.k > 0).any()
    lab = O.labels(m, rays, np.nan_to_num(seg.t01))
    terms, grads, gt = O.forward_backward(obj, rays, lab, seg)
    keep = seg.k > 0
    sub = rays[:, keep]
    seg2 = O.ray_segments(obj, sub)
    lab2 = O.Labels(lab.occ[keep], lab.t_local[keep], lab.normal[keep], lab.albedo[keep], lab.mat[keep])
    terms2, grads2, gt2 = O.forward_backward(obj, sub, lab2, seg2)
    assert abs(terms["total"] - terms2["total"]) < 1e-13
    for (a, b), (c, d) in zip(grads, grads2):
        assert np.allclose(a, c, atol=1e-15) and np.allclose(b, d, atol=1e-15)
    assert np.allclose(gt, gt2, atol=1e-15)
