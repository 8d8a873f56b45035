"""GPU parity of the streamed FP16 fused query -- the FP16 path for networks
whose weights do not fit shared memory, here the stress configuration's
shape (16 levels x 4 features, 1152 -> 128 x 4 -> 12) -- against the
oracle's FP16 network mode: FP16 rounding of the interpolated features, the
weights and the hidden activations, FP64 sums.

The kernel interpolates in FP32 (the oracle in FP64) and rounds each feature
once to FP16, like the oracle, so the two differ only where an FP32 and an
FP64 value round to neighbouring FP16 values (2^-11 of a value) and where the
FP32 boundary points move lattice coordinates (the FP32 path's bound at this
lattice resolution). The logits are held to the FP16 path's bound: 2^-9 of
the largest logit plus the FP32 bound; decisions with a margin of four (hit)
or eight (material) times that agree."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2504_21627_gb300 import inputs as I  # noqa: E402
from paper_2504_21627_gb300 import lsnif  # noqa: E402


def fp32_tol(cfg):
    return max(1e-4, 8 * 2.0 ** -24 * cfg.N_max)


@pytest.fixture(scope="module")
def ctx():
    c = lsnif.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def stress(ctx):
    """The stress shape with 2^18 entries per level (the oracle holds an FP64
    copy of the tables)."""
    cfg = I.cfg_stress_object(log2_T=18)
    mesh = I.noise_torus(seed=2, nu=200, nv=80)
    p = I.random_params(cfg, 7, table_range=0.05, bias_range=0.1)
    orc = O.build_object(mesh, cfg, p)
    h = ctx.load_object(mesh, cfg, tables=p.tables, mlp=p.packed_mlp())
    return dict(h=h, orc=orc, cfg=cfg)


def _compare(ctx, o, rays):
    out = ctx.query_rays(torch.from_numpy(np.ascontiguousarray(rays)).cuda(), obj=o["h"],
                         precision=lsnif.FP16_FUSED, logits=True)
    ctx.check()
    ref, seg = O.query(o["orc"], rays, precision="fp16")
    ok = ~seg.near
    live = ref.live & ok
    assert live.sum() > 500
    lg = out.logits.cpu().numpy()
    scale = np.abs(ref.logits[live]).max()
    tol = 2.0 ** -9 + fp32_tol(o["cfg"])
    err = np.abs(lg[live] - ref.logits[live]).max() / scale
    print(f"streamed FP16: logit error {err:.3g} of the largest (bound {tol:.3g}) over {live.sum()} rays")
    assert err < tol
    hit = out.hit.cpu().numpy().astype(bool)
    miss = ~ref.live & ok
    assert not hit[miss].any()
    assert np.all(np.isinf(out.t.cpu().numpy()[miss]))
    firm = np.abs(ref.logits[live, 0]) > 4 * tol * scale
    assert np.array_equal(hit[live][firm], ref.hit[live][firm])
    zm = np.sort(ref.logits[live, 8:], axis=1)
    firm_m = (zm[:, -1] - zm[:, -2]) > 8 * tol * scale
    assert np.array_equal(out.mat.cpu().numpy()[live][firm_m], ref.mat[live][firm_m])


def test_streamed_fp16_matches_oracle_camera_rays(ctx, stress):
    g = np.random.default_rng(5)
    cam = I.rays_pinhole(I.seeded_camera(2, width=512, height=512))
    _compare(ctx, stress, cam[:, g.choice(cam.shape[1], 3000, replace=False)])


def test_streamed_fp16_matches_oracle_sphere_rays(ctx, stress):
    rays = I.rays_sphere_to_box(3000, 3.0, stress["orc"].bmin, stress["orc"].bmax, seed=9)
    _compare(ctx, stress, rays)


def test_bf16_on_the_stress_shape_is_refused(ctx, stress):
    """BF16 keeps every weight resident (two-term later layers) and does not
    cover this shape: refused, not run."""
    r = torch.from_numpy(I.rays_sphere_to_box(100, 3.0, stress["orc"].bmin, stress["orc"].bmax, seed=1)).cuda()
    with pytest.raises(lsnif.LsnifError) as e:
        ctx.query_rays(r, obj=stress["h"], precision=lsnif.BF16_FUSED)
    assert e.value.code == -10
