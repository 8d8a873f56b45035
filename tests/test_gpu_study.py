"""Directions of the paper's parameter study (Sec. 6.1) on a synthetic mesh:
networks trained on the GPU by the library's own training step, evaluated on
held-out rays against the oracle's FP64 brute-force judge (nearest triangle
over the whole mesh). Only the directions are pinned, with the base
configuration of the paper (V 32, H 18, two levels 64..128, 2^17 entries,
2 x 128; F = 4 so that H L F is a multiple of 16):

  a larger hash map lowers the hit-distance error and raises material accuracy,
  more training steps lower the hit-distance error,
  more points per ray (H) raise visibility accuracy."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2504_21627_gb300 import inputs as I  # noqa: E402
from paper_2504_21627_gb300 import lsnif  # noqa: E402

BASE = dict(V=32, H=18, L=2, F=4, log2_T=17, N_min=64, N_max=128, n_hidden=2, width=128, n_mat=4)


@pytest.fixture(scope="module")
def study():
    mesh = I.noise_torus_tris(11, 20000, amplitude=0.08, n_mat=4)
    lo, hi = O.bbox(mesh.verts)
    diag = float(np.linalg.norm(hi.astype(np.float64) - lo))
    rays = I.rays_sphere_to_box(8000, 1.25 * diag, lo, hi, seed=77)
    judge = O.judge(mesh, rays)
    ctx = lsnif.Context(0)
    results = {}

    def run(name, steps=2000, **over):
        cfg = I.Config(**dict(BASE, **over))
        h = ctx.load_object(mesh, cfg, keep_mesh=True)
        n_pool, B = 1 << 19, 1 << 14
        u = torch.rand((n_pool, lsnif.TRAIN_UNIFORMS), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
        pool, _ = ctx.make_training_rays(h, u, n_outside=n_pool // 2)
        lab = ctx.label_rays(pool, h)
        keep = lab["k"] > 0
        pool = pool[:, keep].contiguous()
        lab = {k: v[keep].contiguous() for k, v in lab.items()}
        gen = torch.Generator("cuda").manual_seed(5)
        for _ in range(steps):
            idx = torch.randint(0, pool.shape[1], (B,), device="cuda", generator=gen)
            ctx.train_step(pool[:, idx].contiguous(), {k: v[idx].contiguous() for k, v in lab.items()}, h,
                           lr=0.01, stats=False)
        q = ctx.query_rays(torch.from_numpy(rays).cuda(), obj=h, precision=lsnif.FP32_PLAIN)
        ctx.check()
        hit = q.hit.cpu().numpy().astype(bool)
        t = q.t.cpu().numpy().astype(np.float64)
        mat = q.mat.cpu().numpy()
        truth = judge.tri >= 0
        both = hit & truth
        terr = np.abs(t[both] - judge.t[both]) / diag
        ref_mat = mesh.tri_mat[judge.tri[both]]
        results[name] = dict(vis=float((hit == truth).mean()), t_p50=float(np.median(terr)),
                             mat=float((mat[both] == ref_mat).mean()))
        print(f"{name}: {results[name]}")
        ctx.unload_object(h)

    run("base")
    run("T 2^11", log2_T=11)
    run("100 steps", steps=100)
    run("H 6", H=6)
    yield results
    ctx.close()


def test_larger_hash_map_is_more_accurate(study):
    # 2^11 entries per level collide heavily at 128^3: material suffers most
    assert study["base"]["mat"] > study["T 2^11"]["mat"] + 0.1
    assert study["base"]["t_p50"] < study["T 2^11"]["t_p50"]


def test_more_training_steps_are_more_accurate(study):
    assert study["base"]["t_p50"] < study["100 steps"]["t_p50"]
    assert study["base"]["mat"] > study["100 steps"]["mat"]


def test_more_points_per_ray_see_more(study):
    assert study["base"]["vis"] > study["H 6"]["vis"]
