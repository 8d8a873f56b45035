"""The oracle's host threading changes timing only: segments, encodings and
judge answers are identical on one thread and on all of them."""
import numpy as np

from oracle import oracle as O
from paper_2504_21627_gb300 import inputs as I


def _run():
    cfg = I.Config(V=16, H=8, L=4, F=2, log2_T=10, N_min=4, N_max=32, n_hidden=2, width=64, n_mat=2)
    mesh = I.noise_icosphere(seed=4, target_tris=1280, amplitude=0.08, n_mat=2)
    orc = O.build_object(mesh, cfg, I.random_params(cfg, seed=3))
    rays = I.rays_sphere_to_box(3000, 3.0, orc.bmin, orc.bmax, seed=5)
    seg = O.ray_segments(orc, rays)
    hits, _ = O.query(orc, rays, seg=seg)
    j = O.judge(mesh, rays)
    return seg.k, seg.pts, hits.logits, j.t, j.tri


def test_results_do_not_depend_on_the_thread_count():
    before = O.threads()
    try:
        O.threads(1)
        one = _run()
        O.threads(max(2, before))
        many = _run()
    finally:
        O.threads(before)
    for a, b in zip(one, many):
        assert np.array_equal(a, b, equal_nan=True)
