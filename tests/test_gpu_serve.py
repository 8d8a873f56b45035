"""Serving loop (lsnif_submit / lsnif_poll): continuous batching over a
stream pool with memory admission. Each request's result must equal the
same rays queried alone."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2504_21627_gb300 import inputs as I  # noqa: E402
from paper_2504_21627_gb300 import lsnif  # noqa: E402


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _objects(ctx):
    objs = []
    for s in range(3):
        cfg = I.Config(V=64, H=18, L=16, F=2, log2_T=16, N_min=16, N_max=512, n_hidden=4, width=64, n_mat=4, seed=s)
        mesh = I.noise_icosphere(seed=10 + s, target_tris=5000, n_mat=4)
        params = I.random_params(cfg, 20 + s, table_range=0.05, bias_range=0.1)
        objs.append(ctx.load_object(mesh, cfg, tables=params.tables, mlp=params.packed_mlp()))
    return objs


def _requests(objs, seed, n_req=24):
    """Uneven request sizes (log-uniform 256..65536), a mix of primary rays,
    shadow rays towards a point light (tmax = distance) and random rays."""
    g = np.random.default_rng(seed)
    out = []
    for i in range(n_req):
        n = int(np.exp(g.uniform(np.log(256), np.log(65536))))
        kind = i % 3
        o = objs[g.integers(0, len(objs))]
        if kind == 0:
            cam = I.seeded_camera(int(g.integers(0, 1 << 30)), radius=3.0, width=256, height=256)
            r = I.rays_pinhole(cam)[:, :n]
        elif kind == 1:
            p = g.uniform(-1, 1, (n, 3))
            light = np.array([3.0, 2.0, 4.0])
            d = light - p
            dist = np.linalg.norm(d, axis=1)
            r = I.pack_rays(p, d / dist[:, None], 1e-3, dist)
        else:
            r = I.rays_sphere_to_box(n, 3.0, (-1, -1, -1), (1, 1, 1), seed=int(g.integers(0, 1 << 30)))
        out.append((o, _cuda(np.ascontiguousarray(r))))
    return out


@pytest.mark.parametrize("prec", [lsnif.FP32_PLAIN, lsnif.BF16_FUSED, lsnif.FP16_FUSED])
def test_results_alone_and_in_the_mix_are_identical(prec):
    with lsnif.Context(0) as ctx:
        objs = _objects(ctx)
        reqs = _requests(objs, seed=prec)
        alone = []
        for o, r in reqs:
            alone.append(ctx.query_rays(r, obj=o, precision=prec))
        torch.cuda.synchronize()
        outs, tickets = [], []
        for o, r in reqs:
            res = ctx._alloc_hits(r.shape[1], 0, False)
            outs.append(res)
            tickets.append(ctx.submit(r, res, obj=o, precision=prec))
        lat = []
        for t in tickets:
            st = ctx.poll(t, timeout_us=20_000_000)
            assert st is not None
            lat.append(st.done_us - st.submit_us)
        assert ctx.pending() == 0
        for a, b in zip(alone, outs):
            for f in ("hit", "t", "mat", "normal", "albedo"):
                assert torch.equal(getattr(a, f), getattr(b, f)), f
        print(f"precision {prec}: p50 {np.percentile(lat, 50) / 1e3:.3f} ms, p99 {np.percentile(lat, 99) / 1e3:.3f} ms")


def test_requests_overlap_on_the_device():
    """Requests admitted while others run execute concurrently: the span of
    all requests is shorter than the sum of their device times."""
    with lsnif.Context(0) as ctx:
        objs = _objects(ctx)
        cam = I.seeded_camera(3, radius=3.0, width=512, height=512)
        r = _cuda(I.rays_pinhole(cam))
        for _ in range(2):
            ctx.query_rays(r, obj=objs[0], precision=lsnif.BF16_FUSED)
        torch.cuda.synchronize()
        res = [ctx._alloc_hits(r.shape[1], 0, False) for _ in range(8)]
        tk = [ctx.submit(r, res[i], obj=objs[i % 3], precision=lsnif.BF16_FUSED) for i in range(8)]
        sts = [ctx.poll(t, timeout_us=20_000_000) for t in tk]
        span = max(s.done_us for s in sts) - min(s.start_us for s in sts)
        busy = sum(s.gpu_ms for s in sts) * 1e3
        print(f"span {span:.0f} us, summed device time {busy:.0f} us")
        assert all(s.start_us <= s.done_us for s in sts)
        assert span < busy


def test_poll_semantics_and_bad_tickets():
    with lsnif.Context(0) as ctx:
        objs = _objects(ctx)
        r = _cuda(I.rays_sphere_to_box(1 << 18, 3.0, (-1, -1, -1), (1, 1, 1), seed=5))
        res = ctx._alloc_hits(r.shape[1], 0, False)
        t = ctx.submit(r, res, obj=objs[0], precision=lsnif.FP32_PLAIN)
        t0 = time.perf_counter()
        st = ctx.poll(t, timeout_us=0)          # never blocks
        assert time.perf_counter() - t0 < 0.05
        if st is None:
            st = ctx.poll(t, timeout_us=20_000_000)
        assert st is not None and st.n_rays == r.shape[1]
        with pytest.raises(lsnif.LsnifError) as e:
            ctx.poll(t, timeout_us=0)          # already reported
        assert e.value.code == -2
        with pytest.raises(lsnif.LsnifError) as e:
            ctx.poll(987654, timeout_us=0)
        assert e.value.code == -2


def test_admission_respects_the_memory_budget():
    cfg = I.Config(V=32, H=18, L=8, F=2, log2_T=14, N_min=8, N_max=128, n_hidden=3, width=64, n_mat=2)
    mesh = I.icosphere(3)
    big = _cuda(I.rays_sphere_to_box(1 << 20, 3.0, (-1, -1, -1), (1, 1, 1), seed=6))
    small = _cuda(I.rays_sphere_to_box(1 << 16, 3.0, (-1, -1, -1), (1, 1, 1), seed=7))
    # scratch of one small request ~ 16 MB; budget admits a few at a time
    with lsnif.Context(0, budget_bytes=96 << 20) as ctx:
        h = ctx.load_object(mesh, cfg)
        res = ctx._alloc_hits(big.shape[1], 0, False)
        with pytest.raises(lsnif.LsnifError) as e:
            ctx.submit(big, res, obj=h, precision=lsnif.BF16_FUSED)
        assert e.value.code == -4
        outs = [ctx._alloc_hits(small.shape[1], 0, False) for _ in range(10)]
        tk = [ctx.submit(small, outs[i], obj=h, precision=lsnif.BF16_FUSED) for i in range(10)]
        for t in tk:
            assert ctx.poll(t, timeout_us=20_000_000) is not None
        assert ctx.device_bytes() <= 96 << 20
    with lsnif.Context(0) as free:   # same seeded object, no budget
        ref = free.query_rays(small, obj=free.load_object(mesh, cfg), precision=lsnif.BF16_FUSED)
        for o in outs:
            assert torch.equal(o.t, ref.t)


def test_a_failed_request_is_charged_to_its_own_ticket():
    """One request in a mix names an object handle that was never loaded (a
    failure made on the host and caught by the kernels' own check, with no
    fault): it alone gets LSNIF_ERR_DEVICE_CHECK, and every other request
    still equals its result alone."""
    with lsnif.Context(0) as ctx:
        objs = _objects(ctx)
        reqs = _requests(objs, seed=7, n_req=12)
        alone = [ctx.query_rays(r, obj=o, precision=lsnif.BF16_FUSED) for o, r in reqs]
        torch.cuda.synchronize()
        bad_at = 5
        unknown = max(objs) + 977
        outs, tickets = [], []
        for i, (o, r) in enumerate(reqs):
            res = ctx._alloc_hits(r.shape[1], 0, False)
            outs.append(res)
            if i == bad_at:
                ids = torch.full((r.shape[1],), unknown, dtype=torch.int32, device="cuda")
                ids[::2] = o
                tickets.append(ctx.submit(r, res, obj_per_ray=ids, precision=lsnif.BF16_FUSED))
            else:
                tickets.append(ctx.submit(r, res, obj=o, precision=lsnif.BF16_FUSED))
        for i, t in enumerate(tickets):
            if i == bad_at:
                with pytest.raises(lsnif.LsnifError) as e:
                    ctx.poll(t, timeout_us=20_000_000)
                assert e.value.code == -8, e.value
            else:
                assert ctx.poll(t, timeout_us=20_000_000) is not None
                for f in ("hit", "t", "mat", "normal", "albedo"):
                    assert torch.equal(getattr(alone[i], f), getattr(outs[i], f)), (i, f)
        assert ctx.pending() == 0
        # the context stays usable and the error was not left for later calls
        again = ctx.query_rays(reqs[0][1], obj=reqs[0][0], precision=lsnif.BF16_FUSED)
        ctx.check()
        assert torch.equal(again.t, alone[0].t)


def test_requests_progress_without_polling():
    """Each stream takes up to two requests, the second behind the first in
    stream order: eight equal requests on four streams are all admitted when
    they are submitted, and the device finishes them without any poll in
    between -- the results are complete before the first poll."""
    with lsnif.Context(0) as ctx:
        objs = _objects(ctx)
        r = _cuda(I.rays_sphere_to_box(1 << 16, 3.0, (-1, -1, -1), (1, 1, 1), seed=8))
        alone = ctx.query_rays(r, obj=objs[1], precision=lsnif.BF16_FUSED)
        torch.cuda.synchronize()
        outs = [ctx._alloc_hits(r.shape[1], 0, False) for _ in range(8)]
        tickets = [ctx.submit(r, outs[i], obj=objs[1], precision=lsnif.BF16_FUSED) for i in range(8)]
        t_submitted = time.perf_counter()
        torch.cuda.synchronize()      # the device drains with no call into the queue
        drained = time.perf_counter()
        for o in outs:                # every result is already in place
            assert torch.equal(o.t, alone.t) and torch.equal(o.hit, alone.hit)
        sts = [ctx.poll(t, timeout_us=0) for t in tickets]
        assert all(st is not None for st in sts)
        # each request was admitted inside its own submit call, not at a later poll
        assert all(st.start_us - st.submit_us < 500.0 for st in sts), [st.start_us - st.submit_us for st in sts]
        print(f"8 requests drained {1e3 * (drained - t_submitted):.2f} ms after the last submit")
