"""Benchmark of the LSNIF per-ray query on GB300.

Workload: a seeded 200k-triangle noise-displaced torus (R=1, r=0.35, 4
materials), 128^3 voxels, 16 hash-grid levels x 2 FP16 features, 2^19
entries per level, resolutions 16..2048, MLP 576 -> 64 x 4 -> 12, queried by
2048 x 2048 pinhole primary rays (45 degree FOV, camera on a radius-4
sphere). One step = one query of all 4,194,304 rays.

Prints one JSON line. `value` is the BF16 fused path's whole-job Mrays/s
with rays resident on the device; FP32 plain, p50/p99 step latency, the
end-to-end number through the host-buffer C-ABI call, the roofline of the
dominant kernel and the oracle's CPU throughput are reported beside it.

--impl reference times the FP64 oracle on a bounded sample of the same
workload on the host cores (the paper ships no code to run).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2504_21627_gb300 import inputs as I  # noqa: E402

METRIC = "Mrays/s LSNIF query, BF16 fused vs FP32 plain; p50/p99 batch latency"
WORKLOAD = ("noise torus 200k tris; V=128^3; hash grid L=16 F=2 T=2^19 N=16..2048 (FP16); "
            "MLP 576-64x4-12; 2048x2048 pinhole primary rays")
PROFILE_MD = os.path.join(ROOT, "profiles", "fused_kernel_torus_4m.md")
FUSED_SOURCES = ["paper_2504_21627_gb300/csrc/fused.cu", "paper_2504_21627_gb300/csrc/encode.cuh",
                 "paper_2504_21627_gb300/csrc/device.cuh", "paper_2504_21627_gb300/csrc/tc_common.cuh"]


def fused_source_hash() -> str:
    h = hashlib.sha256()
    for f in FUSED_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_profile(key: str):
    """A figure of the committed ncu summary of the fused kernel (DRAM bytes
    per launch, L2 sectors per gathered point, tensor-pipe activity), or None
    when the kernel sources changed after the capture."""
    if not os.path.exists(PROFILE_MD):
        return None
    txt = open(PROFILE_MD).read()
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_hash") != fused_source_hash():
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload(side: int = 2048, seed_mesh=2, seed_cam=2):
    """side < 2048 keeps the same camera and scene at a lower resolution
    (profiling captures only)."""
    cfg = I.cfg_torus_4m()
    mesh = I.noise_torus(seed=seed_mesh)
    params = I.random_params(cfg, seed=5, table_range=0.05, bias_range=0.1)
    cam = I.seeded_camera(seed_cam, width=side, height=side)
    rays = I.rays_pinhole(cam)
    return cfg, mesh, params, rays


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = os.path.join("/tmp", f"lsnif_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


_ORC = {}


def oracle_rate(cfg, mesh, params, rays, n_sample: int, seed: int = 0, keep: bool = False):
    """The FP64 oracle, as it stands, on a seeded sample of the workload's rays.
    keep: also return the sample, the oracle's results and the box diagonal."""
    from oracle import oracle as O
    if "obj" not in _ORC:
        _ORC["obj"] = O.build_object(mesh, cfg, params)
    orc = _ORC["obj"]
    g = np.random.default_rng(seed)
    idx = np.sort(g.choice(rays.shape[1], n_sample, replace=False))
    sub = np.ascontiguousarray(rays[:, idx])
    t0 = time.perf_counter()
    ref, seg = O.query(orc, sub)
    dt = time.perf_counter() - t0
    cores = O.threads()
    if keep:
        diag = float(np.linalg.norm(orc.bmax.astype(np.float64) - orc.bmin))
        return n_sample / dt / 1e6, cores, dt, (sub, ref, seg, diag)
    return n_sample / dt / 1e6, cores, dt


# the query's acceptance bounds for the half-precision paths (against the FP64
# oracle): visibility mismatch, hit distance (of the box diagonal, 99th
# percentile of the rays both call a hit), material agreement
BOUNDS = {"visibility_mismatch_max": 1e-3, "hit_t_p99_max": 1e-3, "material_min": 0.999}


def precision_errors(ctx, obj, sample, precisions):
    """Each precision's results on the oracle's sample rays against the
    oracle's FP64 results (near-face rays left out), and whether the bounds
    hold."""
    import torch
    sub, ref, seg, diag = sample
    rays = torch.from_numpy(sub).cuda()
    ok = ~seg.near
    out = {}
    for name, prec in precisions:
        q = ctx.query_rays(rays, obj=obj, precision=prec)
        ctx.check()
        hit = q.hit.cpu().numpy().astype(bool)
        t = q.t.cpu().numpy().astype(np.float64)
        mat = q.mat.cpu().numpy()
        both = ok & hit & ref.hit
        dt = np.abs(t[both] - ref.t[both]) / diag
        e = {"visibility_mismatch": float((hit[ok] != ref.hit[ok]).mean()),
             "hit_t_p50": float(np.median(dt)) if both.any() else None,
             "hit_t_p99": float(np.quantile(dt, 0.99)) if both.any() else None,
             "material": float((mat[both] == ref.mat[both]).mean()) if both.any() else None,
             "rays": int(ok.sum()), "hits": int(both.sum()), "near_face_left_out": int(seg.near.sum())}
        e["meets_bounds"] = bool(both.any() and e["visibility_mismatch"] <= BOUNDS["visibility_mismatch_max"]
                                 and e["hit_t_p99"] <= BOUNDS["hit_t_p99_max"]
                                 and e["material"] >= BOUNDS["material_min"])
        out[name] = e
    return out


def train_object(ctx, obj, steps: int, batch: int, n_pool: int, seed: int):
    """Train an object from its seeded initialisation on GPU-generated
    balanced rays and ray-cast labels (Sec. 5.2): Adam, lr 0.01."""
    import torch
    from paper_2504_21627_gb300 import lsnif
    t0 = time.perf_counter()
    u = torch.rand((n_pool, lsnif.TRAIN_UNIFORMS), device="cuda", generator=torch.Generator("cuda").manual_seed(seed))
    pool, _ = ctx.make_training_rays(obj, u, n_outside=n_pool // 2)
    lab = ctx.label_rays(pool, obj)
    keep = lab["k"] > 0
    pool = pool[:, keep].contiguous()
    lab = {k: v[keep].contiguous() for k, v in lab.items()}
    gen = torch.Generator("cuda").manual_seed(seed + 1)
    losses = []
    for s in range(steps):
        idx = torch.randint(0, pool.shape[1], (batch,), device="cuda", generator=gen)
        st = ctx.train_step(pool[:, idx].contiguous(), {k: v[idx].contiguous() for k, v in lab.items()}, obj,
                            lr=0.01, stats=(s == 0 or s == steps - 1))
        if st is not None:
            losses.append(st.total)
    torch.cuda.synchronize()
    return {"steps": steps, "batch": batch, "pool_rays": int(pool.shape[1]), "loss_first": losses[0],
            "loss_last": losses[-1], "seconds": time.perf_counter() - t0}


def corner_loads(ctx, obj, rays, cfg, res):
    """Corner loads the fused kernel's default gather issues for these rays:
    per gathered point and level one 8-byte load per (y, z) row of the cell
    (the aligned pair that holds corner x0, and x1 when the cell's x index is
    even), plus a 4-byte load per row for x1 when the x index is odd and the
    x weight is not 0. Points shared with the previous segment's exit are
    copied, not gathered. Counted from the traversal's own points."""
    import torch
    k, _, pts, _ = ctx.trace(rays, obj)
    H = cfg.H
    slot = torch.arange(H, device=pts.device)[None, :] < 2 * k[:, None].long()
    shared = torch.zeros_like(slot)
    shared[:, 2::2] = (pts[:, 2::2, :] == pts[:, 1:-1:2, :]).all(-1)
    x = pts[slot & ~shared][:, 0]
    del pts
    loads = 0
    for N in res:
        xs = x * float(N)
        cx = torch.floor(xs)
        odd = ((cx.to(torch.int64) & 1) == 1) & (xs != cx)
        loads += 4 * (x.numel() + int(odd.sum()))
    return loads, int(x.numel())


def oracle_rate_single_thread(cfg, mesh, params, rays, n_sample: int, seed: int = 1):
    """oracle_rate with the oracle's loops on one host thread."""
    from oracle import oracle as O
    before = O.threads(1)
    try:
        rate, _, dt = oracle_rate(cfg, mesh, params, rays, n_sample, seed)
    finally:
        O.threads(before)
    return rate, dt


def run_reference(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg, mesh, params, rays = workload()
    per_step = args.ref_sample
    times = []
    for s in range(args.warmup + args.steps):
        rate, cores, dt = oracle_rate(cfg, mesh, params, rays, per_step, seed=1000 + s)
        if s >= args.warmup:
            times.append(dt)
    ms = float(np.mean(times)) * 1e3
    value = per_step / (ms / 1e3) / 1e6
    sample = f"{per_step} seeded rays of the 2048x2048 workload per step (full oracle: traversal, encoding, MLP)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rays_per_step": per_step, "parallelism": "host cores (OpenMP)"},
        "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    del torch


# ---------------------------------------------------------------------------
# other workloads (not the headline line): many objects in one launch,
# serving, training
# ---------------------------------------------------------------------------

def _timed_graph(ctx, torch, rays, handles, precision, steps, warmup, stream, flush):
    out = ctx._alloc_hits(rays.shape[1], 0, False)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            ctx.query_rays(rays, obj_per_ray=handles, precision=precision, out=out, stream=stream)
        for s in range(steps):
            flush.zero_()
            evs[s][0].record(stream)
            ctx.query_rays(rays, obj_per_ray=handles, precision=precision, out=out, stream=stream)
            evs[s][1].record(stream)
    stream.synchronize()
    ctx.check(stream)
    return np.array([a.elapsed_time(b) for a, b in evs])


def bench_batched(args):
    print(json.dumps(batched_run(args.steps, args.warmup, 16 << 20)))


def batched_run(steps: int, warmup: int, total_rays: int):
    """64 objects (5k..500k triangles, V 64..256, T 2^16..2^20, 4 x 64 BF16
    network), power-law rays per object, about total_rays shuffled together,
    queried by one grouped launch sequence replayed as a CUDA graph."""
    import torch
    from paper_2504_21627_gb300 import lsnif
    t_setup = time.perf_counter()
    spec = I.batched_objects(total_rays=total_rays)
    ctx = lsnif.Context(0)
    rays_l, hand_l = [], []
    for i, (mesh, cfg, n) in enumerate(spec):
        p = I.random_params(cfg, seed=1000 + i, table_range=0.05, bias_range=0.1)
        h = ctx.load_object(mesh, cfg, tables=p.tables, mlp=p.packed_mlp())
        lo, hi = mesh.verts.min(0), mesh.verts.max(0)
        rays_l.append(I.rays_sphere_to_box(n, 3.0, lo, hi, seed=2000 + i))
        hand_l.append(np.full(n, h, np.uint32))
    perm = I.rng(7).permutation(sum(r.shape[1] for r in rays_l))
    rays = torch.from_numpy(np.ascontiguousarray(np.concatenate(rays_l, 1)[:, perm])).cuda()
    handles = torch.from_numpy(np.concatenate(hand_l)[perm].view(np.int32)).cuda()
    n = rays.shape[1]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    variant = ctx.autotune(rays, obj_per_ray=handles, reps=2)
    ctx.set_profiling(True)
    ctx.query_rays(rays, obj_per_ray=handles, precision=lsnif.BF16_FUSED)
    prof = ctx.last_profile()
    ctx.set_profiling(False)
    ctx.set_graph_mode(True)
    t_setup = time.perf_counter() - t_setup
    ms16 = _timed_graph(ctx, torch, rays, handles, lsnif.BF16_FUSED, steps, warmup, stream, flush)
    ms32 = _timed_graph(ctx, torch, rays, handles, lsnif.FP32_PLAIN, max(3, steps // 2), 3, stream, flush)
    out = {
        "workload": "batched", "metric": "Mrays/s, 64 objects in one grouped launch sequence (CUDA graph)",
        "objects": len(spec), "rays_per_step": n, "value": n / (ms16.mean() / 1e3) / 1e6, "unit": "Mrays/s",
        "value_fp32": n / (ms32.mean() / 1e3) / 1e6, "ms_bf16": float(ms16.mean()), "ms_fp32": float(ms32.mean()),
        "p50_ms_bf16": float(np.percentile(ms16, 50)), "p99_ms_bf16": float(np.percentile(ms16, 99)),
        "live_frac": prof.n_live / n, "mean_points_per_live_ray": prof.n_points / max(prof.n_live, 1),
        "fused_variant": lsnif.Context.variants()[variant], "trace_mode": ctx.tuning()[1],
        "group_mode": ctx.tuning()[2],
        "device_gb": ctx.device_bytes() / 1e9,
        "l2": "flushed before every timed step", "graph": True, "setup_s": t_setup}
    ctx.close()
    return out


def _serving_requests(ctx, torch, objs, n_req, seed):
    """Uneven requests: 40% primary pinhole, 30% shadow rays to a point light
    (tmax = distance), 30% cosine bounce rays from surface hit points; sizes
    log-uniform in [256, 262144]."""
    from paper_2504_21627_gb300 import lsnif
    g = I.rng(seed)
    reqs = []
    for i in range(n_req):
        n = int(math.exp(g.uniform(math.log(256), math.log(262144))))
        h, mesh = objs[int(g.integers(0, len(objs)))]
        lo, hi = mesh.verts.min(0).astype(np.float64), mesh.verts.max(0).astype(np.float64)
        c, rad = 0.5 * (lo + hi), 0.5 * np.linalg.norm(hi - lo)
        u = g.random()
        side = int(math.ceil(math.sqrt(n)))
        cam = I.seeded_camera(int(g.integers(0, 1 << 30)), radius=2.5 * rad, width=side, height=side)
        cam.eye = cam.eye + c
        prim = I.rays_pinhole(cam)[:, :n]
        if u < 0.4:
            r = prim
        else:
            pr = torch.from_numpy(np.ascontiguousarray(prim)).cuda()
            lab = ctx.label_rays(pr, h)
            hit = lab["tri"].cpu().numpy() >= 0
            th = lab["t_hit"].cpu().numpy()
            nrm = lab["normal"].cpu().numpy().astype(np.float64)
            o = prim[0:3].T.astype(np.float64)
            d = prim[3:6].T.astype(np.float64)
            p = np.where(hit[:, None], o + np.nan_to_num(th, posinf=0)[:, None] * d, g.uniform(lo, hi, (n, 3)))
            nrm = np.where(hit[:, None], nrm, np.array([0.0, 0.0, 1.0]))
            nrm *= -np.sign(np.sum(nrm * d, 1, keepdims=True) + 1e-30)      # face the incoming ray
            p = p + 1e-4 * rad * nrm
            if u < 0.7:   # shadow rays
                light = c + np.array([3.0, 2.0, 4.0]) * rad
                dl = light - p
                dist = np.linalg.norm(dl, axis=1)
                r = I.pack_rays(p, dl / dist[:, None], 0.0, dist)
            else:         # cosine bounce rays about the facing normal
                uu = g.random((n, 2))
                rr, ph = np.sqrt(uu[:, 0]), 2 * np.pi * uu[:, 1]
                sgn = np.where(nrm[:, 2] >= 0, 1.0, -1.0)
                a = -1.0 / (sgn + nrm[:, 2])
                bb = nrm[:, 0] * nrm[:, 1] * a
                t = np.stack([1 + sgn * nrm[:, 0] ** 2 * a, sgn * bb, -sgn * nrm[:, 0]], 1)
                b = np.stack([bb, sgn + nrm[:, 1] ** 2 * a, -nrm[:, 1]], 1)
                dd = (rr * np.cos(ph))[:, None] * t + (rr * np.sin(ph))[:, None] * b + \
                    np.sqrt(1 - uu[:, 0])[:, None] * nrm
                r = I.pack_rays(p, dd)
        rt = torch.from_numpy(np.ascontiguousarray(r)).cuda()
        reqs.append((h, rt, ctx._alloc_hits(n, 0, False)))
    del lsnif
    return reqs


def _serve(ctx, reqs, precision, rate_rps, seed):
    """Open loop (Poisson arrivals at rate_rps) or closed loop (rate None):
    returns per-request latency (us) and throughput (Mrays/s)."""
    g = I.rng(seed)
    t_start = time.perf_counter()
    arrivals = np.cumsum(g.exponential(1.0 / rate_rps, len(reqs))) if rate_rps else np.zeros(len(reqs))
    pending, lat, done_rays = {}, [], 0
    i = 0
    while i < len(reqs) or pending:
        now = time.perf_counter() - t_start
        while i < len(reqs) and arrivals[i] <= now:
            h, r, out = reqs[i]
            pending[ctx.submit(r, out, obj=h, precision=precision)] = r.shape[1]
            i += 1
        for tk in list(pending):
            st = ctx.poll(tk, timeout_us=0)
            if st is not None:
                lat.append(st.done_us - st.submit_us)
                done_rays += pending.pop(tk)
    wall = time.perf_counter() - t_start
    return np.array(lat), done_rays / wall / 1e6, wall


def bench_serving(args):
    print(json.dumps(serving_run(args.requests)))


def serving_run(n_requests: int):
    """16 resident objects, requests of uneven size and kind, admission under
    an 8 GB budget; p50/p99 latency at 0.5x and 0.9x of the saturation rate."""
    import torch
    from paper_2504_21627_gb300 import lsnif
    t_setup = time.perf_counter()
    spec = I.batched_objects()[:16]
    ctx = lsnif.Context(0, budget_bytes=8 << 30)
    objs = []
    for i, (mesh, cfg, _) in enumerate(spec):
        p = I.random_params(cfg, seed=1000 + i, table_range=0.05, bias_range=0.1)
        objs.append((ctx.load_object(mesh, cfg, tables=p.tables, mlp=p.packed_mlp(), keep_mesh=True), mesh))
    reqs = _serving_requests(ctx, torch, objs, n_requests, seed=11)
    torch.cuda.synchronize()
    res = {"workload": "serving", "metric": "request latency (submit -> done) and Mrays/s, 16 resident objects",
           "requests": len(reqs), "rays": int(sum(r[1].shape[1] for r in reqs)), "budget_gb": 8,
           "setup_s": time.perf_counter() - t_setup}
    for name, prec in (("bf16", lsnif.BF16_FUSED), ("fp32", lsnif.FP32_PLAIN)):
        _serve(ctx, reqs[:8], prec, None, 0)                      # warm the streams
        lat, thr, wall = _serve(ctx, reqs, prec, None, 1)          # saturation (closed loop)
        sat_rps = len(reqs) / wall
        res[name] = {"saturation_mrays_s": thr, "saturation_req_s": sat_rps}
        for frac in (0.5, 0.9):
            lat, thr, _ = _serve(ctx, reqs, prec, frac * sat_rps, 2)
            res[name][f"at_{frac}x"] = {"p50_ms": float(np.percentile(lat, 50)) / 1e3,
                                        "p99_ms": float(np.percentile(lat, 99)) / 1e3, "mrays_s": thr}
    res["device_gb"] = ctx.device_bytes() / 1e9
    # the serving path's headline: BF16 at 0.9x of its saturation rate
    res["p50_ms"] = res["bf16"]["at_0.9x"]["p50_ms"]
    res["p99_ms"] = res["bf16"]["at_0.9x"]["p99_ms"]
    ctx.close()
    return res


def bench_train(args):
    """Training step throughput at the paper's batch of 2^18 rays (the paper
    trains 2000 steps in about 15 s on its GPU) for the icosphere and torus
    objects, from GPU-generated balanced rays and labels."""
    import torch
    from paper_2504_21627_gb300 import lsnif
    out = {"workload": "train", "metric": "training steps/s at batch 2^18 (forward, loss, backward, Adam); "
                                          "network products on the tensor cores and, for reference, FP32 SIMT"}
    objects = (("icosphere", I.cfg_icosphere_small(), I.icosphere(3)),
               ("torus", I.cfg_torus_4m(), I.noise_torus(seed=2)))
    if args.profile_step:   # profiling captures: the torus only, one step in a profiler range
        objects = objects[1:]
    for name, cfg, mesh in objects:
        ctx = lsnif.Context(0)
        h = ctx.load_object(mesh, cfg, keep_mesh=True)
        n_pool, B = 1 << 22, 1 << 18
        u = torch.rand((n_pool, lsnif.TRAIN_UNIFORMS), device="cuda", generator=torch.Generator("cuda").manual_seed(1))
        t0 = time.perf_counter()
        pool, _ = ctx.make_training_rays(h, u, n_outside=n_pool // 2)
        lab = ctx.label_rays(pool, h)
        torch.cuda.synchronize()
        t_data = time.perf_counter() - t0
        keep = lab["k"] > 0
        pool = pool[:, keep].contiguous()
        lab = {k: v[keep].contiguous() for k, v in lab.items()}
        gen = torch.Generator("cuda").manual_seed(2)
        batches = []
        for _ in range(8):
            idx = torch.randint(0, pool.shape[1], (B,), device="cuda", generator=gen)
            batches.append((pool[:, idx].contiguous(), {k: v[idx].contiguous() for k, v in lab.items()}))
        first = ctx.train_step(*batches[0], h).total
        if args.profile_step:
            for s in range(3):
                ctx.train_step(*batches[s % 8], h, stats=False)
            torch.cuda.synchronize()
            torch.cuda.cudart().cudaProfilerStart()
            ctx.train_step(*batches[3], h, stats=False)
            torch.cuda.synchronize()
            torch.cuda.cudart().cudaProfilerStop()
            print(json.dumps({"profile_step": "torus training step", "batch": B}))
            ctx.close()
            return
        out[name] = {"data_generation_s": t_data, "pool_rays": int(pool.shape[1]), "loss_first": first}
        steps = max(20, args.steps)
        for label, products in (("tensor_cores", lsnif.TRAIN_TENSOR_CORES), ("fp32_simt", lsnif.TRAIN_FP32_SIMT)):
            for s in range(3):
                ctx.train_step(*batches[s % 8], h, stats=False, products=products)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for s in range(steps):
                ctx.train_step(*batches[s % 8], h, stats=False, products=products)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            out[name][label] = {"steps_per_s": steps / dt, "ms_per_step": dt / steps * 1e3,
                                "seconds_for_2000_steps": 2000 * dt / steps}
        out[name]["loss_after"] = ctx.train_step(*batches[0], h).total
        ctx.close()
    print(json.dumps(out))


def bench_sweep(args):
    """Parameter and quality sweeps (Sec. 6.1 parameter study; Table 1 low /
    high quality) on a synthetic mesh: each configuration is trained on the
    GPU from its seeded initialisation (balanced rays, labels by ray casting,
    2000 steps of batch 2^14 unless swept) and evaluated on held-out rays
    against the exact answers of the same mesh kept as a mesh object (BVH):
    visibility accuracy, hit-distance error (median and 90th percentile, in
    units of the box diagonal), normal angle (median, degrees) and material
    accuracy. Memory from the storage model (bits + FP16 tables + FP16
    network). Geometric error stands in for the paper's FLIP image error."""
    import torch
    from paper_2504_21627_gb300 import lsnif
    mesh = I.noise_torus_tris(11, 50000, amplitude=0.08, n_mat=4)
    base = dict(V=32, H=18, L=2, F=4, log2_T=17, N_min=64, N_max=128, n_hidden=2, width=128, n_mat=4)
    runs = [("base (paper's V 32, H 18, T 2^17, 2 x 128)", {}, 2000)]
    runs += [(f"V {v}", {"V": v}, 2000) for v in (8, 16, 64)]
    runs += [(f"H {h}", {"H": h}, 2000) for h in (6, 10, 26)]
    runs += [(f"T 2^{t}", {"log2_T": t}, 2000) for t in (11, 13, 15, 19)]
    runs += [(f"{st} training steps", {}, st) for st in (100, 700)]
    runs += [("low quality (width 64, H 10)", {"width": 64, "H": 10}, 2000)]
    if args.steps < 20:   # a shortened sweep for smoke runs
        runs = runs[:2]
    ctx = lsnif.Context(0)
    hm = ctx.load_mesh(mesh)
    lo, hi = mesh.verts.min(0), mesh.verts.max(0)
    diag = float(np.linalg.norm(hi.astype(np.float64) - lo))
    test = torch.from_numpy(I.rays_sphere_to_box(200000, 2.5 * diag / 2, lo, hi, seed=77)).cuda()
    ref = ctx.query_rays(test, obj=hm, precision=lsnif.FP32_PLAIN)
    torch.cuda.synchronize()
    r_hit = ref.hit.bool()
    rows = []
    for name, over, steps in runs:
        c = dict(base, **over)
        cfg = I.Config(**c)
        h = ctx.load_object(mesh, cfg, keep_mesh=True)
        n_pool, B = 1 << 20, 1 << 14
        u = torch.rand((n_pool, lsnif.TRAIN_UNIFORMS), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
        pool, _ = ctx.make_training_rays(h, u, n_outside=n_pool // 2)
        lab = ctx.label_rays(pool, h)
        keep = lab["k"] > 0
        pool = pool[:, keep].contiguous()
        lab = {k: v[keep].contiguous() for k, v in lab.items()}
        gen = torch.Generator("cuda").manual_seed(5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(steps):
            idx = torch.randint(0, pool.shape[1], (B,), device="cuda", generator=gen)
            ctx.train_step(pool[:, idx].contiguous(), {k: v[idx].contiguous() for k, v in lab.items()}, h,
                           lr=0.01, stats=False)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        q = ctx.query_rays(test, obj=h, precision=lsnif.FP32_PLAIN)
        torch.cuda.synchronize()
        q_hit = q.hit.bool()
        both = q_hit & r_hit
        terr = ((q.t - ref.t).abs()[both] / diag).cpu().numpy()
        cosang = (q.normal[:, both] * ref.normal[:, both]).sum(0).clamp(-1, 1).cpu().numpy()
        info = ctx.object_info(h)
        rows.append({"run": name, "V": c["V"], "H": c["H"], "log2_T": c["log2_T"], "width": c["width"],
                     "train_steps": steps, "train_s": t_train,
                     "visibility_acc": float((q_hit == r_hit).float().mean().item()),
                     "t_err_p50": float(np.median(terr)), "t_err_p90": float(np.quantile(terr, 0.9)),
                     "normal_deg_p50": float(np.degrees(np.median(np.arccos(cosang)))),
                     "material_acc": float((q.mat[both] == ref.mat[both]).float().mean().item()),
                     "memory_fp16_kb": info.footprint_fp16_bytes / 1024})
        ctx.unload_object(h)
    out = {"workload": "sweep", "mesh_triangles": int(mesh.tris.shape[0]), "test_rays": int(test.shape[1]),
           "reference_hits": int(r_hit.sum().item()), "base": base, "rows": rows}
    print(json.dumps(out))
    ctx.close()


def bench_stress1(args):
    """One object of the stress scene's network shape (L 16, F 4, T 2^21,
    1152-128x4-12) on the torus workload's mesh and camera: FP16 fused
    (streamed weights), FP8 fused and FP32 plain queries of side x side
    primary rays, with their stage times. A single-object case of the stress network, small enough
    for full profiler captures at side 1024."""
    import torch
    from paper_2504_21627_gb300 import lsnif
    cfg = I.cfg_stress_object()
    mesh = I.noise_torus(seed=2)
    params = I.random_params(cfg, seed=5, table_range=0.05, bias_range=0.1)
    rays = torch.from_numpy(I.rays_pinhole(I.seeded_camera(2, width=args.side, height=args.side))).cuda()
    n = rays.shape[1]
    ctx = lsnif.Context(0)
    obj = ctx.load_object(mesh, cfg, tables=params.tables, mlp=params.packed_mlp())
    if args.variant8 is not None:
        ctx.set_variant8(args.variant8)
    if args.group_mode is not None:
        ctx.set_group_mode(args.group_mode)
    if args.trace_mode is not None:
        ctx.set_trace_mode(args.trace_mode)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    out = {"workload": "stress1", "network": "L=16 F=4 T=2^21, 1152-128x4-12", "rays": n,
           "trace_mode": ctx.tuning()[1], "group_mode": ctx.tuning()[2]}
    for name, prec, steps in (("fp16", lsnif.FP16_FUSED, args.steps), ("fp8", lsnif.FP8_FUSED, args.steps),
                              ("fp32", lsnif.FP32_PLAIN, 3)):
        res = ctx.query_rays(rays, obj=obj, precision=prec)
        for _ in range(args.warmup):
            ctx.query_rays(rays, obj=obj, precision=prec, out=res)
        ctx.set_profiling(True)
        ms, prof = [], []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.query_rays(rays, obj=obj, precision=prec, out=res)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            prof.append(ctx.last_profile())
        ctx.set_profiling(False)
        ctx.check()
        p = prof[-1]
        out[name] = {"mrays_s": n / (np.mean(ms) / 1e3) / 1e6, "ms_per_step": float(np.mean(ms)),
                     "stages_ms": {"trace": float(np.mean([q.ms_trace for q in prof])),
                                   "group": float(np.mean([q.ms_group for q in prof])),
                                   "network": float(np.mean([q.ms_mlp for q in prof]))},
                     "live": int(p.n_live), "points": int(p.n_points)}
    print(json.dumps(out))
    ctx.close()


def _scene_raster(args, ctx, spec, handles, insts, stress):
    """The paper's hybrid frame (Sec. 4, Fig. 4): primary visibility by
    rasterising the meshes into a G-buffer (lsnif_raster_gbuffer; spp
    samples per pixel as a sqrt(spp)-times supersampled G-buffer), first
    bounce rays from the G-buffer, then 2 bounces of LSNIF queries."""
    import torch
    from paper_2504_21627_gb300 import lsnif
    s = int(round(math.sqrt(args.scene_spp)))
    W, H = args.scene_width * s, args.scene_height * s
    cam = I.seeded_camera(4, radius=14.0, width=W, height=H, fov_deg=50.0)
    tan = math.tan(math.radians(cam.fov_deg) / 2.0)
    prim = torch.from_numpy(I.rays_pinhole(cam)).cuda()
    n = prim.shape[1]
    gen = torch.Generator("cuda").manual_seed(11)
    us = [torch.rand((n, 2), device="cuda", generator=gen) for _ in range(3)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    gbuf = ctx.raster_gbuffer(cam.eye, cam.forward, cam.right, cam.up, tan, W, H, insts)

    def raster():
        return ctx.raster_gbuffer(cam.eye, cam.forward, cam.right, cam.up, tan, W, H, insts, out=gbuf)

    def frame(prec, stats=None):
        g = raster()
        res = lsnif.QueryResult(g.hit.view(-1), g.dist.view(-1), g.normal.view(3, -1), None, None, None)
        if stats is not None:
            stats.append((int(g.hit.sum().item()), n))
        rays = ctx.bounce_rays(prim, res, us[0], 1e-3)
        for b in range(2):
            res, _ = ctx.query_scene(rays, insts, precision=prec)
            if stats is not None:
                stats.append((int(res.hit.sum().item()), int((rays[3:6].abs().sum(0) > 0).sum().item())))
            if b < 1:
                rays = ctx.bounce_rays(rays, res, us[b + 1], 1e-3)
        return res

    def timed(fn, steps):
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return np.array(ms)

    nt_of = {h: int(spec[i][0].nt) for i, h in enumerate(handles)}
    n_tri = sum(nt_of[h] for h, _, _ in insts)
    for _ in range(3):
        raster()
    ms_r = timed(raster, max(5, args.steps))
    out = {"workload": "scene-raster", "metric": "hybrid frame: raster G-buffer + 2 LSNIF bounces",
           "instances": len(insts), "unique_objects": len(spec), "gbuffer": [W, H], "triangles": n_tri,
           "network": "L=16 F=4 T=2^21, 1152-128x4-12" if stress else "L=16 F=2 T=2^21, 576-64x4-12",
           "raster": {"ms": float(ms_r.mean()), "mpixels_s": W * H / (ms_r.mean() / 1e3) / 1e6,
                      "gtris_s": n_tri / (ms_r.mean() / 1e3) / 1e9}}
    prec, name = (lsnif.FP8_FUSED, "fp8") if stress else (lsnif.BF16_FUSED, "bf16")
    stats = []
    frame(prec, stats)
    for _ in range(2):
        frame(prec)
    ms = timed(lambda: frame(prec), max(3, args.steps // 4))
    out[name] = {"ms_per_frame": float(ms.mean()), "lsnif_mrays_s": 2 * n / ((ms.mean() - ms_r.mean()) / 1e3) / 1e6,
                 "hits": [h for h, _ in stats], "live_rays": [l for _, l in stats]}
    out["device_gb"] = ctx.device_bytes() / 1e9
    print(json.dumps(out))
    ctx.close()


def bench_mesh1(args):
    """The torus workload's mesh (200k triangles) kept as a mesh object --
    triangles and a BVH, the hybrid pipeline's non-LSNIF objects (Sec. 4) --
    queried with the same 2048 x 2048 primary rays: exact nearest hits by
    BVH traversal, beside the LSNIF query of the same mesh."""
    import torch
    from paper_2504_21627_gb300 import lsnif
    cfg, mesh, params, rays_np = workload(args.side)
    n = rays_np.shape[1]
    ctx = lsnif.Context(0)
    hm = ctx.load_mesh(mesh)
    hl = ctx.load_object(mesh, cfg, tables=params.tables, mlp=params.packed_mlp())
    rays = torch.from_numpy(rays_np).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    out = {"workload": "mesh1", "triangles": int(mesh.tris.shape[0]), "rays": n}
    for name, h, prec in (("bvh", hm, lsnif.FP32_PLAIN), ("lsnif_bf16", hl, lsnif.BF16_FUSED)):
        res = ctx.query_rays(rays, obj=h, precision=prec)
        for _ in range(args.warmup):
            ctx.query_rays(rays, obj=h, precision=prec, out=res)
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.query_rays(rays, obj=h, precision=prec, out=res)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        ctx.check()
        info = ctx.object_info(h)
        out[name] = {"mrays_s": n / (np.mean(ms) / 1e3) / 1e6, "ms_per_step": float(np.mean(ms)),
                     "hits": int(res.hit.sum().item()), "device_mb": info.device_bytes / 2 ** 20}
        if name == "bvh":
            out[name]["bvh_nodes"] = int(info.bvh_nodes)
    print(json.dumps(out))
    ctx.close()


def bench_scene(args):
    """Path-tracer-shaped stress: 32 instances of 8 unique objects (50k..1M
    triangles, V 128, L 16, F 4, T 2^21, 4 x 128 network; `--scene-net
    small` takes F 2 and 4 x 64 instead) with seeded rigid transforms and
    scales, 1920 x 1080 x 4 jittered primary rays, 3 bounces: each bounce is
    one lsnif_query_scene (broad phase over the instances' boxes, pairs
    grouped by object, nearest hit) and one lsnif_bounce_rays. Mrays/s
    counts every submitted ray (dead rays included), as the query's own
    metric does. The F 4, 4 x 128 network runs on the FP16 path (the
    streamed-weights kernel: its weights do not fit shared memory; the
    accepted half-precision path of this shape), the FP8 path and the FP32
    path."""
    import torch
    from paper_2504_21627_gb300 import lsnif
    stress = args.scene_net == "stress"
    spec = I.scene_objects(features=4, width=128) if stress else I.scene_objects()
    spec = spec[:args.scene_objects]
    ctx = lsnif.Context(0)
    handles = []
    for i, (mesh, cfg) in enumerate(spec):
        p = I.random_params(cfg, seed=3000 + i, table_range=0.05, bias_range=0.1)
        p.weights[-1][1][0] = 1.0   # occupancy logit biased towards hits, so bounces continue
        handles.append(ctx.load_object(mesh, cfg, tables=p.tables, mlp=p.packed_mlp(),
                                       keep_mesh=args.primary == "raster", bvh_below_faces=args.bvh_below_faces))
    if args.variant8 is not None:
        ctx.set_variant8(args.variant8)
    # bounce rays arrive in no spatial order and pairs mix 8 objects: the
    # presorted traversal and the spatial grouping (62.5 against 74 ms per
    # FP16 frame with the in-order kernels)
    ctx.set_group_mode(2 if args.group_mode is None else args.group_mode)
    ctx.set_trace_mode(2 if args.trace_mode is None else args.trace_mode)
    insts = [(handles[o], A, b) for o, A, b in I.seeded_instances(args.scene_instances, len(spec), seed=9,
                                                                   spread=10.0)]
    if args.primary == "raster":
        return _scene_raster(args, ctx, spec, handles, insts, stress)
    cam = I.seeded_camera(4, radius=14.0, width=args.scene_width, height=args.scene_height, fov_deg=50.0)
    rays0 = torch.from_numpy(I.camera_rays_spp(cam, args.scene_spp, seed=10)).cuda()
    n = rays0.shape[1]
    gen = torch.Generator("cuda").manual_seed(11)
    us = [torch.rand((n, 2), device="cuda", generator=gen) for _ in range(3)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def frame(prec, stats=None):
        rays = rays0
        for b in range(3):
            res, inst = ctx.query_scene(rays, insts, precision=prec)
            if stats is not None:
                stats.append((int(res.hit.sum().item()), int((rays[3:6].abs().sum(0) > 0).sum().item())))
            if b < 2:
                rays = ctx.bounce_rays(rays, res, us[b], 1e-3)
        return res

    out = {"workload": "scene", "metric": "Mrays/s over 3 bounces of an instanced scene (misses included)",
           "instances": len(insts), "unique_objects": len(spec), "rays_per_bounce": n,
           "mesh_objects": int(sum(ctx.object_info(h).kind == 1 for h in handles)),
           "trace_mode": ctx.tuning()[1], "group_mode": ctx.tuning()[2],
           "network": "L=16 F=4 T=2^21, 1152-128x4-12" if stress else "L=16 F=2 T=2^21, 576-64x4-12"}
    fast = (("fp16", lsnif.FP16_FUSED, max(3, args.steps // 4)), ("fp8", lsnif.FP8_FUSED, max(3, args.steps // 4))) \
        if stress else \
        (("bf16", lsnif.BF16_FUSED, max(3, args.steps // 4)), ("fp8", lsnif.FP8_FUSED, max(3, args.steps // 4)))
    for name, prec, steps in fast + (("fp32", lsnif.FP32_PLAIN, 2),):
        stats = []
        frame(prec, stats)
        for _ in range(2):
            frame(prec)
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            frame(prec)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        ms = np.array(ms)
        out[name] = {"mrays_s": 3 * n / (ms.mean() / 1e3) / 1e6, "ms_per_frame": float(ms.mean()),
                     "hits_per_bounce": [h for h, _ in stats], "live_rays_per_bounce": [l for _, l in stats]}
    out["device_gb"] = ctx.device_bytes() / 1e9
    print(json.dumps(out))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--ref-sample", type=int, default=2048)
    ap.add_argument("--cpu-sample", type=int, default=65536)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", type=int, default=None,
                    help="fused-kernel variant to time instead of the autotuner's choice")
    ap.add_argument("--side", type=int, default=2048, help="image side; below 2048 only for profiling captures")
    ap.add_argument("--workload", default="torus4m", choices=["torus4m", "batched", "serving", "train", "scene", "stress1", "mesh1", "sweep"],
                    help="torus4m is the headline; the others print their own line")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--no-train", action="store_true",
                    help="time random-init weights (profiling captures: no training kernels before the query)")
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--no-extras", action="store_true", help="leave the serving and batched entries out")
    ap.add_argument("--profile-step", action="store_true",
                    help="profiling captures: run one BF16 query step inside cudaProfilerStart/Stop and exit")
    ap.add_argument("--serving-requests", type=int, default=60)
    ap.add_argument("--batched-rays", type=int, default=4 << 20)
    ap.add_argument("--scene-width", type=int, default=1920)
    ap.add_argument("--scene-height", type=int, default=1080)
    ap.add_argument("--scene-net", default="stress", choices=["stress", "small"])
    ap.add_argument("--variant8", type=int, default=None, help="FP8 fused-kernel variant for --workload scene")
    ap.add_argument("--group-mode", type=int, default=None,
                    help="stress1 / scene: live rays grouped by (object, point count) (0), kept in ray order (1) "
                         "or sorted by the cell of their first point (2; the scene's default)")
    ap.add_argument("--trace-mode", type=int, default=None,
                    help="stress1 / scene: traversal in ray order (1) or over rays presorted by entry cell (2; the scene's "
                         "default)")
    ap.add_argument("--scene-objects", type=int, default=8, help="unique objects (below 8 only for profiling)")
    ap.add_argument("--scene-instances", type=int, default=32)
    ap.add_argument("--scene-spp", type=int, default=4)
    ap.add_argument("--bvh-below-faces", type=int, default=0,
                    help="scene workload: objects with fewer triangles stay mesh objects (BVH), Sec. 4")
    ap.add_argument("--primary", default="lsnif", choices=["lsnif", "raster"],
                    help="scene workload: primary rays by LSNIF, or by the rasterised G-buffer (Sec. 4)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return bench_batched(args)
    if args.workload == "serving":
        return bench_serving(args)
    if args.workload == "train":
        return bench_train(args)
    if args.workload == "scene":
        return bench_scene(args)
    if args.workload == "stress1":
        return bench_stress1(args)
    if args.workload == "mesh1":
        return bench_mesh1(args)
    if args.workload == "sweep":
        return bench_sweep(args)

    import torch
    import torch.distributed as dist
    from paper_2504_21627_gb300 import lsnif

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    cfg, mesh, params, rays_np = workload(args.side)
    n = rays_np.shape[1]
    ctx = lsnif.Context(local)
    train_info = None
    if args.no_train:   # random-init weights of the architecture (profiling captures)
        obj = ctx.load_object(mesh, cfg, tables=params.tables, mlp=params.packed_mlp())
    else:
        # the network trained by the library's own training step from its seeded
        # initialisation (the query's cost does not depend on the weights; the
        # precision figures below need a trained network)
        obj = ctx.load_object(mesh, cfg, keep_mesh=True)
        train_info = train_object(ctx, obj, steps=args.train_steps, batch=1 << 16, n_pool=1 << 21, seed=5)
        params = I.Params(ctx.read_params(obj, lsnif.PARAM_TABLES),
                          I.unpack_mlp(cfg, ctx.read_params(obj, lsnif.PARAM_MLP)))
    rays = torch.from_numpy(rays_np).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)
    # pick the fused kernel's tile shape on this workload (outside the timed region)
    if args.profile_step and args.variant is not None:
        variant = args.variant
    else:
        variant = ctx.autotune(rays, obj=obj, reps=3)
    if args.variant is not None:   # fixed shape (profiling runs, whose timings differ)
        variant = args.variant
        ctx.set_variant(variant)   # for BF16 and FP16 (else FP16 keeps its own autotuned shape)
    vshape = lsnif.Context.variants()[variant]
    stream = torch.cuda.current_stream()
    if args.profile_step:
        # one BF16 step inside a profiler range (ncu --profile-from-start off):
        # the kernels of exactly one query, after warm-up, L2 flushed before it
        out = ctx.query_rays(rays, obj=obj, precision=lsnif.BF16_FUSED)
        for _ in range(3):
            ctx.query_rays(rays, obj=obj, precision=lsnif.BF16_FUSED, out=out)
        flush.zero_()
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        ctx.query_rays(rays, obj=obj, precision=lsnif.BF16_FUSED, out=out)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        ctx.check()
        print(json.dumps({"profile_step": "BF16 query", "rays": n, "variant": vshape}))
        ctx.close()
        return

    def timed(precision, steps, warmup, profile=False):
        out = ctx.query_rays(rays, obj=obj, precision=precision)
        for _ in range(warmup):
            ctx.query_rays(rays, obj=obj, precision=precision, out=out)
        ctx.check()
        ctx.set_profiling(profile)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        kern = []
        barrier()
        t_wall = time.perf_counter()
        for s in range(steps):
            flush.zero_()
            evs[s][0].record(stream)
            ctx.query_rays(rays, obj=obj, precision=precision, out=out)
            evs[s][1].record(stream)
            if profile:
                p = ctx.last_profile()
                kern.append(p)
        barrier()
        wall = time.perf_counter() - t_wall
        ctx.set_profiling(False)
        ctx.check()
        ms = np.array([a.elapsed_time(b) for a, b in evs])
        return ms, kern, wall

    # ---- BF16 fused (headline), clocks sampled during its timed region ----
    with ClockSampler(local) as clk:
        ms16, prof16, wall16 = timed(lsnif.BF16_FUSED, args.steps, args.warmup, profile=True)
    clocks = clk.summary()
    ms32, prof32, wall32 = timed(lsnif.FP32_PLAIN, max(3, args.steps // 2), 3, profile=True)
    ms8, prof8, wall8 = timed(lsnif.FP8_FUSED, max(3, args.steps // 2), 3, profile=True)
    msh, profh, wallh = timed(lsnif.FP16_FUSED, max(3, args.steps // 2), 3, profile=True)

    from paper_2504_21627_gb300 import replicas

    def reduce_max(x: float) -> float:
        return replicas.aggregate(x, n)[0]

    mean16, _, value = replicas.aggregate(float(ms16.mean()), n)
    mean32, _, v32 = replicas.aggregate(float(ms32.mean()), n)
    mean8, _, v8 = replicas.aggregate(float(ms8.mean()), n)
    meanh, _, vh = replicas.aggregate(float(msh.mean()), n)

    # ---- end to end through the host-buffer C-ABI call ----
    # page-locked host buffers; the kernels read the rays and write the results
    # there directly (lsnif_set_host_mode DIRECT), and, for reference, the
    # staged copies of the default mode
    host_rays = torch.from_numpy(rays_np).pin_memory()
    hres = ctx._alloc_hits(n, 0, False, device=False)

    def e2e_time(mode):
        ctx.set_host_mode(mode)
        for _ in range(3):
            ctx.query_rays_host(host_rays, obj=obj, precision=lsnif.BF16_FUSED, out=hres)
        ts = []
        barrier()
        for _ in range(max(3, args.steps // 2)):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.query_rays_host(host_rays, obj=obj, precision=lsnif.BF16_FUSED, out=hres)
            ts.append(time.perf_counter() - t0)
        barrier()
        return reduce_max(float(np.mean(ts)) * 1e3)

    e2e_staged_ms = e2e_time(lsnif.HOST_STAGED)
    e2e_ms = e2e_time(lsnif.HOST_DIRECT)
    ctx.set_host_mode(lsnif.HOST_STAGED)
    h2d = n * 8 * 4
    d2h = n * (1 + 4 + 12 + 4 + 12)

    # ---- roofline of the dominant kernel (fused gather + MLP + decode) ----
    p = prof16[-1]
    L, F = cfg.L, cfg.F
    live, pts = p.n_live, p.n_points
    # algorithmic bytes: 8 corners x F FP16 features per point and level, the
    # point itself, per live ray its record in (order, k, t0/t1, tmin/tmax)
    # and its results out (hit, t, normal, material, albedo)
    alg_bytes = pts * (L * 8 * F * 2 + 12) + live * (4 + 1 + 8 + 8 + 33)
    fused_ms = float(np.mean([q.ms_mlp for q in prof16]))
    achieved = alg_bytes / (fused_ms / 1e3) / 1e9
    peak, peak_src = measured_peaks()
    # the committed capture is of the 2048 x 2048 workload
    traffic = recorded_profile("dram_bytes_per_launch") if args.side == 2048 else None
    launches_per_step = int(prof16[-1].launches)
    # The tables (32 MB) stay in L2, so the gather's roof is the rate at which
    # L2 answers small random requests: measured here by the library's own
    # kernel on this object's tables (untimed), in 32-byte sectors. The fused
    # kernel's L2 sectors per launch: ncu's L2 <- L1 read sectors per gathered
    # point (committed capture of the same kernel sources) times this run's
    # gathered points. Its corner loads hit L1 too, so loads issued per second
    # (also reported) exceed what reaches L2.
    gather_rate = ctx.gather_rate(obj)
    info = ctx.object_info(obj)
    loads, gathered_points = corner_loads(ctx, obj, rays, cfg, list(info.res[:L]))
    sectors_per_point = recorded_profile("l2_sectors_per_gathered_point")
    l2_sectors = sectors_per_point * gathered_points if sectors_per_point else None
    l2_achieved = l2_sectors * 32 / (fused_ms / 1e3) / 1e9 if l2_sectors else None
    l2_peak = gather_rate * 32 / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean16, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rays_per_step": n, "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "fused_variant": {"threads": vshape[0], "levels_in_flight": vshape[1]}},
        "latency_ms": {"bf16_p50": float(np.percentile(ms16, 50)), "bf16_p99": float(np.percentile(ms16, 99)),
                       "fp32_p50": float(np.percentile(ms32, 50)), "fp32_p99": float(np.percentile(ms32, 99))},
        "fp32_plain": {"value": v32, "unit": "Mrays/s", "ms_per_step": mean32},
        "fp8_fused": {"value": v8, "unit": "Mrays/s", "ms_per_step": mean8,
                      "fused_ms": float(np.mean([q.ms_mlp for q in prof8]))},
        "fp16_fused": {"value": vh, "unit": "Mrays/s", "ms_per_step": meanh,
                       "fused_ms": float(np.mean([q.ms_mlp for q in profh])),
                       "note": "the BF16 kernel with FP16 operands (three more significand bits)"},
        "rays": {"live": int(live), "live_frac": live / n, "points": int(pts),
                 "mean_points_per_live_ray": pts / max(live, 1)},
        "stages_ms_bf16": {"trace": float(np.mean([q.ms_trace for q in prof16])),
                           "group": float(np.mean([q.ms_group for q in prof16])), "fused": fused_ms},
        "stages_ms_fp32": {"trace": float(np.mean([q.ms_trace for q in prof32])),
                           "group": float(np.mean([q.ms_group for q in prof32])),
                           "gather+mlp": float(np.mean([q.ms_mlp for q in prof32]))},
        "roofline": {"bound": "l2", "achieved": l2_achieved, "peak": l2_peak, "unit": "GB/s",
                     "frac": l2_achieved / l2_peak if l2_achieved else None,
                     "l2_frac": l2_achieved / l2_peak if l2_achieved else None, "traffic": traffic,
                     "kernel": "fused gather+MLP+decode (BF16 tcgen05)",
                     "peak_source": "measured in this run: lsnif_gather_rate, random 8-byte loads over the "
                                    "object's FP16 tables (L2-resident), 32 B sectors",
                     "l2_sectors_per_launch": l2_sectors, "gathered_points": gathered_points,
                     # ncu sm__pipe_tensor_cycles_active of the same kernel sources (1024^2
                     # capture): the MLP on tcgen05 is not what bounds the kernel
                     "tensor_pipe_active_pct": recorded_profile("tensor_pipe_active_pct"),
                     "l2_peak_requests_per_s": gather_rate, "corner_loads_per_launch": loads,
                     "corner_loads_per_s": loads / (fused_ms / 1e3),
                     "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                             "peak_source": peak_src,
                             "bytes": "every corner of every point as if from HBM (the tables are L2-resident)"},
                     # the query's memory ceiling: every corner of every point from HBM, plus
                     # 32 B of ray in and 33 B of results per submitted ray
                     "memory_ceiling_mrays_s": peak * 1e9 / ((alg_bytes - live * 54) / n + 65) / 1e6},
        "e2e": {"value": world * n / (e2e_ms / 1e3) / 1e6, "unit": "Mrays/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "host_mode": "direct: the kernels read the page-locked rays and write the page-locked results",
                "staged": {"value": world * n / (e2e_staged_ms / 1e3) / 1e6, "ms_per_step": e2e_staged_ms}},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "wall_s": {"bf16_timed": wall16, "fp32_timed": wall32, "fp8_timed": wall8},
    }
    if train_info is not None:
        line["config"]["weights"] = f"trained {train_info['steps']} steps on the GPU from the seeded initialisation"
        line["training"] = train_info
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, dt, sample = oracle_rate(cfg, mesh, params, rays_np, args.cpu_sample, keep=True)
        line["cpu_baseline"] = {"value": rate, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
                                "sample": f"{args.cpu_sample} seeded rays of the workload ({dt:.1f} s)"}
        # every path's results on the same sample rays against the oracle's
        errs = precision_errors(ctx, obj, sample, (("bf16", lsnif.BF16_FUSED), ("fp16", lsnif.FP16_FUSED),
                                                   ("fp32", lsnif.FP32_PLAIN), ("fp8", lsnif.FP8_FUSED)))
        line["precision"] = {"against": "FP64 oracle on the cpu_baseline sample, near-face rays left out",
                             "weights": "trained" if train_info is not None else "random-init",
                             "bounds": BOUNDS, **errs}
        line["accepted_precision"] = [k for k in ("bf16", "fp16", "fp8") if errs[k]["meets_bounds"]]
        n1 = max(256, args.cpu_sample // 16)
        rate1, dt1 = oracle_rate_single_thread(cfg, mesh, params, rays_np, n1)
        line["cpu_baseline"]["single_thread"] = {
            "value": rate1, "unit": "Mrays/s", "cores": 1,
            "sample": f"{n1} seeded rays of the workload ({dt1:.1f} s)"}
    ctx.close()
    if rank == 0 and not args.no_extras:
        # the serving loop and the many-object graph launch, compact
        line["serving"] = serving_run(args.serving_requests)
        line["batched"] = batched_run(5, 3, args.batched_rays)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
