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
                 "paper_2504_21627_gb300/csrc/device.cuh"]


def fused_source_hash() -> str:
    h = hashlib.sha256()
    for f in FUSED_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per fused-kernel launch from the committed ncu summary, or
    None when the kernel sources changed after the capture."""
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
        return float(vals["dram_bytes_per_launch"])
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


def oracle_rate(cfg, mesh, params, rays, n_sample: int, seed: int = 0):
    """The FP64 oracle, as it stands, on a seeded sample of the workload's rays."""
    from oracle import oracle as O
    if "obj" not in _ORC:
        _ORC["obj"] = O.build_object(mesh, cfg, params)
    orc = _ORC["obj"]
    g = np.random.default_rng(seed)
    idx = np.sort(g.choice(rays.shape[1], n_sample, replace=False))
    sub = np.ascontiguousarray(rays[:, idx])
    t0 = time.perf_counter()
    O.query(orc, sub)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return n_sample / dt / 1e6, cores, dt


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--ref-sample", type=int, default=2048)
    ap.add_argument("--cpu-sample", type=int, default=65536)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--side", type=int, default=2048, help="image side; below 2048 only for profiling captures")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

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
    obj = ctx.load_object(mesh, cfg, tables=params.tables, mlp=params.packed_mlp())
    rays = torch.from_numpy(rays_np).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)
    # pick the fused kernel's tile shape on this workload (outside the timed region)
    variant = ctx.autotune(rays, obj=obj, reps=3)
    vshape = lsnif.Context.variants()[variant]
    stream = torch.cuda.current_stream()

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

    from paper_2504_21627_gb300 import replicas

    def reduce_max(x: float) -> float:
        return replicas.aggregate(x, n)[0]

    mean16, _, value = replicas.aggregate(float(ms16.mean()), n)
    mean32, _, v32 = replicas.aggregate(float(ms32.mean()), n)

    # ---- end to end through the host-buffer C-ABI call ----
    host_rays = torch.from_numpy(rays_np).pin_memory()
    hres = ctx._alloc_hits(n, 0, False, device=False)
    for _ in range(3):
        ctx.query_rays_host(host_rays, obj=obj, precision=lsnif.BF16_FUSED, out=hres)
    e2e_t = []
    barrier()
    for _ in range(max(3, args.steps // 2)):
        t0 = time.perf_counter()
        ctx.query_rays_host(host_rays, obj=obj, precision=lsnif.BF16_FUSED, out=hres)
        e2e_t.append(time.perf_counter() - t0)
    barrier()
    e2e_ms = reduce_max(float(np.mean(e2e_t)) * 1e3)
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
    traffic = recorded_traffic()
    launches_per_step = int(prof16[-1].launches)
    l2_requests = pts * L * 5.0  # ~1.25 16-byte requests per x-pair, 4 pairs per point and level

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
        "rays": {"live": int(live), "live_frac": live / n, "points": int(pts),
                 "mean_points_per_live_ray": pts / max(live, 1)},
        "stages_ms_bf16": {"trace": float(np.mean([q.ms_trace for q in prof16])),
                           "group": float(np.mean([q.ms_group for q in prof16])), "fused": fused_ms},
        "stages_ms_fp32": {"trace": float(np.mean([q.ms_trace for q in prof32])),
                           "group": float(np.mean([q.ms_group for q in prof32])),
                           "gather+mlp": float(np.mean([q.ms_mlp for q in prof32]))},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": "fused gather+MLP+decode (BF16 tcgen05)",
                     "peak_source": peak_src,
                     "l2_request_rate_gps": l2_requests / (fused_ms / 1e3) / 1e9},
        "e2e": {"value": world * n / (e2e_ms / 1e3) / 1e6, "unit": "Mrays/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "wall_s": {"bf16_timed": wall16, "fp32_timed": wall32},
    }
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, dt = oracle_rate(cfg, mesh, params, rays_np, args.cpu_sample)
        line["cpu_baseline"] = {"value": rate, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
                                "sample": f"{args.cpu_sample} seeded rays of the workload ({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
