#!/usr/bin/env python
"""Benchmark of the GB300 Domain Transform Solver.

One step = one complete DTS solve (distances + K iterations of N horizontal and
N vertical recursive-filter passes + the data-term update) of the stereo-shaped
workload: a 2880 x 1988 RGB guide, 20 iterations, sigma_s = 16, sigma_r = 0.1,
lambda = 0.99, FP32 (seeded synthetic data shaped like the paper's Middlebury
stereo refinement; the dataset itself is not available).

Prints ONE JSON line (rank 0).  ``value`` is megapixels solved per second over
all ranks with inputs resident in HBM; ``e2e`` is the same metric through the
Python binding with host-resident (pinned) inputs copied in and the result
copied out every step; ``roofline`` is the dominant kernel's algorithmic bytes
per launch over its event-timed duration, against the measured HBM copy
bandwidth; ``cpu_baseline`` is the FP64 oracle timed on the host cores.

``--impl reference`` times the oracle itself (the CPU program the GPU path is
checked against) on the same workload and metric.

Multi-GPU (torchrun): every rank solves its own replica (the solve of one image
does not shard here); the value is the images of all ranks over the slowest
rank's time.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "megapixels/sec per DTS solve (fwd, fwd+bwd) and % of GB300 HBM roofline at stated error"
UNIT = "MP/s"
TOL = 1e-4
PROFILE_EVERY = 10

# algorithmic bytes per pixel of each kernel (s_d distance storage, s_t target storage, C guide
# channels of s_g bytes): every input element read once, every output element written once
def bytes_per_pixel(name, s_d, s_t, C=3, s_g=4):
    return {
        "distance_kernel": C * s_g + 2 * s_d + s_t + 4,
        "copy_plane_kernel": s_t + 4,
        "row_pass_kernel": 8 + s_d,
        "col_pass_kernel": 8 + s_d,
        "col_pass_kernel<update>": 16 + s_d + s_t,
        "row_pass_kernel<support>": s_d + 4,
        "col_pass_kernel<support>": 12 + s_d,
    }.get(name)


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--dist-dtype", choices=["f32", "f16"], default="f32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    return ap.parse_args()


def workload():
    from paper_1805_04590_gb300 import workloads
    wl = workloads.make(1)
    return wl, wl.problems[0], wl.params


def workload_config(p, q, extra=None):
    H, W = p.target.shape
    cfg = {"workload": f"stereo-shaped {W}x{H} RGB guide, {q.iterations} iterations, sigma_s={q.sigma_s:g}, "
                       f"sigma_r={q.sigma_r:g}, lambda={q.lam:g}, N={q.passes} passes, GD step {q.step:g}",
           "width": W, "height": H, "channels": int(p.guide.shape[0]), "iterations": q.iterations,
           "passes": q.passes, "megapixels_per_step": round(H * W / 1e6, 6)}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu_index), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        reasons = []
        for i, name in ((5, "hw_slowdown"), (6, "hw_thermal_slowdown"), (7, "sw_thermal_slowdown"),
                        (8, "sw_power_cap")):
            if any(r[i].lower().startswith("active") for r in self.rows):
                reasons.append(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def rejected(clk):
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if set(clk.get("reasons", [])) & bad:
        return True
    if clk.get("sm_mhz") and clk.get("sm_max_mhz") and not clk["reasons"]:
        return clk["sm_mhz"] < 0.5 * clk["sm_max_mhz"]
    return False


# ---------------------------------------------------------------- roofline helpers
def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_for(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, when that
    summary was taken on the current kernel source (else None)."""
    src = os.path.join(ROOT, "paper_1805_04590_gb300", "csrc", "dts_forward.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    pat = re.compile(r"^traffic\s+(\S+)\s+bytes_per_launch=(\d+)\s+source_sha=([0-9a-f]+)", re.M)
    for fn in sorted(os.listdir(pdir)):
        if fn.endswith((".md", ".txt")):
            for m in pat.finditer(open(os.path.join(pdir, fn)).read()):
                if m.group(1) == kernel and m.group(3) == sha:
                    return int(m.group(2))
    return None


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1805_04590_gb300 import dts

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl, p, q = workload()
    H, W = p.target.shape
    mp = H * W / 1e6
    s_d = 2 if args.dist_dtype == "f16" else 4
    prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, step=q.step, iterations=q.iterations,
                     passes=q.passes, dist_dtype=dts.F16 if s_d == 2 else dts.F32)
    g = torch.from_numpy(p.guide).to(dev)
    t = torch.from_numpy(p.target).to(dev)
    c = torch.from_numpy(p.conf).to(dev)
    ws = dts.workspace(g, prm)
    out = torch.empty_like(t)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        dts.dts_solve(g, t, c, prm, out=out, ws=ws)
    torch.cuda.synchronize()
    if dts.dts_last_status() != 0:
        raise RuntimeError("device status not clean after warm-up")

    def timed_loop():
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        clk = ClockSampler(local_rank)
        barrier()
        torch.cuda.synchronize()
        clk.start()
        time.sleep(0.15)
        dts.dts_profile(1)
        dts.dts_profile(0)
        wall0 = time.perf_counter()
        for i, (e0, e1) in enumerate(evs):
            # per-kernel events on every PROFILE_EVERY-th step (events between kernels cost a little)
            dts.dts_profile(2 if i % PROFILE_EVERY == 0 else 0)
            flush.zero_()
            e0.record(stream)
            dts.dts_solve(g, t, c, prm, out=out, ws=ws)
            e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        barrier()
        dts.dts_profile(0)
        clk.stop()
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms, wall, clk.summary(), dts.dts_profile_read()

    ms, wall, clk, recs = timed_loop()
    if rejected(clk):
        ms, wall, clk, recs = timed_loop()
        clk["remeasured"] = True
    total_ms = float(np.sum(ms))
    if world > 1:
        tt = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
    value = world * args.steps * mp / (total_ms / 1e3)
    if dts.dts_last_status() != 0:
        raise RuntimeError("device status not clean after the timed region")

    # per-kernel durations inside the timed region (sampled steps)
    profiled_steps = len(range(0, args.steps, PROFILE_EVERY))
    launches_per_step = len(recs) // profiled_steps
    kern = {}
    for name, _, px, fl, t_ms in recs:
        k = kern.setdefault(name, {"launches": 0, "ms": 0.0, "pixels": 0})
        k["launches"] += 1
        k["ms"] += t_ms
        k["pixels"] += px
    dom = max(kern, key=lambda n: kern[n]["ms"])
    kd = kern[dom]
    bpp = bytes_per_pixel(dom, s_d, 4, C=int(p.guide.shape[0]))
    alg_bytes = bpp * kd["pixels"] / kd["launches"]
    avg_s = kd["ms"] / kd["launches"] / 1e3
    peak, peak_kind = measured_peak()
    achieved = alg_bytes / avg_s / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": f"{peak_kind} hbm_gbs (copy)",
            "algorithmic_bytes_per_launch": int(alg_bytes), "bytes_per_pixel": bpp,
            "avg_launch_us": round(avg_s * 1e6, 2), "traffic": traffic_for(dom),
            "share_of_step": round(kd["ms"] / sum(v["ms"] for v in kern.values()), 4)}
    kernels = {n: {"launches": v["launches"], "avg_us": round(v["ms"] / v["launches"] * 1e3, 2),
                   "share": round(v["ms"] / sum(x["ms"] for x in kern.values()), 4)} for n, v in kern.items()}

    # end to end through the binding with host-resident inputs and output
    gh = torch.from_numpy(p.guide).pin_memory()
    th = torch.from_numpy(p.target).pin_memory()
    ch = torch.from_numpy(p.conf).pin_memory()
    zh = torch.empty((H, W), dtype=torch.float32).pin_memory()
    gd, td, cd = torch.empty_like(g), torch.empty_like(t), torch.empty_like(c)
    n_e2e = max(1, min(args.e2e_steps, args.steps))
    for _ in range(2):
        gd.copy_(gh, non_blocking=True); td.copy_(th, non_blocking=True); cd.copy_(ch, non_blocking=True)
        dts.dts_solve(gd, td, cd, prm, out=out, ws=ws)
        zh.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n_e2e):
        gd.copy_(gh, non_blocking=True); td.copy_(th, non_blocking=True); cd.copy_(ch, non_blocking=True)
        dts.dts_solve(gd, td, cd, prm, out=out, ws=ws)
        zh.copy_(out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    if world > 1:
        tt = torch.tensor([e2e_ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(tt.item())
    h2d = gh.numel() * 4 + th.numel() * 4 + ch.numel() * 4
    e2e = {"value": round(world * n_e2e * mp / (e2e_ms / 1e3), 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": zh.numel() * 4, "steps": n_e2e}

    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded PCG64 Voronoi guide with colour gradients, piecewise-planar disparity "
                    "target with 10% outliers; stands in for Middlebury stereo)",
            "config": workload_config(p, q, {"direction": "fwd", "distance_storage": args.dist_dtype,
                                             "l2": "flushed between steps (512 MiB write)",
                                             "parallelism": f"replicas x{world}"}),
            "roofline": roof, "kernels": kernels, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": clk, "wall_s_timed_region": round(wall, 4),
            "kernel_timing": f"CUDA events around each kernel on every {PROFILE_EVERY}th timed step"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        zgpu = out.cpu().numpy()
        t0 = time.perf_counter()
        zref = oracle.solve(p.guide, p.target, p.conf, lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, step=q.step,
                            iterations=q.iterations, passes=q.passes)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": round(mp / dt, 4), "unit": UNIT, "cores": oracle.num_threads(),
                                "kind": "oracle",
                                "sample": f"one full FP64 oracle solve of the same {W}x{H} workload "
                                          f"({q.iterations} iterations), {dt:.2f} s"}
        err = float(np.abs(zgpu - zref).max())
        rng = float(p.target.max() - p.target.min())
        line["error"] = {"max_abs_vs_oracle": err, "rel_to_target_range": err / rng, "tolerance": TOL,
                         "within": err <= TOL * rng}
    return line


# ---------------------------------------------------------------- reference arm (the oracle)
def run_reference(args):
    import oracle
    _, p, q = workload()
    H, W = p.target.shape
    # bounded sample: the centre quarter (half width, half height) of the same image, full solve
    h0, w0 = H // 4, W // 4
    sl = (slice(h0, h0 + H // 2), slice(w0, w0 + W // 2))
    gi = np.ascontiguousarray(p.guide[:, sl[0], sl[1]])
    ti = np.ascontiguousarray(p.target[sl])
    ci = np.ascontiguousarray(p.conf[sl])
    mp = ti.size / 1e6

    def step():
        oracle.solve(gi, ti, ci, lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, step=q.step,
                     iterations=q.iterations, passes=q.passes)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = args.steps * mp / dt
    sample = (f"centre {ti.shape[1]}x{ti.shape[0]} crop of the {W}x{H} workload, full {q.iterations}-iteration "
              f"FP64 solve per step")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (same seeded workload)",
            "config": workload_config(p, q, {"direction": "fwd", "sample": sample, "parallelism": "host cores"}),
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)), flush=True)
        return 0
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        line = run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
