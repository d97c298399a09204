#!/usr/bin/env python
"""Benchmark of the GB300 Domain Transform Solver.

One step = one complete DTS solve (distances + K iterations of N horizontal and
N vertical recursive-filter passes + the data-term update) of the default
workload: the 10000 x 10000 multispectral image with 16 bands, 10 iterations,
sigma_s = 32, sigma_r = 0.1, lambda = 0.99, FP32 (seeded synthetic data shaped
like satellite imagery; the largest configuration that fits one GPU).  The
line's value is the forward solve; ``fwdbwd`` holds the same measurement for
the forward solve followed by its reverse mode (dts_solve_backward, gradients
for target, confidence and guide).  ``--workload`` picks the stereo-shaped,
depth-SR, batched or 256 x 256 workload instead.

Prints ONE JSON line (rank 0).  ``value`` is megapixels solved per second over
all ranks with inputs resident in HBM; ``e2e`` is the same metric through the
Python binding with host-resident (pinned) inputs copied in and the result
copied out every step; ``roofline`` is the dominant kernel's algorithmic bytes
per launch over its event-timed duration, against the measured HBM copy
bandwidth, with the whole step's on the method's byte count; ``cpu_baseline`` is
the FP64 oracle timed on the host cores on a bounded sample, and ``error`` the
GPU's distance from it on that sample.

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

UPDATES = {"gd": 0, "jacobi": 1, "cg": 2}


def update_desc(update, step):
    return {"gd": f"GD step {step:g} (Eq. 3)", "jacobi": "fixed-point update (Eq. 4)",
            "cg": "conjugate gradients on Eq. 2"}[update]


def oracle_solve(update, I, t, c, kw):
    """The oracle's solve for this update rule (kw: lam, sigma_s, sigma_r, step, iterations, passes)."""
    import oracle
    if update == "cg":
        k = {n: v for n, v in kw.items() if n not in ("step", "charbonnier_eps")}
        return oracle.solve_cg(I, t, c, **k)
    return oracle.solve(I, t, c, update=UPDATES[update], **kw)


# algorithmic bytes per pixel of each kernel (s_d distance storage, s_t target storage, C guide
# channels of s_g bytes): every input element read once, every output element written once
def bytes_per_pixel(name, s_d, s_t, C=3, s_g=4, N=3, K=10):
    return {
        # the persistent batched kernel runs a whole solve per launch: the distances, per iteration
        # 2N passes, the update fused into K - 1 of the horizontal ones, and the last update
        "batched_solve_kernel": (C * s_g + 2 * s_d + s_t + 4 + K * 2 * N * (8 + s_d) + (K - 1) * (12 + s_t)
                                 + 16 + s_t),
        "distance_kernel": C * s_g + 2 * s_d + s_t + 4,
        # per pixel and iteration: the distances once per pass, z_k, t and c read and z_{k+1}
        # written by the update; the iterate itself stays in shared memory between passes
        "resident_solve_kernel": 2 * N * s_d + 12 + s_t,
        "copy_plane_kernel": s_t + 4,
        "row_pass_kernel": 8 + s_d,
        "col_pass_kernel": 8 + s_d,
        "col_strip_kernel": 8 + s_d,
        "col_chain_kernel": 8 + s_d,
        "col_tall_kernel": 8 + s_d,
        "col_bwd_chain_kernel": 24 + s_d,
        # the two-phase vertical adjoint: chunk totals (pass input, adjoint, distances), then the
        # replay (those again, the pass output and the distance adjoint read; two planes written)
        "col_bwd_agg_kernel": 8 + s_d,
        "col_bwd_apply_kernel": 24 + s_d,
        # the chunk tuples in and the carries out (nine floats each way per column and chunk of
        # the default 128 rows): the implementation's bytes, none of the method's
        "col_bwd_carry_kernel": 72 / 128,
        "row_pass_kernel<support>": s_d + 4,
        "col_pass_kernel<support>": 12 + s_d,
        "row_pass_kernel<update>": 20 + s_t + s_d,
        "row_stream_kernel": 8 + s_d,
        "row_stream_kernel<update>": 20 + s_t + s_d,
        "update_kernel": 16 + s_t,
        "row_bwd_kernel": 24 + s_d,
        "row_bwd_kernel<final>": 28 + s_d,
        "col_bwd_kernel": 24 + s_d,
        "guide_grad_kernel": C * s_g + 2 * s_d + 8 + 4 * C,
        "guide_grad_kernel<x4>": C * s_g + 2 * s_d + 8 + 4 * C,
        "axpy_plane_kernel": 12,
        "update_adjoint_kernel": 36 + s_t,
        "row_pass_kernel<transpose>": 8 + s_d,
        # the first transposed vertical pass of a product also reads the minuend plane
        "col_pass_kernel<transpose>": 8 + s_d + 4.0 / N,
        "col_strip_kernel<transpose>": 8 + s_d + 4.0 / N,
        "col_chain_kernel<transpose>": 8 + s_d + 4.0 / N,
        "col_tall_kernel<transpose>": 8 + s_d + 4.0 / N,
        "square_plane_kernel": 8,
        "confidence_kernel": 12,
        "box_line_kernel": 12,
        "transpose_kernel": 8,
        "cg_apply_kernel": 20,
        "cg_step_kernel": 24,
        "cg_direction_kernel": 12,
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
    ap.add_argument("--workload", choices=["stereo", "plain", "depth_sr", "batched", "multispectral"],
                    default="multispectral")
    ap.add_argument("--storage", choices=["f32", "bf16"], default="f32", help="guide and target storage")
    ap.add_argument("--direction", choices=["fwd", "fwdbwd", "both"], default="both",
                    help="both: forward as the line's value, forward + backward under 'fwdbwd'")
    ap.add_argument("--update", choices=["gd", "jacobi", "cg"], default="gd",
                    help="Eq. 3 gradient step, Eq. 4 fixed point, or conjugate gradients on Eq. 2")
    ap.add_argument("--sweep", choices=["iterations", "sigma", "size"], default=None,
                    help="one JSON line per point instead of the bench line: accuracy and time against "
                         "iterations (GD, Jacobi, CG), time against sigma_s / sigma_r, time against megapixels")
    ap.add_argument("--filter-kernel", choices=["rf", "box"], default="rf",
                    help="recursive-filter kernel, or the box kernel Eq. 10 prints")
    ap.add_argument("--batch-policy", choices=["auto", "persistent", "graph"], default="auto",
                    help="batched workload: the persistent kernel, the graph of per-image launch sequences, "
                         "or (auto) whichever dts_autotune_batched measures faster before the warm-up")
    ap.add_argument("--ncu-case", choices=sorted(NCU_CASES), default=None,
                    help="run one small case of a kernel's launch plan (for a profiler capture) and print the "
                         "per-kernel event times instead of the bench line")
    ap.add_argument("--charbonnier-eps", type=float, default=0.0,
                    help="> 0: Charbonnier loss on the target term (the paper's stereo loss uses 0.001)")
    return ap.parse_args()


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


BACKWARD_KERNELS = ("row_bwd_kernel", "col_bwd_kernel", "col_bwd_chain_kernel", "col_bwd_agg_kernel",
                    "col_bwd_apply_kernel", "col_bwd_carry_kernel", "update_adjoint_kernel",
                    "guide_grad_kernel", "axpy_plane_kernel")


def kernel_source(kernel):
    """Path of the library source file that holds `kernel` (a name the per-launch timer reports)."""
    fn = ("dts_backward.cu" if kernel.startswith(BACKWARD_KERNELS) else "dts_cg.cu" if kernel.startswith("cg_")
          else "dts_box.cu" if kernel.startswith(("box_", "transpose_"))
          else "dts_resident.cu" if kernel.startswith("resident_")
          else "dts_batched.cu" if kernel.startswith("batched_")
          else "dts_rows.cu" if kernel.startswith("row_stream_")
          else "dts_confidence.cu" if kernel.startswith(("square_plane_", "confidence_"))
          else "dts_forward.cu")
    return os.path.join(ROOT, "paper_1805_04590_gb300", "csrc", fn)


def source_hash(path):
    """SHA-256 (first 16 hex digits) of a library source file together with every local header it
    includes, recursively (a change to any of them changes the kernel)."""
    seen, h = set(), hashlib.sha256()

    def add(fn):
        fn = os.path.normpath(fn)
        if fn in seen or not os.path.exists(fn):
            return
        seen.add(fn)
        text = open(fn, "rb").read()
        h.update(text)
        for inc in re.findall(rb'#include\s+"([^"]+)"', text):
            add(os.path.join(os.path.dirname(fn), inc.decode()))

    add(path)
    return h.hexdigest()[:16]


def traffic_key(args):
    """The workload key of a committed traffic line: workload, guide and target storage, distance
    storage (each changes what a launch moves)."""
    return f"{args.workload}:{args.storage}:{args.dist_dtype}"


def traffic_for(kernel, key):
    """DRAM bytes per launch of `kernel` on the workload `key` (traffic_key) from the committed ncu
    summary, when that summary was taken on the current source of the kernel's translation unit
    (its .cu file and the headers it includes), else None."""
    sha = source_hash(kernel_source(kernel))
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    pat = re.compile(r"^traffic\s+(\S+)\s+workload=(\S+)\s+bytes_per_launch=(\d+)\s+source_sha=([0-9a-f]+)", re.M)
    for fn in sorted(os.listdir(pdir)):
        if fn.endswith((".md", ".txt")):
            for m in pat.finditer(open(os.path.join(pdir, fn)).read()):
                if m.group(1) == kernel and m.group(2) == key and m.group(4) == sha:
                    return int(m.group(3))
    return None


# ---------------------------------------------------------------- our arm
WORKLOAD_INDEX = {"plain": 0, "stereo": 1, "depth_sr": 2, "batched": 3, "multispectral": 4}
WORKLOAD_DATA = {
    "plain": "synthetic (seeded PCG64 Voronoi guide, per-cell depth target with noise and 5% outliers)",
    "stereo": "synthetic (seeded PCG64 Voronoi guide with colour gradients, piecewise-planar disparity target "
              "with 10% outliers; stands in for Middlebury stereo)",
    "depth_sr": "synthetic (seeded PCG64 guides, 128x96 depth bilinearly upsampled x16; stands in for the "
                "Ferstl depth super-resolution benchmark)",
    "batched": "synthetic (64 seeded images of uneven sizes built like the plain workload)",
    "multispectral": "synthetic (seeded 16-band smooth fields with Voronoi edges; satellite-shaped imagery)",
}


class Inputs:
    """A workload's inputs resident on the device (guides and targets in the storage dtype)."""

    def __init__(self, args, dev):
        import torch
        from paper_1805_04590_gb300 import workloads
        self.name = args.workload
        self.wl = workloads.make(WORKLOAD_INDEX[self.name])
        self.sdt = torch.bfloat16 if args.storage == "bf16" else torch.float32
        self.s_io = 2 if args.storage == "bf16" else 4
        probs = self.wl.problems
        self.mp = sum(p.target.size for p in probs) / 1e6
        self.g = [torch.from_numpy(p.guide).to(dev).to(self.sdt) for p in probs]
        self.t = [torch.from_numpy(p.target).to(dev).to(self.sdt) for p in probs]
        self.c = [torch.from_numpy(p.conf).to(dev) for p in probs]


class Case:
    """One step of a workload in one direction on the GPU: inputs resident, outputs, gradients and
    the workspace preallocated."""

    def __init__(self, args, dev, inputs, direction):
        import torch
        from paper_1805_04590_gb300 import dts
        self.torch, self.dts = torch, dts
        self.args, self.dev, self.inp = args, dev, inputs
        self.name = inputs.name
        self.wl = inputs.wl
        self.mp = inputs.mp
        self.g, self.t, self.c = inputs.g, inputs.t, inputs.c
        self.s_io = inputs.s_io
        self.direction = direction
        self.bwd = direction == "fwdbwd"
        q = self.wl.params
        self.s_d = 2 if args.dist_dtype == "f16" else 4
        self.prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, step=q.step, iterations=q.iterations,
                              passes=q.passes, dist_dtype=dts.F16 if self.s_d == 2 else dts.F32,
                              save_checkpoints=0, update=UPDATES[args.update],
                              charbonnier_eps=args.charbonnier_eps,
                              filter_kernel=dts.KERNEL_BOX if args.filter_kernel == "box" else dts.KERNEL_RF)
        probs = self.wl.problems
        big = max(range(len(probs)), key=lambda i: probs[i].target.size)
        if self.bwd:  # what the autograd path picks: every pass input kept when memory allows
            self.prm.save_checkpoints = dts.backward_checkpoint_mode(self.g[big], self.prm)
        self.out = [torch.empty(p.target.shape, dtype=torch.float32, device=dev) for p in probs]
        rng = np.random.default_rng(77)
        self.gz = [torch.from_numpy(rng.standard_normal(p.target.shape).astype(np.float32)).to(dev) for p in probs] \
            if self.bwd else None
        if self.name == "batched":
            self.ws = [dts.batched_workspace(self.g, self.prm)]
        else:
            self.ws = [dts.workspace(self.g[big], self.prm, with_backward=self.bwd)]
        self.grads = None

    def step(self, g=None, t=None, c=None):
        dts = self.dts
        g, t, c = g or self.g, t or self.t, c or self.c
        if self.name == "batched":
            dts.dts_solve_batched(g, t, c, self.prm, outs=self.out, ws=self.ws[0])
            return
        self.grads = []
        for i in range(len(g)):
            dts.dts_solve(g[i], t[i], c[i], self.prm, out=self.out[i], ws=self.ws[0])
            if self.bwd:
                self.grads.append(dts.dts_solve_backward(g[i], t[i], c[i], self.prm, self.ws[0], self.gz[i])[:3])

    def solve_into(self, dev_in, dev_out):
        """The forward solve of every image from device inputs [guides.., targets.., confs..]
        into device outputs (one per image), on the current stream."""
        n = len(dev_out)
        g, t, c = dev_in[:n], dev_in[n:2 * n], dev_in[2 * n:]
        if self.name == "batched":
            self.dts.dts_solve_batched(g, t, c, self.prm, outs=dev_out, ws=self.ws[0])
            return
        for i in range(n):
            self.dts.dts_solve(g[i], t[i], c[i], self.prm, out=dev_out[i], ws=self.ws[0])

    def io_bytes(self):
        h2d = sum(x.numel() * x.element_size() for x in self.g + self.t + self.c)
        d2h = sum(x.numel() * 4 for x in self.out)
        if self.bwd:
            h2d += sum(x.numel() * 4 for x in self.gz)
            d2h += sum(x.numel() * 4 * (2 + g.shape[0]) for x, g in zip(self.out, self.g))
        return h2d, d2h

    def config(self, world):
        p = self.wl.problems[0]
        q = self.wl.params
        shapes = sorted({tuple(x.target.shape) for x in self.wl.problems})
        desc = {"plain": "plain 256x256 RGB", "stereo": "stereo-shaped 2880x1988 RGB",
                "depth_sr": "depth SR x16, batch 8 x 2048x1536 RGB", "batched": "64 uneven RGB images",
                "multispectral": "multispectral 10000x10000 x 16 bands"}[self.name]
        return {"workload": f"{desc}, {q.iterations} iterations, sigma_s={q.sigma_s:g}, sigma_r={q.sigma_r:g}, "
                            f"lambda={q.lam:g}, N={q.passes} passes, {update_desc(self.args.update, q.step)}",
                "images": len(self.wl.problems), "channels": int(p.guide.shape[0]),
                "shape_hw": list(shapes[0]) if len(shapes) == 1 else "uneven",
                "iterations": q.iterations, "passes": q.passes, "megapixels_per_step": round(self.mp, 6),
                "direction": self.direction, "storage": self.args.storage, "update": self.args.update,
                "target_loss": (f"charbonnier eps={self.args.charbonnier_eps:g}" if self.args.charbonnier_eps > 0
                                else "square"),
                "filter_kernel": {"rf": "recursive filter", "box": "box (Eq. 10 as printed)"}[self.args.filter_kernel],
                "distance_storage": self.args.dist_dtype,
                "l2": "flushed between steps (512 MiB write), in the device-timed and the end-to-end loops",
                "backward_checkpoints": ({1: "iterates (pass inputs recomputed)", 2: "every pass input"}
                                         .get(self.prm.save_checkpoints) if self.bwd else None),
                "parallelism": f"replicas x{world}"}


def cpu_sample(args, inp, case):
    """The oracle on a bounded sample of the workload: (megapixels, seconds, description, error).
    The error compares the GPU's solve of the same sample (for the multispectral image: a solve of
    its 2500 x 2500 crop) with the oracle's on the inputs as stored on the GPU, and for 16-bit
    storage also with the oracle's on the unrounded inputs."""
    import oracle
    import torch
    q = inp.wl.params
    probs = inp.wl.problems
    idx = list(range(min(len(probs), 8 if inp.name == "batched" else 1)))
    kw = dict(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, step=q.step, iterations=q.iterations,
              passes=q.passes, charbonnier_eps=args.charbonnier_eps)
    crop = inp.name == "multispectral"
    sl = (slice(0, 2500), slice(0, 2500)) if crop else (slice(None), slice(None))
    mp, dt, rels, rels0 = 0.0, 0.0, [], []
    for i in idx:
        p = probs[i]
        gd = inp.g[i][:, sl[0], sl[1]].contiguous()
        td = inp.t[i][sl].contiguous()
        cd = inp.c[i][sl].contiguous()
        I = gd.float().cpu().numpy()  # the values the GPU saw (rounded when stored in bf16)
        t = td.float().cpu().numpy()
        cc = cd.cpu().numpy()
        t0 = time.perf_counter()
        z = oracle_solve(args.update, I, t, cc, kw)
        dt += time.perf_counter() - t0
        mp += t.size / 1e6
        zg = (case.dts.dts_solve(gd, td, cd, case.prm) if crop else case.out[i]).float().cpu().numpy()
        rng = max(float(np.ptp(t)), 1e-30)
        rels.append(float(np.abs(zg - z).max()) / rng)
        if args.storage != "f32":
            z0 = oracle_solve(args.update, np.ascontiguousarray(p.guide[:, sl[0], sl[1]]),
                              np.ascontiguousarray(p.target[sl]), cc, kw)
            rels0.append(float(np.abs(zg - z0).max()) / rng)
    what = ("a 2500x2500 crop (16 bands)" if crop else
            f"{len(idx)} of {len(probs)} images" if len(probs) > 1 else "the full image")
    desc = f"FP64 oracle, {what}, all {q.iterations} iterations forward, {dt:.2f} s"
    error = {"rel_to_target_range": max(rels), "tolerance": TOL, "within": max(rels) <= TOL,
             "inputs": "as stored on the GPU", "sample": what}
    if rels0:
        error["rel_to_target_range_unrounded_inputs"] = max(rels0)
    return mp, dt, desc, error


def measure(args, case, world, local_rank, flush):
    """Warm-up, the timed region (max over ranks), the dominant kernel's roofline and the whole
    step's, and the end-to-end leg through the binding with host buffers, for one Case."""
    import torch
    dts = case.dts
    dev = case.dev
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        case.step()
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
            case.step()
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
    total_ms = max_over_ranks(float(np.sum(ms)), world, dev)
    value = job_value(world, args.steps, case.mp, total_ms)
    if dts.dts_last_status() != 0:
        raise RuntimeError("device status not clean after the timed region")
    res = {"value": round(value, 2), "ms_per_step": round(total_ms / args.steps, 4), "clocks": clk,
           "wall_s_timed_region": round(wall, 4)}
    res.update(roofline_of(args, case, recs, total_ms))
    res["e2e"] = e2e_of(args, case, world, flush)
    return res


def roofline_of(args, case, recs, total_ms):
    """The dominant kernel's algorithmic bytes per launch over its mean event-timed duration, and
    the whole step's algorithmic bytes (the method's, by the per-pixel count of each pass, not the
    implementation's) over the step time, against the measured HBM copy bandwidth."""
    profiled_steps = len(range(0, args.steps, PROFILE_EVERY))
    launches_per_step = len(recs) // profiled_steps if recs else None
    kern = {}
    C = int(case.g[0].shape[0])
    s_g = case.s_io
    for name, _, px, fl, t_ms in recs:
        k = kern.setdefault(name, {"launches": 0, "ms": 0.0, "pixels": 0})
        k["launches"] += 1
        k["ms"] += t_ms
        k["pixels"] += px
    out = {"roofline": None, "kernels": None,
           "gpu_launches": launches_per_step * args.steps if launches_per_step else None}
    if not kern:
        return out
    N, K = case.prm.passes, case.prm.iterations
    dom = max(kern, key=lambda n: kern[n]["ms"])
    kd = kern[dom]
    bpp = bytes_per_pixel(dom, case.s_d, case.s_io, C=C, s_g=s_g, N=N, K=K)
    alg_bytes = bpp * kd["pixels"] / kd["launches"]
    avg_s = kd["ms"] / kd["launches"] / 1e3
    peak, peak_kind = measured_peak()
    achieved = alg_bytes / avg_s / 1e9
    tot_ms = sum(v["ms"] for v in kern.values())
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": f"{peak_kind} hbm_gbs (copy)",
            "algorithmic_bytes_per_launch": int(alg_bytes), "bytes_per_pixel": round(bpp, 3),
            "avg_launch_us": round(avg_s * 1e6, 2), "traffic": traffic_for(dom, traffic_key(args)),
            "share_of_step": round(kd["ms"] / tot_ms, 4)}
    step_bytes = step_algorithmic_bytes(case, C, s_g)
    step_s = total_ms / args.steps / 1e3
    profiled = len(range(0, args.steps, PROFILE_EVERY))
    bpps = {n: bytes_per_pixel(n, case.s_d, case.s_io, C=C, s_g=s_g, N=N, K=K) for n in kern}
    moved = sum(bpps[n] * v["pixels"] for n, v in kern.items() if bpps[n] is not None) / profiled
    roof["step"] = {"algorithmic_bytes": int(step_bytes), "achieved": round(step_bytes / step_s / 1e9, 1),
                    "frac": round(step_bytes / step_s / 1e9 / peak, 4),
                    "bytes_per_pixel": round(step_bytes / (case.mp * 1e6), 2),
                    "count": "the method's bytes per pixel: distances C s_g + 2 s_d once, then per iteration "
                             "2N (8 + s_d) for the passes and 8 + s_t for the update (z_k, t, c read)"
                             + ("; backward per iteration the forward recompute, 8N for saving the pass "
                                "inputs, 2N (20 + s_d) for the adjoint passes and 24 for the update "
                                "adjoint, then 8 + C s_g + 4C for the guide gradient" if case.bwd else ""),
                    "kernel_bytes": int(moved),
                    "kernel_frac": round(moved / step_s / 1e9 / peak, 4),
                    "kernels_without_bytes": sorted(n for n in kern if bpps[n] is None)}
    out["roofline"] = roof
    out["kernels"] = {n: {"launches": v["launches"], "avg_us": round(v["ms"] / v["launches"] * 1e3, 2),
                          "share": round(v["ms"] / tot_ms, 4)} for n, v in kern.items()}
    return out


def step_algorithmic_bytes(case, C, s_g):
    """The method's algorithmic bytes of one step (the per-pixel count of the path's design, not
    of this implementation's kernels): the distances once (C s_g in, 2 s_d out); per iteration
    2N passes of 8 + s_d (iterate read and written, distances read) and the update reading z_k, t
    and c (8 + s_t); conjugate gradients run 4N passes and three vector kernels (20, 24 and 12 bytes)
    per step; the backward adds per iteration the forward's bytes again (the pass inputs
    recomputed), 8N for keeping them, 2N adjoint passes of 20 + s_d (adjoint and pass input read,
    input adjoint written, distance adjoint updated) and 24 for the update adjoint, and once
    8 + C s_g + 4C for the guide gradient."""
    q = case.wl.params
    N, K, s_d, s_t = case.prm.passes, q.iterations, case.s_d, case.s_io
    if case.args.update == "cg":
        per_iter = 4 * N * (8 + s_d) + 20 + 24 + 12
    else:
        per_iter = 2 * N * (8 + s_d) + 8 + s_t
    bpp = C * s_g + 2 * s_d + K * per_iter
    if case.bwd:
        bpp += K * (per_iter + 8 * N + 2 * N * (20 + s_d) + 24) + 8 + C * s_g + 4 * C
    return bpp * case.mp * 1e6


def e2e_of(args, case, world, flush):
    """The same metric through the binding with pinned host inputs copied in and the result (and
    the gradients) copied out every step, L2 flushed before every solve as in the timed region."""
    import torch
    dts = case.dts
    stream = torch.cuda.current_stream()
    gh = [x.cpu().pin_memory() for x in case.g]
    th = [x.cpu().pin_memory() for x in case.t]
    ch = [x.cpu().pin_memory() for x in case.c]
    zh = [torch.empty(x.shape, dtype=torch.float32).pin_memory() for x in case.out]
    gzh = [x.cpu().pin_memory() for x in case.gz] if case.bwd else []
    n_e2e = max(1, min(args.e2e_steps, args.steps))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the binding's host pipeline overlaps each step's copies with the neighbouring steps' work
    # (every step still copies its inputs in and its results out)
    if case.bwd:
        n = len(case.g)
        gth = [torch.empty(x.shape, dtype=torch.float32).pin_memory() for x in case.out]
        gch = [torch.empty(x.shape, dtype=torch.float32).pin_memory() for x in case.out]
        ggh = [torch.empty(tuple(x.shape), dtype=torch.float32).pin_memory() for x in case.g]

        def solve_flushed(din, dout):
            flush.zero_()
            g, t, c, gz = din[:n], din[n:2 * n], din[2 * n:3 * n], din[3 * n:]
            for i in range(n):
                dts.dts_solve(g[i], t[i], c[i], case.prm, out=dout[i], ws=case.ws[0])
                dts.dts_solve_backward(g[i], t[i], c[i], case.prm, case.ws[0], gz[i],
                                       outs=(dout[n + i], dout[2 * n + i], dout[3 * n + i], None))

        hin, hout = gh + th + ch + gzh, zh + gth + gch + ggh
        copies = ("dts.HostPipeline: step i+1's host-to-device and step i-1's device-to-host copies (inputs, "
                  "incoming gradient; result and the target, confidence and guide gradients) overlap step i's "
                  "solve and backward")
    else:
        def solve_flushed(din, dout):
            flush.zero_()
            case.solve_into(din, dout)

        hin, hout = gh + th + ch, zh
        copies = ("dts.HostPipeline: step i+1's host-to-device and step i-1's device-to-host copies overlap "
                  "step i's solve")
    pipe = dts.HostPipeline(solve_flushed)
    pipe.run([hin] * 2, [hout] * 2)
    torch.cuda.synchronize()
    e0.record(stream)
    pipe.run([hin] * n_e2e, [hout] * n_e2e, start_event=e0)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    if world > 1:
        tt = torch.tensor([e2e_ms], device=case.dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        e2e_ms = float(tt.item())
    h2d, d2h = case.io_bytes()
    return {"value": round(world * n_e2e * case.mp / (e2e_ms / 1e3), 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": n_e2e, "copies": copies,
            "l2": "flushed before every solve (512 MiB write), as in the device-timed loop"}


def directions_for(args):
    """The directions a run measures: forward, and forward plus backward when the solve has a
    backward (not the batched entry point, conjugate gradients or the box kernel)."""
    has_bwd = args.workload != "batched" and args.update != "cg" and args.filter_kernel == "rf"
    if args.direction == "both":
        return ["fwd", "fwdbwd"] if has_bwd else ["fwd"]
    if args.direction == "fwdbwd" and not has_bwd:
        raise SystemExit("this solve has no backward (batched entry point, conjugate gradients or box kernel)")
    return [args.direction]


def run_ours(args, rank, world, local_rank):
    import torch

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    inp = Inputs(args, dev)
    dirs = directions_for(args)
    from paper_1805_04590_gb300 import dts as _dts
    _dts.autotune_import("batch %d\n" % (1 if args.batch_policy == "graph" else 0))
    case = Case(args, dev, inp, dirs[0])
    batch_policy = args.batch_policy
    if case.name == "batched" and batch_policy == "auto":
        batch_policy = _dts.dts_autotune_batched(case.g, case.t, case.c, case.prm, outs=case.out, ws=case.ws[0])
    main = measure(args, case, world, local_rank, flush)
    line = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": WORKLOAD_DATA[case.name],
            "config": case.config(world), "roofline": main["roofline"], "kernels": main["kernels"],
            "e2e": main["e2e"], "gpu_launches": main["gpu_launches"], "clocks": main["clocks"],
            "wall_s_timed_region": main["wall_s_timed_region"],
            "kernel_timing": f"CUDA events around each kernel on every {PROFILE_EVERY}th timed step"}
    if case.name == "batched":
        line["config"]["batch_policy"] = (batch_policy + " (measured faster by dts_autotune_batched)"
                                          if args.batch_policy == "auto" else batch_policy)
        line["gpu_launches_note"] = "one CUDA graph launch per step; its kernels are not bracketed by events"
        if batch_policy == "graph" and line["roofline"]:
            # the graph's per-image kernels run on several streams at once, so one event-timed
            # launch overlaps others and its duration says nothing of its bandwidth: the unit is
            # the whole graph, one launch per step, on the step's algorithmic bytes
            r = line["roofline"]
            st = r["step"]
            r["per_kernel_overlapped"] = {k: r[k] for k in ("kernel", "achieved", "frac", "avg_launch_us",
                                                            "algorithmic_bytes_per_launch")}
            r.update({"kernel": "graph of per-image launches (one per step)", "achieved": st["achieved"],
                      "frac": st["frac"], "algorithmic_bytes_per_launch": st["algorithmic_bytes"],
                      "bytes_per_pixel": st["bytes_per_pixel"], "avg_launch_us": round(main["ms_per_step"] * 1e3, 2),
                      "traffic": None, "share_of_step": 1.0})

    # the oracle's box filter tests every sample of a line for every position (quadratic in the
    # line length): no bounded sample of a full-size image, so no CPU baseline for that kernel
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.filter_kernel == "rf":
        import oracle
        mp, dt, desc, error = cpu_sample(args, inp, case)
        line["cpu_baseline"] = {"value": round(mp / dt, 4), "unit": UNIT, "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": desc}
        line["error"] = error
    if len(dirs) > 1:
        del case
        torch.cuda.empty_cache()
        case_b = Case(args, dev, inp, dirs[1])
        sub = measure(args, case_b, world, local_rank, flush)
        line["fwdbwd"] = {"value": sub["value"], "unit": UNIT, "ms_per_step": sub["ms_per_step"],
                          "direction": "forward solve and dts_solve_backward (gradients for target, "
                                       "confidence and guide)",
                          "backward_checkpoints": case_b.config(world)["backward_checkpoints"],
                          "roofline": sub["roofline"], "kernels": sub["kernels"], "e2e": sub["e2e"],
                          "gpu_launches": sub["gpu_launches"], "clocks": sub["clocks"],
                          "wall_s_timed_region": sub["wall_s_timed_region"]}
    return line


# ---------------------------------------------------------------- reference arm (the oracle)
def run_reference(args):
    """The FP64 oracle timed on the host cores, each step a bounded sample of the workload."""
    import oracle
    from paper_1805_04590_gb300 import workloads
    if args.update == "cg" and args.direction == "fwdbwd":
        raise SystemExit("conjugate gradients have no backward")
    if args.filter_kernel == "box":
        raise SystemExit("the reference arm times the recursive-filter solve (the oracle's box filter is quadratic "
                         "in the line length)")
    wl = workloads.make(WORKLOAD_INDEX[args.workload])
    q = wl.params
    p = wl.problems[0]
    H, W = p.target.shape
    if args.workload == "stereo":  # the centre quarter (half width, half height) of the image
        h0, w0 = H // 4, W // 4
        sl = (slice(h0, h0 + H // 2), slice(w0, w0 + W // 2))
        what = f"centre {W // 2}x{H // 2} crop of the {W}x{H} image"
    elif args.workload == "multispectral":
        sl = (slice(0, 1250), slice(0, 1250))
        what = f"1250x1250 crop (16 bands) of the {W}x{H} image"
    else:
        sl = (slice(0, H), slice(0, W))
        what = f"image 1 of {len(wl.problems)} ({W}x{H})" if len(wl.problems) > 1 else f"the {W}x{H} image"
    gi = np.ascontiguousarray(p.guide[:, sl[0], sl[1]])
    ti = np.ascontiguousarray(p.target[sl])
    ci = np.ascontiguousarray(p.conf[sl])
    if args.storage == "bf16":  # the oracle sees the same rounded values the GPU arm stores
        import torch
        gi = torch.from_numpy(gi).to(torch.bfloat16).float().numpy()
        ti = torch.from_numpy(ti).to(torch.bfloat16).float().numpy()
    mp = ti.size / 1e6
    kw = dict(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, step=q.step, iterations=q.iterations,
              passes=q.passes, charbonnier_eps=args.charbonnier_eps)
    rng = np.random.default_rng(77)
    gz = rng.standard_normal(ti.shape)

    def step():
        if args.direction == "fwdbwd":
            oracle.solve_backward(gi, ti, ci, gz, **kw)  # recomputes the forward inside
        else:
            oracle_solve(args.update, gi, ti, ci, kw)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = args.steps * mp / dt
    sample = f"{what}, full {q.iterations}-iteration FP64 {'forward+backward' if args.direction == 'fwdbwd' else 'forward'} per step"
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": WORKLOAD_DATA[args.workload],
            "config": {"workload": args.workload, "sample": sample, "iterations": q.iterations,
                       "direction": args.direction, "update": args.update, "storage": args.storage, "parallelism": "host cores"},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------- replicas across ranks
def max_over_ranks(x, world, device=None):
    """The largest x over the ranks of the process group (the slowest replica's time)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, mp_per_step, total_ms):
    """Whole-job throughput: every rank's megapixels over the slowest rank's time (MP/s)."""
    return world * steps * mp_per_step / (total_ms / 1e3)


# ---------------------------------------------------------------- sweeps
def _time_solve(torch, dts, g, t, c, prm, out, ws, flush, reps=3):
    """Median device time (ms) of one solve, L2 flushed before each."""
    dts.dts_solve(g, t, c, prm, out=out, ws=ws)
    times = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dts.dts_solve(g, t, c, prm, out=out, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    if dts.dts_last_status() != 0:
        raise RuntimeError("device status not clean")
    return sorted(times)[len(times) // 2]


def run_sweep(args):
    """The paper's scaling experiments on the stereo-shaped workload (synthetic): accuracy (MAE and
    RMSE against the generator's true disparity, and the objective of Eq. 2) and time against the
    number of iterations for the three update rules; time against sigma_s and sigma_r; time against
    the image size."""
    import torch
    from paper_1805_04590_gb300 import dts, workloads
    dev = torch.device("cuda", 0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    lines = []

    def load(wl):
        p = wl.problems[0]
        return (p, torch.from_numpy(p.guide).to(dev), torch.from_numpy(p.target).to(dev),
                torch.from_numpy(p.conf).to(dev))

    if args.sweep == "iterations":
        wl = workloads.make(1)
        q = wl.params
        p, g, t, c = load(wl)
        truth = torch.from_numpy(p.truth).to(dev).double()
        out = torch.empty_like(t)
        for upd in ("gd", "jacobi", "cg"):
            for K in (1, 2, 5, 10, 20, 50, 100, 200):
                prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, step=q.step, iterations=K,
                                 passes=q.passes, update=UPDATES[upd])
                ws = dts.workspace(g, prm)
                ms = _time_solve(torch, dts, g, t, c, prm, out, ws, flush)
                z = out.double()
                Az = dts.dts_filter(g, out, prm).double()
                F = float(0.5 * q.lam * ((z - Az) ** 2).sum() + (c.double() * (z - t.double()) ** 2).sum())
                err = z - truth
                lines.append({"sweep": "iterations", "update": upd, "iterations": K, "ms_per_solve": round(ms, 4),
                              "mae_px": round(float(err.abs().mean()), 5),
                              "rmse_px": round(float((err ** 2).mean().sqrt()), 5), "objective_eq2": F})
    elif args.sweep == "sigma":
        wl = workloads.make(1)
        q = wl.params
        _, g, t, c = load(wl)
        out = torch.empty_like(t)
        for ss, sr in [(s_, 0.1) for s_ in (16.0, 32.0, 128.0, 256.0)] + [(16.0, r_) for r_ in (0.3, 0.5, 0.7, 0.9)]:
            prm = dts.Params(lam=q.lam, sigma_s=ss, sigma_r=sr, iterations=q.iterations, passes=q.passes)
            ms = _time_solve(torch, dts, g, t, c, prm, out, dts.workspace(g, prm), flush)
            lines.append({"sweep": "sigma", "sigma_s": ss, "sigma_r": sr, "iterations": q.iterations,
                          "ms_per_solve": round(ms, 4)})
    else:
        for f in (0.25, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0, 4.18):
            H, W = int(round(1988 * f)), int(round(2880 * f))
            wl = workloads.workload_stereo(H=H, W=W)
            q = wl.params
            _, g, t, c = load(wl)
            out = torch.empty_like(t)
            prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, iterations=q.iterations, passes=q.passes)
            ms = _time_solve(torch, dts, g, t, c, prm, out, dts.workspace(g, prm), flush)
            lines.append({"sweep": "size", "H": H, "W": W, "megapixels": round(H * W / 1e6, 4),
                          "iterations": q.iterations, "ms_per_solve": round(ms, 4),
                          "mp_per_s": round(H * W / 1e6 / (ms / 1e3), 1)})
    return lines


# Small cases of the large workloads' launch plans, for profiler captures of a few launches on a
# GPU holding about a gigabyte: (H, W, channels, what runs).  tall: the 10000-row vertical plan;
# row / rowupd: the 10000-column horizontal plan (plain passes; a 2-iteration solve whose fourth
# horizontal launch is the first update pass); bwd: a solve and its reverse mode with every pass
# input kept (the 10000-row adjoint plan); stereo: 2 iterations of the stereo-shaped solve;
# batched: the first 8 images of the batched workload in one persistent launch.
NCU_CASES = {"tall": (10000, 2048, 3, "filter"), "row": (2048, 10000, 3, "filter"),
             "rowupd": (2048, 10000, 3, "solve"), "bwd": (10000, 1024, 3, "backward"),
             "stereo": (1988, 2880, 3, "solve"), "batched": (0, 0, 3, "batched"),
             "bwd16": (2048, 10000, 16, "backward")}


def run_ncu_case(args):
    import torch
    from paper_1805_04590_gb300 import dts, workloads
    H, W, C, what = NCU_CASES[args.ncu_case]
    dev = torch.device("cuda:0")
    if what == "batched":
        wl = workloads.make(3)
        q = wl.params
        probs = wl.problems[:8]
        g = [torch.from_numpy(p.guide).to(dev) for p in probs]
        t = [torch.from_numpy(p.target).to(dev) for p in probs]
        c = [torch.from_numpy(p.conf).to(dev) for p in probs]
        prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, iterations=q.iterations, passes=q.passes)
        ws = dts.batched_workspace(g, prm)
        dts.autotune_import("batch 0\n")
        run = lambda: dts.dts_solve_batched(g, t, c, prm, ws=ws)
    else:
        gen = torch.Generator(device=dev).manual_seed(0)
        g = torch.rand(C, H, W, device=dev, generator=gen)
        t = torch.rand(H, W, device=dev, generator=gen)
        c = torch.rand(H, W, device=dev, generator=gen) * 0.9 + 0.1
        prm = dts.Params(lam=0.99, sigma_s=32.0, sigma_r=0.1, passes=3, iterations=2,
                         save_checkpoints=2 if what == "backward" else 0)
        ws = dts.workspace(g, prm, with_backward=what == "backward")
        gz = torch.randn(H, W, device=dev, generator=gen)
        if what == "filter":
            run = lambda: dts.dts_filter(g, t, prm, ws=ws)
        elif what == "solve":
            run = lambda: dts.dts_solve(g, t, c, prm, ws=ws)
        else:
            run = lambda: (dts.dts_solve(g, t, c, prm, ws=ws), dts.dts_solve_backward(g, t, c, prm, ws, gz))
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    dts.dts_profile(1)
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    recs = dts.dts_profile_read()
    dts.dts_profile(0)
    status = dts.dts_last_status()
    agg = {}
    for name, _, px, fl, ms in recs:
        a = agg.setdefault(name, [0, 0.0])
        a[0] += 1
        a[1] += ms
    return {"ncu_case": args.ncu_case, "status": status,
            "kernels_us": {n: round(ms / k * 1e3, 2) for n, (k, ms) in sorted(agg.items(), key=lambda kv: -kv[1][1])}}


def main():
    args = parse_args()
    if args.ncu_case:
        line = run_ncu_case(args)
        print(json.dumps(line), flush=True)
        return 0 if line["status"] == 0 else 1
    if args.sweep:
        for line in run_sweep(args):
            print(json.dumps(line), flush=True)
        return 0
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
