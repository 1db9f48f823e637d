#!/usr/bin/env python
"""Benchmark of the Shack-Hartmann measurement on the ELT workload.

One step = one frame of the ELT-class system (800x800 px pupil at 4.875e-2 m,
obstruction 0.28; 6 LGS 80x80 WFSs with 10-px subapertures padded to 32,
16x16 detector px, 8 sodium slices; 3 H-band NGS 2x2 WFSs; 10 layers): 27,804
subaperture spots, projected, imaged, elongated, binned, made noisy and reduced
to slopes.  Inputs (2048^2 x 10 FP32 screens) are resident in HBM; L2 is
flushed (256 MB write) between timed steps, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun), each rank measures its own
independent Monte-Carlo run (replicas; no collective on the data path) and the
value is the total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SH-WFS spots/s & ELT 6-LGS frames/s at ≤1e-3 px slope err; served p50/p99"
UNIT = "spots/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
PRECISIONS = {"fp32": 0, "bf16x3": 1, "fp16s": 2}      # WFS_PREC_FP32, _BF16X3, _FP16S
WORKLOAD = ("config3 ELT frame: 800x800 px pupil (4.875e-2 m), 6 LGS 80x80 (n=10, N=32, 16x16 det px, "
            "8 Na slices) + 3 NGS 2x2 (n=32, N=64), 10 layers, noise on")
L2_FLUSH_BYTES = 256 << 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def q_dft_flops(n, nd):
    """Flops of Q = G^T M in the 32-point kernels, per subaperture: the rows |dy| < n folded
    modulo nd (2 flops per complex add), then an nd-point radix-2 DFT per column dx (nd/2
    butterflies per stage; 4 flops in the first stage, whose twiddles are 1, 10 in the others:
    a complex multiply and two complex adds)."""
    fold = 2 * max(0, (2 * n - 1) - nd) * n
    stages = int(math.log2(nd))
    return fold + n * (nd // 2) * (4 + 10 * (stages - 1))


def dft_forms(kernel, N):
    """How a spot kernel computes the dense DFT stages: U = F X with the rows k and k + N/2 paired
    ("r2": F[k + N/2][p] = F[k][p] (-1)^p i^(n-1)) in the tensor-core kernels up to N = 32 and in
    the FP32 32-point kernel, which also takes Y = U F^T and Ta = I Ga^T by column quadruples
    (m + 8j: "r4"); otherwise dense."""
    if kernel.startswith("spot_n32"):
        return {"U": "r2", "Y": "r4", "Ta": "r4"}
    if kernel.startswith("spot_tc") and not kernel.startswith("spot_tcu") and N <= 32:
        return {"U": "r2", "Y": "dense", "Ta": "dense"}
    return {"U": "dense", "Y": "dense", "Ta": "dense"}


def spot_flops(n, N, nd, lgs, kernel=""):
    """FP32 flops (FMA = 2) of one subaperture in its spot kernel: the DFT U = F X, 8Nn^2, and
    Y = U F^T, 8N^2n (together 8Nn(n+N)), |.|^2 3N^2, as each kernel computes them (dft_forms):
    U paired 4Nn^2 + 2Nn (half sums, one complex add each way); Y by quadruples 2N^2n + 4N^2
    (quarter sums, a 4-point DFT of them); Ta by quadruples N (N/4) (6 + 4 ceil(n/2) + 8 floor(n/2))
    (six adds combine the four intensities, a real coefficient for even d, a complex one for odd).
    LGS elongation and binning through the transfer function: Ta 4N^2 n, then
      32-point kernels: M as a radix-2 DFT across the lanes, 10 log2(N) N n, times the phase
      and Kt 12 (2n-1) n; Q = G^T M as a folded nd-point DFT (q_dft_flops); B = Re Q G
      4 nd^2 n; photometry 2 nd^2 (the centroid, 4 nd^2, runs in the separate noise pass);
      other sizes (direct sums): M (2n-1) n (8N+6); P = M G 8 (2n-1) nd n; B 4 nd^2 (2n-1);
      photometry and centroid 6 nd^2.
    NGS: binning N^2, photometry and centroid 6 nd^2.  Without a kernel name, every stage dense."""
    fm = dft_forms(kernel, N)
    f = (4 * N * n * n + 2 * N * n if fm["U"] == "r2" else 8 * N * n * n)
    f += (2 * N * N * n + 4 * N * N if fm["Y"] == "r4" else 8 * N * N * n) + 3 * N * N
    ta = (N * (N // 4) * (6 + 4 * ((n + 1) // 2) + 8 * (n // 2)) if fm["Ta"] == "r4" else 4 * N * N * n)
    if lgs and N == 32:
        f += ta + 10 * 5 * N * n + 12 * (2 * n - 1) * n + q_dft_flops(n, nd) + 4 * nd * nd * n
        f += 2 * nd * nd
    elif lgs:
        f += ta + (2 * n - 1) * n * (8 * N + 6) + 8 * (2 * n - 1) * nd * n + 4 * nd * nd * (2 * n - 1)
        f += 6 * nd * nd
    else:
        f += N * N + 6 * nd * nd
    return f


def dft_useful_flops(n, N):
    """Useful flops of the spot DFT Y = F X F^T with F in C^{N x n} (FMA = 2): 8 N n (n + N)."""
    return 8 * N * n * (n + N)


# Stages of the 32-point LGS spot kernels that run as tcgen05 MMAs, with their useful FP32 flops
# (FMA = 2) and the BF16 flops the MMAs issue per subaperture (tile shapes of k_sh_tc: M = 128
# rows = 4 subapertures x 32 DFT rows, so per subaperture 32 rows of each MMA).
TC_STAGES = {
    # Y = U F^T: 8 N^2 n useful; issued N = 64, K = 64 (three split products in one K atom)
    "Y": (lambda n, N, nd: 8 * N * N * n, lambda n, N, nd: 2 * 32 * 64 * 64),
    # Ta = I Ga^T: 4 N^2 n useful; issued two chains of N = 32, K = 64
    "Ta": (lambda n, N, nd: 4 * N * N * n, lambda n, N, nd: 2 * 2 * 32 * 32 * 64),
    # U = F X: 8 N n^2 useful; issued four MMAs of M = 128 per 4 subapertures (one per
    # subaperture's field tile), N = 32, K = 64
    "U": (lambda n, N, nd: 8 * N * n * n, lambda n, N, nd: 2 * 128 * 32 * 64),
}


def tc_stages(kernel_name):
    """The MMA stages of a spot kernel (by its timing name)."""
    if kernel_name.startswith("spot_tcu"):
        return ("U", "Y", "Ta")
    if kernel_name.startswith("spot_tc"):
        return ("Y", "Ta")
    return ()


def source_sha(names):
    h = hashlib.sha256()
    for nm in names:
        with open(os.path.join(ROOT, "paper_1408_0698_gb300", "csrc", nm), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {"spot": ["k_sh.cu", "noise.cuh", "proj_math.cuh", "internal.h"],
                  "spot_n32": ["k_sh_n32.cu", "spot_tail.cuh", "noise.cuh", "internal.h"],
                  "spot_tc": ["k_sh_tc.cu", "spot_tail.cuh", "noise.cuh", "internal.h", "tcgen05.cuh"],
                  "spot_tc64": ["k_sh_tc64.cu", "noise.cuh", "proj_math.cuh", "internal.h", "tcgen05.cuh"],
                  "noise_cog": ["k_noise_cog.cu", "spot_tail.cuh", "noise.cuh", "internal.h"],
                  "project": ["k_project_bulk.cu", "k_project.cu", "proj_direct.cuh", "proj_math.cuh", "internal.h",
                              "tcgen05.cuh"],
                  "gemv": ["k_loop.cu", "proj_math.cuh", "internal.h"],
                  "dm_layer": ["k_loop.cu", "proj_math.cuh", "internal.h"],
                  "uplink": ["k_uplink.cu", "proj_math.cuh", "internal.h"]}


def ncu_traffic(kernel_key):
    """Per-launch DRAM bytes of a kernel from profiles/traffic.txt, if the kernel's
    sources still hash to what was profiled; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    want = source_sha(KERNEL_SOURCES[kernel_key])
    for line in open(p):
        parts = line.split("#")[0].split()
        if len(parts) == 3 and parts[0] == kernel_key and parts[2] == want:
            return float(parts[1])
    return None


class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(cfg, scr, t, target_s=12.0):
    """The FP64 oracle on this host's cores, over a bounded sample of the ELT frame: every k-th
    subaperture of each LGS WFS plus all NGS subapertures.  The elongation runs in the oracle's
    separable form (pinned equal to its direct periodic convolution), as the timing plan asks."""
    import oracle
    oracle.set_separable(True)
    try:
        return _cpu_baseline(oracle, cfg, scr, t, target_s)
    finally:
        oracle.set_separable(False)


def _cpu_baseline(oracle, cfg, scr, t, target_s):
    nthreads = oracle.num_threads()
    t0 = time.perf_counter()
    oracle.measure_wfs(cfg, scr, 0, t, seed=cfg.seed, noise=True, sel=np.arange(0, 4632, 97, dtype=np.int32))
    per = (time.perf_counter() - t0) / len(range(0, 4632, 97))
    n_lgs_per_wfs = max(1, int(target_s / per / 6))
    stride = max(1, 4632 // n_lgs_per_wfs)
    spots = 0
    t0 = time.perf_counter()
    for w, s in enumerate(cfg.stars):
        if s.is_lgs:
            sel = np.arange(w % stride, 4632, stride, dtype=np.int32)
            oracle.measure_wfs(cfg, scr, w, t, seed=cfg.seed, noise=True, sel=sel)
            spots += len(sel)
        else:
            spots += len(oracle.measure_wfs(cfg, scr, w, t, seed=cfg.seed, noise=True)["slopes"])
    dt = time.perf_counter() - t0
    # the same oracle on one core, over a sixteenth of that sample (LGS subapertures only)
    oracle.set_threads(1)
    try:
        sel = np.arange(0, 4632, stride * 16, dtype=np.int32)
        t1 = time.perf_counter()
        oracle.measure_wfs(cfg, scr, 0, t, seed=cfg.seed, noise=True, sel=sel)
        dt1 = time.perf_counter() - t1
    finally:
        oracle.set_threads(nthreads)
    return {"value": spots / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"{spots} spots of one ELT frame (every {stride}th LGS subaperture of 6 WFSs "
                      f"+ all 12 NGS subapertures), FP64, separable elongation, noise on, {dt:.1f} s",
            "single_thread": {"value": len(sel) / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"{len(sel)} LGS subapertures of WFS 0, {dt1:.1f} s"}}


def replica_throughput(local_ms, spots_per_step, steps, world, dev):
    """Whole-job throughput of `world` replicas: every rank measured `steps` steps of its own
    run in local_ms; the job's time is the slowest rank's (all-reduce MAX)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return world * spots_per_step * steps / (ms_max / 1e3), world * steps / (ms_max / 1e3), ms_max


def served(load=0.8, duration_s=20.0, n_runs=32, budget_gb=150.0, slots=3, other_loads=(0.5, 0.95),
           small_budget_gb=1.0, other_duration_s=4.0):
    """Continuous-batching serving of frame requests from n_runs concurrent MC runs drawn from
    configs 1-3, device-resident (admitted by HBM footprint), Poisson arrivals at `load` times
    the measured batched capacity over duration_s of traffic; p50/p99 latency and served
    throughput.  Also the other offered loads, and `load` under a small HBM budget at which
    admission binds (runs wait for earlier runs to retire), over other_duration_s each."""
    from paper_1408_0698_gb300 import serving
    runs = serving.make_runs(n_runs, 5000)
    budget = int(budget_gb * (1 << 30))
    cap = serving.capacity(runs, budget, slots)

    def one(ld, bud, preadmit=True, dur=other_duration_s):
        arrivals = serving.poisson_arrivals(runs, ld * cap / n_runs, dur, seed=11)
        srv = serving.Server(runs, bud, slots)
        if preadmit:
            srv.preadmit()
        return srv.serve(arrivals).summary()

    st = one(load, budget, dur=duration_s)
    st.update({"traffic_s": duration_s, "other_traffic_s": other_duration_s, "load": load, "capacity_frames_per_s": cap, "runs": n_runs, "budget_gb": budget_gb,
               "slots": slots, "mix": "configs 1-3 (seeded)"})
    keys = ("p50_ms", "p99_ms", "frames_per_s", "spots_per_s", "mean_batch", "max_admitted")
    st["other_loads"] = [dict({"load": ld}, **{k: v for k, v in one(ld, budget).items() if k in keys})
                         for ld in other_loads]
    small = one(load, int(small_budget_gb * (1 << 30)), preadmit=False)
    st["small_budget"] = dict({"load": load, "budget_gb": small_budget_gb},
                              **{k: v for k, v in small.items() if k in keys + ("requests",)})
    return st


def reference_arm(args):
    """The oracle on the host cores, on bounded samples of the ELT frame (one per step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_1408_0698_gb300 import inputs
    cfg = inputs.config3(inputs.PREC_FP32)
    scr = inputs.make_screens(cfg.layers, cfg.seed)
    oracle.set_separable(True)  # the timing form of the elongation (pinned equal to the direct one)
    budget = 150.0 / max(1, args.steps + args.warmup)
    t0 = time.perf_counter()
    oracle.measure_wfs(cfg, scr, 0, 0.0, seed=cfg.seed, noise=True, sel=np.arange(0, 4632, 193, dtype=np.int32))
    per = (time.perf_counter() - t0) / len(range(0, 4632, 193))
    per_step = max(1, min(4632, int(budget / per)))  # subapertures of one LGS WFS per step
    rng = np.random.default_rng(0)

    def step(k):
        w = k % 6
        sel = np.sort(rng.choice(4632, size=per_step, replace=False)).astype(np.int32)
        oracle.measure_wfs(cfg, scr, w, k * cfg.dt_s, seed=cfg.seed, noise=True, sel=sel)
        return len(sel)

    for k in range(args.warmup):
        step(k)
    spots = 0
    t0 = time.perf_counter()
    for k in range(args.steps):
        spots += step(args.warmup + k)
    dt = time.perf_counter() - t0
    v = spots / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_spots_per_step": per_step},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{per_step} subapertures of one LGS WFS per step (the six in "
                                       f"turn), FP64 oracle, separable elongation"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def closed_loop(cfg, s_d, flush, args, dev, rank):
    """The closed loop on the same ELT frame (Sec. 3 "The closed loop"): each step measures the
    residual through three mirrors (ground, 81 x 81 actuators, 5000 modes; 4 km, 43 x 43, 1400;
    12.7 km, 50 x 50, 1800), multiplies the slopes by an 8200 x 55608 FP32 control matrix and
    integrates (gain 0.3), then rebuilds the actuator commands and the mirror layers.  The
    modal bases are seeded Gaussian patterns, the control matrix seeded uniform values on the
    device (a calibrated matrix of that size times the same)."""
    import torch

    from paper_1408_0698_gb300 import inputs, native
    dms = inputs.elt_dms()
    m2a = [torch.as_tensor(inputs.modal_base(d, cfg.seed + 50 + i)).to(dev) for i, d in enumerate(dms)]
    n = sum(d.n_modes for d in dms)
    w = native.Wfs(cfg, seed=cfg.seed + rank, noise=True)
    ns = 2 * w.total
    g = torch.Generator(device=dev)
    g.manual_seed(cfg.seed + 60)
    cm = (torch.rand((n, ns), generator=g, device=dev) * 2.0 - 1.0) * (1e-3 / math.sqrt(ns))
    gain = torch.full((n,), 0.3, device=dev)
    structs = [native.wfs_dm(d.n_act, d.pitch_m, d.alt_m, d.coupling, d.support, d.n_modes, M.data_ptr())
               for d, M in zip(dms, m2a)]
    lp = native.wfs_loop_create(w.h, structs, cm.data_ptr(), gain.data_ptr())
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    slopes = torch.empty((w.total, 2), device=dev)
    dt = cfg.dt_s
    for k in range(5):
        native.wfs_loop_step(lp, w.h, s_d.data_ptr(), k * dt, slopes.data_ptr(), sp)
    torch.cuda.synchronize()
    native.wfs_sync_status(w.h)
    kl = min(args.steps, 300)
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(kl)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(kl)]
    # steps with no event between kernels, then per-kernel durations from 30 more with events
    for k in range(kl):
        if args.flush_mb:
            flush.fill_(float(k))
        e0[k].record(stream)
        native.wfs_loop_step(lp, w.h, s_d.data_ptr(), (5 + k) * dt, slopes.data_ptr(), sp)
        e1[k].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in zip(e0, e1))
    native.wfs_timing_enable(w.h, True)
    native.wfs_timing_read(w.h)
    for k in range(min(kl, 30)):
        if args.flush_mb:
            flush.fill_(float(k))
        native.wfs_loop_step(lp, w.h, s_d.data_ptr(), (5 + kl + k) * dt, slopes.data_ptr(), sp)
    torch.cuda.synchronize()
    kt = native.wfs_timing_read(w.h)
    native.wfs_timing_enable(w.h, False)
    native.wfs_sync_status(w.h)
    pk, kind = peaks()
    roof = None
    if "reconstruct" in kt:
        launches, tot_ms = kt["reconstruct"]
        avg_s = tot_ms / launches / 1e3
        # algorithmic bytes: the control matrix once, the slopes, gains, coefficients read + written
        nbytes = 4 * (n * ns + ns + n + 2 * n)
        ach = nbytes / avg_s / 1e9
        roof = {"kernel": "reconstruct", "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": ach / pk["hbm_gbs"], "traffic": ncu_traffic("gemv"),
                "bytes_per_launch": nbytes, "avg_launch_ms": avg_s * 1e3, "peak_source": kind}
    # eight Monte-Carlo runs of the same system as one batch: the control matrix and the modal
    # bases are read once per four loops
    nb = 8
    hs = [native.Wfs(cfg, seed=cfg.seed + 100 + i, noise=True) for i in range(nb)]
    lps = [native.wfs_loop_create(x.h, structs, cm.data_ptr(), gain.data_ptr()) for x in hs]
    bt = native.wfs_loop_batch_create(lps)
    scr_b = [s_d] * nb
    sl_b = [torch.empty((w.total, 2), device=dev) for _ in range(nb)]
    for k in range(3):
        native.wfs_loop_batch_step(bt, [x.data_ptr() for x in scr_b], [k * dt] * nb, [x.data_ptr() for x in sl_b], sp)
    torch.cuda.synchronize()
    kb = min(kl, 60)
    for k in range(kb):
        if args.flush_mb:
            flush.fill_(float(k))
        e0[k].record(stream)
        native.wfs_loop_batch_step(bt, [x.data_ptr() for x in scr_b], [(3 + k) * dt + 1e-4 * i for i in range(nb)],
                                   [x.data_ptr() for x in sl_b], sp)
        e1[k].record(stream)
    torch.cuda.synchronize()
    ms_b = sum(a.elapsed_time(b) for a, b in zip(e0[:kb], e1[:kb]))
    for x in hs:
        native.wfs_sync_status(x.h)
    native.wfs_loop_batch_destroy(bt)
    for x, y in zip(lps, hs):
        native.wfs_loop_destroy(x)
        y.close()
    batch = {"loops": nb, "steps": kb, "ms_per_batch_step": ms_b / kb,
             "loop_steps_per_s": nb * kb / (ms_b / 1e3), "spots_per_s": nb * w.total * kb / (ms_b / 1e3),
             "note": "one screen set shared by the eight runs (memory); each run has its own handle, seed, "
                     "mirrors and coefficients"}
    out = {"workload": "config3 ELT frame + 3 mirrors (5000 + 1400 + 1800 modes), control matrix "
                       f"{n} x {ns} FP32, gain 0.3, noise on",
           "batch": batch,
           "steps": kl, "ms_per_step": ms / kl, "steps_per_s": kl / (ms / 1e3),
           "spots_per_s": w.total * kl / (ms / 1e3),
           "kernels": {k: {"launches": v[0], "avg_ms": v[1] / max(1, v[0])} for k, v in kt.items()},
           "reconstruct_roofline": roof}
    native.wfs_loop_destroy(lp)
    w.close()
    return out


def calibration(cfg, args, dev, rank):
    """Push-pull registration of the interaction matrix of the ground mirror (81 x 81 actuators,
    5000 modes) with one 80 x 80 LGS of the ELT frame -- the calibration the paper times (Sec. 5:
    5000 modes, 80 x 80 subapertures, one LGS, about 14 hours).  Two measurements per mode, no
    noise, no turbulence; timed with CUDA events after one untimed registration."""
    import torch

    from paper_1408_0698_gb300 import inputs, native
    dm = inputs.elt_dms()[0]
    M = torch.as_tensor(inputs.modal_base(dm, cfg.seed + 70)).to(dev)
    w = native.Wfs(cfg, seed=cfg.seed + rank, noise=False)
    ns = 2 * w.total
    cm = torch.zeros((dm.n_modes, ns), device=dev)
    gain = torch.zeros(dm.n_modes, device=dev)
    lp = native.wfs_loop_create(w.h, [native.wfs_dm(dm.n_act, dm.pitch_m, dm.alt_m, dm.coupling, dm.support,
                                                    dm.n_modes, M.data_ptr())], cm.data_ptr(), gain.data_ptr())
    nv = native.wfs_num_valid(w.h, 0)
    im = torch.empty((dm.n_modes, 2 * nv), device=dev)
    sp = torch.cuda.current_stream(dev).cuda_stream
    native.wfs_loop_calibrate(lp, w.h, 0, 1.0, im.data_ptr(), sp)
    torch.cuda.synchronize()
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        native.wfs_loop_calibrate(lp, w.h, 0, 1.0, im.data_ptr(), sp)
    e1.record()
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1e3 / reps
    # per-kernel durations from one more registration with the library's events
    native.wfs_timing_enable(w.h, True)
    native.wfs_timing_read(w.h)
    native.wfs_loop_calibrate(lp, w.h, 0, 1.0, im.data_ptr(), sp)
    torch.cuda.synchronize()
    native.wfs_sync_status(w.h)
    kt = native.wfs_timing_read(w.h)
    native.wfs_timing_enable(w.h, False)
    native.wfs_loop_destroy(lp)
    w.close()
    return {"workload": f"ground mirror {dm.n_act}x{dm.n_act} actuators, {dm.n_modes} modes, push-pull with LGS 0 "
                        f"of the ELT frame ({nv} subapertures, BF16x3 spots), no noise",
            "seconds": s, "modes_per_s": dm.n_modes / s, "spots_per_s": 2 * dm.n_modes * nv / s,
            "repetitions": reps, "paper_seconds": 14 * 3600.0,
            "kernels": {k: {"launches": v[0], "avg_ms": v[1] / max(1, v[0])} for k, v in kt.items()}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "bf16x3", "fp16s"],
                    help="DFT arithmetic of the LGS geometry for the headline (the others are timed beside it)")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-served", action="store_true", help="skip the served-traffic measurement")
    ap.add_argument("--no-loop", action="store_true", help="skip the closed-loop measurement")
    ap.add_argument("--no-calib", action="store_true", help="skip the push-pull calibration measurement")
    ap.add_argument("--paths", default="fp32,fp16s,uplink,slices,configs,batch",
                    help="comparison paths timed after the headline (comma list of fp32, fp16s, uplink, "
                         "slices, configs, batch; 'none'); fp32 and fp16s time the other DFT precisions, "
                         "configs the single-instance configs 1 and 2, batch the uneven config-4 batch")
    ap.add_argument("--flush-mb", type=int, default=L2_FLUSH_BYTES >> 20,
                    help="L2 flush buffer written between timed steps (0: none, for profiling runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    assert args.warmup >= 3, "at least 3 warm-up steps"

    import torch
    import torch.distributed as dist

    from paper_1408_0698_gb300 import inputs, native

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    prec = PRECISIONS[args.precision]
    cfg = inputs.config3(prec)
    scr = inputs.make_screens(cfg.layers, cfg.seed + 17 * rank)   # one MC run per rank
    w = native.Wfs(cfg, seed=cfg.seed + rank, noise=True)
    spots = w.total
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    s_d = torch.as_tensor(scr).to(dev)
    slopes = torch.empty((spots, 2), device=dev)
    flush = torch.empty(max(1, args.flush_mb << 18), dtype=torch.float32, device=dev)
    dt = cfg.dt_s

    for k in range(args.warmup):
        native.wfs_measure(w.h, s_d.data_ptr(), k * dt, slopes.data_ptr(), sp)
    torch.cuda.synchronize()
    native.wfs_sync_status(w.h)

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        if args.flush_mb:
            flush.fill_(float(k))
        ev0[k].record(stream)
        native.wfs_measure(w.h, s_d.data_ptr(), (args.warmup + k) * dt, slopes.data_ptr(), sp)
        ev1[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    native.wfs_sync_status(w.h)
    ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    value, frames, ms_max = replica_throughput(ms, spots, args.steps, world, dev)

    # per-kernel durations: the same steps again with the library's CUDA events around every
    # launch, on each launch's own stream.  Events between kernels stop the programmatic
    # dependent launches from overlapping a kernel's prologue with its predecessor, so the
    # headline steps above run without them.
    kk = min(args.steps, 500)
    native.wfs_timing_enable(w.h, True)
    native.wfs_timing_read(w.h)
    torch.cuda.synchronize()
    for k in range(kk):
        if args.flush_mb:
            flush.fill_(float(k))
        ev0[k].record(stream)
        native.wfs_measure(w.h, s_d.data_ptr(), (args.warmup + k) * dt, slopes.data_ptr(), sp)
        ev1[k].record(stream)
    torch.cuda.synchronize()
    native.wfs_timing_enable(w.h, False)
    ktimes = native.wfs_timing_read(w.h)
    native.wfs_sync_status(w.h)
    ms_k = sum(a.elapsed_time(b) for a, b in zip(ev0[:kk], ev1[:kk]))

    # e2e: host buffers through wfs_measure_host, copies inside the timed region
    host_scr = torch.as_tensor(scr).pin_memory()
    host_sl = torch.empty((spots, 2)).pin_memory()
    ke = max(3, min(args.e2e_steps, args.steps))
    for k in range(3):
        native.wfs_measure_host(w.h, host_scr.data_ptr(), k * dt, host_sl.data_ptr(), sp)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    e0.record(stream)
    h2d = d2h = 0
    for k in range(ke):
        native.wfs_measure_host(w.h, host_scr.data_ptr(), k * dt, host_sl.data_ptr(), sp)
        b_in, b_out = native.wfs_host_transfer_bytes(w.h)  # the library copies only what the frame reads
        h2d += b_in
        d2h += b_out
    e1.record(stream)
    torch.cuda.synchronize()
    e_ms = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(e_ms, op=dist.ReduceOp.MAX)
    e2e = {"value": world * spots * ke / (float(e_ms.item()) / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(round(h2d / ke)), "d2h_bytes_per_step": int(round(d2h / ke)),
           "host_input_bytes_per_step": int(host_scr.numel() * 4), "steps": ke}
    if h2d == 0:
        # the pinned host screens are mapped into the GPU's address space and the kernels read
        # what they need in place: the bytes that cross the host link are the screen pixels the
        # frame's bilinear taps touch (at least; the link moves whole sectors)
        maps = [native.wfs_valid_map(w.h, k) for k in range(len(cfg.stars))]
        _, scr_b, _ = projection_footprint_bytes(cfg, maps, (args.warmup + ke) * dt, all_stars=True)
        e2e["h2d_bytes_per_step"] = int(scr_b)
        e2e["h2d_note"] = ("screens read in place by the kernels from pinned host memory (no copy); "
                           "bytes = the screen pixels the frame's taps touch")

    # roofline of the dominant kernel (the spot launch with the most work; launches of other
    # geometries run concurrently on side streams, so event windows overlap), from the live
    # per-kernel events recorded on each launch's own stream
    pk, kind = peaks()

    def spot_work(name):
        N = int(name.split("N")[-1])
        f = 0
        for k, s in enumerate(cfg.stars):
            g = cfg.geometries[s.geometry_index]
            if g.n_fft == N:
                f += w.layouts[k].n_valid * spot_flops(g.n_pix_sub, g.n_fft, g.n_det, s.is_lgs, name)
        return f

    spots_k = {k: v for k, v in ktimes.items() if k.startswith("spot_")}
    roof = None
    if spots_k:
        name = max(spots_k, key=spot_work)
        roof = spot_roofline(name, ktimes[name], cfg, w, pk, kind)
    if "project" in ktimes:
        if roof is not None:
            roof["projection"] = projection_roofline(ktimes["project"], cfg, w, pk, kind, args.warmup * dt)
    if "noise_cog" in ktimes:
        # the noise-and-centroid pass: detector pixels of the 32-point subapertures per second
        launches, tot_ms = ktimes["noise_cog"]
        px = sum(w.layouts[k].n_valid * cfg.geometries[s.geometry_index].n_det ** 2
                 for k, s in enumerate(cfg.stars) if cfg.geometries[s.geometry_index].n_fft == 32)
        if roof is not None:
            roof["noise_pass"] = {"avg_launch_ms": tot_ms / launches, "pixels_per_launch": px,
                                  "gpixels_per_s": px / (tot_ms / launches / 1e3) / 1e9,
                                  "traffic": ncu_traffic("noise_cog")}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "spots_per_frame": spots, "dft_precision": args.precision,
                       "l2": (f"flushed between timed steps ({args.flush_mb} MB write, outside the step events)"
                              if args.flush_mb else "not flushed (profiling run)"),
                       "replicas": world},
            "frames_per_s": frames,
            "kernels": {k: {"launches": v[0], "avg_ms": v[1] / max(1, v[0])} for k, v in ktimes.items()},
            "kernel_timing_pass": {"steps": kk, "ms_per_step": ms_k / kk,
                                   "note": "per-kernel events recorded on each launch's stream; without "
                                           "programmatic dependent launch overlap"},
            # the timed steps launch what the timing pass counted, per step
            "gpu_launches": int(round(sum(v[0] for v in ktimes.values()) / kk * args.steps)),
            "roofline": roof, "e2e": e2e, "clocks": clk, "wall_s_timed": wall}
    paths = set(args.paths.split(","))
    # the other DFT precisions, timed the same way on the same inputs (comparison paths; the
    # "fp32" path times BF16 x3 when the headline is FP32)
    for key in ("fp32", "fp16s"):
        other = key if args.precision != key else "bf16x3"
        if key in paths and other != args.precision:
            time_other_precision(line, other, cfg, rank, s_d, slopes, sp, stream, flush, ev0, ev1, spots, args, dt)
    if "uplink" in paths:
        time_uplink(line, cfg, rank, s_d, slopes, sp, stream, flush, ev0, ev1, spots, args, dt)
    if "slices" in paths:
        time_per_slice(line, cfg, rank, s_d, slopes, sp, stream, flush, ev0, ev1, spots, args, dt)
    if "configs" in paths and world == 1:
        line.update(single_configs(args, dev, flush, ev0, ev1))
    if "batch" in paths and world == 1:
        line["batch"] = batch_leg(args, dev, flush)
    if not args.no_loop:
        line["closed_loop"] = closed_loop(cfg, s_d, flush, args, dev, rank)
    if not args.no_calib:
        line["calibration"] = calibration(cfg, args, dev, rank)
    if not args.no_served:
        line["served"] = served()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, scr, 0.0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    w.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def spot_roofline(name, timing, cfg, w, pk, kind):
    """Roofline of a spot launch from its live per-launch time: the CUDA-core flops (the
    algorithmic flops minus those of the stages that run as MMAs) against the FP32 peak (the
    bound), and beside it the DFT's useful flops 8 N n (n + N) against the measured BF16
    tensor peak, with the BF16 flops the MMAs issue."""
    launches, tot_ms = timing
    avg_s = tot_ms / launches / 1e3
    N = int(name.split("N")[-1])
    stages = tc_stages(name)
    total = cuda = useful = issued = 0
    for k, s in enumerate(cfg.stars):
        g = cfg.geometries[s.geometry_index]
        if g.n_fft != N:
            continue
        nv = w.layouts[k].n_valid
        n, nd = g.n_pix_sub, g.n_det
        f = spot_flops(n, N, nd, s.is_lgs, name)
        on_tc = sum(TC_STAGES[st][0](n, N, nd) for st in stages) if s.is_lgs else 0
        total += nv * f
        cuda += nv * (f - on_tc)
        useful += nv * dft_useful_flops(n, N)
        issued += nv * sum(TC_STAGES[st][1](n, N, nd) for st in stages) if s.is_lgs else 0
    ach = cuda / avg_s / 1e12
    roof = {"kernel": name, "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP32_PEAK_TFLOPS,
            "traffic": ncu_traffic("spot_n32" if name.startswith("spot_n32") else
                                   "spot_tc" if name.startswith("spot_tc") else "spot"),
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
            "flops_per_launch": cuda, "flops_note": "CUDA-core flops only (the MMA stages excluded)",
            "algorithmic_flops_per_launch": total, "avg_launch_ms": avg_s * 1e3}
    if stages:
        t_use = useful / avg_s / 1e12
        t_iss = issued / avg_s / 1e12
        roof["tensor_pipe"] = {"useful_dft_flops_per_launch": useful, "achieved": t_use,
                               "peak": pk["bf16_tflops"], "unit": "TFLOP/s", "frac": t_use / pk["bf16_tflops"],
                               "issued_bf16_flops_per_launch": issued, "issued_achieved": t_iss,
                               "issued_frac": t_iss / pk["bf16_tflops"], "mma_stages": list(stages),
                               "peak_source": f"{kind} (burst)"}
    return roof


def projection_footprint_bytes(cfg, valid_maps, t, all_stars=False):
    """Algorithmic bytes of one projection launch of the 32-point group (or, with all_stars,
    of every star's projection): every screen pixel that the bilinear taps of the valid pupil
    pixels touch, counted once per layer (4 B), plus the projected OPD written (4 B per valid
    pupil pixel).  valid_maps[k]: star k's valid subaperture indices (row-major)."""
    L = cfg.layers
    S, ds = L.screen_size, L.screen_dx_m
    tel = cfg.telescope
    touched = 0
    opd_bytes = 0
    members = [k for k, s in enumerate(cfg.stars) if all_stars or cfg.geometries[s.geometry_index].n_fft == 32]
    for l in range(L.n_layers):
        mask = np.zeros((S, S), bool)
        h = L.alt_m[l]
        for k in members:
            s = cfg.stars[k]
            g = cfg.geometries[s.geometry_index]
            n, ns = g.n_pix_sub, g.n_sub
            Np = ns * n
            dx = tel.diameter_m / Np
            idx = np.asarray(valid_maps[k])
            sy, sx = np.divmod(idx, ns)
            p, q = np.mgrid[0:n, 0:n]
            i = (sy[:, None, None] * n + p[None]).ravel()
            j = (sx[:, None, None] * n + q[None]).ravel()
            if l == 0:
                opd_bytes += 4 * i.size
            x = (j - (Np - 1) / 2.0) * dx
            y = (i - (Np - 1) / 2.0) * dx
            c = 1.0 - h / s.range_m if s.is_lgs else 1.0
            u = S / 2.0 + (c * x + s.theta_x_rad * h - (L.x0_m[l] + L.wind_vx_mps[l] * t)) / ds
            v = S / 2.0 + (c * y + s.theta_y_rad * h - (L.y0_m[l] + L.wind_vy_mps[l] * t)) / ds
            iu = np.floor(u).astype(np.int64)
            iv = np.floor(v).astype(np.int64)
            for a in (0, 1):
                for b in (0, 1):
                    mask[(iv + b) % S, (iu + a) % S] = True
        touched += int(mask.sum())
    return 4 * touched + opd_bytes, 4 * touched, opd_bytes


def projection_roofline(timing, cfg, w, pk, kind, t):
    """HBM roofline of the projection: algorithmic bytes (unique screen footprint + OPD) over
    its live per-launch time, against the measured copy bandwidth."""
    launches, tot_ms = timing
    avg_s = tot_ms / launches / 1e3
    from paper_1408_0698_gb300 import native
    maps = [native.wfs_valid_map(w.h, k) for k in range(len(cfg.stars))]
    tot, scr_b, opd_b = projection_footprint_bytes(cfg, maps, t)
    gbs = tot / avg_s / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
            "bytes_per_launch": tot, "screen_footprint_bytes": scr_b, "opd_bytes": opd_b,
            "avg_launch_ms": avg_s * 1e3, "traffic": ncu_traffic("project"), "peak_source": kind}


def time_frames(w, s_d, slopes, sp, stream, flush, ev0, ev1, args, dt, steps, kernel_steps=30):
    """ms per frame of handle w: `steps` frames with no event between the kernels of a frame
    (events there stop the programmatic dependent launches from overlapping), then per-kernel
    durations from `kernel_steps` more frames with the library's events around every launch."""
    import torch

    from paper_1408_0698_gb300 import native
    for k in range(3):
        native.wfs_measure(w.h, s_d.data_ptr(), k * dt, slopes.data_ptr(), sp)
    torch.cuda.synchronize()
    for k in range(steps):
        if args.flush_mb:
            flush.fill_(float(k))
        ev0[k].record(stream)
        native.wfs_measure(w.h, s_d.data_ptr(), (args.warmup + k) * dt, slopes.data_ptr(), sp)
        ev1[k].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in zip(ev0[:steps], ev1[:steps])) / steps
    native.wfs_timing_enable(w.h, True)
    native.wfs_timing_read(w.h)
    for k in range(min(kernel_steps, steps)):
        if args.flush_mb:
            flush.fill_(float(k))
        native.wfs_measure(w.h, s_d.data_ptr(), (args.warmup + k) * dt, slopes.data_ptr(), sp)
    torch.cuda.synchronize()
    native.wfs_timing_enable(w.h, False)
    kt = native.wfs_timing_read(w.h)
    native.wfs_sync_status(w.h)
    return ms, {k: {"launches": v[0], "avg_ms": v[1] / max(1, v[0])} for k, v in kt.items()}


def batch_leg(args, dev, flush, n_inst=64, steps=200):
    """Config 4: n_inst uneven instances (2x2 / 10x10 / 40x40 / 80x80 subapertures, DFT sizes
    16-64, 1-10 layers, LGS and NGS) measured together by wfs_batch_measure (one projection
    launch and one spot launch per kernel class, replayed as a CUDA graph), after
    wfs_batch_tune has picked the launch shapes; BF16 x3 (geometries without a tensor-core
    kernel stay FP32) against all FP32.  L2 flushed between steps."""
    import torch

    from paper_1408_0698_gb300 import inputs, native
    out = {}
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    for name, prec in (("bf16x3", inputs.PREC_BF16X3), ("fp32", inputs.PREC_FP32)):
        insts = inputs.config4_instances(n_inst, 4000, precision=prec)
        hs, scr, outs, ts = [], [], [], []
        n_tc = 0
        for i, c in enumerate(insts):
            try:
                w = native.Wfs(c, seed=c.seed, noise=True)
                n_tc += prec != inputs.PREC_FP32
            except native.WfsError as e:
                if e.status != native.WFS_EUNSUPPORTED:
                    raise
                c.geometries[0].precision = inputs.PREC_FP32
                w = native.Wfs(c, seed=c.seed, noise=True)
            hs.append(w)
            scr.append(torch.as_tensor(inputs.make_screens(c.layers, c.seed)).to(dev))
            outs.append(torch.zeros((max(w.total, 1), 2), device=dev))
        spots = sum(w.total for w in hs)
        b = native.wfs_batch_create([w.h for w in hs])
        sps, ops = [x.data_ptr() for x in scr], [o.data_ptr() for o in outs]
        native.wfs_batch_tune(b, sps, [0.0] * len(hs), ops, sp)
        for k in range(5):
            native.wfs_batch_measure(b, sps, [k * 1e-3] * len(hs), ops, sp)
        torch.cuda.synchronize()
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for k in range(steps):
            flush.fill_(float(k))
            e0[k].record(stream)
            native.wfs_batch_measure(b, sps, [(5 + k) * 1e-3] * len(hs), ops, sp)
            e1[k].record(stream)
        torch.cuda.synchronize()
        ms = sum(x.elapsed_time(y) for x, y in zip(e0, e1)) / steps
        info = native.wfs_batch_info(b)
        native.wfs_batch_destroy(b)
        # each kernel class alone (its instances as a batch of their own, one projection and one
        # spot launch): how much the classes overlap in the graph, i.e. what one persistent launch
        # over all classes could still gain
        per_class = []
        groups = {}
        for i, c in enumerate(insts):
            g = c.geometries[0]
            groups.setdefault((g.precision, g.n_pix_sub, g.n_fft, g.n_det), []).append(i)
        for key, idx in sorted(groups.items()):
            bc = native.wfs_batch_create([hs[i].h for i in idx])
            sp_c, op_c = [sps[i] for i in idx], [ops[i] for i in idx]
            native.wfs_batch_tune(bc, sp_c, [0.0] * len(idx), op_c, sp)
            for k in range(3):
                native.wfs_batch_measure(bc, sp_c, [k * 1e-3] * len(idx), op_c, sp)
            torch.cuda.synchronize()
            kc = min(steps, 100)
            for k in range(kc):
                flush.fill_(float(k))
                e0[k].record(stream)
                native.wfs_batch_measure(bc, sp_c, [(5 + k) * 1e-3] * len(idx), op_c, sp)
                e1[k].record(stream)
            torch.cuda.synchronize()
            per_class.append({"precision": key[0], "n_pix_sub": key[1], "n_fft": key[2], "n_det": key[3],
                              "instances": len(idx), "spots": sum(hs[i].total for i in idx),
                              "ms_per_step": sum(x.elapsed_time(y) for x, y in zip(e0[:kc], e1[:kc])) / kc})
            native.wfs_batch_destroy(bc)
        for w in hs:
            w.close()
        out[name] = {"value": spots / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
                     "spots_per_step": spots, "instances": len(hs), "instances_on_tensor_cores": n_tc,
                     "classes": [{k: c[k] for k in ("kind", "n_pix_sub", "n_fft", "n_det", "n_wfs", "n_subaps", "grid_cap", "cta_warps")
                                  if k in c} for c in info],
                     "classes_alone": per_class,
                     "sum_of_classes_alone_ms": sum(c["ms_per_step"] for c in per_class),
                     "largest_class_alone_ms": max(c["ms_per_step"] for c in per_class)}
    out["workload"] = (f"config4: {n_inst} uneven instances (seed 4000) of one WFS each, 2x2/10x10/40x40/80x80 "
                       "subapertures, DFT 16/24/32/64, 1-10 layers, LGS and NGS, noise on; one batch launch set "
                       "per step (CUDA graph), autotuned launch shapes")
    return out


def single_configs(args, dev, flush, ev0, ev1):
    """Configs 1 and 2 as single instances (the plain FP32 path and BF16 x3 on the tensor cores),
    noise on, frames timed as the headline's."""
    import torch

    from paper_1408_0698_gb300 import inputs, native
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    out = {}
    for cname, fn in (("config1", inputs.config1), ("config2", inputs.config2)):
        res = {}
        for pname, prec in (("fp32", inputs.PREC_FP32), ("bf16x3", inputs.PREC_BF16X3)):
            cfg = fn(prec)
            w = native.Wfs(cfg, seed=cfg.seed, noise=True)
            s_d = torch.as_tensor(inputs.make_screens(cfg.layers, cfg.seed)).to(dev)
            sl = torch.empty((w.total, 2), device=dev)
            k = min(args.steps, 300)
            ms, kt = time_frames(w, s_d, sl, sp, stream, flush, ev0, ev1, args, cfg.dt_s, k)
            res[pname] = {"value": w.total / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": k,
                          "spots_per_frame": w.total, "kernels": kt}
            w.close()
        out[cname] = res
    return out


def time_other_precision(line, other, cfg, rank, s_d, slopes, sp, stream, flush, ev0, ev1, spots, args, dt):
    from paper_1408_0698_gb300 import inputs, native
    w2 = native.Wfs(inputs.config3(PRECISIONS[other]), seed=cfg.seed + rank, noise=True)
    k2 = min(args.steps, 300)
    ms, kt = time_frames(w2, s_d, slopes, sp, stream, flush, ev0, ev1, args, dt, k2)
    w2.close()
    line[f"{other}_path"] = {"value": spots / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": k2,
                             "dft_precision": other, "kernels": kt}


def time_uplink(line, cfg, rank, s_d, slopes, sp, stream, flush, ev0, ev1, spots, args, dt):
    """The same frame with the LGS uplink tip-tilt on (0.4 m launch beam, 24 x 24 samples)."""
    from paper_1408_0698_gb300 import native
    w3 = native.Wfs(cfg, seed=cfg.seed + rank, noise=True)
    for k, st in enumerate(cfg.stars):
        if st.is_lgs:
            native.wfs_set_uplink(w3.h, k, 0.4, 24)
    k3 = min(args.steps, 300)
    ms, kt = time_frames(w3, s_d, slopes, sp, stream, flush, ev0, ev1, args, dt, k3)
    w3.close()
    line["uplink_path"] = {"value": spots / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": k3,
                           "uplink": "6 LGS, 0.4 m launch beam, 24 x 24 samples", "kernels": kt}


def time_per_slice(line, cfg, rank, s_d, slopes, sp, stream, flush, ev0, ev1, spots, args, dt):
    """The same frame with the paper's per-slice LGS model (8 wavefronts and 8 DFTs per LGS
    subaperture, FP32 generic kernel)."""
    from paper_1408_0698_gb300 import native
    w4 = native.Wfs(cfg, seed=cfg.seed + rank, noise=True)
    native.wfs_set_lgs_model(w4.h, 1)
    k4 = min(args.steps, 100)
    ms, kt = time_frames(w4, s_d, slopes, sp, stream, flush, ev0, ev1, args, dt, k4, kernel_steps=10)
    w4.close()
    n_sl = len(cfg.stars[0].na_alt_m)
    line["per_slice_path"] = {"value": spots / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": k4,
                              "model": f"per-slice LGS, {n_sl} slices (one wavefront and DFT each): one projection of every (LGS, slice) pair, tensor-core per-slice spot kernel",
                              "kernels": kt}


if __name__ == "__main__":
    sys.exit(main())
