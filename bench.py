"""Benchmark: XTRG beta-doubling steps on one GB300 (or N replicas).

A step is one doubling rho <- compress(rho^T rho) of the 64-site Heisenberg
chain at D* = 256 with 4 full sweeps, followed by the trace and the
thermodynamic observables (the whole hot path after initialisation).  Steps
are timed once the bonds have saturated at D*.  Prints one JSON line.

  python bench.py [--steps K] [--warmup W] [--prec bf16x6|bf16x3|fp64]
                  [--impl native|reference] [--fp64-sample]

Multi-GPU (torchrun, one rank per GPU): every rank runs an independent
replica (the doubling of one instance does not shard); value is the sum of
the ranks' doublings divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

METRIC = ("XTRG doubling steps/s & TFLOP/s @D*=256,L=64: mixed vs FP64, "
          "|Δf|/site≤1e-6")
UNIT = "doubling steps/s"
W = wl.CHAIN_L64_XXX
DESC = ("Heisenberg XXX chain, L=64 open, J=1, Delta=1, D*=256, 4 sweeps/doubling, "
        "tau0=2^-12 doubled to beta=64; the last steps of that schedule are timed")
L2_NOTE = ("no flush: every update streams operands far larger than L2 (one environment "
           "~100 MB, one resident half ~400 MB per plane set; ~75 GB working set)")


def set_workload(L, dstar):
    """Replace the timed chain by a smaller one of the same family (for
    profiler captures that must stay small); the defaults are the headline
    workload."""
    global W, DESC
    if (L, dstar) != (W.L, W.dstar):
        W = W.with_(name=f"xxx_L{L}_D{dstar}", L=L, dstar=dstar)
        DESC = (f"Heisenberg XXX chain, L={L} open, J=1, Delta=1, D*={dstar}, 4 sweeps/doubling, "
                f"tau0=2^-12 doubled to beta=64 (profiling case)")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--id={self.index}",
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------- CPU oracle
def oracle_update_seconds(n_updates=2, D=256, seed=0):
    """Time two-site updates of the oracle at the saturated shape of the
    workload (all bonds D): C_E, SVD split, environment update.  Seeded
    synthetic tensors of the workload's shapes."""
    from oracle import xtrg as xo
    rng = np.random.default_rng(seed)
    VL = rng.standard_normal((D, D, D)) / D
    VR = rng.standard_normal((D, D, D)) / D
    A = rng.standard_normal((D, 2, 2, D)) / D
    B = rng.standard_normal((D, 2, 2, D)) / D
    ts = []
    for _ in range(n_updates):
        t = time.perf_counter()
        CE = xo.two_site_overlap(VL, A, A, B, B, VR)
        Ci, Cj, _, _ = xo.split_two_site(CE, "right", D, 1e-15)
        xo.left_env_update(VL, A, A, Ci)
        ts.append(time.perf_counter() - t)
    return float(np.median(ts))


def cpu_baseline(n_updates=2):
    t = oracle_update_seconds(n_updates)
    updates = 2 * W.sweeps * (W.L - 1)
    return {"value": 1.0 / (t * updates), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"{n_updates} oracle two-site updates (C_E, SVD split, environment update) at "
                       f"bond 256 of the L=64 D*=256 doubling, median {t:.3f} s/update, scaled by the "
                       f"{updates} updates of one doubling (4 full sweeps)")}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    oracle_update_seconds(1)          # warm-up of BLAS threads
    for _ in range(max(0, args.warmup - 1)):
        pass
    times = []
    for _ in range(args.steps):
        times.append(oracle_update_seconds(1, seed=len(times) + 1))
    t = float(np.median(times))
    updates = 2 * W.sweeps * (W.L - 1)
    value = 1.0 / (t * updates)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t * updates * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": DESC, "L": W.L, "dstar": W.dstar, "sweeps": W.sweeps,
                      "tau0": W.tau0, "prec": "fp64 (oracle)", "l2": L2_NOTE,
                      "parallelism": "rank 0 only"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"one oracle two-site update per step at bond 256, median "
                                      f"{t:.3f} s, x{updates} updates per doubling"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def aggregate(ms_local, steps_local, dist=None, device=None):
    """Whole-job throughput of independent replicas: the slowest rank's timed
    interval (max over ranks) and the sum of all ranks' steps.  Returns
    (ms_max, steps_total, value in steps/s)."""
    import torch
    ms, steps = float(ms_local), float(steps_local)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        n = torch.tensor([steps], dtype=torch.float64, device=device)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
        ms, steps = float(t.item()), float(n.item())
    return ms, steps, steps / (ms / 1e3)


# ---------------------------------------------------------------- GPU path
def run_native(args):
    import torch
    from paper_1801_00142_gb300 import _lib
    from paper_1801_00142_gb300.engine import XTRG

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    eng = XTRG.xxz(W.L, W.J, W.Delta, tau0=W.tau0, dstar=W.dstar, sweeps=W.sweeps,
                   order=W.order, prec=args.prec, beta_switch=0.0, device=str(dev))
    st = eng.stream
    eng.init()
    # the full schedule tau0 -> 2^n_doublings tau0; the last W + K doublings
    # are the warm-up and the timed steps, the ones before them are set-up
    n_setup = max(0, W.n_doublings - args.warmup - args.steps)
    for _ in range(n_setup + args.warmup):
        eng.double()
        eng.observables()
    assert eng.observables()["max_bond"] == W.dstar

    clocks = ClockSampler(local)
    eng.set_profiling(True)
    s0 = eng.counters()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    if args.ncu_region:
        torch.cuda.profiler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    rows = []
    for _ in range(args.steps):
        eng.double()
        rows.append(eng.observables())
    e1.record(st)
    torch.cuda.synchronize(dev)
    if args.ncu_region:
        torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    s1 = eng.counters()
    eng.set_profiling(False)
    ms, steps_total, value = aggregate(e0.elapsed_time(e1), args.steps, dist, dev)

    # end to end through the C ABI with host buffers: upload rho, double,
    # observables, download rho, every step
    sites, lnc, beta = eng.get_state()
    h2d = sum(w.nbytes for w in sites)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(max(1, args.steps)):
        eng.set_state(sites, lnc, beta, right_canonical=True)
        eng.double()
        eng.observables()
        sites, lnc, beta = eng.get_state()
        d2h = sum(w.nbytes for w in sites)
    torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / max(1, args.steps)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks, src = measured_peaks()
    nprod = {"bf16x6": 6, "bf16x3": 3}.get(args.prec, 0)
    tc_ms = s1["tc_ms"] - s0["tc_ms"]
    tc_fl = s1["tc_flops"] - s0["tc_flops"]
    contr = s1["contraction_flops"] - s0["contraction_flops"]
    tc_tflops = tc_fl / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else None
    roof = None
    if nprod:
        bf16_peak = peaks["bf16_tflops_sustained"]
        peak = bf16_peak / nprod
        roof = {"bound": "tensor", "achieved": tc_tflops, "peak": peak, "unit": "TFLOP/s",
                "frac": (tc_tflops / peak) if tc_tflops else None, "traffic": None,
                "kernel": "tc_gemm_kernel (tcgen05 BF16 split-plane GEMM)",
                "peak_note": (f"{src} bf16 sustained {bf16_peak} TFLOP/s / {nprod} BF16 products per "
                              f"algorithmic FP32-class multiply-add; issued "
                              f"{tc_tflops * nprod if tc_tflops else None:.1f} TFLOP/s"),
                "launches": s1["tc_launches"] - s0["tc_launches"],
                "avg_launch_ms": tc_ms / max(1, s1["tc_launches"] - s0["tc_launches"])}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
           "config": {"workload": DESC, "L": W.L, "dstar": W.dstar, "sweeps": W.sweeps,
                      "tau0": W.tau0, "prec": args.prec,
                      "beta": [rows[0]["beta"], rows[-1]["beta"]],
                      "l2": L2_NOTE,
                      "parallelism": f"replicas x{ws}"},
           "tflops": contr / (ms / 1e3) / 1e12 * ws,
           "tflops_note": "algorithmic 2MNK of the contraction GEMMs per second (whole job)",
           "roofline": roof,
           "clocks": clk,
           "e2e": {"value": ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h},
           "gpu_launches": s1["kernel_launches"] - s0["kernel_launches"],
           "exact_split_fallbacks": s1["exact_split_fallbacks"] - s0["exact_split_fallbacks"],
           "truncation_ms_per_step": (s1["split_ms"] - s0["split_ms"]) / args.steps,
           "orth_cluster_calls": s1["orth_cluster_calls"] - s0["orth_cluster_calls"],
           "observables_last": {k: rows[-1][k] for k in ("beta", "lnZ", "f", "u", "max_bond")}}
    if not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(2)
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--prec", default="bf16x6", choices=["bf16x6", "bf16x3", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-region", action="store_true",
                    help="bracket the timed region with cudaProfilerStart/Stop")
    ap.add_argument("--L", type=int, default=W.L,
                    help="chain length (smaller chains only for profiler captures)")
    ap.add_argument("--dstar", type=int, default=W.dstar,
                    help="bond cap D* (smaller caps only for profiler captures)")
    args = ap.parse_args()
    set_workload(args.L, args.dstar)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
