"""Benchmark: XTRG beta-doubling steps on one GB300 (or N replicas).

A step is one doubling rho <- compress(rho^T rho) of the 64-site XX chain at
D* = 256 with 4 full sweeps, followed by the trace and the thermodynamic
observables (the whole hot path after initialisation).  The timed steps are
the saturated doublings of the schedule tau0 = 2^-12 -> beta = 64, repeated
from a device checkpoint when more steps are asked for than the schedule
has.  Prints one JSON line with the accuracy of the run against the XX
chain's closed form, the FP64 GPU path on the same state, the roofline of
the tensor-core GEMM and the CPU oracle.

  python bench.py [--steps K] [--warmup W] [--prec bf16x6|bf16x3|fp64]
                  [--impl native|reference] [--no-fp64-arm] [--no-cpu-baseline]

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
W = wl.CHAIN_L64_XX
# doublings that start below this beta run in FP64 (the precision schedule
# under which the tensor-core path meets |df|/site <= 1e-6)
BETA_SWITCH = 0.25
DESC = ("Heisenberg XX chain (XXZ, Delta=0), L=64 open, J=1, D*=256, 4 sweeps/doubling, "
        "tau0=2^-12 doubled to beta=64; the saturated doublings of that schedule are timed")
L2_NOTE = ("no flush: every update streams operands far larger than L2 (one environment "
           "~100 MB, one resident half ~400 MB per plane set; ~75 GB working set)")


def set_workload(L, dstar):
    """Replace the timed chain by a smaller one of the same family (for
    profiler captures that must stay small); the defaults are the headline
    workload."""
    global W, DESC
    if (L, dstar) != (W.L, W.dstar):
        W = W.with_(name=f"xxx_L{L}_D{dstar}", L=L, dstar=dstar)
        DESC = (f"Heisenberg XX chain, L={L} open, J=1, Delta=0, D*={dstar}, 4 sweeps/doubling, "
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
           "config": {"workload": DESC, "L": W.L, "Delta": W.Delta, "dstar": W.dstar,
                      "sweeps": W.sweeps, "tau0": W.tau0, "prec": "fp64 (oracle)",
                      "beta_switch": BETA_SWITCH, "l2": L2_NOTE,
                      "timed_window": ("per step: one oracle two-site update at the saturated "
                                       "bond 256 of the doubling (C_E, SVD split, environment "
                                       "update), scaled by the doubling's updates"),
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
def free_fermion_f(L, beta, J=1.0):
    """Free energy per site of the open XX chain (Delta = 0) in closed form:
    Jordan-Wigner fermions with eps_k = J cos(k pi / (L+1)),
    ln Z = sum_k ln(1 + e^{-beta eps_k}) (App. F of the paper).  Used only to
    state the accuracy of the timed run next to its throughput."""
    k = np.arange(1, L + 1)
    eps = J * np.cos(k * np.pi / (L + 1))
    lnZ = float(np.sum(np.logaddexp(0.0, -beta * eps)))
    return -lnZ / (L * beta)


def traffic_from_profile(kernel_src):
    """DRAM bytes per C_E launch of tc_gemm_kernel from the committed ncu
    summary, if that summary was taken of the current kernel source (its
    sha256 is recorded in the summary); otherwise None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_tc_gemm_ce_L64_D256_bf16x6.md")
    try:
        text = open(path).read()
        src = open(kernel_src, "rb").read()
    except OSError:
        return None, None
    sha = hashlib.sha256(src).hexdigest()
    fields = {}
    for ln in text.splitlines():
        key, sep, val = ln.partition(":")
        if sep and key.strip() in ("source_sha256", "traffic_bytes_per_launch", "launch_shape"):
            fields[key.strip()] = val.strip().strip("`")
    if fields.get("source_sha256") != sha:
        return None, "ncu summary is of another kernel source"
    try:
        return float(fields["traffic_bytes_per_launch"]), fields.get("launch_shape")
    except (KeyError, ValueError):
        return None, None


def run_native(args):
    import torch
    from paper_1801_00142_gb300.engine import XTRG

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    beta_end = W.betas[-1]
    xx = W.Delta == 0.0

    eng = XTRG.xxz(W.L, W.J, W.Delta, tau0=W.tau0, dstar=W.dstar, sweeps=W.sweeps,
                   order=W.order, prec=args.prec, beta_switch=BETA_SWITCH, device=str(dev))
    st = eng.stream
    # set-up: initialisation and the doublings up to the first state that the
    # timed doublings start from (mixed arithmetic, bonds saturated at D*)
    eng.init()
    rows_sched = [eng.observables()]
    while True:
        o = rows_sched[-1]
        if o["max_bond"] == W.dstar and (args.prec == "fp64" or o["beta"] >= BETA_SWITCH):
            break
        if o["beta"] >= beta_end:
            raise RuntimeError("bonds did not saturate inside the schedule")
        eng.double()
        rows_sched.append(eng.observables())
    beta0 = rows_sched[-1]["beta"]
    ckpt = eng.checkpoint()

    cur = {"beta": beta0}

    def step():
        # the timed doublings walk beta0 -> beta_end and start over from the
        # checkpoint, so every timed step is a saturated doubling of the schedule
        if cur["beta"] >= beta_end:
            eng.restore(ckpt)
        eng.double()
        o = eng.observables()
        cur["beta"] = o["beta"]
        return o

    # a step is the doubling and the thermodynamics of Eq. ThermalQuan; the
    # FP64 Hermiticity diagnostic is taken once, on the last state (below)
    eng.set_herm_check(False)
    for _ in range(args.warmup):
        rows_sched.append(step())
    clocks = ClockSampler(local)
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
        rows.append(step())
    e1.record(st)
    torch.cuda.synchronize(dev)
    if args.ncu_region:
        torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    s1 = eng.counters()
    ms, steps_total, value = aggregate(e0.elapsed_time(e1), args.steps, dist, dev)
    timed_betas = sorted({r["beta"] for r in rows})

    # profiled pass over the same doublings (beta0 -> beta_end): every
    # tensor-core GEMM launch and truncation bracketed by CUDA events on the
    # context's stream; kept out of the timed region above
    eng.restore(ckpt)
    cur["beta"] = beta0
    eng.set_profiling(True)
    p0 = eng.counters()
    n_cycle = int(round(math.log2(beta_end / beta0)))
    for _ in range(n_cycle):
        step()
    p1 = eng.counters()
    eng.set_profiling(False)

    # end to end through the C ABI with host buffers, over the same doublings:
    # upload rho, double, observables, download rho, every step
    eng.restore(ckpt)
    host0 = eng.get_state()
    sites, lnc, beta = host0
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    h2d = d2h = 0
    for _ in range(max(1, args.steps)):
        if beta >= beta_end:
            sites, lnc, beta = host0
        h2d = sum(w.nbytes for w in sites)
        eng.set_state(sites, lnc, beta, right_canonical=True)
        eng.double()
        eng.observables()
        sites, lnc, beta = eng.get_state()
        d2h = sum(w.nbytes for w in sites)
    torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / max(1, args.steps)

    eng.set_herm_check(True)
    herm_last = eng.observables()
    fp64 = None
    if args.prec != "fp64" and not args.no_fp64_arm and rank == 0:
        fp64 = fp64_arm(XTRG, host0, dev)
    eng.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks, src = measured_peaks()
    nprod = {"bf16x6": 6, "bf16x3": 3}.get(args.prec, 0)
    tc_ms = p1["tc_ms"] - p0["tc_ms"]
    tc_fl = p1["tc_flops"] - p0["tc_flops"]
    tc_n = p1["tc_launches"] - p0["tc_launches"]
    contr = s1["contraction_flops"] - s0["contraction_flops"]
    tc_tflops = tc_fl / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else None
    roof = None
    if nprod:
        bf16_peak = peaks["bf16_tflops_sustained"]
        peak = bf16_peak / nprod
        traffic, shape = traffic_from_profile(
            os.path.join(ROOT, "paper_1801_00142_gb300", "csrc", "tc_gemm.cu"))
        roof = {"bound": "tensor", "achieved": tc_tflops, "peak": peak, "unit": "TFLOP/s",
                "frac": (tc_tflops / peak) if tc_tflops else None, "traffic": traffic,
                "traffic_note": shape,
                "kernel": "tc_gemm_kernel (tcgen05 BF16 split-plane GEMM)",
                "peak_note": (f"{src} bf16 sustained {bf16_peak} TFLOP/s / {nprod} BF16 products per "
                              f"algorithmic FP32-class multiply-add (of measured); issued "
                              f"{tc_tflops * nprod if tc_tflops else 0:.1f} TFLOP/s"),
                "timing": (f"CUDA events around each of the {tc_n} launches of a profiled pass "
                           f"over the timed doublings (beta {beta0:g} -> {beta_end:g})"),
                "launches": tc_n, "avg_launch_ms": tc_ms / max(1, tc_n)}
    df_sched = [abs(r["f"] - free_fermion_f(W.L, r["beta"], W.J)) for r in rows_sched] if xx else []
    df_timed = [abs(r["f"] - free_fermion_f(W.L, r["beta"], W.J)) for r in rows] if xx else []
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
           "config": {"workload": DESC, "L": W.L, "Delta": W.Delta, "dstar": W.dstar,
                      "sweeps": W.sweeps, "tau0": W.tau0, "prec": args.prec,
                      "beta_switch": BETA_SWITCH,
                      "timed_betas": [timed_betas[0], timed_betas[-1]],
                      "timed_window": (f"doublings beta {beta0:g} -> {beta_end:g} of the schedule "
                                       f"(bonds saturated at D*), restarted from a device "
                                       f"checkpoint at beta {beta0:g} after beta {beta_end:g}"),
                      "l2": L2_NOTE,
                      "parallelism": f"replicas x{ws}"},
           "accuracy": ({"vs_exact_max_abs_df_per_site_setup": max(df_sched),
                         "vs_exact_max_abs_df_per_site_timed": max(df_timed),
                         "exact": "free-fermion closed form of the XX chain",
                         "vs_fp64_one_doubling_abs_df_per_site":
                             fp64.get("mixed_vs_fp64_abs_df") if fp64 else None,
                         "gate": "|df|/site <= 1e-6 against the FP64 path at the same D*",
                         "note": ("the exact result differs from XTRG at D*=256 by the "
                                  "truncation error both paths share; the FP64 comparison is "
                                  "one doubling of both paths from the same state")}
                        if xx else None),
           "tflops": contr / (ms / 1e3) / 1e12 * ws,
           "tflops_note": "algorithmic 2MNK of the contraction GEMMs per second (whole job)",
           "roofline": roof,
           "clocks": clk,
           "e2e": {"value": ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h},
           "gpu_launches": s1["kernel_launches"] - s0["kernel_launches"],
           "exact_split_fallbacks": s1["exact_split_fallbacks"] - s0["exact_split_fallbacks"],
           "truncation_ms_per_step": (p1["split_ms"] - p0["split_ms"]) / n_cycle,
           "tc_gemm_ms_per_step": tc_ms / n_cycle,
           "orth_cluster_calls": s1["orth_cluster_calls"] - s0["orth_cluster_calls"],
           "orth_fallbacks": s1["orth_fallbacks"] - s0["orth_fallbacks"],
           "orth_full_second_pass": s1["orth_full_second_pass"] - s0["orth_full_second_pass"],
           "orth_deflated_columns": s1["orth_deflated_columns"] - s0["orth_deflated_columns"],
           "graph_replays_timed": s1["graph_replays"] - s0["graph_replays"],
           "fp64_arm": fp64,
           "observables_last": {k: rows[-1][k] for k in ("beta", "lnZ", "f", "u", "max_bond")},
           "herm_defect_last": {"beta": herm_last["beta"], "herm_defect": herm_last["herm_defect"],
                                "note": "||rho - rho^T||_F / ||rho||_F of the state after the e2e "
                                        "leg (FP64 transfers), taken outside the timed steps"}}
    if fp64 and fp64.get("ms_per_step"):
        out["fp64_ms_per_step"] = fp64["ms_per_step"]
        out["speedup_vs_fp64"] = fp64["ms_per_step"] / (ms / args.steps)
    if not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(2)
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def fp64_arm(XTRG, host_state, dev):
    """The FP64 GPU path on the same saturated state: one doubling with one
    full sweep, every two-site update and the initial environment pass timed
    by CUDA events inside the library; a 4-sweep doubling is that doubling
    plus the measured mean update time for the 3 further sweeps.  (A full
    4-sweep FP64 doubling at D* = 256, L = 64 takes several minutes.)"""
    import torch
    sites, lnc, beta = host_state
    e = XTRG.xxz(W.L, W.J, W.Delta, tau0=W.tau0, dstar=W.dstar, sweeps=1, order=W.order,
                 prec="fp64", device=str(dev))
    e.set_state(sites, lnc, beta, right_canonical=True)
    e.set_profiling(True)
    c0 = e.counters()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    a.record(e.stream)
    e.double()
    e.observables()
    b.record(e.stream)
    torch.cuda.synchronize(dev)
    c1 = e.counters()
    o64 = e.observables()
    e.close()
    t1 = a.elapsed_time(b)
    # the tensor-core path doubles the same state with the same single sweep
    m = XTRG.xxz(W.L, W.J, W.Delta, tau0=W.tau0, dstar=W.dstar, sweeps=1, order=W.order,
                 prec="bf16x6", device=str(dev), keep_parts=False)
    m.set_state(sites, lnc, beta, right_canonical=True)
    m.double()
    om = m.observables()
    m.close()
    n_upd = c1["fp64_updates_timed"] - c0["fp64_updates_timed"]
    upd_ms = (c1["fp64_update_ms"] - c0["fp64_update_ms"]) / max(1, n_upd)
    extra = (W.sweeps - 1) * 2 * (W.L - 1)
    # FP64 denominator: cuBLAS DGEMM (torch.matmul, 4096^3) on this GPU; the
    # FP64 path's contractions per update are 88 D*^4 flops (both halves)
    x = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    for _ in range(2):
        torch.matmul(x, x)
    a.record()
    for _ in range(5):
        torch.matmul(x, x)
    b.record()
    torch.cuda.synchronize(dev)
    dgemm_tflops = 5 * 2 * 4096.0 ** 3 / (a.elapsed_time(b) / 1e3) / 1e12
    upd_tflops = 88.0 * W.dstar ** 4 / (upd_ms / 1e3) / 1e12 if upd_ms > 0 else None
    return {"ms_per_step": t1 + extra * upd_ms, "measured_ms_1_sweep": t1,
            "dgemm_tflops_measured": dgemm_tflops,
            "update_contraction_tflops": upd_tflops,
            "update_frac_of_dgemm": upd_tflops / dgemm_tflops if upd_tflops else None,
            "updates_timed": n_upd, "ms_per_update": upd_ms,
            "env_pass_ms": c1["fp64_env_pass_ms"] - c0["fp64_env_pass_ms"],
            "beta": beta, "mixed_vs_fp64_abs_df": abs(om["f"] - o64["f"]),
            "method": (f"one FP64 doubling with 1 sweep from the timed window's start state "
                       f"(CUDA events), plus {extra} further two-site updates at the measured "
                       f"mean FP64 update time for the {W.sweeps}-sweep doubling")}


def run_gemm_microbench(args):
    """The tensor-core contraction primitive alone at the C_E shape of a
    saturated two-site update (M = N = 4 D*, K = D*^2, 3 planes, 6 products,
    the split-K given), through xtrg_tc_gemm: CUDA events around whole calls
    (BF16 plane conversion of the FP64 inputs, the GEMM kernel, the FP64
    split-K sum; the engine's own C_E reads planes that are already
    converted, so its rate is the kernel's).  One JSON line; used for small
    profiler captures of the GEMM launch, whose kernel time ncu reports."""
    import torch
    from paper_1801_00142_gb300 import _lib
    D = W.dstar
    M = N = 4 * D
    K = D * D
    splitk = args.splitk
    planes, nprod = args.planes, args.nprod
    rng = np.random.default_rng(0)
    A = torch.from_numpy(rng.standard_normal((M, K)) / D).cuda()
    B = torch.from_numpy(rng.standard_normal((N, K)) / D).cuda()
    C = torch.empty((M, N), dtype=torch.float64, device="cuda")
    nb = _lib.xtrg_tc_gemm_workspace_bytes(M, N, K, 1, planes, splitk)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    p = (ws.data_ptr() + 255) // 256 * 256
    st = torch.cuda.current_stream().cuda_stream
    for _ in range(max(1, args.warmup)):
        _lib.xtrg_tc_gemm(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, 1, planes, nprod,
                          splitk, p, nb, st)
    ts = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        _lib.xtrg_tc_gemm(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, 1, planes, nprod,
                          splitk, p, nb, st)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.median(ts))
    peaks, src = measured_peaks()
    flops = 2.0 * M * N * K
    print(json.dumps({"microbench": "tc_gemm C_E", "M": M, "N": N, "K": K, "splitk": splitk,
                      "planes": planes, "nprod": nprod, "ms_median_call": ms,
                      "algorithmic_tflops_call": flops / ms / 1e9,
                      "note": "call = plane conversion of A and B + GEMM + FP64 split-K sum",
                      "peak_bf16_sustained_over_6": peaks["bf16_tflops_sustained"] / 6}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--prec", default="bf16x6", choices=["bf16x6", "bf16x3", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--microbench", choices=["ce"], default=None,
                    help="time the tensor-core GEMM alone at the C_E shape of the workload")
    ap.add_argument("--splitk", type=int, default=7, help="split-K of --microbench ce")
    ap.add_argument("--planes", type=int, default=3, help="BF16 planes of --microbench ce")
    ap.add_argument("--nprod", type=int, default=6, help="plane products of --microbench ce")
    ap.add_argument("--no-fp64-arm", action="store_true",
                    help="skip the FP64 GPU comparison arm (several minutes at L=64)")
    ap.add_argument("--ncu-region", action="store_true",
                    help="bracket the timed region with cudaProfilerStart/Stop")
    ap.add_argument("--L", type=int, default=W.L,
                    help="chain length (smaller chains only for profiler captures)")
    ap.add_argument("--dstar", type=int, default=W.dstar,
                    help="bond cap D* (smaller caps only for profiler captures)")
    args = ap.parse_args()
    set_workload(args.L, args.dstar)
    if args.microbench:
        run_gemm_microbench(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
