#!/usr/bin/env python
"""Adam iterations per second of the deep-FBSDE training step on GB300.

One step = one pass of the whole hot path on one batch: Philox increments and
Euler-Maruyama paths for M paths x N steps, the network and Z = grad_x u at
every point, the loss and its Theta-gradient (tangent + adjoint sweeps and
weight-gradient contractions), and the Adam update.  The default workload is
100-D Black-Scholes-Barenblatt with M = 4096 paths, N = 64 steps and a ResNet
of 5 blocks x 256 tanh, in the BF16 tensor-core form, with the FP32 CUDA-core
form timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica (its own seed) of the
workload; the job value is all ranks' steps / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Adam iters/sec, 100-D BSB M=4096 N=64, BF16 vs FP32 form at Y0 rel err ≤1%"
DEFAULT_WORKLOAD = "bsb_d100_n64_m4096_resnet5x256_tanh"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["bf16", "fp32"], default="bf16")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--fp32-steps", type=int, default=10,
                    help="timed steps of the FP32 form beside a BF16 run (0: skip)")
    ap.add_argument("--accuracy-steps", type=int, default=5000,
                    help="Adam steps of each BF16 accuracy run (0: skip)")
    ap.add_argument("--accuracy-seeds", type=int, default=3,
                    help="seeds of the accuracy runs (each form)")
    ap.add_argument("--fp32-accuracy-steps", type=int, default=3000,
                    help="at most this many steps of each FP32-form accuracy run under the decayed learning "
                         "rate (it stops once the 1%% band is held; 0: skip)")
    ap.add_argument("--fp32-accuracy-seeds", type=int, default=1,
                    help="seeds of the FP32-form accuracy runs")
    ap.add_argument("--lr-decay-step", type=int, default=2000,
                    help="accuracy runs with the learning rate multiplied by --lr-decay-factor after this step "
                         "(beside the paper's constant rate; 0: skip)")
    ap.add_argument("--lr-decay-factor", type=float, default=0.1)
    ap.add_argument("--decay-accuracy-steps", type=int, default=3000,
                    help="steps of each BF16 run with the decayed learning rate")
    ap.add_argument("--cpu-iters", type=int, default=1,
                    help="whole-workload FP64 oracle steps timed for the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--loss-steps", type=int, default=20,
                    help="timed loss-only evaluations (forward sweep + residuals), 0: skip")
    ap.add_argument("--fp8-steps", type=int, default=1000,
                    help="Adam steps of the FP8-hidden-layer form (timed for speed, then trained; 0: skip)")
    ap.add_argument("--nais-steps", type=int, default=5,
                    help="timed steps of the HJB NAIS-Net workload in both forms (0: skip)")
    ap.add_argument("--nais-accuracy-steps", type=int, default=0,
                    help="> 0: also train the NAIS-Net HJB workload (BF16) until |Y0 - u(0,0)| <= 1%% "
                         "(at most this many steps)")
    ap.add_argument("--wide-steps", type=int, default=3,
                    help="train steps timed per form on the NAIS-Net 6 x 512 network (BSB, M = 16384); 0 skips")
    ap.add_argument("--wide-accuracy-steps", type=int, default=0,
                    help="> 0: also train that network single-level and multilevel to |Y0 err| <= 1%% "
                         "(at most this many steps on the N = 64 grid)")
    ap.add_argument("--batched-steps", type=int, default=3,
                    help="timed group steps of the 32 uneven instances (0: skip)")
    ap.add_argument("--M", type=int, default=0,
                    help="override the number of paths (small cases for profiler captures)")
    return ap.parse_args()


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id, self.rows, self.proc = gpu_id, [], None

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "100"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(self.rows)}


def gpu_id_of(dev_index: int) -> str:
    import torch
    try:
        p = torch.cuda.get_device_properties(dev_index)
        return "%08X:%02X:%02X.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        return ""


# ----------------------------------------------------------------- peaks / traffic

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# Sources of the fused point-contraction kernels (FC / ResNet: the pipelined
# kernels): a committed DRAM-traffic figure is reported only while the
# sources it names are unchanged since its capture.
KERNEL_SOURCES = ("fused_pipe.cu", "fused_common.cuh", "tc_common.cuh", "bf16_work.cuh")


def source_hash(files=KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1910_11623_gb300", "csrc")
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(form: str, workload: str):
    """DRAM bytes per launch of the dominant kernel from a committed ncu
    summary, or None when none exists for the current sources."""
    path = os.path.join(ROOT, "profiles", f"traffic_{form}_{workload}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("source_hash") != source_hash(tuple(d.get("hash_of", KERNEL_SOURCES))):
        return None
    return d.get("dram_bytes_per_launch")


def fused_algorithmic_bytes(w):
    """Bytes one fused forward and one fused backward launch must move (their
    mean), or None when the workload is not served by the fused kernels.
    Forward: the e_l (L + 1) and g_l (L) BF16 operand blocks, Z and Y written,
    the BF16 X rows read.  Backward: the g_l blocks and the BF16 X and v rows
    read; written, for FC / ResNet (the pipelined kernel) h'_l and h_l for
    l < L and abar_l for l <= L (3L + 1 blocks) and the read-out gradient's
    per-tile partial sums, for NAIS-Net h'_l, h_l and abar_l (3 (L + 1))."""
    p, a = w.problem, w.arch
    if a.prec == "fp32" or a.width > 256 or a.depth > 8 or p.D > 256:
        return None
    P, L = p.M * (p.N + 1), a.depth
    stack = P * (-(-a.width // 64) * 64) * 2
    rows = P * (-(-p.D // 64) * 64) * 2
    fwd = (2 * L + 1) * stack + rows + P * p.D * 4 + P * 4
    if a.kind == "nais" or a.prec not in ("bf16", None):
        bwd = 3 * (L + 1) * stack + L * stack + 2 * rows
    else:
        bwd = (3 * L + 1) * stack + L * stack + 2 * rows + (-(-P // 128)) * 4 * a.width * 4
    return (fwd + bwd) / 2.0


# ----------------------------------------------------------------- CPU oracle

def cpu_oracle_rate(workload, iters: int):
    """The FP64 oracle's train step on the whole workload (all M paths), as it
    stands, timed over `iters` steps on the host cores (no warm-up: NumPy has
    nothing to compile)."""
    import numpy as np
    from oracle import fbsde as F
    from tests.helpers import oracle_specs
    op, oa = oracle_specs(workload.problem, workload.arch)
    theta = F.init_params(op, oa, workload.seed)
    m, v = np.zeros_like(theta), np.zeros_like(theta)
    t0 = time.perf_counter()
    for s in range(1, 1 + iters):
        _, _, theta, m, v = F.train_step(op, oa, theta, m, v, workload.seed, s, workload.lr)
    dt = (time.perf_counter() - t0) / iters
    threads = _blas_threads()
    return {"value": 1.0 / dt, "unit": "it/s", "cores": threads, "kind": "oracle", "seconds_per_step": dt,
            "sample": f"{iters} full FP64 train step(s) of the workload ({workload.problem.M} paths x "
                      f"{workload.problem.N} steps, {dt:.2f} s each), no extrapolation; NumPy with its BLAS "
                      f"on {threads} of {os.cpu_count()} host cores"}


def _blas_threads() -> int:
    """Threads the BLAS under NumPy runs on (the oracle's only parallel part)."""
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count() or 1


def run_reference(args):
    import paper_1910_11623_gb300 as P
    w = P.workloads.WORKLOADS[args.workload]
    # each timed step is one whole FP64 train step (about 20 s on 16 cores);
    # at most two are timed so that the run ends within a few minutes
    steps = max(1, min(args.steps, 2))
    base = cpu_oracle_rate(w, steps)
    line = {"metric": METRIC, "value": base["value"], "unit": "it/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": 0, "ms_per_step": 1000.0 / base["value"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (Philox Brownian paths, seeded Xavier init)",
            "config": {"workload": args.workload}, "impl": "reference",
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": "it/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------- GPU arm

def time_steps(solver, theta, m, v, first_step, K, lr):
    import torch
    st = solver.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for s in range(first_step, first_step + K):
        solver.train_step(theta, m, v, s, lr)
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1)


def batched_run(P, steps: int, lr: float):
    """32 independent uneven instances (half BSB, half HJB; D, N, M, width
    drawn with a seed) trained together, the group step captured as one CUDA
    graph and the SM split between the instances autotuned, in both group
    modes: grouped launches (the fused instances' forward and backward
    kernels as one launch each) and streams (every instance's step on its own
    stream).  Against: the same instances trained one after another with
    direct calls."""
    import torch
    from paper_1910_11623_gb300 import _lib as L
    ws = P.workloads.batched_instances()
    solvers, th, mm, vv, streams = [], [], [], [], []
    for w in ws:
        # a stream of its own per instance (torch's stream pool would hand out shared ones)
        st = torch.cuda.ExternalStream(L.fbsde_stream_create())
        streams.append(st)
        s = P.Solver(w.problem, w.arch, seed=w.seed, stream=st)
        t = s.init_params()
        solvers.append(s); th.append(t); mm.append(torch.zeros_like(t)); vv.append(torch.zeros_like(t))
    n = len(solvers)
    # one after another, direct calls on one stream
    seq = torch.cuda.Stream()
    for s, t, m, v in zip(solvers, th, mm, vv):
        with torch.cuda.stream(seq):
            s.train_step(t, m, v, 1, lr)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per = []
    for s, t, m, v in zip(solvers, th, mm, vv):
        e0.record(s.stream)
        for k in range(steps):
            s.train_step(t, m, v, 2 + k, lr)
        e1.record(s.stream)
        e1.synchronize()
        per.append(e0.elapsed_time(e1) / steps)
    seq_ms = sum(per)
    G = P.Group(solvers)
    modes = {}
    for mode in ("grouped", "streams"):
        G.set_mode(mode)
        caps, tune_ms, _ = G.autotune(th, lr, trial_steps=1)
        step_dev = torch.full((n,), 2 + steps, dtype=torch.int64, device="cuda")
        graph = G.capture(th, mm, vv, step_dev, lr, steps=1)
        graph.launch()
        torch.cuda.synchronize()
        e0.record(G.stream)
        for _ in range(steps):
            graph.launch()
        e1.record(G.stream)
        e1.synchronize()
        modes[mode] = {"ms_per_round": e0.elapsed_time(e1) / steps,
                       "autotune": {"caps": caps, "ms_per_step": tune_ms}}
        graph.close()
    g_ms = modes["grouped"]["ms_per_round"]
    pts = sum(w.problem.M * (w.problem.N + 1) for w in ws)
    res = {"instances": n, "points_per_round": pts,
           "shapes": [[w.problem.kind, w.problem.D, w.problem.N, w.problem.M, w.arch.width] for w in ws],
           "sequential_ms_per_round": seq_ms, "grouped_ms_per_round": g_ms,
           "streams_ms_per_round": modes["streams"]["ms_per_round"],
           "speedup_grouped_vs_sequential": seq_ms / g_ms,
           "instance_steps_per_s": n / (g_ms / 1000.0), "modes": modes,
           "timing": f"{steps} group steps replayed from one CUDA graph per step, after one warm replay"}
    G.close()
    for s in solvers:
        s.close()
    torch.cuda.synchronize()
    for st in streams:
        L.fbsde_stream_destroy(st.cuda_stream)
    del solvers, th, mm, vv
    torch.cuda.empty_cache()
    return res


CHECK_EVERY = 50   # steps between Y0 checks
HOLD_CHECKS = 10   # consecutive checks within 1% that count as having reached it
TAIL_STEPS = 250   # Y0 averaged over the last steps of a run


class Held:
    """Tracks |Y0 - target| / target <= tol at the checks: the first check
    inside, and the first check of a run of `hold` consecutive checks inside
    (the step and wall time at which Y0 entered the band it then stayed in)."""

    def __init__(self, target, tol=0.01, hold=HOLD_CHECKS):
        self.target, self.tol, self.hold = target, tol, hold
        self.first = None     # (step, wall_s)
        self.entry = None     # candidate start of a run inside the band
        self.run = 0
        self.held = None      # (step, wall_s) of the start of the first held run
        self.checks = []      # (step, rel_err)

    def check(self, step, wall, y0):
        err = abs(y0 - self.target) / self.target
        self.checks.append((step, err))
        if err <= self.tol:
            if self.first is None:
                self.first = (step, wall)
            if self.run == 0:
                self.entry = (step, wall)
            self.run += 1
            if self.held is None and self.run >= self.hold:
                self.held = self.entry
        else:
            self.run = 0
        return self.held is not None


def accuracy_run(P, w, target, seed, max_steps, stop_when_held=False, keep=False, decay=None):
    """Train from Theta_0 of `seed` on the workload's grid in schedule calls
    of CHECK_EVERY steps (one Y0 read-back per call), checking |Y0 - target|
    after each call.  Reports the first check within 1%, the start of the
    first run of HOLD_CHECKS consecutive checks within 1% (steps and wall
    time), the share of later checks still within 1%, and Y0 averaged over
    the last TAIL_STEPS steps.  With stop_when_held, training ends once the
    held run is established.  With keep, also returns the solver and the
    trained Theta (the caller closes the solver).  decay = (step, factor):
    the learning rate is multiplied by factor after that step (not in the
    paper, which trains at a constant 1e-3)."""
    import numpy as np
    import torch
    N = w.problem.N
    s = P.Solver(w.problem, w.arch, seed=seed)
    th = s.init_params()
    m, v = torch.zeros_like(th), torch.zeros_like(th)
    torch.cuda.synchronize()
    hd = Held(target)
    trace = []
    t0 = time.perf_counter()
    step = 1
    while step <= max_steps:
        k = min(CHECK_EVERY, max_steps - step + 1)
        lr = w.lr
        if decay and step > decay[0]:
            lr = w.lr * decay[1]
        elif decay:
            k = min(k, decay[0] - step + 1)
        _, y0 = s.train_schedule(th, m, v, [N], [k], step, lr)
        y0 = y0.cpu().numpy().astype(np.float64)
        trace.extend(y0.tolist())
        step += k
        if hd.check(step - 1, time.perf_counter() - t0, float(y0[-1])) and stop_when_held:
            break
    wall = time.perf_counter() - t0
    if not keep:
        s.close()
    tail = float(np.mean(trace[-TAIL_STEPS:]))
    after = [e for st, e in hd.checks if hd.held and st >= hd.held[0]]
    res = {"seed": seed, "steps": len(trace), "wall_s": wall,
            "first_within_1pct": {"step": hd.first[0], "s": hd.first[1]} if hd.first else None,
            "held_within_1pct": {"step": hd.held[0], "s": hd.held[1]} if hd.held else None,
            "share_of_checks_within_1pct_after_held": (sum(e <= 0.01 for e in after) / len(after)) if after else None,
            "y0_last": trace[-1], "y0_tail_mean": tail, "y0_tail_rel_err": abs(tail - target) / target,
            "max_rel_err_last_1000_steps": float(np.max(np.abs(np.array(trace[-1000:]) - target)) / target)}
    return (res, s, th) if keep else res


def accuracy_study(P, w, target, seeds, bf16_steps, fp32_steps, decay=None, fp32_seeds=None, keep_first=True):
    """accuracy_run for `seeds` seeds in both forms: the BF16 form for
    bf16_steps steps, the FP32 form until its held run is established (at
    most fp32_steps).  The speed-up at that accuracy is the ratio of the
    median times to the held 1% band.  Returns the summary and (solver,
    Theta) of the BF16 run of the workload's own seed (to be closed by the
    caller)."""
    import statistics as st
    trained = None
    out = {"criterion": f"|Y0 - {target:.6f}| / {target:.6f} <= 1% at {HOLD_CHECKS} consecutive checks "
                        f"{CHECK_EVERY} steps apart; time and step of the first check of that run",
           "tail_mean_over_steps": TAIL_STEPS}
    if decay:
        out["lr_schedule"] = f"{w.lr:g} for steps 1..{decay[0]}, then {w.lr * decay[1]:g}"
    for form, steps, stop in (("bf16", bf16_steps, False), ("fp32", fp32_steps, True)):
        if steps <= 0:
            continue
        wf = w.with_prec(form)
        runs = []
        for k in range(seeds if form == "bf16" or fp32_seeds is None else fp32_seeds):
            if form == "bf16" and k == 0 and keep_first:
                r, s0, th0 = accuracy_run(P, wf, target, w.seed, steps, stop, keep=True, decay=decay)
                trained = (s0, th0)
            else:
                r = accuracy_run(P, wf, target, w.seed + k, steps, stop, decay=decay)
            runs.append(r)
        held = [r["held_within_1pct"]["s"] for r in runs if r["held_within_1pct"]]
        out[form] = {"runs": runs, "seeds_held": len(held),
                     "median_time_to_held_1pct_s": st.median(held) if len(held) == len(runs) else None}
    b, f = out.get("bf16", {}), out.get("fp32", {})
    if b.get("median_time_to_held_1pct_s") and f.get("median_time_to_held_1pct_s"):
        out["speedup_bf16_vs_fp32_to_held_1pct"] = f["median_time_to_held_1pct_s"] / b["median_time_to_held_1pct_s"]
    return out, trained


def multilevel_run(P, w, target, max_steps, decay=None):
    """Multilevel training (Section 3.2) from the same Theta_0 as the
    single-level accuracy run: fixed Adam steps on the coarse grids, then the
    target grid until |Y0 - closed form| stays within 1% (Held, as in the
    single-level runs).  Wall time includes every level.  decay = (step,
    factor): the learning rate is multiplied by factor after that (global)
    step, as in the single-level runs with decay."""
    import torch
    levels = list(P.workloads.MULTILEVEL_LEVELS)
    N = w.problem.N
    s = P.Solver(w.problem, w.arch, seed=w.seed, N_max=N)
    th = s.init_params()
    m, v = torch.zeros_like(th), torch.zeros_like(th)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step, per_level = 1, []
    hd = Held(target)
    for lv in levels:
        budget = P.workloads.MULTILEVEL_COARSE_STEPS if lv < N else max_steps
        done = 0
        tl = time.perf_counter()
        while done < budget:
            k = min(CHECK_EVERY, budget - done)
            lr = w.lr
            if decay and step > decay[0]:
                lr = w.lr * decay[1]
            elif decay:
                k = min(k, decay[0] - step + 1)
            _, y0 = s.train_schedule(th, m, v, [lv], [k], step, lr)
            step += k
            done += k
            err = abs(y0[-1].item() - target) / target
            if lv == N and hd.check(step - 1, time.perf_counter() - t0, y0[-1].item()):
                break
        per_level.append({"N": lv, "steps": done, "wall_s": time.perf_counter() - tl, "y0_rel_err": err})
        if hd.held:
            break
    res = {"levels": levels, "coarse_steps_per_level": P.workloads.MULTILEVEL_COARSE_STEPS,
           "per_level": per_level,
           "criterion": f"{HOLD_CHECKS} consecutive checks within 1% on the N = {N} grid (time of the first)",
           "time_to_held_1pct_s": hd.held[1] if hd.held else None,
           "steps_to_held_1pct": hd.held[0] if hd.held else None,
           "time_to_first_1pct_s": hd.first[1] if hd.first else None, "wall_s": time.perf_counter() - t0}
    s.close()
    return res


def single_level_run(P, w, target, max_steps):
    """Training on the target grid alone from Theta_0 until |Y0 - closed form|
    stays within 1% (Held: checked every CHECK_EVERY steps), in schedule
    calls of CHECK_EVERY steps."""
    import torch
    N = w.problem.N
    s = P.Solver(w.problem, w.arch, seed=w.seed)
    th = s.init_params()
    m, v = torch.zeros_like(th), torch.zeros_like(th)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step, err = 1, None
    hd = Held(target)
    while step <= max_steps:
        k = min(CHECK_EVERY, max_steps - step + 1)
        _, y0 = s.train_schedule(th, m, v, [N], [k], step, w.lr)
        step += k
        err = abs(y0[-1].item() - target) / target
        if hd.check(step - 1, time.perf_counter() - t0, y0[-1].item()):
            break
    res = {"N": N, "criterion": f"{HOLD_CHECKS} consecutive checks within 1% (time of the first)",
           "time_to_held_1pct_s": hd.held[1] if hd.held else None,
           "steps_to_held_1pct": hd.held[0] if hd.held else None,
           "time_to_first_1pct_s": hd.first[1] if hd.first else None,
           "y0_rel_err": err, "wall_s": time.perf_counter() - t0}
    s.close()
    return res


# ----------------------------------------------------------------- replicas

def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank trains an independent replica: its own noise and Theta_0."""
    return base_seed + rank


def job_throughput(world: int, steps_per_rank: int, ms_max: float) -> float:
    """Whole-job iterations/s: all ranks' steps over the slowest rank's time."""
    return world * steps_per_rank / (ms_max / 1000.0)


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import torch
    import torch.distributed as dist
    import paper_1910_11623_gb300 as P
    from paper_1910_11623_gb300 import _lib as L

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    w = P.workloads.WORKLOADS[args.workload].with_prec(args.form)
    if args.M:
        from dataclasses import replace as _replace
        w = _replace(w, problem=_replace(w.problem, M=args.M))
    stream = torch.cuda.Stream()
    solver = P.Solver(w.problem, w.arch, seed=replica_seed(w.seed, rank), stream=stream)
    theta = solver.init_params()
    m, v = torch.zeros_like(theta), torch.zeros_like(theta)
    with torch.cuda.stream(stream):
        for s in range(1, args.warmup + 1):
            solver.train_step(theta, m, v, s, w.lr)
    barrier()

    # kernel classes: direct calls with the library profiler on
    L.fbsde_profile_enable(solver.ctx, True)
    n0 = L.fbsde_launch_count(solver.ctx)
    prof_steps = max(1, min(args.steps, 20))
    first = args.warmup + 1
    ms_direct = time_steps(solver, theta, m, v, first, prof_steps, w.lr)
    launches_per_step = (L.fbsde_launch_count(solver.ctx) - n0) / prof_steps
    prof = [L.fbsde_profile_read(solver.ctx, c) for c in range(3)]
    L.fbsde_profile_enable(solver.ctx, False)
    first += prof_steps

    # the timed region: the whole training step replayed from one CUDA graph
    # (device step counter), GRAPH_STEPS steps per graph launch
    GRAPH_STEPS = 10
    step_dev = torch.full((1,), first, dtype=torch.int64, device="cuda")
    graph = solver.capture_train_steps(theta, m, v, step_dev, w.lr, steps=GRAPH_STEPS)
    n_launch = (args.steps + GRAPH_STEPS - 1) // GRAPH_STEPS
    graph.launch()  # warm replay
    barrier()
    clocks = ClockSampler(gpu_id_of(local))
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n_launch):
        graph.launch()
    e1.record(stream)
    e1.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    timed_steps = n_launch * GRAPH_STEPS
    launches = int(round(launches_per_step * timed_steps))
    graph.close()

    t = torch.tensor([ms], device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = job_throughput(world, timed_steps, ms_max)

    # end to end through the public API: per step, x0 from pinned host memory
    # to the device, the training step, and the loss / Y0 back to the host.
    D = w.problem.D
    x0_host = torch.tensor(w.problem.x0, dtype=torch.float32).pin_memory()
    x0_dev = torch.empty(D, device="cuda")
    out_host = torch.empty(2, dtype=torch.float32).pin_memory()
    out_dev = torch.empty(2, device="cuda")
    e2e_steps = max(1, min(args.steps, 50))
    # one training step per replay of a one-step graph (the same public API
    # the timed region uses), x0 staged from pinned host memory before it and
    # the step's loss and Y0 read back after it
    g1 = solver.capture_train_steps(theta, m, v, step_dev, w.lr, steps=1)
    with torch.cuda.stream(solver.stream):
        g1.launch()
    barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(solver.stream):
        for _ in range(e2e_steps):
            x0_dev.copy_(x0_host, non_blocking=True)
            L.fbsde_set_x0_device(solver.ctx, x0_dev.data_ptr())
            g1.launch()
            out_dev[0:1].copy_(g1.loss, non_blocking=True)
            out_dev[1:2].copy_(g1.y0, non_blocking=True)
            out_host.copy_(out_dev, non_blocking=True)
            solver.stream.synchronize()
    e2e_s = time.perf_counter() - t0
    g1.close()
    te = torch.tensor([e2e_s], device="cuda")
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e = {"value": job_throughput(world, e2e_steps, 1000.0 * float(te.item())), "unit": "it/s",
           "h2d_bytes_per_step": D * 4, "d2h_bytes_per_step": 8}

    out = None
    if rank == 0:
        peaks, peak_src = measured_peaks()
        dom = max(range(2), key=lambda c: prof[c][0])
        dms, dn, dfl = prof[dom]
        if args.form == "bf16":
            peak = peaks["bf16_tflops_sustained"]
            bound, unit = "tensor", "TFLOP/s"
            achieved = dfl / (dms / 1000.0) / 1e12 if dms > 0 else None
        else:
            # FP32 FFMA: 152 SMs x 128 lanes x 2 flop x max SM clock
            peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            bound, unit = "alu", "TFLOP/s"
            achieved = dfl / (dms / 1000.0) / 1e12 if dms > 0 else None
        traffic = ncu_traffic(args.form, args.workload)
        # the same kernels against HBM: the algorithmic bytes of a launch over
        # its measured duration
        hbm_view = None
        ab = fused_algorithmic_bytes(w)
        if ab and dom == 0 and dms > 0 and dn > 0:
            gbs = ab / (dms / dn / 1000.0) / 1e9
            hbm_view = {"algorithmic_bytes_per_launch": ab, "achieved_gbs": gbs, "peak_gbs": peaks["hbm_gbs"],
                        "frac": gbs / peaks["hbm_gbs"]}
        out = {
            "metric": METRIC, "value": value, "unit": "it/s", "n_gpus": world,
            "steps": timed_steps, "warmup": args.warmup, "ms_per_step": ms_max / timed_steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if args.form == "bf16" else "f32",
            "data": "synthetic (Philox Brownian paths, seeded Xavier init)",
            "config": {"workload": args.workload, "form": args.form, "D": w.problem.D,
                       "N": w.problem.N, "M": w.problem.M, "arch": w.arch.kind,
                       "width": w.arch.width, "depth": w.arch.depth, "act": w.arch.act,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "working set per step >> 126 MB L2 (no flush needed)",
                       "timing": f"CUDA graph of {GRAPH_STEPS} whole training steps, replayed",
                       "direct_call_ms_per_step": ms_direct / prof_steps},
            "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                         "frac": (achieved / peak) if achieved else None,
                         "traffic": traffic,
                         "kernel": ["point contractions", "weight-gradient contractions"][dom],
                         "launches": dn, "ms_total": dms, "flops_total": dfl, "hbm_view": hbm_view,
                         "peak_source": (peak_src + (" sustained bf16" if args.form == "bf16"
                                                     else " FP32 FFMA from SM count and max clock"))},
            "kernel_classes": {name: {"ms": p[0], "launches": p[1], "flops": p[2]}
                               for name, p in zip(["points", "wgrad", "other"], prof)},
            "clocks": clk, "e2e": e2e, "gpu_launches": int(launches),
        }

    # loss only (paths, network forward and Z, residuals): the forward half of a step
    if args.loss_steps > 0:
        loss_buf, y0_buf = torch.empty(1, device="cuda"), torch.empty(1, device="cuda")
        for i in range(3):
            L.fbsde_rollout_loss(solver.ctx, theta.data_ptr(), 10**6 + i, loss_buf.data_ptr(), y0_buf.data_ptr())
        barrier()
        L.fbsde_profile_enable(solver.ctx, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(solver.stream)
        for i in range(args.loss_steps):
            L.fbsde_rollout_loss(solver.ctx, theta.data_ptr(), 2 * 10**6 + i, loss_buf.data_ptr(), y0_buf.data_ptr())
        e1.record(solver.stream)
        e1.synchronize()
        pl = L.fbsde_profile_read(solver.ctx, 0)
        L.fbsde_profile_enable(solver.ctx, False)
        if out is not None:
            lms = e0.elapsed_time(e1) / args.loss_steps
            out["loss_only"] = {"ms_per_eval": lms, "points_ms_per_eval": pl[0] / args.loss_steps,
                                "points_launches_per_eval": pl[1] / args.loss_steps,
                                "points_tflops": pl[2] / (pl[0] / 1000.0) / 1e12 if pl[0] > 0 else None}

    # FP32 form beside the BF16 form (same workload, same GPU)
    if args.form == "bf16" and args.fp32_steps > 0:
        del solver
        torch.cuda.empty_cache()
        w32 = w.with_prec("fp32")
        s32 = P.Solver(w32.problem, w32.arch, seed=replica_seed(w.seed, rank))
        th32 = s32.init_params()
        m32, v32 = torch.zeros_like(th32), torch.zeros_like(th32)
        for s in range(1, 3):
            s32.train_step(th32, m32, v32, s, w.lr)
        barrier()
        ms32 = time_steps(s32, th32, m32, v32, 3, args.fp32_steps, w.lr)
        t = torch.tensor([ms32], device="cuda")
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if out is not None:
            v32rate = job_throughput(world, args.fp32_steps, float(t.item()))
            out["fp32_form"] = {"value": v32rate, "unit": "it/s", "steps": args.fp32_steps}
            out["speedup_vs_fp32_form"] = value / v32rate
        del s32
        torch.cuda.empty_cache()

    # FP8 hidden layers (E4M3 forward contractions of layers 1..L): speed and
    # the Y0 reached after a bounded training run
    if args.form == "bf16" and args.fp8_steps > 0:
        try:
            w8 = w.with_prec("fp8")
            s8 = P.Solver(w8.problem, w8.arch, seed=replica_seed(w.seed, rank), stream=torch.cuda.Stream())
            th8 = s8.init_params()
            m8, v8 = torch.zeros_like(th8), torch.zeros_like(th8)
            with torch.cuda.stream(s8.stream):
                for s in range(1, 4):
                    s8.train_step(th8, m8, v8, s, w.lr)
            ms8 = time_steps(s8, th8, m8, v8, 4, args.fp32_steps or 10, w.lr)
            res8 = {"value": (args.fp32_steps or 10) / (ms8 / 1000.0), "unit": "it/s"}
            if w.problem.kind == "bsb" and w.problem.D == 100:
                target = P.workloads.BSB_Y0_D100
                with torch.cuda.stream(s8.stream):
                    for s in range(4 + (args.fp32_steps or 10), args.fp8_steps + 1):
                        _, y08 = s8.train_step(th8, m8, v8, s, w.lr)
                s8.stream.synchronize()
                res8.update({"train_steps": args.fp8_steps, "y0": y08.item(),
                             "y0_rel_err": abs(y08.item() - target) / target})
            if out is not None:
                out["fp8_hidden_form"] = res8
            s8.close()
        except Exception as exc:
            if out is not None:
                out["fp8_hidden_form"] = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.empty_cache()

    # accuracy: train from Theta_0 and track |Y0 - closed form| / closed form,
    # several seeds, both forms
    if args.accuracy_steps > 0 and out is not None and w.problem.kind == "bsb" and w.problem.D == 100:
        target = P.workloads.BSB_Y0_D100
        # the paper's constant learning rate, BF16 form (the FP32 form is
        # compared under the decayed schedule below, where the band can hold)
        out["accuracy"], (sa, th) = accuracy_study(P, w, target, args.accuracy_seeds, args.accuracy_steps, 0)
        if args.lr_decay_step > 0:
            out["accuracy_lr_decay"], _ = accuracy_study(
                P, w, target, args.accuracy_seeds, args.decay_accuracy_steps, args.fp32_accuracy_steps,
                decay=(args.lr_decay_step, args.lr_decay_factor), fp32_seeds=args.fp32_accuracy_seeds,
                keep_first=False)
        # the trained Theta of the workload's own seed, for the generalisation check
        # generalisation (Section 4.2): the trained Theta at perturbed x0
        x0 = list(w.problem.x0)
        rng = __import__("random").Random(w.seed)
        cases = {f"scale{e:+.2f}": [(1.0 + e) * c for c in x0] for e in (-0.1, -0.05, 0.05, 0.1)}
        cases["random0.05"] = [c * (1.0 + 0.05 * rng.gauss(0.0, 1.0)) for c in x0]
        got = sa.generalisation(th, list(cases.values()))
        out["generalisation"] = {
            name: {"y0": g, "closed_form": P.workloads.bsb_y0(xc),
                   "rel_err": abs(g - P.workloads.bsb_y0(xc)) / P.workloads.bsb_y0(xc)}
            for (name, xc), g in zip(cases.items(), got)}
        sa.close()
        del sa
        decay = (args.lr_decay_step, args.lr_decay_factor) if args.lr_decay_step > 0 else None
        out["multilevel"] = multilevel_run(P, w, target, args.accuracy_steps, decay)
        if decay:
            out["multilevel"]["lr_schedule"] = out["accuracy_lr_decay"]["lr_schedule"]

    # the stable network of the paper (NAIS-Net, HJB, Section 4): BF16 form
    # (fused per-tile kernels) and FP32 form
    if out is not None and args.nais_steps > 0:
        try:
            wn = P.workloads.WORKLOADS["hjb_d100_n64_m8192_nais6x256_tanh"]
            res_n = {"workload": wn.name}
            for prec in ("bf16", "fp32"):
                wp_ = wn.with_prec(prec)
                sn = P.Solver(wp_.problem, wp_.arch, seed=wn.seed, stream=torch.cuda.Stream())
                thn = sn.init_params()
                mn, vn = torch.zeros_like(thn), torch.zeros_like(thn)
                with torch.cuda.stream(sn.stream):
                    for s_ in range(1, 3):
                        sn.train_step(thn, mn, vn, s_, wn.lr)
                msn = time_steps(sn, thn, mn, vn, 3, args.nais_steps, wn.lr)
                res_n[prec] = {"value": args.nais_steps / (msn / 1000.0), "unit": "it/s"}
                sn.close()
                torch.cuda.empty_cache()
            res_n["speedup_bf16_vs_fp32"] = res_n["bf16"]["value"] / res_n["fp32"]["value"]
            if args.nais_accuracy_steps > 0:
                # u(0, 0) of the HJB problem by Cole-Hopf (chi-square quadrature)
                res_n["accuracy"] = single_level_run(P, wn.with_prec("bf16"), P.workloads.HJB_U00_D100,
                                                     args.nais_accuracy_steps)
            out["nais_hjb"] = res_n
        except Exception as exc:
            out["nais_hjb"] = {"error": f"{type(exc).__name__}: {exc}"}

    # the wide NAIS-Net of the multilevel study (BSB, D = 100, M = 16384,
    # NAIS-Net 6 x 512): width 512 runs on the layered tensor-core path
    if out is not None and args.wide_steps > 0:
        try:
            ww = P.workloads.WORKLOADS["bsb_d100_n64_m16384_nais6x512_tanh"]
            res_w = {"workload": ww.name}
            for prec, n in (("bf16", args.wide_steps), ("fp32", 1)):
                wp_ = ww.with_prec(prec)
                sw = P.Solver(wp_.problem, wp_.arch, seed=ww.seed, stream=torch.cuda.Stream())
                thw = sw.init_params()
                mw, vw = torch.zeros_like(thw), torch.zeros_like(thw)
                with torch.cuda.stream(sw.stream):
                    sw.train_step(thw, mw, vw, 1, ww.lr)
                msw = time_steps(sw, thw, mw, vw, 2, n, ww.lr)
                res_w[prec] = {"value": n / (msw / 1000.0), "unit": "it/s", "steps": n}
                sw.close()
                del thw, mw, vw
                torch.cuda.empty_cache()
            res_w["speedup_bf16_vs_fp32"] = res_w["bf16"]["value"] / res_w["fp32"]["value"]
            if args.wide_accuracy_steps > 0:
                wb = ww.with_prec("bf16")
                target = P.workloads.bsb_y0(wb.problem.x0)
                res_w["single_level"] = single_level_run(P, wb, target, args.wide_accuracy_steps)
                res_w["multilevel"] = multilevel_run(P, wb, target, args.wide_accuracy_steps)
            out["wide_nais"] = res_w
        except Exception as exc:
            out["wide_nais"] = {"error": f"{type(exc).__name__}: {exc}"}

    if out is not None and args.batched_steps > 0 and world == 1:
        try:
            out["batched"] = batched_run(P, args.batched_steps, w.lr)
        except Exception as exc:  # report, keep the main line
            out["batched"] = {"error": f"{type(exc).__name__}: {exc}"}

    if out is not None and not args.no_cpu_baseline:
        try:
            out["cpu_baseline"] = cpu_oracle_rate(P.workloads.WORKLOADS[args.workload], args.cpu_iters)
        except Exception as exc:  # report, keep the main line
            out["cpu_baseline"] = {"error": f"{type(exc).__name__}: {exc}", "kind": "oracle"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
