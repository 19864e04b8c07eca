#!/usr/bin/env python3
"""Benchmark of the batched evolutionary hot path (one JSON line on stdout).

Workload (the batched-evaluation configuration, N = 4096 individuals x
D = 100 on six seeded shifted-rotated families: ellipsoid (1e6 conditioning),
Rosenbrock, Rastrigin, Schwefel, Ackley, Griewank): three batched run states
-- DE/rand/1/bin, DE/current-to-pbest/1/bin with archive, inertia PSO with
ring topology -- each holding one population of NP = 4096 per family.
One step = one generation of all three states: Philox draws, trial /
velocity update, crossover and repair, TF32 tensor-core evaluation with FP64
refinement below 1e-4, selection / archive / pbest and guides.  Evaluations
per step: 3 x 6 x 4096 = 73,728.  Inputs are synthetic (seeded uniform
initial populations), resident in HBM; the working set (X, trials, archive,
velocities, pbest: ~160 MB) exceeds the 129 MB L2, so every step streams
from HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own replica with its own seeds
(runs are independent: weak scaling, no collective on the data path); the
step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fitness evals/s at D=100/1000, mixed vs FP64 GPU; run-grid wall time vs oracle"
D, NP, FAMILIES = 100, 4096, 6
ALGS = [("de_rand1_bin", 0), ("de_ctpb1_bin_archive", 1), ("pso_ring", 3)]
WORKLOAD = "batched evaluation N=4096 x D=100, 6 shifted-rotated families, one DE/rand/1 + DE/ctpb/1 + PSO-ring generation per step"


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- our arm
GROUPS = 2  # groups of states stepped by one sevo_state_step_many call each


def make_states(S, prec, seed0, torch, groups=None):
    """One batched state per algorithm and group of families, each on its
    own CUDA stream; a group holds one state per algorithm over FAMILIES /
    groups of the six problems.  Each step advances every state by one
    generation: one sevo_state_step_many call per group, so that one group's
    joint evaluation (tensor cores, FP32) runs while the other group's DE and
    PSO operators (FP64 pipe) run.  The work per step is the same for any
    number of groups: 3 algorithms x 6 populations of NP rows."""
    groups = groups or GROUPS
    probs = [S.Problem(0x5EB00000 + f, f, D) for f in range(FAMILIES)]
    per = FAMILIES // groups
    states = []
    for gi in range(groups):
        fams = list(range(gi * per, (gi + 1) * per))
        for k, (name, alg) in enumerate(ALGS):
            params = S.alg_params(alg, NP, 10 ** 12, prec=prec)
            seeds = [seed0 + 1000 * k + f for f in fams]
            stream = torch.cuda.Stream()
            st = S.State([probs[f] for f in fams], params, seeds, stream=stream)
            st.torch_stream = stream  # keep the stream alive with its state
            st.group = gi
            states.append(st)
    torch.cuda.synchronize()
    return probs, states


RESTART_EVERY = 25


def groups_of(states):
    """The states of each group, in group order."""
    out = {}
    for st in states:
        out.setdefault(getattr(st, "group", 0), []).append(st)
    return [out[k] for k in sorted(out)]


def run_steps(states, first_gen, n, serial=False):
    """Generations first_gen .. first_gen + n - 1 of every state, one
    sevo_state_step_many call per group and generation (each state's
    operators on its own stream, the group's rows evaluated in one fused
    launch).  Every
    RESTART_EVERY generations each run restarts from a fresh uniform
    population (sevo_state_restart, new seeds; its work is inside the timed
    region, its evaluations are not counted), so the timed generations stay
    in the early phase the microbench describes (X ~ U[-100, 100]) instead
    of drifting into the refinement-heavy end of converged runs, which the
    run-grid measurement covers.  serial: the device drains after every
    generation, so generations do not overlap one another."""
    import torch
    import paper_2505_17430_gb300 as S
    for g in range(first_gen, first_gen + n):
        if g % RESTART_EVERY == 0:
            for k, st in enumerate(states):
                st.restart([(g * 7919 + 1000 * k + r) & 0xFFFFFFFF for r in range(st.R)])
        for grp in groups_of(states):
            rc = S.sevo_state_step_many(grp, g)
            if rc != 0:
                raise RuntimeError(f"step failed: {rc}")
        if serial:
            torch.cuda.synchronize()
    return first_gen + n


def write_timeline(S, torch, states, gen, K, path):
    """K steps traced launch by launch (each launch bracketed by events on
    its stream): the spans go to path as JSON, with the step count and the
    wall span of the K steps."""
    torch.cuda.synchronize()
    S.trace_enable(True, timeline=True)
    gen = run_steps(states, gen, K)
    torch.cuda.synchronize()
    spans = S.trace_timeline()
    S.trace_enable(False)
    with open(path, "w") as f:
        json.dump({"steps": K, "spans": spans}, f)
    return gen


def time_steps(torch, states, gen, K):
    """K steps between two events on the current stream: the states' streams
    start after the first event and the second waits for all of them."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for st in states:
        st.torch_stream.wait_event(e0)
    gen = run_steps(states, gen, K)
    for st in states:
        done = torch.cuda.Event()
        done.record(st.torch_stream)
        stream.wait_event(done)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), gen


def _source_hash(files):
    """Hash of the kernels' code: comments and whitespace are left out, so
    that a change to a comment does not retire a profile of the same code."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2505_17430_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(name, files):
    """DRAM bytes per row of a kernel from its committed ncu summary: the
    summary's 'traffic_bytes_per_row' and 'source_hash' lines; None if the
    kernel's sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    per_row = src = None
    for line in open(path):
        if line.startswith("traffic_bytes_per_row:"):
            per_row = float(line.split(":", 1)[1])
        elif line.startswith("source_hash:"):
            src = line.split(":", 1)[1].strip()
    if per_row is None or src != _source_hash(files):
        return None
    return per_row


FUSED_SOURCES = ("eval_tc.cu", "tc_walk.cuh", "bodies.cuh", "tc_ptx.cuh")


def traced_step_kernels(S, torch, states, gen, K, serial=False):
    """Per-kernel device time from a traced repeat of the timed steps (CUDA
    events recorded on the launching stream around every launch); serial:
    the device drains after every generation.  Returns (trace, next gen,
    restarts in the window: each adds one evaluation of every state's rows)."""
    S.trace_enable(True)
    g0 = gen
    gen = run_steps(states, gen, K, serial=serial)
    torch.cuda.synchronize()
    t = S.trace_read()
    S.trace_enable(False)
    restarts = sum(1 for g in range(g0, g0 + K) if g % RESTART_EVERY == 0)
    return {k: v for k, v in t.items() if v[0] > 0}, gen, restarts


def rooflines(trace, states, peaks, K, fp64=None, restarts=0):
    """Dominant kernel (fused tcgen05 evaluation) and the streaming DE/PSO
    kernels against the measured HBM copy bandwidth.  Rows per launch: every
    state's rows for the fused evaluation (one launch per step), one state's
    for a DE trial or PSO move launch."""
    peak = peaks.get("hbm_gbs")
    src = "measured (MEASURED_PEAKS.json hbm_gbs)" if not peaks.get("fallback") else "fallback"
    total_ms = sum(ms for _, ms in trace.values())
    step_rows = sum(st.R * NP for st in states)

    def entry(kind, bytes_per_row, bound="hbm", restart_bytes_per_row=None):
        n, ms = trace.get(kind, (0, 0.0))
        if not n:
            return None
        per = ms / n
        rows = (step_rows * (K + restarts) // n if kind == "eval_tc_fused"
                else states[0].R * NP)
        algo = rows * bytes_per_row
        if restart_bytes_per_row is not None:  # the restarts' evaluations read FP64 rows
            algo = (step_rows * K * bytes_per_row +
                    step_rows * restarts * restart_bytes_per_row) // n
        ach = algo / (per * 1e-3) / 1e9
        return {"kernel": kind, "bound": bound, "achieved": round(ach, 1), "peak": peak,
                "unit": "GB/s", "frac": round(ach / peak, 4) if peak else None,
                "rows_per_launch": rows,
                "algorithmic_bytes_per_launch": algo, "launch_ms": round(per, 4),
                "launches": n, "share_of_step": round(ms / total_ms, 4), "peak_source": src}

    # the fused evaluation of a generation reads the TF32 operand its rows'
    # operator wrote (4 B per coordinate) and writes the fitness; evaluations
    # of fresh populations (restarts) read the FP64 rows instead
    main = entry("eval_tc_fused", D * 4 + 8, restart_bytes_per_row=D * 8 + 8)
    per_row = profiled_traffic("eval_tc_fused_tf32_d100.md", FUSED_SOURCES)
    main["traffic"] = round(per_row * main["rows_per_launch"]) if per_row else None
    # DE trial: target + three donors read, trial written (FP64 rows) + 16 B
    # of partner indices; PSO move: x, v, pbest read, x, v written (the guide
    # row is one per run or neighbourhood and is served from L2); both also
    # write the rows' TF32 operand for the evaluation (4 B per coordinate)
    stream = {k: entry(k, b) for k, b in (("de_trial", 5 * 8 * D + 16 + 4 * D),
                                            ("pso_move", 5 * 8 * D + 4 * D))}
    # the FP64 pipe, which binds both: the formula's FP64 operations per
    # coordinate (DE/rand/1 2, current-to-pbest 4 -- one launch of each per
    # step -- and the PSO move 8) against the DGEMM rate measured here
    if fp64:
        for k, ops in (("de_trial", (2 + 4) / 2), ("pso_move", 8)):
            n, ms = trace.get(k, (0, 0.0))
            if n and stream.get(k):
                ach = n * states[0].R * NP * D * ops / (ms * 1e-3)
                stream[k]["fp64_pipe"] = {"bound": "alu", "unit": "FP64 op/s",
                                          "ops_per_coordinate": ops,
                                          "achieved": round(ach / 1e9, 2) * 1e9,
                                          "peak": round(fp64 / 1e9, 2) * 1e9,
                                          "frac": round(ach / fp64, 4),
                                          "peak_source": "cuBLAS DGEMM 4096^3 timed here, one "
                                                         "op per multiply-add"}
    shares = {k: {"launches": n, "ms": round(ms, 3), "share": round(ms / total_ms, 4)}
              for k, (n, ms) in sorted(trace.items(), key=lambda kv: -kv[1][1])}
    return main, stream, shares


STREAM_SOURCES = ("evo.cu", "ops.cuh", "bounds.cuh", "sevo_internal.cuh", "u53.cuh")


def dominant_roofline(shares, eval_roof, stream_roof):
    """The roofline of the kernel with the largest measured share of the step's
    device time among the fused evaluation, the DE trials and the PSO move:
    the evaluation against HBM, the operators against the FP64 rate that binds
    them (bound "alu"; their HBM figures kept under "hbm")."""
    cands = {k: shares.get(k, {}).get("ms", 0.0) for k in ("eval_tc_fused", "de_trial", "pso_move")}
    k = max(cands, key=cands.get)
    if k == "eval_tc_fused" or not (stream_roof.get(k) or {}).get("fp64_pipe"):
        return eval_roof
    r, f = stream_roof[k], stream_roof[k]["fp64_pipe"]
    per_row = profiled_traffic("streaming_fp64_de_trial_pso_move_d100.md", STREAM_SOURCES)
    return {"kernel": k, "bound": "alu", "achieved": f["achieved"], "peak": f["peak"],
            "unit": "FP64 op/s", "frac": f["frac"], "ops_per_coordinate": f["ops_per_coordinate"],
            "rows_per_launch": r["rows_per_launch"], "launch_ms": r["launch_ms"],
            "launches": r["launches"], "share_of_step": r["share_of_step"],
            "peak_source": f["peak_source"],
            "traffic": round(per_row * r["rows_per_launch"]) if per_row else None,
            "hbm": {"achieved": r["achieved"], "peak": r["peak"], "unit": "GB/s", "frac": r["frac"],
                    "algorithmic_bytes_per_launch": r["algorithmic_bytes_per_launch"]}}


def mode_eval_rates(S, torch, probs):
    """Evaluation-only throughput per precision mode on the step's rows."""
    rows = FAMILIES * NP
    X = torch.empty((rows, D), dtype=torch.float64, device="cuda").uniform_(-100, 100)
    out = torch.empty(rows, dtype=torch.float64, device="cuda")
    res = {}
    for name, prec in (("fp64", S.FP64), ("fp32", S.FP32), ("tf32", S.TF32),
                       ("bf16x3", S.BF16X3)):
        reps = 2 if prec == S.FP64 else 10
        for p in probs:
            p.evaluate(X, out, prec=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            for p in probs:
                p.evaluate(X, out, prec=prec)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        res[name] = round(rows * len(probs) / dt, 1)
    return res


def large_d_rates(S, torch, peaks):
    """Mixed precision at large D (N = 1024 rows, D in {1000, 5000}; and
    16,384 rows at D = 1000 to fill the GPU): evaluation rate per mode on a
    shifted-rotated Rastrigin, a hybrid and a composition instance, against
    the FP64 GPU path; the rotation GEMM's own tensor rate from traced launch
    times (2 N D^2 flops per component; BF16X3 counts its three bf16
    products against the bf16 peak, TF32 is held against the bf16 peak x
    1.1 / 2.25, the nominal dense TF32 : BF16 ratio)."""
    bf16 = peaks.get("bf16_tflops")
    res = []
    for Dl, N in ((1000, 1024), (5000, 1024), (1000, 16384)):
        X = torch.empty((N, Dl), dtype=torch.float64, device="cuda").uniform_(-100, 100)
        out = torch.empty(N, dtype=torch.float64, device="cuda")
        fams = (2, 6, 7) if N == 1024 else (2,)
        for fam in fams:
            p = S.Problem(0x5EB10000 + 16 * fam + Dl, fam, Dl)
            row = {"D": Dl, "N": N, "family": ["ellipsoid", "rosenbrock", "rastrigin", "schwefel",
                                               "ackley", "griewank", "hybrid", "composition"][fam],
                   "components": p.ncomp}
            for name, prec in (("tf32", S.TF32), ("bf16x3", S.BF16X3), ("fp64", S.FP64)):
                if prec == S.FP64 and (Dl > 1000 or fam == 7 or N > 1024):
                    continue
                reps = 3 if prec == S.FP64 else 10
                p.evaluate(X, out, prec=prec)
                torch.cuda.synchronize()
                # the call's time untraced; the GEMM's launch time from a
                # traced repeat (tracing adds an event pair per launch)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    p.evaluate(X, out, prec=prec)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                t = {}
                if prec != S.FP64:
                    S.trace_enable(True)
                    for _ in range(reps):
                        p.evaluate(X, out, prec=prec)
                    torch.cuda.synchronize()
                    t = S.trace_read()
                    S.trace_enable(False)
                row[name] = {"evals_per_s": round(N / (ms * 1e-3), 1), "ms_per_call": round(ms, 4)}
                n, gms = t.get("gemm_big", (0, 0.0))
                if n and prec != S.FP64:
                    fl = 2.0 * N * Dl * Dl  # per launch (one component)
                    tf = fl / (gms / n * 1e-3) / 1e12
                    pk = (bf16 * 1.1 / 2.25) if prec == S.TF32 else bf16 / 3.0
                    row[name]["gemm_tflops"] = round(tf, 1)
                    row[name]["gemm_frac_of_tensor_peak"] = round(tf / pk, 4) if bf16 else None
                    row[name]["gemm_share_of_call"] = round(gms / reps / ms, 3)
            res.append(row)
        del X, out
    return res


def c4_sample(S):
    """Bounded sample of the large-scale grid (D = 1000; PSO NP = 1000 and DE
    current-to-pbest NP = 200 on hybrid and composition instances, 3e6
    evaluations per run in full): 2 hybrid + 2 composition instances x 2 runs
    x both algorithms at a budget of 2e4, mixed (TF32 + FP64 refinement)
    against the FP64 GPU path through sevo_run_grid."""
    import numpy as np
    Dl, budget = 1000, 20000
    probs = [S.Problem(0xC4000000 + k, 6 if k < 2 else 7, Dl) for k in range(4)]
    out = {"workload": "2 hybrid + 2 composition instances x 2 runs x {PSO NP=1000, DE ctpb NP=200}, "
                       "D=1000, budget 2e4 (of 3e6)", "evals": None}
    for name, prec in (("tf32", S.TF32), ("fp64", S.FP64)):
        algs = [S.alg_params(2, 1000, budget, prec=prec), S.alg_params(1, 200, budget, prec=prec)]
        tasks = [(pi, ai, 1 + r) for pi in range(4) for ai in range(2) for r in range(2)]
        r = S.sevo_run_grid(probs, algs, tasks)
        out["evals"] = int(r["evals"])
        out[name] = {"wall_s": round(r["wall_ms"] / 1e3, 3),
                     "evals_per_s": round(r["evals"] / (r["wall_ms"] / 1e3), 1),
                     "median_final_error": float(np.median(r["best"]))}
    out["tf32_speedup"] = round(out["fp64"]["wall_s"] / out["tf32"]["wall_s"], 1)
    return out


def shade_sec31(S):
    """The paper's SHADE timing shape (Sec. 3.1): population 100, 30,000
    evaluations, 10 independent runs on the 30-D Rosenbrock (shifted and
    rotated here) -- the 10 runs batched through sevo_run_grid in FP32 (the
    paper's float) and FP64, against the oracle running the same 10 runs one
    after another on one host core; mean time per run."""
    import numpy as np
    import oracle as O
    D, NP, budget, runs = 30, 100, 30000, 10
    p = S.Problem(0x5EB00001, 1, D)
    out = {"workload": "SHADE NP=100, 30,000 evals, 10 runs, shifted-rotated Rosenbrock D=30"}
    for name, prec in (("fp32", S.FP32), ("fp64", S.FP64)):
        a = S.alg_params(S.DE_SHADE, NP, budget, prec=prec)
        S.sevo_run_grid([p], [a], [(0, 0, 1)])  # warm-up
        t0 = time.perf_counter()
        r = S.sevo_run_grid([p], [a], [(0, 0, s) for s in range(1, runs + 1)])
        wall = time.perf_counter() - t0
        out[name] = {"wall_s_10_runs": round(wall, 4), "mean_s_per_run": round(wall / runs, 5),
                     "median_final_error": float(np.median(r["best"]))}
    q = O.Problem(0x5EB00001, 1, D)
    t0 = time.perf_counter()
    ob = [O.run(q, O.make_alg(O.ALG_DE_SHADE, NP, budget), s)["best"] for s in range(1, runs + 1)]
    owall = time.perf_counter() - t0
    out["oracle"] = {"wall_s_10_runs": round(owall, 4), "mean_s_per_run": round(owall / runs, 5),
                     "median_final_error": float(np.median(ob)), "cores": 1}
    return out


def psode_case1(S):
    """The paper's PSODE case study shape (Sec. 4, Listing 4): population 100,
    D = 30, 1000 D evaluations, bounds [-100, 100], Rosenbrock, float -- 10
    runs batched through sevo_run_grid in FP32 and FP64, against the oracle
    running the same 10 runs one after another on one host core."""
    import numpy as np
    import oracle as O
    D, NP, budget, runs = 30, 100, 30000, 10
    p = S.Problem(0x5EB00003, 1, D)
    out = {"workload": "PSODE (ring PSO + SHADE, pairwise/3) NP=100, 30,000 evals, 10 runs, "
                       "shifted-rotated Rosenbrock D=30"}
    for name, prec in (("fp32", S.FP32), ("fp64", S.FP64)):
        a = S.alg_params(S.PSODE, NP, budget, prec=prec)
        S.sevo_run_grid([p], [a], [(0, 0, 1)])  # warm-up
        t0 = time.perf_counter()
        r = S.sevo_run_grid([p], [a], [(0, 0, s) for s in range(1, runs + 1)])
        wall = time.perf_counter() - t0
        out[name] = {"wall_s_10_runs": round(wall, 4), "mean_s_per_run": round(wall / runs, 5),
                     "median_final_error": float(np.median(r["best"]))}
    q = O.Problem(0x5EB00003, 1, D)
    t0 = time.perf_counter()
    ob = [O.run(q, O.make_alg(O.ALG_PSODE, NP, budget), s)["best"] for s in range(1, runs + 1)]
    owall = time.perf_counter() - t0
    out["oracle"] = {"wall_s_10_runs": round(owall, 4), "mean_s_per_run": round(owall / runs, 5),
                     "median_final_error": float(np.median(ob)), "cores": 1}
    return out


def cso_sec33(S):
    """The paper's CSO shape (Sec. 3.3): swarm 300, 1e6 evaluations, 1000-D,
    5 runs, float -- here on the shifted-rotated Rastrigin (the trigonometric
    group), the 5 runs batched through sevo_run_grid in FP32 CUDA-core mode
    with FP64 refinement, against the oracle on one host core timed over a
    bounded sample of 2,000 evaluations and extrapolated per evaluation."""
    import numpy as np
    import oracle as O
    D, NP, budget, runs = 1000, 300, 1000000, 5
    p = S.Problem(0x5EB00002, 2, D)
    a = S.alg_params(S.CSO, NP, budget, w=0.1, prec=S.FP32)
    t0 = time.perf_counter()
    r = S.sevo_run_grid([p], [a], [(0, 0, s) for s in range(1, runs + 1)])
    wall = time.perf_counter() - t0
    q = O.Problem(0x5EB00002, 2, D)
    sample = 2000
    t0 = time.perf_counter()
    O.run(q, O.make_alg(O.ALG_CSO, NP, sample, w=0.1), 1)
    osec = time.perf_counter() - t0
    per_eval = osec / sample
    return {"workload": "CSO swarm 300, phi 0.1, 1e6 evals, D=1000, 5 runs, shifted-rotated "
                        "Rastrigin, FP32 + FP64 refinement",
            "gpu_wall_s_5_runs": round(wall, 3), "gpu_evals_per_s": round(r["evals"] / wall, 1),
            "median_final_error": float(np.median(r["best"])),
            "oracle": {"sample_evals": sample, "sample_wall_s": round(osec, 3), "cores": 1,
                       "extrapolated_wall_s_5_runs": round(per_eval * runs * budget, 1)},
            "speedup_vs_oracle_extrapolated": round(per_eval * runs * budget / wall, 1)}


def c0_single_run(S):
    """The smallest configuration: DE/rand/1/bin, NP = 50, D = 10, FP64, one
    run of 1e5 evaluations on shifted-rotated Rastrigin, seed 1 -- GPU run
    through sevo_run_grid (graph-captured generations) and the oracle's own
    run on one host core."""
    import oracle as O
    p = S.Problem(0x5EB00002, 2, 10)
    a = S.alg_params(S.DE_RAND1, 50, 100000)
    S.sevo_run_grid([p], [a], [(0, 0, 1)])  # warm-up (instance upload, graph build)
    t0 = time.perf_counter()
    r = S.sevo_run_grid([p], [a], [(0, 0, 1)])
    wall = time.perf_counter() - t0
    q = O.Problem(0x5EB00002, 2, 10)
    t0 = time.perf_counter()
    ro = O.run(q, O.make_alg(O.ALG_DE_RAND1, 50, 100000), 1)
    owall = time.perf_counter() - t0
    return {"workload": "DE/rand/1/bin NP=50 D=10 F=0.5 CR=0.9 FP64, 1e5 evals, shifted-rotated "
                        "Rastrigin, seed 1",
            "gpu_wall_s": round(wall, 4), "gpu_device_ms": round(r["wall_ms"], 3),
            "gpu_best": r["best"][0], "oracle_wall_s": round(owall, 4), "oracle_best": ro["best"],
            "oracle_cores": 1, "gens": int(r["gens"][0])}


def e2e_rate(S, torch, states, gen, K):
    """Same step through the C ABI with host buffers: every step each state's
    population is copied in from pinned host memory, the generation runs and
    the fitness of all its rows is copied out to pinned host memory; the
    states' copies and generations are enqueued on their own streams
    (sevo_state_set_async / sevo_state_get_async).  The host reads every
    step's results one step late: after enqueuing step g it waits for step
    g - 1's fitness (double-buffered pinned result buffers) and takes its
    minimum, so that step g's input copies overlap step g - 1's tail.  The
    timed region ends when the last step's results are on the host; every
    copy is inside it."""
    import numpy as np
    rows = [st.R * NP for st in states]
    hostX = [torch.empty((r, D), dtype=torch.float64).pin_memory() for r in rows]
    hostF = [[torch.empty(r, dtype=torch.float64).pin_memory() for r in rows] for _ in range(2)]
    for st, hx in zip(states, hostX):
        hx.copy_(torch.from_numpy(st.get()["X"]))
    lib = S.lib()
    import ctypes as C
    dp = C.POINTER(C.c_double)
    best = float("inf")

    def consume(evs, buf):
        nonlocal best
        for ev in evs:
            ev.synchronize()
        best = min(best, min(float(np.min(h.numpy())) for h in buf))

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prev = None
    for k, g in enumerate(range(gen, gen + K)):
        buf = hostF[k % 2]
        for st, hx in zip(states, hostX):
            S.check(lib.sevo_state_set_async(st.h, C.cast(C.c_void_p(hx.data_ptr()), dp), None,
                                             None, 0, None, None, None, -1), "sevo_state_set_async")
        for grp in groups_of(states):
            S.check(S.sevo_state_step_many(grp, g), "sevo_state_step_many")
        evs = []
        for st, hf in zip(states, buf):
            S.check(lib.sevo_state_get_async(st.h, None, C.cast(C.c_void_p(hf.data_ptr()), dp),
                                             None, None, None, None, None, None),
                    "sevo_state_get_async")
            ev = torch.cuda.Event()
            ev.record(st.torch_stream)
            evs.append(ev)
        if prev is not None:
            consume(*prev)
        prev = (evs, buf)
    consume(*prev)
    dt = (time.perf_counter() - t0) / K
    evals = sum(rows)
    return {"value": round(evals / dt, 1), "unit": "evals/s",
            "h2d_bytes_per_step": sum(r * D * 8 for r in rows),
            "d2h_bytes_per_step": sum(r * 8 for r in rows),
            "path": "sevo_state_set_async (pinned X in) per state on its own stream, "
                    "sevo_state_step_many, sevo_state_get_async (pinned fitness out) per state; "
                    "the host reads each step's results (their minimum) while the next step "
                    "runs, double-buffered",
            "best_seen": best}, gen + K


# ---------------------------------------------------------------- grid
GRID_DIMS = (10, 30, 50, 100)
GRID_RUNS = 51


def grid_problems(S_or_O, D, make):
    """30 seeded problems of dimension D: 10 single-family (the six families
    cycled), 10 hybrid, 10 composition."""
    out = []
    for i in range(10):
        out.append(make(0xC3000000 + 1000 * D + i, i % 6, D))
    for i in range(10):
        out.append(make(0xC3100000 + 1000 * D + i, 6, D))
    for i in range(10):
        out.append(make(0xC3200000 + 1000 * D + i, 7, D))
    return out


def grid_algs(S, D, prec):
    b = 10000 * D
    return [S.alg_params(1, 18 * D, b, prec=prec),   # DE current-to-pbest/1/bin + archive
            S.alg_params(2, 40, b, prec=prec),       # PSO gbest
            S.alg_params(3, 40, b, prec=prec)]       # PSO ring


def run_grid_bench(S, dims, prec, runs=GRID_RUNS):
    """The whole grid in one sevo_run_grid call: one bucket per (algorithm,
    D), all buckets running side by side."""
    names = ("de_ctpb", "pso_gbest", "pso_ring")
    probs, algs, tasks = [], [], []
    for D in dims:
        p0, a0 = len(probs), len(algs)
        ps = grid_problems(S, D, lambda seed, fam, d: S.Problem(seed, fam, d))
        probs += ps
        algs += grid_algs(S, D, prec)
        tasks += [(p0 + pi, a0 + ai, 1 + r + 1000 * pi) for pi in range(len(ps)) for ai in range(3)
                  for r in range(runs)]
    r = S.sevo_run_grid(probs, algs, tasks)
    succ = {n: [0, 0] for n in names}
    for (pi, ai, _), ok in zip(tasks, r["success"]):
        succ[names[ai % 3]][0] += int(ok)
        succ[names[ai % 3]][1] += 1
    return {"wall_ms": r["wall_ms"], "evals": int(r["evals"]), "tasks": len(tasks),
            "success": {k: round(v[0] / max(v[1], 1), 4) for k, v in succ.items()}}


def wilson(k, n, z=1.959963984540054):
    """95 % Wilson score interval of a success proportion k / n."""
    if n == 0:
        return [0.0, 1.0]
    p = k / n
    den = 1.0 + z * z / n
    mid = (p + z * z / (2 * n)) / den
    half = z * ((p * (1 - p) / n + z * z / (4 * n * n)) ** 0.5) / den
    return [round(mid - half, 4), round(mid + half, 4)]


def success_vs_fp64(S, large=True):
    """Mixed precision (TF32 rotation + FP64 refinement) against the plain
    FP64 GPU path on the same runs (same seeds): success rate at 1e-8 with
    its 95 % interval, median final error and evaluations per second.
    D = 100: 5 problems (Rastrigin, Griewank, Ackley, hybrid, composition)
    x 11 seeds x {DE current-to-pbest NP = 18 D, PSO ring NP = 40} at the
    full budget 1e4 D.  D = 1000: 2 hybrid + 2 composition instances x 3
    seeds x {DE NP = 200, PSO NP = 1000} at 1e5 evaluations (1/30 of the 3e6
    budget, so that the FP64 path's runs -- about 7e4 evaluations per second
    at this size -- fit the benchmark's time; at this budget no run of either
    path reaches 1e-8, so the final-error medians are the comparison)."""
    import numpy as np
    out = {}
    cases = [(100, [(0x5EB10000 + f, f) for f in (2, 5, 4, 6, 7)], 11,
              [(1, 18 * 100), (3, 40)], 10 ** 6)]
    if large:
        cases.append((1000, [(0x5EB20000 + i, 6) for i in range(2)] +
                      [(0x5EB20100 + i, 7) for i in range(2)], 3, [(1, 200), (3, 1000)], 100000))
    for D, plist, seeds, alg_np, budget in cases:
        probs = [S.Problem(sd, f, D) for sd, f in plist]
        tasks = [(pi, ai, 7 + s + 100 * pi) for pi in range(len(probs)) for ai in range(len(alg_np))
                 for s in range(seeds)]
        row = {"problems": len(probs), "seeds": seeds, "budget": budget}
        for name, prec in (("tf32", S.TF32), ("fp64", S.FP64)):
            algs = [S.alg_params(a, npop, budget, prec=prec) for a, npop in alg_np]
            r = S.sevo_run_grid(probs, algs, tasks)
            per = {}
            for ai, (a, npop) in enumerate(alg_np):
                idx = [t for t, (_, aj, _) in enumerate(tasks) if aj == ai]
                ok = int(np.sum(np.asarray(r["success"])[idx]))
                key = ("de_ctpb" if a == 1 else "pso_ring") + f"_np{npop}"
                per[key] = {"success": ok, "runs": len(idx), "ci95": wilson(ok, len(idx)),
                            "median_final_error": float(np.median(np.asarray(r["best"])[idx]))}
            row[name] = {"wall_s": round(r["wall_ms"] / 1e3, 3),
                         "evals_per_s": round(r["evals"] / (r["wall_ms"] / 1e3), 1), "algs": per}
        row["tf32_speedup"] = round(row["tf32"]["evals_per_s"] / row["fp64"]["evals_per_s"], 2)
        out[f"d{D}"] = row
    return out


def fp64_peak(torch):
    """FP64 instruction rate of this GPU, measured here: a cuBLAS DGEMM of
    4096^3 timed with CUDA events (best of 5), n^3 multiply-adds, each one
    FP64 instruction (the unit the operators' per-coordinate counts use: a
    DADD, DMUL or DFMA is one operation)."""
    n = 4096
    a = torch.rand((n, n), dtype=torch.float64, device="cuda")
    b = torch.rand((n, n), dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return float(n) ** 3 / (best * 1e-3)


def oracle_grid_sample(dims, frac=0.1):
    """The oracle's thread pool on 3 problems (single, hybrid, composition)
    per (algorithm, D) with one run each at frac of the budget; extrapolated
    to the full grid (30 problems x 51 runs, whole budget) by evaluations."""
    import oracle as O
    probs, algs, seeds, full_evals, sample_evals = [], [], [], 0, 0
    for D in dims:
        gp = grid_problems(O, D, lambda seed, fam, d: O.Problem(seed, fam, d))
        for pi in (0, 10, 20):
            for kind, NP in ((O.ALG_DE_CTPB, 18 * D), (O.ALG_PSO_GBEST, 40),
                             (O.ALG_PSO_RING, 40)):
                probs.append(gp[pi])
                algs.append(O.make_alg(kind, NP, int(frac * 10000 * D)))
                seeds.append(1 + pi)
                sample_evals += int(frac * 10000 * D)
                full_evals += 10 * GRID_RUNS * 10000 * D  # 10 problems of this type x 51 runs
    t0, c0 = time.perf_counter(), time.process_time()
    O.run_many(probs, algs, seeds, nthreads=oracle_cores())
    dt, cpu = time.perf_counter() - t0, time.process_time() - c0
    cores = oracle_cores()
    # CPU seconds scale with evaluations; a full grid keeps every core busy
    full_cpu = cpu * full_evals / sample_evals
    return {"sample_wall_s": round(dt, 3), "sample_cpu_s": round(cpu, 3),
            "sample_evals": sample_evals, "cores": cores,
            "extrapolated_full_wall_s": round(full_cpu / cores, 1),
            "sample": f"3 problems (single, hybrid, composition) x 3 algorithms x D in {list(dims)}, "
                      f"one run each at {frac:g} of the budget, thread pool on all host cores; "
                      "extrapolated to 30 problems x 51 runs at the full budget by evaluation count"}


# ---------------------------------------------------------------- oracle arm
class OracleStep:
    """The oracle's own operators on a bounded sample of the workload: the
    same three algorithms x six families at D = 100 with NP = npop."""

    def __init__(self, npop, seed0=1):
        import numpy as np
        import oracle as O
        self.O, self.np = O, np
        self.npop = npop
        self.probs = [O.Problem(0x5EB00000 + f, f, D) for f in range(FAMILIES)]
        self.st = []
        for k, (_, alg) in enumerate(ALGS):
            for f, q in enumerate(self.probs):
                seed = seed0 + 1000 * k + f
                X = O.init_population(seed, npop, D)
                fx = q.eval(X)
                s = {"alg": alg, "q": q, "seed": seed, "X": X, "fx": fx,
                     "A": np.zeros((npop, D)), "asize": 0}
                if alg >= 2:
                    s.update(V=np.zeros_like(X), P=X.copy(), fp=fx.copy(),
                             guide=O.pso_guides(fx, alg - 2))
                self.st.append(s)
        self.gen = 0

    def step(self):
        O = self.O
        self.gen += 1
        g = self.gen
        for s in self.st:
            q = s["q"]
            if s["alg"] == 0:
                U, _ = O.de_rand1_trials(s["seed"], g, s["X"])
                fu = q.eval(U)
                s["X"], s["fx"], _, _, _ = O.de_select(s["seed"], g, s["X"], s["fx"], U, fu)
            elif s["alg"] == 1:
                U, _ = O.de_ctpb_trials(s["seed"], g, s["X"], s["fx"], s["A"], s["asize"])
                fu = q.eval(U)
                s["X"], s["fx"], s["A"], s["asize"], _ = O.de_select(
                    s["seed"], g, s["X"], s["fx"], U, fu, s["A"], s["asize"])
            else:
                s["X"], s["V"] = O.pso_move(s["seed"], g, s["X"], s["V"], s["P"], s["guide"])
                s["fx"] = q.eval(s["X"])
                s["P"], s["fp"], _ = O.pso_update(s["X"], s["fx"], s["P"], s["fp"])
                s["guide"] = O.pso_guides(s["fp"], s["alg"] - 2)
        return len(self.st) * self.npop


def oracle_cores():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


def cpu_baseline(npop=NP, steps=30):
    o = OracleStep(npop)
    o.step()
    t0 = time.perf_counter()
    ev = 0
    for _ in range(steps):
        ev += o.step()
    dt = time.perf_counter() - t0
    return {"value": round(ev / dt, 1), "unit": "evals/s", "cores": oracle_cores(),
            "kind": "oracle",
            "sample": f"{steps} generations of the 3 algorithms x 6 families at D={D} with "
                      f"NP={npop} (the workload's operators and evaluation, {ev} evals)"}


def max_over_ranks(ms, dist=None):
    """The timed region's milliseconds, the maximum over all ranks (every
    rank receives it); the ranks then meet at a barrier.  One process: ms."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def whole_job_rate(evals_per_step, world, ms_per_step):
    """Evaluations per second of the whole job: every rank runs its own
    replica of the step's evaluations, timed by the slowest rank."""
    return evals_per_step * world / (ms_per_step * 1e-3)


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    # each step is the workload's generation on a population sample sized so
    # that the whole run takes about a minute on the host cores
    npop = max(64, min(NP, int(NP * 24 / max(args.steps + args.warmup, 1))))
    o = OracleStep(npop)
    for _ in range(args.warmup):
        o.step()
    t0 = time.perf_counter()
    ev = 0
    for _ in range(args.steps):
        ev += o.step()
    dt = time.perf_counter() - t0
    v = ev / dt
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": NP, "D": D, "families": FAMILIES,
                       "sample_np": npop},
            "cpu_baseline": {"value": round(v, 1), "unit": "evals/s", "cores": oracle_cores(),
                             "kind": "oracle",
                             "sample": f"each step: one generation of the 3 algorithms x 6 "
                                       f"families at D={D}, NP={npop}"},
            "e2e": {"value": round(v, 1), "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def eval_only(spec):
    """Three evaluation calls of ROWS x D rows ~ U[-100, 100] (a small fixed
    workload for profiler captures of one evaluation kernel)."""
    import torch
    import paper_2505_17430_gb300 as S
    rows, Dv, prec, fam = int(spec[0]), int(spec[1]), spec[2].upper(), int(spec[3])
    S.build()
    X = torch.empty((rows, Dv), dtype=torch.float64, device="cuda").uniform_(-100, 100)
    out = torch.empty(rows, dtype=torch.float64, device="cuda")
    p = S.Problem(0x5EB00000 + fam, fam, Dv)
    for _ in range(3):
        p.evaluate(X, out, prec=getattr(S, prec))
    torch.cuda.synchronize()
    print(json.dumps({"eval_only": True, "rows": rows, "D": Dv, "prec": prec, "family": fam,
                      "checksum": float(out.sum())}))
    return 0


# ---------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-grid", action="store_true", help="skip the run-grid measurement")
    ap.add_argument("--no-large-d", action="store_true", help="skip the D=1000/5000 rates")
    ap.add_argument("--eval-only", nargs=4, metavar=("ROWS", "D", "PREC", "FAMILY"),
                    help="evaluate ROWS x D uniform rows three times with one mode "
                         "(tf32|bf16x3|fp32|fp64) on one family (0-7); for profiling")
    ap.add_argument("--only-steps", action="store_true",
                    help="time the steps only (for launch-list profiling)")
    ap.add_argument("--timeline", metavar="PATH",
                    help="after the timed steps, trace 20 more steps launch by launch and "
                         "write the spans (kind, stream, start ms, end ms) to PATH as JSON")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.eval_only:
        return eval_only(args.eval_only)

    import torch
    import paper_2505_17430_gb300 as S

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    S.build()
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))
    if "hbm_gbs" not in peaks:
        peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}

    seed0 = 1 + 100000 * rank
    probs, states = make_states(S, S.TF32, seed0, torch)
    gen = run_steps(states, 1, args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = S.lib().sevo_kernel_launches()
    ms, gen = time_steps(torch, states, gen, args.steps)
    launches = S.lib().sevo_kernel_launches() - l0
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist)
    evals_per_step = sum(st.R * NP for st in states)
    ms_per_step = ms / args.steps
    value = whole_job_rate(evals_per_step, world, ms_per_step)

    if args.timeline and rank == 0:
        gen = write_timeline(S, torch, states, gen, 20, args.timeline)
    if rank != 0 or args.only_steps:
        if args.only_steps and rank == 0:
            print(json.dumps({"only_steps": True, "value": round(value, 1),
                              "ms_per_step": round(ms_per_step, 4), "gpu_launches": launches}))
        if dist:
            dist.destroy_process_group()
        return 0

    # FP64 GPU path, same step (plain DFMA rotation, FP64 bodies)
    _, st64 = make_states(S, S.FP64, seed0, torch)
    g64 = run_steps(st64, 1, 1)
    ms64, _ = time_steps(torch, st64, g64, 2)
    fp64 = {"value": round(evals_per_step / (ms64 / 2 * 1e-3), 1),
            "ms_per_step": round(ms64 / 2, 3)}
    del st64
    KT = min(args.steps, 200)
    f64peak = fp64_peak(torch)
    traced, gen, rs = traced_step_kernels(S, torch, states, gen, KT)
    roof, stream_roof, shares = rooflines(traced, states, peaks, KT, f64peak, rs)
    traced1, gen, rs1 = traced_step_kernels(S, torch, states, gen, KT, serial=True)
    roof1, stream1, shares1 = rooflines(traced1, states, peaks, KT, f64peak, rs1)
    roof["alone"] = {k: roof1[k] for k in ("achieved", "frac", "launch_ms")}
    for k in stream_roof:
        if stream_roof[k] and stream1.get(k):
            stream_roof[k]["alone"] = {q: stream1[k][q] for q in ("achieved", "frac", "launch_ms")}
            if stream1[k].get("fp64_pipe"):
                stream_roof[k]["alone"]["fp64_frac"] = stream1[k]["fp64_pipe"]["frac"]
    dom = dominant_roofline(shares, roof, stream_roof)
    if dom is not roof and stream_roof[dom["kernel"]].get("alone"):
        a = stream_roof[dom["kernel"]]["alone"]
        dom["alone"] = {"frac": a.get("fp64_frac"), "launch_ms": a["launch_ms"]}
    e2e, gen = e2e_rate(S, torch, states, gen, max(3, min(args.steps // 4, 400)))
    modes = mode_eval_rates(S, torch, probs)
    large = None if args.no_large_d else large_d_rates(S, torch, peaks)
    c4 = None if args.no_large_d else c4_sample(S)
    c0 = c0_single_run(S)
    sh31 = shade_sec31(S)
    psode4 = psode_case1(S)
    cso33 = None if args.no_large_d else cso_sec33(S)
    svf = success_vs_fp64(S, large=not args.no_large_d)
    cpu = None if args.no_cpu_baseline else cpu_baseline()
    grid = None
    if not args.no_grid:
        g = run_grid_bench(S, GRID_DIMS, S.TF32)
        g64 = run_grid_bench(S, (10,), S.FP64)
        g32 = run_grid_bench(S, (10,), S.TF32)
        og = None if args.no_cpu_baseline else oracle_grid_sample(GRID_DIMS)
        grid = {"workload": "30 problems (10 single, 10 hybrid, 10 composition) x D in "
                            "{10,30,50,100} x 51 runs x {DE ctpb/1/bin+archive NP=18D, PSO gbest "
                            "NP=40, PSO ring NP=40}, budget 10000*D, TF32 + FP64 refinement",
                "gpu_wall_s": round(g["wall_ms"] / 1e3, 3), "evals": g["evals"],
                "evals_per_s": round(g["evals"] / (g["wall_ms"] / 1e3), 1),
                "tasks": g["tasks"], "success_rate_tf32": g["success"],
                "d10_success_fp64_vs_tf32": {"fp64": g64["success"], "tf32": g32["success"],
                                             "fp64_wall_s": round(g64["wall_ms"] / 1e3, 3),
                                             "tf32_wall_s": round(g32["wall_ms"] / 1e3, 3)},
                "oracle": og}
        if og:
            grid["speedup_vs_oracle_extrapolated"] = round(
                og["extrapolated_full_wall_s"] / (g["wall_ms"] / 1e3), 1)
    line = {"metric": METRIC, "value": round(value, 1), "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "tf32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": NP, "D": D, "families": FAMILIES,
                       "algorithms": [a for a, _ in ALGS], "evals_per_step": evals_per_step,
                       "prec": "tf32 rotation, fp32 bodies, fp64 shift/refine/positions",
                       "l2": "working set ~160 MB per step > 129 MB L2 (no flush needed)",
                       "kernel_times": "per-kernel CUDA-event times from a traced repeat of "
                                       "the timed steps (events on the launching stream); "
                                       "'alone': a second repeat in which the device "
                                       "drains after every generation",
                       "restart_every": RESTART_EVERY,
                       "streams": f"{GROUPS} groups of 3 states (one per algorithm, "
                                  f"{FAMILIES // GROUPS} populations each), one CUDA stream "
                                  "per state; each step one sevo_state_step_many call per "
                                  "group (operators on each state's stream, one fused "
                                  "evaluation of the group's rows, selections on each "
                                  "stream); the timed region is forked from and joined to "
                                  "one stream by events",
                       "parallelism": f"replicas x{world}"},
            "roofline": dom, "eval_roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk, "fp64_path": fp64, "streaming_rooflines": stream_roof,
            "kernel_shares": shares, "kernel_shares_alone": shares1,
            "eval_only_evals_per_s": modes, "large_d": large,
            "c4_sample": c4, "shade_sec31": sh31, "psode_case1": psode4, "cso_sec33": cso33,
            "c0_single_run": c0, "grid": grid, "success_vs_fp64": svf,
            "fp64_peak_op_per_s": round(f64peak / 1e9, 2) * 1e9}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
