#!/usr/bin/env python
"""Benchmark of synchronous parallel simulated annealing on one GB300 (or N replicas).

Default workload (one "step" = one full annealing run): normalised Schwefel,
n = 256, box [-500, 500]^n, 262144 chains, L = 1000 Metropolis steps per level,
200 levels, T0 = 100, rho = 0.95, sigma = 0.1 width sqrt(T/T0), FP32 state with
FP64 argmin, seed 0 -- 5.24e10 Metropolis steps per run.  ``--workload`` selects
the other workloads (measurement lines for the other rows; the default line is
the headline).

Prints one JSON line: Metropolis steps/s (device-timed, inputs resident), the
same through the public C ABI with host buffers (e2e), time-to-target, the
roofline of the sweep kernel, sampled clocks, and the FP64 CPU oracle timed on
this host's cores as a baseline.  ``--impl reference`` times the oracle alone.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Metropolis steps/s and time-to-target (best f within 1e-6 rel) on 1 GB300"
UNIT = "Metropolis steps/s"
MUFU_PER_CLK_SM = 16
# Algorithmic SFU operations per Metropolis step, per cost: the proposal needs
# log2 and sqrt (Box-Muller radius) and cos (angle); the acceptance test one
# log2 (tau = -T ln u3); the energy difference the transcendental terms of the
# new coordinate value only (the old one's term can be kept): Schwefel sqrt +
# sin, Rastrigin cos, Ackley cos + sqrt + 2 exp, Rosenbrock none.
# Rotated costs: every rotated coordinate changes, so n transcendental terms
# per step (Rastrigin: one sine per coordinate in the product-to-sum form;
# Schwefel: sqrt and sine of the new term) plus the 4 of the proposal and test.
SFU_PER_STEP = {"schwefel": 6, "rastrigin": 5, "ackley": 8, "rosenbrock": 4}


def sfu_per_step(cost, n, proposal="gaussian"):
    # a uniform redraw of the coordinate needs none of the Gaussian step's lg2, sqrt and cos
    less = 3 if proposal == "uniform" else 0
    if cost == "rot_rastrigin":
        return n + 4 - less
    if cost == "rot_schwefel":
        return 2 * n + 4 - less
    return SFU_PER_STEP[cost] - less


def step_ops(cost, n, proposal="gaussian"):
    """Algorithmic operations of one Metropolis step per measured pipe: the SFU
    functions by kind (their sum is sfu_per_step), and one Philox4x32-10 block
    (the step's four random words: coordinate, the two uniforms of the move, the
    acceptance uniform), whose 32x32 -> 64-bit products run on the integer
    multiply pipe."""
    ops = {"lg2": 1, "sqrt": 0, "sin": 0, "cos": 0, "ex2": 0, "philox": 1}  # lg2: tau = -T ln u3
    if proposal != "uniform":
        ops["lg2"] += 1   # Box-Muller radius sqrt(-2 ln u1) ...
        ops["sqrt"] += 1
        ops["cos"] += 1   # ... and angle cos(2 pi u2)
    if cost == "schwefel":
        ops["sqrt"] += 1
        ops["sin"] += 1
    elif cost == "rastrigin":
        ops["cos"] += 1
    elif cost == "ackley":
        ops["cos"] += 1
        ops["sqrt"] += 1
        ops["ex2"] += 2
    elif cost == "rot_rastrigin":
        ops["sin"] += n
    elif cost == "rot_schwefel":
        ops["sqrt"] += n
        ops["sin"] += n
    assert sum(v for k, v in ops.items() if k != "philox") == sfu_per_step(cost, n, proposal)
    return ops


PIPE_OPS_MEASURED = ("lg2", "sqrt", "sin", "cos", "ex2", "philox", "imad_wide", "imad_hi", "imad_lo", "lop3", "ffma")


def measure_pipes(sa):
    """Operations per clock per SM of each pipe the step uses, measured on this GPU (sa_pipe_rate)."""
    return {op: sa.pipe_rate(op, 4096)[0] for op in PIPE_OPS_MEASURED}


def pipe_roofline(w, pipes, sms, sm_mhz, sweep_ms):
    """Roofline of the sweep: steps/s that each pipe allows (its measured rate over the
    algorithmic operations of a level's steps), the binding (lowest) one, and the sweep's
    achieved steps/s against it."""
    per_level = {k: 0.0 for k in ("lg2", "sqrt", "sin", "cos", "ex2", "philox")}
    for p in w.problems:
        for k, v in step_ops(p["cost"], p["n"], w.proposal).items():
            per_level[k] += v * p["chains"] * w.L
    steps_level = sum(p["chains"] for p in w.problems) * w.L
    clk = sm_mhz * 1e6 * sms
    t_sfu = sum(per_level[k] / (pipes[k] * clk) for k in ("lg2", "sqrt", "sin", "cos", "ex2"))
    t_philox = per_level["philox"] / (pipes["philox"] * clk)
    roofs = {"sfu": steps_level / t_sfu, "philox_imad": steps_level / t_philox}
    binding = min(roofs, key=roofs.get)
    achieved = steps_level / (sweep_ms * 1e-3)
    return achieved, roofs, binding


SWEEP_SOURCES = ["sweep_f32.cu", "sweep_f32w.cu", "sweep_rot.cu", "sa_device.cuh", "sa_internal.h"]
WARMUP_MIN_S = 4.0
WORKLOADS = ("schwefel_n256", "schwefel_n2", "batched", "rot_rastrigin_n1024", "rot_schwefel_n128")
ROT_WORKLOADS = {"rot_rastrigin_n1024": "ROT_RASTRIGIN_N1024", "rot_schwefel_n128": "ROT_SCHWEFEL_N128"}
# The delayed-acceptance level's launch count: training steps per level and kernels per
# training step (batch draw, weights' cast, forward, loss, backward, Adam), buffer insertions.
DA_TRAIN_STEPS, DA_LAUNCHES_PER_TRAIN_STEP, DA_INSERTS = 128, 22, 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=WORKLOADS, default="schwefel_n256")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--levels", type=int, default=0, help="override the level count (profiling runs only)")
    ap.add_argument("--polish-k", type=int, default=0,
                    help="the hybrid SA: polish the k best final states by projected gradients after the last "
                         "level (its time counts in the run; time-to-target may then be reached at the run's end)")
    ap.add_argument("--proposal", choices=["gaussian", "uniform"], default="gaussian",
                    help="the move: the workloads' Gaussian step, or the paper's reading (a uniform redraw of the "
                         "chosen coordinate)")
    ap.add_argument("--surrogate", action="store_true",
                    help="rotated workloads: the delayed-acceptance sweep with the learned surrogate (two-stage "
                         "acceptance, the network trained between levels) instead of the plain rotated sweep")
    ap.add_argument("--independent", action="store_true",
                    help="asynchronous chains (no exchange between levels; the paper's V1), single-problem workloads")
    ap.add_argument("--gemm-route", action="store_true",
                    help="time the rotated costs' GEMM route at the rotated Rastrigin n = 1024 workload's shape "
                         "(every step's candidates Y' = X' Q^T on the tensor cores) against the rank-1 sweep")
    ap.add_argument("--paper-schwefel", action="store_true",
                    help="the paper's Schwefel accuracy and timing tables instead (T0 = 1000, rho = 0.99, 1146 levels "
                         "of N = 100, 16384 chains, n = 8 .. 512, uniform redraw moves): V2 and V1 per n")
    ap.add_argument("--suite", action="store_true",
                    help="the paper's 41-problem test suite (Tables 8-9) instead: one synchronous run per problem, "
                         "then the hybrid's Nelder-Mead polish (one JSON line per problem and a summary)")
    ap.add_argument("--convergence", action="store_true",
                    help="the convergence study of Sec. 4.1 (Figures 4-5) instead: relative error of the best value "
                         "against explored points for V0, V1 and V2 at equal numbers of explored points, n = 8 .. 256 "
                         "(one JSON line per n)")
    ap.add_argument("--surrogate-vs-plain", action="store_true",
                    help="the learned-surrogate workload (rotated Schwefel n = 128, 131072 chains, L = 2000, 150 "
                         "levels) in full, plain Metropolis and delayed acceptance, each with the hybrid's projected "
                         "gradients from the 64 best final states: time-to-target against the best FP64 value found")
    ap.add_argument("--surrogate-forward", action="store_true",
                    help="time the surrogate's forward pass at the delayed-acceptance step's shape (131072 rows of "
                         "n = 128): the one-kernel tensor-core pass against the two GEMMs with fused epilogues")
    ap.add_argument("--seeds", type=int, default=1,
                    help="--surrogate-vs-plain: run the comparison for this many seeds (one JSON line each)")
    ap.add_argument("--hybrid", action="store_true",
                    help="the hybrid SA of Table 10 instead: annealing stopped early, then Nelder-Mead or projected "
                         "gradients from its best final states (one JSON line per function)")
    return ap.parse_args()


# ------------------------------------------------------------------ workloads
class Workload:
    """One workload: how to build its handle and what one run amounts to."""

    def __init__(self, name, levels_override=0, independent=False, proposal="gaussian", polish_k=0, surrogate=False):
        from paper_2408_00018_gb300 import inputs
        self.name = name
        self.surrogate = bool(surrogate)
        if self.surrogate and name not in ROT_WORKLOADS:
            raise SystemExit("--surrogate: rotated workloads only")
        self.independent = bool(independent)
        self.proposal = proposal
        self.polish_k = int(polish_k)
        if name in ("schwefel_n256", "schwefel_n2") or name in ROT_WORKLOADS:
            if name in ROT_WORKLOADS:
                cfg = dict(getattr(inputs, ROT_WORKLOADS[name]))
            else:
                cfg = dict(inputs.SCHWEFEL_N256_FP32 if name == "schwefel_n256" else inputs.SCHWEFEL_N2_FP64)
            if levels_override:
                cfg["levels"] = levels_override
            lo, hi = inputs.box(cfg["cost"], cfg["n"])
            Q = inputs.rotation(cfg["n"], cfg["q_seed"]) if "q_seed" in cfg else None
            self.problems = [{"cost": cfg["cost"], "n": cfg["n"], "chains": cfg["chains"], "lo": lo, "hi": hi, "Q": Q}]
            self.L, self.K, self.T0, self.rho = cfg["L"], cfg["levels"], cfg["T0"], cfg["rho"]
            self.sigma_frac, self.precision, self.seed = cfg["sigma_frac"], cfg["precision"], cfg["seed"]
            self.batch = False
            self.tag = (f"{cfg['cost']}_n{cfg['n']}_c{cfg['chains']}_L{cfg['L']}_K{cfg['levels']}_{cfg['precision']}"
                        + (f"_Q{cfg['q_seed']}" if Q is not None else ""))
        else:  # 512 independent problems of uneven n and chain count
            self.problems = inputs.batch_problems(count=512, seed=0)
            self.L, self.K = 500, levels_override or 100
            self.T0, self.rho, self.sigma_frac, self.precision, self.seed = 100.0, 0.95, 0.1, "fp32", 0
            self.batch = True
            self.tag = f"batched512_L500_K{self.K}_fp32_autotuned"
        self.steps_per_run = sum(p["chains"] for p in self.problems) * self.L * self.K
        self.sfu_per_level = sum(p["chains"] * self.L * sfu_per_step(p["cost"], p["n"], proposal)
                                 for p in self.problems)
        self.f_star = [inputs.F_STAR.get(p["cost"]) for p in self.problems]
        self.rotated = [p["cost"].startswith("rot_") for p in self.problems]

    def schedule(self, sa):
        return sa.Schedule(T0=self.T0, rho=self.rho, levels=self.K, sigma_frac=self.sigma_frac,
                           precision=self.precision, independent=1 if self.independent else 0,
                           proposal=self.proposal, polish_k=self.polish_k, surrogate=1 if self.surrogate else 0)

    def create(self, sa, tune=True):
        if self.batch:
            h = sa.create_batch(self.problems, self.L, self.schedule(sa), seed=self.seed)
            if tune:
                h.autotune()
            return h
        p = self.problems[0]
        return sa.create(p["cost"], p["lo"], p["hi"], p["n"], p["chains"], self.L, self.schedule(sa), seed=self.seed,
                         Q=p.get("Q"))

    def launches_per_run(self, h):
        groups = len(h.describe())
        rot = sum(self.rotated)
        if self.surrogate:
            # per level: the statistics, DA_TRAIN_STEPS training steps of DA_LAUNCHES_PER_TRAIN_STEP
            # kernels, the weights' cast, bits cleared, start states, their f~ (2 GEMMs and the head
            # sum), L steps of (patch, 2 GEMMs, step), the buffer insertions, the level's end; then
            # the argmin/restart, the restart transform and the level advance
            per_level = (1 + DA_TRAIN_STEPS * DA_LAUNCHES_PER_TRAIN_STEP + 1 + 1 + 1 + 3 + 4 * self.L
                         + DA_INSERTS + 1)
            return 1 + 2 * rot + 2 + self.K * (per_level + 2 + rot)  # (+ 2: the network's init and reset)
        if groups == 1 and h.describe()[0]["kind"] == "fp32_batch_level":
            return 1 + self.K  # start stamp, then one launch per level (it ends every problem's level)
        # start stamp (+ initial points and Y0 = X0 Q^T per rotated problem), then per level the
        # group sweeps, the argmin/restart, the restart transform per rotated problem, the level advance
        return 1 + 2 * rot + self.K * (groups + 2 + rot)

    def config(self):
        c = {"workload": self.tag + ("_async" if self.independent else "") +
                         ("_surrogate" if self.surrogate else "") +
                         ("_uniform_moves" if self.proposal == "uniform" else "") +
                         (f"_polish{self.polish_k}" if self.polish_k else ""), "L": self.L, "levels": self.K,
             "T0": self.T0, "rho": self.rho, "seed": self.seed, "steps_per_run": self.steps_per_run, "argmin": "f64",
             "exchange": "none (asynchronous chains)" if self.independent else "restart from the level's best"}
        if self.batch:
            c.update({"problems": len(self.problems), "chains_total": sum(p["chains"] for p in self.problems),
                      "n_range": [min(p["n"] for p in self.problems), max(p["n"] for p in self.problems)],
                      "costs": "uniform over schwefel/rastrigin/ackley/rosenbrock"})
        else:
            p = self.problems[0]
            c.update({"cost": p["cost"], "n": p["n"], "chains": p["chains"]})
            if p.get("Q") is not None:
                c["Q"] = "Q factor of a seeded N(0,1) matrix (inputs.rotation)"
        return c


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
            return
        # wait for the first sample, so that nvidia-smi's start-up is over before any timing
        t0 = time.perf_counter()
        while self.lines() == 0 and time.perf_counter() - t0 < 10.0:
            time.sleep(0.05)

    def lines(self) -> int:
        try:
            with open(self.path) as fh:
                return sum(1 for _ in fh)
        except OSError:
            return 0

    def stop(self, window=None):
        """Median SM clock and active throttle reasons over the samples taken inside
        window = (first line, last line) (plus one sample on each side), else all."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if window is not None:
            rows = rows[max(0, window[0] - 1):window[1] + 1]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_id_for(dev: int) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


# ------------------------------------------------------------------ helpers
def source_hash(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2408_00018_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_from_profile(workload):
    """DRAM bytes per sweep launch from the committed ncu summary, if the profiled
    kernel's source files are unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    try:
        d = json.load(open(p)).get(workload)
        if not d or d.get("src_sha") != source_hash(d.get("files", SWEEP_SOURCES)):
            return None
    except Exception:
        return None
    return d.get("dram_bytes_per_launch")


def time_to_target(logs, t_start_ns, f_stars, final_f=None, run_s=None):
    """Per problem: first level whose incumbent is within 1e-6 max(1, |f*|) of f*; with the
    hybrid's polish, a problem whose polished incumbent (final_f) is within it counts as
    reached at the end of the run (run_s, the run's device time)."""
    if any(fs is None for fs in f_stars):
        return {"reached": None, "note": "no closed-form minimum for this cost (rotated Schwefel in a box)"}
    reached, last_t, gaps, by_polish = 0, 0.0, [], 0
    for p, (log, fs) in enumerate(zip(logs, f_stars)):
        tol = 1e-6 * max(1.0, abs(fs))
        hit = [l for l, f in enumerate(log["f_inc"]) if abs(f - fs) <= tol]
        if hit:
            reached += 1
            last_t = max(last_t, (int(log["t_ns"][hit[0]]) - int(t_start_ns)) * 1e-9)
        elif final_f is not None and abs(final_f[p] - fs) <= tol:
            reached += 1
            by_polish += 1
            last_t = max(last_t, run_s)
        else:
            f_last = float(log["f_inc"][-1])
            gaps.append(abs(f_last - fs) / max(1.0, abs(fs)))
    out = {"reached": reached == len(f_stars), "problems_reached": reached, "problems": len(f_stars),
           "seconds": last_t if reached == len(f_stars) else None}
    if by_polish:
        out["reached_by_polish"] = by_polish
    if gaps:
        out["worst_final_rel_gap"] = max(gaps)
        out["median_final_rel_gap"] = statistics.median(gaps)
    if len(f_stars) == 1 and not gaps and not by_polish:
        out["level"] = next(l for l, f in enumerate(logs[0]["f_inc"])
                            if abs(f - f_stars[0]) <= 1e-6 * max(1.0, abs(f_stars[0])))
    return out


def oracle_sample(w, budget_steps, threads):
    """The FP64 CPU oracle, as it stands, on level 0 (and 1) of a bounded part of the workload."""
    import oracle
    done, t0 = 0, time.perf_counter()
    descr = []
    mode = 0 if w.precision == "fp64" else 1
    for p_idx, p in enumerate(w.problems):
        levels = 1 if w.batch else (w.K if w.steps_per_run <= budget_steps else 2)
        chains = p["chains"]
        steps = chains * w.L * levels
        if done + steps > budget_steps:
            chains = max(1, (budget_steps - done) // (w.L * levels))
            steps = chains * w.L * levels
        op = oracle.Problem(p["cost"], p["n"], p["lo"], p["hi"], chains=chains, L=w.L, T0=w.T0, rho=w.rho,
                            sigma_frac=w.sigma_frac, seed=w.seed, problem=p_idx, mode=mode, threads=threads,
                            Q=p.get("Q"), independent=w.independent, proposal=w.proposal)
        op.run(levels)
        done += steps
        descr.append(p_idx)
        if done >= budget_steps:
            break
    dt = time.perf_counter() - t0
    if w.batch:
        what = f"level 0 of the first {len(descr)} of {len(w.problems)} problems, {done:.3g} steps"
    elif levels == w.K:
        what = f"the full run ({w.K} levels of {w.problems[0]['chains']} chains x L={w.L}), {done:.3g} steps"
    else:
        what = f"levels 0-1 of {w.problems[0]['chains'] if done >= w.problems[0]['chains'] * w.L * 2 else 'part of the'} chains x L={w.L}, {done:.3g} steps"
    return done / dt, dt, what + f" (FP64 oracle, {dt:.1f} s)"


# ------------------------------------------------------------------ our arm
def time_to_target_variant(args, sa, torch, flush, proposal, polish_k, runs=3):
    """Time-to-target of the default workload with another move and the hybrid's polish:
    one untimed run, then `runs` runs each timed on the device after an L2 flush; the
    fastest run's time-to-target (per-level device clock, or the run's end when the
    polished incumbent is what reaches the target)."""
    v = Workload(args.workload, 0, False, proposal, polish_k, False)
    h = v.create(sa)
    h.run()
    torch.cuda.synchronize()
    best = None
    for _ in range(runs):
        flush.fill_(7)
        h.reset()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.run()
        e1.record(stream)
        torch.cuda.synchronize()
        run_s = e0.elapsed_time(e1) * 1e-3
        b = h.best()
        t = time_to_target([h.level_log()], b[2]["t_start_ns"], v.f_star, final_f=[b[1]], run_s=run_s)
        t.update({"run_s": run_s, "best_f": b[1]})
        if best is None or (t.get("seconds") or 1e30) < (best.get("seconds") or 1e30):
            best = t
    h.destroy()
    best.update({"move": "uniform redraw of the chosen coordinate (the paper's Step 2)" if proposal == "uniform"
                 else "Gaussian step", "polish": f"projected gradients from the {polish_k} best final states",
                 "workload": v.config()["workload"], "steps_per_run": v.steps_per_run})
    return best


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2408_00018_gb300 import _build, sa

    torch.cuda.set_device(local_rank)
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    sa.load()
    w = Workload(args.workload, args.levels, args.independent, args.proposal, args.polish_k, args.surrogate)
    h = w.create(sa)
    groups = h.describe()
    pipes = measure_pipes(sa)  # the roofline's pipe rates, measured on this GPU before the timed region
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    flush.fill_(1)  # the first use of torch's fill kernel may JIT-compile it: not inside the timed region
    sampler = ClockSampler(gpu_id_for(local_rank))
    sampler.start()  # before the warm-up: its start-up must not overlap the timed region
    # W warm-up runs, continued until at least WARMUP_MIN_S of device work has
    # passed: the first seconds of work after idle run ~20% slower on this GPU.
    t_warm, warm_runs = time.perf_counter(), 0
    while warm_runs < args.warmup or time.perf_counter() - t_warm < WARMUP_MIN_S:
        flush.fill_(warm_runs & 0xFF)
        h.reset()
        h.run()
        torch.cuda.synchronize()
        warm_runs += 1
    if world > 1:
        torch.distributed.barrier()

    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    line0 = sampler.lines()
    e0.record(stream)
    for k in range(args.steps):
        flush.fill_(k & 0xFF)   # L2 flush between runs
        h.reset()
        h.run()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop((line0, sampler.lines()))
    ms = e0.elapsed_time(e1)
    bests = [h.best(p) for p in range(len(w.problems))]
    logs = [h.level_log(p) for p in range(len(w.problems))]
    ttt = time_to_target(logs, bests[0][2]["t_start_ns"], w.f_star,
                         final_f=[b[1] for b in bests] if w.polish_k else None, run_s=ms * 1e-3 / args.steps)

    t_max = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t_max, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(t_max.item())
    value = w.steps_per_run * args.steps * world / (ms_max * 1e-3)

    # ---- the headline's time-to-target under the paper's reading of a move (a uniform
    # redraw of the chosen coordinate) with the hybrid's projected-gradient polish of the 64
    # best final states: the same schedule, chains and levels, timed the same way
    ttt_variants = []
    if (rank == 0 and args.workload == "schwefel_n256" and not args.levels and w.proposal == "gaussian"
            and not w.polish_k and not w.independent):
        ttt_variants.append(time_to_target_variant(args, sa, torch, flush, "uniform", 64))

    # ---- live per-kernel timing of the sweep (eager launches, CUDA events on the same stream)
    h.reset()
    sweep_ms, level_ms = h.profile()
    launches = w.launches_per_run(h)
    h.destroy()
    sweep_avg = float(np.mean(sweep_ms))
    sm_mhz = clocks["sm_mhz"] or 2070.0
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    achieved, roofs, binding = pipe_roofline(w, pipes, sms, sm_mhz, sweep_avg)
    sfu_achieved = w.sfu_per_level / (sweep_avg * 1e-3) / 1e12
    sfu_peak = MUFU_PER_CLK_SM * sms * sm_mhz * 1e6 / 1e12
    roofline = {"bound": "alu", "achieved": round(achieved, 1), "peak": round(roofs[binding], 1),
                "unit": "Metropolis steps/s", "frac": round(achieved / roofs[binding], 4),
                "binding_pipe": binding,
                "pipes_steps_per_s": {k: round(v, 1) for k, v in roofs.items()},
                "frac_sfu": round(sfu_achieved / sfu_peak, 4),
                "traffic": traffic_from_profile(args.workload),
                "kernel": "sweep (" + ", ".join(g["kind"] for g in groups) + ")",
                "launch_ms": round(sweep_avg, 4),
                "sweep_share_of_level": round(float(np.sum(sweep_ms) / np.sum(level_ms)), 4),
                "algorithmic_ops_per_step": {p["cost"]: step_ops(p["cost"], p["n"], w.proposal)
                                             for p in w.problems[:1]} if not w.batch else "per problem (step_ops)",
                "pipe_rates_per_clk_per_sm": {k: round(v, 3) for k, v in pipes.items()},
                "peak_basis": f"measured pipe rates (sa_pipe_rate, ops/clk/SM) x {sms} SMs x {sm_mhz:.0f} MHz "
                              "(median sampled SM clock); per pipe, steps/s = rate / algorithmic ops per step; "
                              "peak = the lowest (binding) pipe"}
    if w.surrogate:  # the timed "sweep" is the whole delayed-acceptance level: training, GEMMs, steps
        roofline.update({"traffic": None, "kernel": "delayed-acceptance level (training, 2 surrogate GEMMs and "
                                                    "the step kernel per step)",
                         "note": "SFU ops of the true evaluations only; the level is bound by its lockstep "
                                 "kernels' latency, not by the SFU"})

    # ---- end to end through the public API with host buffers, every step
    e2e_times = []
    h2d = d2h = 0
    for k in range(args.steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        hh = w.create(sa, tune=False)
        hh.run()
        for p in range(len(w.problems)):
            xx, ff, stt = hh.best(p)
        hh.destroy()
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t)
        h2d, d2h = stt["h2d_bytes"], stt["d2h_bytes"]
    e2e_s = torch.tensor([sum(e2e_times)], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(e2e_s, op=torch.distributed.ReduceOp.MAX)
    e2e = {"value": w.steps_per_run * args.steps * world / float(e2e_s.item()), "unit": UNIT,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "note": "create (H2D of boxes and descriptors) + run + best (D2H) + destroy per step"
                   + ("; default launch shapes (no autotune)" if w.batch else "")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and w.surrogate:
        cpu = {"value": None, "unit": UNIT, "kind": "oracle",
               "sample": "none: the oracle replays the delayed-acceptance decisions from recorded surrogate values "
                         "(tests) and does not run the sweep itself"}
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        budget = 3e8 if w.batch else 5.3e8 / (w.problems[0]["n"] / 4 if any(w.rotated) else 1)
        v, dt, what = oracle_sample(w, budget, threads)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": what}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64" if w.precision == "fp64" else "f32",
               "data": "synthetic",
               "config": dict(w.config(), parallelism=f"replicas{world}", l2="flushed between runs (256 MiB write)",
                              launch_groups=[{"kind": "delayed_acceptance", "problems": 1,
                                              "n_max": w.problems[0]["n"]}] if w.surrogate else groups,
                              warmup_runs=warm_runs, warmup_min_s=WARMUP_MIN_S),
               "time_to_target": ttt, "best_f": bests[0][1] if len(bests) == 1 else None,
               "time_to_target_variants": ttt_variants or None,
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
               "fp64_rechecks_per_step": (bests[0][2]["rechecks"] / bests[0][2]["steps"]) if any(w.rotated) else None,
               "gpu_launches": launches * args.steps}
        print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.surrogate:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle has no delayed-acceptance sweep of its own "
                                                               "(it replays the GPU's decisions in the tests)"}))
        return
    w = Workload(args.workload, args.levels, args.independent, args.proposal, args.polish_k)
    threads = os.cpu_count() or 1
    budget = 6.5e7 / (w.problems[0]["n"] / 4 if any(w.rotated) else 1)
    for _ in range(args.warmup):
        oracle_sample(w, budget, threads)
    total_steps, total_s, what = 0, 0.0, ""
    for _ in range(args.steps):
        v, dt, what = oracle_sample(w, budget, threads)
        total_steps += v * dt
        total_s += dt
    value = total_steps / total_s
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": dict(w.config(), parallelism="cpu"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": "each step: " + what},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_surrogate_vs_plain(args):
    """The learned-surrogate workload has no closed-form minimum.  Its target is the
    best value found: the lowest of the projected-gradient-polished values of the
    oracle's reduced run (stored by tests/golden/make_oracle_best_f.py) and of the
    two full GPU runs timed here -- plain Metropolis and delayed acceptance, each
    followed by the polish of its 64 best final states.  Each arm's time-to-target
    is its whole run (the polish is the last step) if its polished value is within
    1e-6 relative of the target, else it is not reached and the gap is given; the
    per-level incumbents and device times are printed beside."""
    import torch
    from paper_2408_00018_gb300 import _build, sa

    _build.build()
    sa.load()
    torch.cuda.set_device(0)
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_best_f.json")))["rot_schwefel_n128"]
    seeds = [None] + list(range(1, args.seeds))  # None: the workload's own seed
    for seed in seeds:
        run_surrogate_vs_plain_seed(args, sa, torch, gold, seed)


def run_surrogate_vs_plain_seed(args, sa, torch, gold, seed):
    """One seed of the comparison (the chains' initial points and every draw)."""
    arms = {}
    for name, surrogate in (("plain", False), ("delayed_acceptance", True)):
        w = Workload("rot_schwefel_n128", 0, False, "gaussian", 64, surrogate)
        if seed is not None:
            w.seed = seed
        h = w.create(sa)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.run()
        e1.record(stream)
        torch.cuda.synchronize()
        x, f, st = h.best()
        log = h.level_log()
        arms[name] = {"run_s": e0.elapsed_time(e1) * 1e-3, "f_polished": f, "steps": st["steps"],
                      "true_evaluations": st["true_evals"], "f_inc_by_level": [float(v) for v in log["f_inc"][::10]],
                      "t_by_level_s": [(int(t) - int(st["t_start_ns"])) * 1e-9 for t in log["t_ns"][::10]]}
        h.destroy()
    f_target = min([gold["f_polished"]] + [a["f_polished"] for a in arms.values()])
    tol = 1e-6 * max(1.0, abs(f_target))
    for a in arms.values():
        gap = abs(a["f_polished"] - f_target)
        a["time_to_target"] = {"reached": gap <= tol, "seconds": a["run_s"] if gap <= tol else None,
                               "final_rel_gap": gap / max(1.0, abs(f_target))}
    p, d = arms["plain"]["time_to_target"], arms["delayed_acceptance"]["time_to_target"]
    out = {"metric": "time-to-target of the learned-surrogate workload (1e-6 relative to the best value found)",
           "workload": "rot_schwefel_n128_c131072_L2000_K150_fp32_Q0 + projected gradients from the 64 best",
           "data": "synthetic", "n_gpus": 1, "seed": w.seed, "f_target": f_target,
           "f_target_sources": {"oracle_reduced_run_polished (2048 chains, 10 levels)": gold["f_polished"],
                                "plain_polished": arms["plain"]["f_polished"],
                                "delayed_acceptance_polished": arms["delayed_acceptance"]["f_polished"]},
           "arms": arms,
           "ratio_plain_over_delayed_acceptance": (p["seconds"] / d["seconds"]) if p["seconds"] and d["seconds"] else None}
    print(json.dumps(out), flush=True)


# Table 10's functions at its sizes (F0_g Schwefel n = 512, F1_d Ackley n = 400,
# F13_b Rastrigin n = 400) with f* from their closed forms, moves by the paper's
# reading (a uniform redraw of the chosen coordinate), and the annealing stopped
# early: (cost, n, f*, T0, rho, levels).  A move changes Ackley's f by
# ~1e-3 at n = 400 (the others' by ~1 to 10), hence its lower T0.
HYBRID = [("schwefel", 512, -418.9828872724337, 100.0, 0.9, 100), ("ackley", 400, 0.0, 0.01, 0.9, 100),
          ("rastrigin", 400, 0.0, 100.0, 0.9, 100)]
HYBRID_CHAINS, HYBRID_L, HYBRID_K = 16384, 2000, 16


def run_hybrid(args):
    """Hybrid SA (Sec. 4.2, Table 10): annealing stopped after a few levels, then the
    local minimiser from the HYBRID_K best final states.  Times the annealing alone and
    annealing + polish (wall clock, after one untimed run of each), and reports the
    error |f - f*| of each, plus Nelder-Mead's iterations from the annealing's best point."""
    import numpy as np
    import torch
    from paper_2408_00018_gb300 import _build, inputs, sa

    _build.build()
    sa.load()

    def timed(sch, cost, lo, hi, n):
        with sa.create(cost, lo, hi, n, HYBRID_CHAINS, HYBRID_L, sch, seed=0) as h:
            h.run()  # untimed: graph capture and first-touch
            torch.cuda.synchronize()
            h.reset()
            t = time.perf_counter()
            h.run()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            x, f, _ = h.best()
        return dt, x, f

    for cost, n, fstar, T0, rho, K in HYBRID:
        lo, hi = inputs.box(cost, n)
        base = dict(T0=T0, rho=rho, levels=K, precision="fp32", proposal="uniform")
        t_sa, x_sa, f_sa = timed(sa.Schedule(**base), cost, lo, hi, n)
        out = {"metric": "hybrid SA: seconds and |f - f*| (Table 10 functions)", "workload": f"{cost}_n{n}",
               "data": "synthetic", "n_gpus": 1,
               "sa": {"chains": HYBRID_CHAINS, "L": HYBRID_L, "levels": K, "T0": T0, "rho": rho,
                      "steps": HYBRID_CHAINS * HYBRID_L * K, "s": t_sa, "err": abs(f_sa - fstar)}}
        for method in ("pgd", "nelder_mead", "nelder_mead_adaptive"):
            t, x, f = timed(sa.Schedule(**base, polish_k=HYBRID_K, polish_method=method), cost, lo, hi, n)
            out[method] = {"starts": HYBRID_K, "s": t, "polish_s": t - t_sa, "err": abs(f - fstar)}
        T = T0
        for _ in range(K - 1):
            T = T * rho
        step = min(1.0, 0.1 * (T / T0) ** 0.5)
        sa.nelder_mead(cost, x_sa[None], lo, hi, step_frac=step, max_iter=10)  # untimed
        t = time.perf_counter()
        _, f1, it1 = sa.nelder_mead(cost, x_sa[None], lo, hi, step_frac=step, max_iter=200 * (n + 1),
                                    ftol=1e-12, xtol=1e-10)
        dt = time.perf_counter() - t
        out["nelder_mead_from_best"] = {"s": dt, "iters": int(it1[0]), "us_per_iter": 1e6 * dt / max(1, int(it1[0])),
                                        "err": abs(float(f1[0]) - fstar)}
        t = time.perf_counter()
        _, f2, it2 = sa.nelder_mead(cost, x_sa[None], lo, hi, step_frac=step, max_iter=200 * (n + 1),
                                    ftol=1e-12, xtol=1e-10, adaptive=True)
        dt = time.perf_counter() - t
        out["nelder_mead_adaptive_from_best"] = {"s": dt, "iters": int(it2[0]), "err": abs(float(f2[0]) - fstar)}
        print(json.dumps(out), flush=True)


def run_gemm_route(args):
    """The GEMM route for rotated costs at the rotated Rastrigin n = 1024 workload's shape
    (65536 chains, L = 500): every step forms all chains' candidates X' (C x n) and
    Y' = X' Q^T (2 C n^2 flops) on the tensor cores, which this times with the library's
    tcgen05 BF16 GEMM and with torch.matmul (cuBLAS), CUDA events, after warm-up.  The
    rank-1 route's level (the rotated sweep) is timed live on the same workload."""
    import ctypes
    import numpy as np
    import torch
    from paper_2408_00018_gb300 import _build, inputs, sa

    _build.build()
    lib = sa.load()
    cfg = inputs.ROT_RASTRIGIN_N1024
    C, n, L = cfg["chains"], cfg["n"], cfg["L"]
    g = torch.Generator(device="cpu").manual_seed(0)
    X = (torch.rand(C, n, generator=g) * 10.24 - 5.12).to(torch.bfloat16).cuda()
    Q = torch.as_tensor(inputs.rotation(n, cfg["q_seed"]), dtype=torch.float32).to(torch.bfloat16).cuda()
    D = torch.empty(C, n, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    s_ptr = ctypes.c_void_p(stream.cuda_stream)

    def ours():
        lib.sa_gemm_bf16(ctypes.c_void_p(X.data_ptr()), n, ctypes.c_void_p(Q.data_ptr()), n,
                         ctypes.c_void_p(D.data_ptr()), n, C, n, n, ctypes.c_void_p(status.data_ptr()), s_ptr)

    def cublas():
        torch.mm(X, Q.t())

    flops = 2.0 * C * n * n
    res = {}
    for name, fn in (("tcgen05", ours), ("cublas", cublas)):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms_per_step": ms, "tflops": flops / (ms * 1e-3) / 1e12, "ms_per_level": ms * L}
    assert int(status.item()) == 0
    # the rank-1 route: the rotated sweep's live level time on the same workload
    lo, hi = inputs.box(cfg["cost"], n)
    sch = sa.Schedule(T0=cfg["T0"], rho=cfg["rho"], levels=3, sigma_frac=cfg["sigma_frac"], precision="fp32")
    with sa.create(cfg["cost"], lo, hi, n, C, L, sch, seed=cfg["seed"], Q=inputs.rotation(n, cfg["q_seed"])) as h:
        h.run()
        h.reset()
        sweep_ms, level_ms = h.profile()
    rank1 = float(np.mean(sweep_ms[1:]))  # levels >= 1 (level 0 also reads X0, Y0)
    # level 0 with the run's start-up work (initial states, costs, the transform Y0 = X0 Q^T)
    level0 = {"level_ms_other_levels": float(np.mean(level_ms[1:])), "tensor_split": float(level_ms[0])}
    # the level-0 transform Y0 = X0 Q^T alone (exact BF16 slices, 21 tcgen05 products into
    # double-float pairs), and level 0 of a run whose transform is the FP64 product instead
    X32 = (torch.rand(C, n, generator=g) * 10.24 - 5.12).cuda()
    Q64 = torch.as_tensor(inputs.rotation(n, cfg["q_seed"]), dtype=torch.float64).cuda()
    for _ in range(3):
        Y, st = sa.rotate_rows(X32, Q64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(5):
        Y, st = sa.rotate_rows(X32, Q64)
    e1.record(stream)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    rot_ms = e0.elapsed_time(e1) / 5
    del Y, X32
    prev = os.environ.get("SA_ROT_TC")
    os.environ["SA_ROT_TC"] = "0"
    try:
        with sa.create(cfg["cost"], lo, hi, n, C, L, sch, seed=cfg["seed"], Q=inputs.rotation(n, cfg["q_seed"])) as h:
            h.run()
            h.reset()
            _, ms64 = h.profile()
        level0["fp64"] = float(ms64[0])
    finally:
        if prev is None:
            del os.environ["SA_ROT_TC"]
        else:
            os.environ["SA_ROT_TC"] = prev
    peak = 1736.1
    print(json.dumps({"metric": "rotated costs: GEMM route vs rank-1 route (rotated Rastrigin n = 1024)",
                      "shape": {"C": C, "n": n, "L": L}, "flops_per_step": flops, "gemm": res,
                      "bf16_peak_tflops_sustained": peak,
                      "rank1_sweep_ms_per_level": rank1,
                      "level0_transform": {"ms": rot_ms, "slice_products": 21,
                                           "tflops_bf16": 21 * flops / (rot_ms * 1e-3) / 1e12},
                      "level0_ms": level0,
                      "note": "the GEMM route's time is the BF16 product alone: BF16 inputs carry 8 "
                              "significant bits, so nearly every decision would go to the FP64 re-check; an "
                              "error-free split needs at least 3 products"}), flush=True)


def run_surrogate_forward(args):
    """The surrogate's forward pass f~(X) for the 131072 candidate rows (n = 128) that every
    delayed-acceptance step evaluates: sa_mlp_forward (BF16 cast of the weights, packing of X,
    the forward pass, the head's final sum) with the fused one-kernel pass and with the two
    GEMMs, CUDA events after warm-up.  The forward pass alone is 8.6e10 flops."""
    import numpy as np
    import torch
    from paper_2408_00018_gb300 import _build, sa

    _build.build()
    n, B = 128, 131072
    p = torch.empty(sa.mlp_param_count(n), dtype=torch.float32, device="cuda")
    sa.mlp_init(p, n, seed=1)
    g = torch.Generator(device="cpu").manual_seed(0)
    X = (torch.rand(B, n, generator=g) * 2 - 1).cuda()
    stream = torch.cuda.current_stream()
    res = {}
    prev = os.environ.get("SA_MLP_FUSED")
    try:
        for name, flag in (("fused", "1"), ("two_gemms", "0")):
            os.environ["SA_MLP_FUSED"] = flag
            for _ in range(5):
                y = sa.mlp_forward(p, n, X)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 50
            e0.record(stream)
            for _ in range(reps):
                y = sa.mlp_forward(p, n, X)
            e1.record(stream)
            torch.cuda.synchronize()
            res[name] = {"us_per_call": e0.elapsed_time(e1) / reps * 1e3, "y_checksum": float(y.double().sum())}
    finally:
        if prev is None:
            os.environ.pop("SA_MLP_FUSED", None)
        else:
            os.environ["SA_MLP_FUSED"] = prev
    flops = 2.0 * B * 512 * (n + 512)
    print(json.dumps({"metric": "surrogate forward pass (131072 x 128 -> 512 -> 512 -> 1)", "rows": B, "n": n,
                      "flops": flops, "calls": res,
                      "note": "per sa_mlp_forward call: weight cast, input packing, forward pass, head sum; the "
                              "forward kernels alone are in the ncu launch list"}), flush=True)


def run_paper_schwefel(args):
    """The normalised Schwefel function under the paper's configuration (Sec. 4.1):
    T0 = 1000, T_min = 0.01, rho = 0.99 (1146 levels), N = 100 steps, 16384 chains,
    box [-512, 512]^n, the paper's reading of a move (a uniform redraw of the chosen
    coordinate); FP32 state, FP64 argmin.  Per n and version (V2 synchronous, V1
    asynchronous, V2 with the stochastic crossover instead of the minimum): |f - f*|,
    the relative error of x, the device time of the run (CUDA events, after an
    untimed run) and steps/s."""
    import numpy as np
    import torch
    from paper_2408_00018_gb300 import _build, inputs, sa

    _build.build()
    sa.load()
    xs, fs = 420.968746, inputs.SCHWEFEL_F_STAR
    for n in (8, 16, 32, 64, 128, 256, 512):
        lo, hi = np.full(n, -512.0), np.full(n, 512.0)
        out = {"metric": "paper Schwefel table: |f - f*|, relative x error, seconds", "n": n, "chains": 16384,
               "L": 100, "levels": 1146, "proposal": "uniform", "precision": "fp32"}
        for version, indep, xo in (("V2", 0, 0), ("V1", 1, 0), ("V2_crossover", 0, 1)):
            sch = sa.Schedule(T0=1000.0, rho=0.99, levels=0, T_min=0.01, precision="fp32", independent=indep,
                              proposal="uniform", crossover=xo)
            with sa.create("schwefel", lo, hi, n, 16384, 100, sch, seed=0) as h:
                h.run()  # untimed: graph capture
                h.reset()
                stream = torch.cuda.current_stream()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                h.run()
                e1.record(stream)
                torch.cuda.synchronize()
                x, f, st = h.best()
            dt = e0.elapsed_time(e1) / 1e3
            out[version] = {"err": abs(f - fs), "rel_x": float(np.linalg.norm(x - xs) / np.linalg.norm(np.full(n, xs))),
                            "s": dt, "steps": st["steps"], "steps_per_s": st["steps"] / dt}
        print(json.dumps(out), flush=True)


# The convergence study (Sec. 4.1, Figures 4-5): per level every version explores
# CONV_C * CONV_L points; CONV_R replicas per version, reported as their mean.
CONV_N = (8, 16, 32, 64, 128, 256)
CONV_C, CONV_L, CONV_R = 1024, 100, 8
CONV_CHECKPOINTS = (1, 2, 5, 10, 20, 50, 100, 200, 500, 1000, 1146)


def convergence_curve(f_levels, f_star, checkpoints):
    """Mean over the replicas of the relative error |f - f*| / |f*| of the level's best
    value after each checkpoint's number of levels (a checkpoint past the end of a run
    takes its last level)."""
    import numpy as np
    out = []
    for k in checkpoints:
        errs = [abs(float(f[min(k, len(f)) - 1]) - f_star) / abs(f_star) for f in f_levels]
        out.append(float(np.mean(errs)))
    return out


def run_convergence(args):
    """The convergence study of Sec. 4.1 (Figures 4-5) at equal numbers of explored
    points: V1 (asynchronous) and V2 (synchronous) run CONV_C chains of CONV_L steps per
    level; V0 (sequential: one chain) runs CONV_C * CONV_L steps per level at the same
    temperatures (T0 = 1000, rho = 0.99, T_min = 0.01: 1146 levels), so every version
    explores the same points per level.  Schwefel on [-512, 512]^n, the paper's move (a
    uniform redraw of the chosen coordinate), FP32 state.  Each version runs CONV_R
    replicas as the problems of one batch (each problem draws its own Philox streams);
    for V1 the level's value is the best over all its chains, as in the paper."""
    import numpy as np
    import torch
    from paper_2408_00018_gb300 import _build, inputs, sa

    _build.build()
    sa.load()
    fs = inputs.SCHWEFEL_F_STAR
    for n in CONV_N:
        lo, hi = np.full(n, -512.0), np.full(n, 512.0)
        out = {"metric": "convergence: mean relative error |f - f*| / |f*| of the level's best value vs explored points",
               "cost": "schwefel", "n": n, "chains": CONV_C, "L": CONV_L, "replicas": CONV_R, "levels": 1146,
               "points_per_level": CONV_C * CONV_L, "checkpoint_levels": list(CONV_CHECKPOINTS),
               "points": [k * CONV_C * CONV_L for k in CONV_CHECKPOINTS], "proposal": "uniform", "precision": "fp32"}
        for version, indep, chains, L in (("V0", 0, 1, CONV_C * CONV_L), ("V1", 1, CONV_C, CONV_L),
                                          ("V2", 0, CONV_C, CONV_L)):
            sch = sa.Schedule(T0=1000.0, rho=0.99, levels=0, T_min=0.01, precision="fp32", independent=indep,
                              proposal="uniform")
            probs = [dict(cost="schwefel", n=n, chains=chains, lo=lo, hi=hi) for _ in range(CONV_R)]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with sa.create_batch(probs, L, sch, seed=0) as h:
                h.run()
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                logs = [h.level_log(p)["f_level"] for p in range(CONV_R)]
                steps = h.best(0)[2]["steps"]
            out[version] = {"rel_err": convergence_curve(logs, fs, CONV_CHECKPOINTS), "steps_per_replica": int(steps),
                            "s": dt}
        print(json.dumps(out), flush=True)


# The suite's schedule: one for every problem (the paper tunes per function and
# prints no schedule): T0 = 10, rho = 0.9, 100 levels of L = 500 steps, moves
# by the paper's reading (a uniform redraw of the chosen coordinate).  Costs
# with an O(1) energy difference run FP32 with 65536 chains; the Appendix's other
# tests run the FP64 full evaluation with 16384 chains (4096 above 16 coordinates,
# where every step evaluates n transcendental terms in FP64).
SUITE_L, SUITE_K, SUITE_T0, SUITE_RHO, SUITE_POLISH = 500, 100, 10.0, 0.9, 8


def run_suite(args):
    """Tables 8-9 on this GPU: per problem the steps, the device time of the run
    (CUDA events around sa_run, after an untimed run), |f - f*| and the same after
    the hybrid's Nelder-Mead polish of the 8 best final states."""
    import numpy as np
    import torch
    from paper_2408_00018_gb300 import _build, inputs, sa

    _build.build()
    sa.load()
    base_costs = ("schwefel", "ackley", "rastrigin", "rosenbrock")
    rows = []
    for p in inputs.appendix_suite():
        fp32 = p["cost"] in base_costs
        C = 65536 if fp32 else (16384 if p["n"] <= 16 else 4096)
        out = {"metric": "suite: seconds and |f - f*| per problem (Tables 8-9 problems)", "problem": p["name"],
               "cost": p["cost"], "n": p["n"], "chains": C, "L": SUITE_L, "levels": SUITE_K,
               "precision": "fp32" if fp32 else "fp64", "steps": C * SUITE_L * SUITE_K, "f_star": p["f_star"]}
        for polish in (0, SUITE_POLISH):
            sch = sa.Schedule(T0=SUITE_T0, rho=SUITE_RHO, levels=SUITE_K, precision="fp32" if fp32 else "fp64",
                              polish_k=polish, polish_method="nelder_mead", proposal="uniform")
            with sa.create(p["cost"], p["lo"], p["hi"], p["n"], C, SUITE_L, sch, seed=0, table=p["table"]) as h:
                h.run()  # untimed: graph capture
                h.reset()
                stream = torch.cuda.current_stream()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                h.run()
                e1.record(stream)
                torch.cuda.synchronize()
                _, f, _ = h.best()
            key = "sa" if polish == 0 else "hybrid"
            out[key] = {"s": e0.elapsed_time(e1) / 1e3, "f": f, "err": abs(f - p["f_star"])}
        out["steps_per_s"] = out["steps"] / out["sa"]["s"]
        rows.append(out)
        print(json.dumps(out), flush=True)
    tol = lambda r, k: r[k]["err"] <= 1e-4 * max(1.0, abs(r["f_star"]))  # noqa: E731
    summary = {"metric": "suite summary", "problems": len(rows),
               "sa_seconds": sum(r["sa"]["s"] for r in rows), "hybrid_seconds": sum(r["hybrid"]["s"] for r in rows),
               "steps": sum(r["steps"] for r in rows),
               "sa_within_1e-4": sum(tol(r, "sa") for r in rows), "hybrid_within_1e-4": sum(tol(r, "hybrid") for r in rows)}
    print(json.dumps(summary), flush=True)


def main():
    args = parse()
    if args.gemm_route:
        run_gemm_route(args)
        return
    if args.paper_schwefel:
        run_paper_schwefel(args)
        return
    if args.surrogate_forward:
        run_surrogate_forward(args)
        return
    if args.suite:
        run_suite(args)
        return
    if args.hybrid:
        run_hybrid(args)
        return
    if args.convergence:
        run_convergence(args)
        return
    if args.surrogate_vs_plain:
        run_surrogate_vs_plain(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
