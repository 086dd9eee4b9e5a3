"""Writes tests/golden/oracle_best_f.json: the FP64 CPU oracle's best values on the
benchmark workloads, at the sizes the oracle can run on a host (the full run of the
two Schwefel workloads; a seeded 32-problem subset of the batched workload; 1024 and
2048 chains over 10 levels of the two rotated workloads), with the same seeds,
schedules and Philox streams as the GPU runs of the same inputs.

It calls only the oracle (and the seeded input generators).  Run from the
repository root:  python tests/golden/make_oracle_best_f.py [names...]
(the full n = 256 run takes about ten minutes on eight cores).
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2408_00018_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_best_f.json")
THREADS = os.cpu_count() or 1

# The oracle runs of each workload: (workload config, chains, levels, problems).
RUNS = {
    "schwefel_n2": dict(cfg=inputs.SCHWEFEL_N2_FP64, chains=None, levels=None),
    "schwefel_n256": dict(cfg=inputs.SCHWEFEL_N256_FP32, chains=None, levels=None),
    "rot_rastrigin_n1024": dict(cfg=inputs.ROT_RASTRIGIN_N1024, chains=1024, levels=10),
    "rot_schwefel_n128": dict(cfg=inputs.ROT_SCHWEFEL_N128, chains=2048, levels=10, polish=64),
    "batched32": dict(cfg=None, problems=32, L=500, levels=100),
}


def run_single(name, spec):
    cfg = dict(spec["cfg"])
    n = cfg["n"]
    lo, hi = inputs.box(cfg["cost"], n)
    Q = inputs.rotation(n, cfg["q_seed"]) if "q_seed" in cfg else None
    C = spec["chains"] or cfg["chains"]
    K = spec["levels"] or cfg["levels"]
    mode = 0 if cfg["precision"] == "fp64" else 1
    p = oracle.Problem(cfg["cost"], n, lo, hi, chains=C, L=cfg["L"], T0=cfg["T0"], rho=cfg["rho"],
                       sigma_frac=cfg["sigma_frac"], seed=cfg["seed"], Q=Q, mode=mode, threads=THREADS)
    t = time.perf_counter()
    polish = spec.get("polish", 0)
    r = p.run(K, want_final=bool(polish))
    rec = {"cost": cfg["cost"], "n": n, "chains": C, "L": cfg["L"], "levels": K, "T0": cfg["T0"], "rho": cfg["rho"],
           "seed": cfg["seed"], "mode": mode, "f_inc": r["f_inc"], "x_inc": r["x_inc"].tolist(),
           "argmin": r["argmin"].tolist(), "f_level": r["f_level"].tolist(),
           "seconds": round(time.perf_counter() - t, 1), "threads": THREADS}
    if polish:
        # the hybrid: projected gradients from the `polish` best final states (value, then index)
        order = np.lexsort((np.arange(C), r["F_final"]))[:polish]
        best_f, best_x = np.inf, None
        for c in order:
            x, f, _ = oracle.pgd(cfg["cost"], r["X_final"][c], lo, hi, Q=Q, max_iter=1000, tol=1e-10)
            if f < best_f:
                best_f, best_x = f, x
        g = oracle.grad(cfg["cost"], best_x, Q)
        # projected gradient: zero where a bound is active and the gradient points outward
        pg = np.where((best_x <= lo) & (g > 0), 0.0, np.where((best_x >= hi) & (g < 0), 0.0, g))
        rec.update({"f_polished": float(best_f), "x_polished": best_x.tolist(),
                    "kkt_projected_grad_inf": float(np.abs(pg).max()),
                    "f_polished_fp64_recheck": float(oracle.cost(cfg["cost"], best_x, Q))})
    return rec


def run_batched(spec):
    probs = inputs.batch_problems(count=512, seed=0)[:spec["problems"]]
    out = []
    t = time.perf_counter()
    for pid, pr in enumerate(probs):
        p = oracle.Problem(pr["cost"], pr["n"], pr["lo"], pr["hi"], chains=pr["chains"], L=spec["L"], T0=100.0,
                           rho=0.95, sigma_frac=0.1, seed=0, problem=pid, mode=1, threads=THREADS)
        r = p.run(spec["levels"])
        out.append({"problem": pid, "cost": pr["cost"], "n": pr["n"], "chains": pr["chains"], "f_inc": r["f_inc"],
                    "argmin_last": int(r["argmin"][-1])})
        print(f"  batched problem {pid}: {pr['cost']} n={pr['n']} C={pr['chains']} f={r['f_inc']:.6g}", flush=True)
    return {"problems": out, "L": spec["L"], "levels": spec["levels"], "T0": 100.0, "rho": 0.95, "seed": 0,
            "seconds": round(time.perf_counter() - t, 1), "threads": THREADS}


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names or list(RUNS):
        spec = RUNS[name]
        print(f"{name} ...", flush=True)
        data[name] = run_batched(spec) if name == "batched32" else run_single(name, spec)
        json.dump(data, open(OUT, "w"), indent=1)
        print(f"{name}: done in {data[name]['seconds']} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
