"""FP64 CPU oracle for synchronous parallel simulated annealing -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA library: the C source
``sa_oracle.c`` is compiled on its own with gcc (``-ffp-contract=off``) and loaded
through ctypes.  Every function follows the paper's algorithm step by step
(Sec. 2.1 Steps 1-5, Sec. 2.2.2, Listings 3-4); see the header of ``sa_oracle.c``
for the readings taken where the paper is silent.

Pins: the tests under ``tests/test_oracle_*.py`` check this oracle against
published Philox4x32-10 known-answer vectors, the closed-form normalised
Schwefel minimum, brute-force grids, schedule/evaluation-count identities
printed with Table 1, and Metropolis invariants (acceptance 1 on a constant
cost, zero uphill moves as T -> 0, Boltzmann histogram at fixed T); the
Nelder-Mead of the hybrid SA is pinned iteration for iteration against scipy's
implementation of the same method.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sa_oracle.c")
_LIB = os.path.join(_HERE, "libsaoracle.so")
_lock = threading.Lock()
_lib = None

COSTS = {"schwefel": 0, "rastrigin": 1, "ackley": 2, "rosenbrock": 3,
         "rot_rastrigin": 4, "rot_schwefel": 5,
         "branin": 6, "cosine_mixture": 7, "dekkers_aarts": 8, "easom": 9, "exponential": 10,
         "goldstein_price": 11, "griewank": 12, "himmelblau": 13, "levy_montalvo": 14, "langerman": 15,
         "michalewicz": 16, "salomon": 17, "six_hump_camel": 18, "shubert": 19, "shekel": 20, "foxholes": 21}
TAG_SWEEP, TAG_INIT, TAG_DA = 0, 1, 3


def build(force: bool = False) -> str:
    """Compile the oracle's shared library with gcc (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Cfg(ctypes.Structure):
    _fields_ = [("cost", ctypes.c_int32), ("n", ctypes.c_int32), ("chains", ctypes.c_int64),
                ("L", ctypes.c_int32), ("K", ctypes.c_int32), ("level0", ctypes.c_int32),
                ("boundary", ctypes.c_int32), ("mode", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("problem", ctypes.c_uint32), ("seed", ctypes.c_uint64), ("T0", ctypes.c_double),
                ("rho", ctypes.c_double), ("sigma_frac", ctypes.c_double),
                ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("independent", ctypes.c_int32), ("exchange_every", ctypes.c_int32),
                ("table", ctypes.c_void_p), ("table_rows", ctypes.c_int32), ("proposal", ctypes.c_int32),
                ("crossover", ctypes.c_int32)]


class Out(ctypes.Structure):
    _fields_ = [("x_best", ctypes.c_void_p), ("f_best", ctypes.c_void_p), ("x_inc", ctypes.c_void_p),
                ("f_inc", ctypes.c_void_p), ("argmin", ctypes.c_void_p), ("f_level", ctypes.c_void_p),
                ("accepts", ctypes.c_void_p), ("bits", ctypes.c_void_p), ("trace_levels", ctypes.c_int32),
                ("F_final", ctypes.c_void_p), ("X_final", ctypes.c_void_p), ("xo_src", ctypes.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            vp, i32, i64, u32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
            L.sao_philox4x32_10.argtypes = [vp, vp, vp]
            L.sao_uniform.argtypes = [u32]
            L.sao_uniform.restype = f64
            L.sao_coord.argtypes = [u32, i32]
            L.sao_coord.restype = u32
            L.sao_cost.argtypes = [i32, i32, vp, vp, vp, i32]
            L.sao_cost.restype = f64
            L.sao_grad.argtypes = [i32, i32, vp, vp, vp]
            L.sao_temperature.argtypes = [f64, f64, i32]
            L.sao_temperature.restype = f64
            L.sao_levels_for.argtypes = [f64, f64, f64]
            L.sao_levels_for.restype = i32
            L.sao_init_point.argtypes = [ctypes.POINTER(Cfg), i64, vp]
            L.sao_chain_level.argtypes = [ctypes.POINTER(Cfg), i32, i64, vp, vp, vp]
            L.sao_chain_level.restype = f64
            L.sao_chain_level_steps.argtypes = [ctypes.POINTER(Cfg), i32, i64, vp, vp, vp, vp, vp]
            L.sao_chain_level_steps.restype = f64
            L.sao_da_chain_level.argtypes = [ctypes.POINTER(Cfg), i32, i64, vp, f64, vp, vp, vp, vp]
            L.sao_da_chain_level.restype = f64
            L.sao_da_chain_level_steps.argtypes = [ctypes.POINTER(Cfg), i32, i64, vp, f64, vp, vp, vp, vp, vp]
            L.sao_da_chain_level_steps.restype = f64
            L.sao_rotate.argtypes = [i32, vp, vp, vp]
            L.sao_proposal.argtypes = [ctypes.POINTER(Cfg), i32, i64, i32, vp, vp, vp]
            L.sao_da_chain_level_trace.argtypes = [ctypes.POINTER(Cfg), i32, i64, vp, f64, vp, vp, vp, vp, vp, vp, i32]
            L.sao_da_chain_level_trace.restype = f64
            L.sao_da_chain_level_fn.argtypes = [ctypes.POINTER(Cfg), i32, i64, vp, f64, f64, vp, vp, vp]
            L.sao_da_chain_level_fn.restype = f64
            L.sao_run.argtypes = [ctypes.POINTER(Cfg), ctypes.POINTER(Out)]
            L.sao_run.restype = ctypes.c_int
            L.sao_level_chains.argtypes = [ctypes.POINTER(Cfg), i32, vp, i64, i64, vp, vp, vp, vp]
            L.sao_level_chains.restype = ctypes.c_int
            L.sao_pgd.argtypes = [i32, i32, vp, vp, vp, vp, i32, f64, f64, i32, vp, vp]
            L.sao_pgd.restype = ctypes.c_int
            L.sao_nelder_mead.argtypes = [i32, i32, vp, vp, vp, vp, i32, vp, f64, i32, f64, f64, i32, vp, vp]
            L.sao_nelder_mead.restype = ctypes.c_int
            L.sao_crossover_sources.argtypes = [ctypes.POINTER(Cfg), i32, vp, i64, vp]
            L.sao_crossover_sources.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().sao_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def stream_key(seed: int, tag: int):
    return [seed & 0xFFFFFFFF, ((seed >> 32) & 0xFFFFFFFF) ^ tag]


def uniform(w: int) -> float:
    return lib().sao_uniform(int(w))


def coord(w: int, n: int) -> int:
    return lib().sao_coord(int(w), int(n))


def _table(table):
    """(array, rows) of a table of rows (a_i1 .. a_in, c_i), or (None, 0)."""
    if table is None:
        return None, 0
    t = np.ascontiguousarray(np.atleast_2d(np.asarray(table, np.float64)))
    return t, t.shape[0]


def cost(name_or_id, x, Q=None, table=None) -> float:
    cid = COSTS[name_or_id] if isinstance(name_or_id, str) else int(name_or_id)
    x = np.ascontiguousarray(x, dtype=np.float64)
    Qa = None if Q is None else np.ascontiguousarray(Q, dtype=np.float64)
    t, rows = _table(table)
    return lib().sao_cost(cid, x.size, _p(x), _p(Qa), _p(t), rows)


def rotate(Q, x) -> np.ndarray:
    """y = Q x in FP64, each y_i summed over j in index order (the rotated costs' transform)."""
    Qa = np.ascontiguousarray(Q, dtype=np.float64)
    xa = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(xa.size)
    lib().sao_rotate(xa.size, _p(Qa), _p(xa), _p(y))
    return y


def grad(name_or_id, x, Q=None) -> np.ndarray:
    cid = COSTS[name_or_id] if isinstance(name_or_id, str) else int(name_or_id)
    x = np.ascontiguousarray(x, dtype=np.float64)
    Qa = None if Q is None else np.ascontiguousarray(Q, dtype=np.float64)
    g = np.zeros_like(x)
    lib().sao_grad(cid, x.size, _p(x), _p(Qa), _p(g))
    return g


def temperature(T0: float, rho: float, level: int) -> float:
    return lib().sao_temperature(T0, rho, level)


def levels_for(T0: float, rho: float, T_min: float) -> int:
    return lib().sao_levels_for(T0, rho, T_min)


class Problem:
    """A box-constrained problem plus the schedule of one synchronous SA run."""

    def __init__(self, cost, n, lo, hi, chains, L, T0=100.0, rho=0.9, sigma_frac=0.1,
                 boundary="reflect", seed=0, problem=0, Q=None, mode=0, threads=0, independent=False,
                 exchange_every=1, table=None, proposal="gaussian", crossover=False):
        self.cost = COSTS[cost] if isinstance(cost, str) else int(cost)
        self.n = int(n)
        self.lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, np.float64), (self.n,)))
        self.hi = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, np.float64), (self.n,)))
        self.Q = None if Q is None else np.ascontiguousarray(Q, dtype=np.float64)
        self.chains, self.L = int(chains), int(L)
        self.T0, self.rho, self.sigma_frac = float(T0), float(rho), float(sigma_frac)
        self.boundary = {"reflect": 0, "clip": 1}[boundary] if isinstance(boundary, str) else int(boundary)
        self.seed, self.problem, self.mode, self.threads = int(seed), int(problem), int(mode), int(threads)
        self.independent = 1 if independent else 0
        self.exchange_every = int(exchange_every)
        self.table, self.table_rows = _table(table)
        self.proposal = {"gaussian": 0, "uniform": 1}[proposal] if isinstance(proposal, str) else int(proposal)
        self.crossover = 1 if crossover else 0

    def cfg(self, K=0, level0=0) -> Cfg:
        return Cfg(self.cost, self.n, self.chains, self.L, K, level0, self.boundary, self.mode,
                   self.threads, self.problem, self.seed, self.T0, self.rho, self.sigma_frac,
                   _p(self.lo), _p(self.hi), _p(self.Q), self.independent, self.exchange_every,
                   _p(self.table), self.table_rows, self.proposal, self.crossover)

    def crossover_sources(self, level: int, F) -> np.ndarray:
        """The stochastic crossover's draw of a source chain for every chain, given final values F."""
        F = np.ascontiguousarray(F, np.float64)
        src = np.zeros(F.size, np.int64)
        cfg = self.cfg()
        if lib().sao_crossover_sources(ctypes.byref(cfg), level, _p(F), F.size, _p(src)) != 0:
            raise ValueError("sao_crossover_sources failed")
        return src

    def init_point(self, c: int) -> np.ndarray:
        x = np.zeros(self.n)
        cfg = self.cfg()
        lib().sao_init_point(ctypes.byref(cfg), c, _p(x))
        return x

    def chain_level(self, level, c, x_start=None, trace=False):
        """One chain for one level; returns (F_end, x_end, accepts, bits)."""
        cfg = self.cfg()
        x = self.init_point(c) if x_start is None else np.array(x_start, np.float64)
        words = (self.L + 31) // 32
        bits = np.zeros(words, np.uint32) if trace else None
        acc = np.zeros(1, np.int64)
        F = lib().sao_chain_level(ctypes.byref(cfg), level, c, _p(x), _p(bits), _p(acc))
        return F, x, int(acc[0]), bits

    def chain_steps(self, level, c, x_start=None):
        """One chain for one level with per-step diagnostics: (F_end, x_end, bits, dF[L], tau[L])."""
        cfg = self.cfg()
        x = self.init_point(c) if x_start is None else np.array(x_start, np.float64)
        bits = np.zeros((self.L + 31) // 32, np.uint32)
        acc = np.zeros(1, np.int64)
        dF = np.zeros(self.L)
        tau = np.zeros(self.L)
        F = lib().sao_chain_level_steps(ctypes.byref(cfg), level, c, _p(x), _p(bits), _p(acc), _p(dF), _p(tau))
        return F, x, bits, dF, tau

    def da_chain_level(self, level, c, ft0, ft_prop, x_start=None):
        """One chain, one level of delayed acceptance with given surrogate values
        (ft0 at the start state, ft_prop[s] at step s's proposal); returns
        (F_end, x_end, bits, accepts, true_evaluations)."""
        cfg = self.cfg()
        x = self.init_point(c) if x_start is None else np.array(x_start, np.float64)
        ftp = np.ascontiguousarray(ft_prop, np.float64)
        assert ftp.size == self.L
        bits = np.zeros((self.L + 31) // 32, np.uint32)
        acc = np.zeros(1, np.int64)
        ev = np.zeros(1, np.int64)
        F = lib().sao_da_chain_level(ctypes.byref(cfg), level, c, _p(x), float(ft0), _p(ftp), _p(bits), _p(acc),
                                     _p(ev))
        return F, x, bits, int(acc[0]), int(ev[0])

    def da_chain_level_steps(self, level, c, ft0, ft_prop, x_start=None):
        """As da_chain_level, also returning dF [L]: each step's true difference (NaN
        where stage 1 rejected the move)."""
        cfg = self.cfg()
        x = self.init_point(c) if x_start is None else np.array(x_start, np.float64)
        ftp = np.ascontiguousarray(ft_prop, np.float64)
        bits = np.zeros((self.L + 31) // 32, np.uint32)
        acc = np.zeros(1, np.int64)
        ev = np.zeros(1, np.int64)
        dF = np.zeros(self.L)
        F = lib().sao_da_chain_level_steps(ctypes.byref(cfg), level, c, _p(x), float(ft0), _p(ftp), _p(bits), _p(acc),
                                           _p(ev), _p(dF))
        return F, x, bits, int(acc[0]), int(ev[0]), dF

    def propose_step(self, level, c, s, x):
        """The move (d, x'_d) that chain c at state x proposes at step s of a level."""
        cfg = self.cfg()
        xa = np.ascontiguousarray(x, np.float64)
        d = np.zeros(1, np.int32)
        xp = np.zeros(1)
        lib().sao_proposal(ctypes.byref(cfg), level, c, s, _p(xa), _p(d), _p(xp))
        return int(d[0]), float(xp[0])

    def da_chain_level_trace(self, level, c, ft0, ft_prop, x_start=None, plant=0):
        """As da_chain_level_steps, also returning tau [L]: each step's stage-2 threshold
        -T ln u3 (NaN where stage 1 rejected the move).  plant=1 flips the sign of the
        surrogate difference in stage 2: a planted mistake, for the tests that show the
        parity checks catch it.  Returns (F_end, x_end, bits, accepts, evaluations, dF, tau)."""
        cfg = self.cfg()
        x = self.init_point(c) if x_start is None else np.array(x_start, np.float64)
        ftp = np.ascontiguousarray(ft_prop, np.float64)
        assert ftp.size == self.L
        bits = np.zeros((self.L + 31) // 32, np.uint32)
        acc = np.zeros(1, np.int64)
        ev = np.zeros(1, np.int64)
        dF = np.zeros(self.L)
        tau = np.zeros(self.L)
        F = lib().sao_da_chain_level_trace(ctypes.byref(cfg), level, c, _p(x), float(ft0), _p(ftp), _p(bits), _p(acc),
                                           _p(ev), _p(dF), _p(tau), int(plant))
        return F, x, bits, int(acc[0]), int(ev[0]), dF, tau

    def da_chain_level_fn(self, level, c, a, b, x_start=None):
        """Delayed acceptance with the analytic surrogate a f(x) + b sum_i sin(x_i);
        returns (F_end, x_end, bits, accepts, true_evaluations)."""
        cfg = self.cfg()
        x = self.init_point(c) if x_start is None else np.array(x_start, np.float64)
        bits = np.zeros((self.L + 31) // 32, np.uint32)
        acc = np.zeros(1, np.int64)
        ev = np.zeros(1, np.int64)
        F = lib().sao_da_chain_level_fn(ctypes.byref(cfg), level, c, _p(x), float(a), float(b), _p(bits), _p(acc),
                                        _p(ev))
        return F, x, bits, int(acc[0]), int(ev[0])

    def level_chains(self, level, c0, c1, x_start=None, want_x=False, trace=False):
        """One level for chains [c0, c1); returns dict of per-chain results."""
        cfg = self.cfg()
        m = c1 - c0
        F = np.zeros(m)
        X = np.zeros((m, self.n)) if want_x else None
        words = (self.L + 31) // 32
        bits = np.zeros((m, words), np.uint32) if trace else None
        acc = np.zeros(m, np.int64)
        xs = None if x_start is None else np.ascontiguousarray(x_start, np.float64)
        rc = lib().sao_level_chains(ctypes.byref(cfg), level, _p(xs), c0, c1, _p(F), _p(X), _p(bits), _p(acc))
        if rc != 0:
            raise ValueError("sao_level_chains failed")
        return {"F": F, "X": X, "bits": bits, "accepts": acc}

    def run(self, K, level0=0, x_best=None, f_best=None, x_inc=None, f_inc=None,
            trace_levels=0, want_final=False):
        """Run K levels; returns a dict with the incumbent, per-level argmins and optional traces."""
        n, C = self.n, self.chains
        xb = np.zeros(n) if x_best is None else np.array(x_best, np.float64)
        fb = np.array([np.inf if f_best is None else f_best], np.float64)
        xi = np.zeros(n) if x_inc is None else np.array(x_inc, np.float64)
        fi = np.array([np.inf if f_inc is None else f_inc], np.float64)
        am = np.zeros(max(K, 1), np.int64)
        fl = np.zeros(max(K, 1))
        ac = np.zeros(max(K, 1), np.int64)
        words = (self.L + 31) // 32
        tl = min(trace_levels, K)
        bits = np.zeros((max(tl, 1), C, words), np.uint32) if tl > 0 else None
        Ff = np.zeros(C) if want_final else None
        Xf = np.zeros((C, n)) if want_final else None
        xs = np.zeros((max(K, 1), C), np.int64) if self.crossover else None
        out = Out(_p(xb), _p(fb), _p(xi), _p(fi), _p(am), _p(fl), _p(ac), _p(bits), tl, _p(Ff), _p(Xf), _p(xs))
        cfg = self.cfg(K, level0)
        rc = lib().sao_run(ctypes.byref(cfg), ctypes.byref(out))
        if rc != 0:
            raise ValueError(f"sao_run failed ({rc})")
        return {"x_best": xb, "f_best": float(fb[0]), "x_inc": xi, "f_inc": float(fi[0]),
                "argmin": am[:K], "f_level": fl[:K], "accepts": ac[:K], "bits": bits,
                "F_final": Ff, "X_final": Xf, "xo_src": None if xs is None else xs[:K]}


def pgd(name_or_id, x0, lo, hi, Q=None, max_iter=1000, tol=1e-10, armijo_c=1e-4, max_halvings=30):
    """Box-projected gradient descent with Armijo backtracking from x0."""
    cid = COSTS[name_or_id] if isinstance(name_or_id, str) else int(name_or_id)
    x = np.array(x0, np.float64)
    n = x.size
    lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, np.float64), (n,)))
    hi = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, np.float64), (n,)))
    Qa = None if Q is None else np.ascontiguousarray(Q, dtype=np.float64)
    f = np.zeros(1)
    it = np.zeros(1, np.int32)
    rc = lib().sao_pgd(cid, n, _p(lo), _p(hi), _p(Qa), _p(x), max_iter, tol, armijo_c, max_halvings, _p(f), _p(it))
    if rc != 0:
        raise ValueError("sao_pgd failed")
    return x, float(f[0]), int(it[0])


def nelder_mead(name_or_id, x0, lo, hi, Q=None, step_frac=0.05, max_iter=20000, ftol=1e-12, xtol=1e-10,
                table=None, adaptive=False):
    """Nelder-Mead with box clipping from x0 (adaptive: Gao & Han's coefficients); returns (x, f, iterations)."""
    cid = COSTS[name_or_id] if isinstance(name_or_id, str) else int(name_or_id)
    x = np.array(x0, np.float64)
    n = x.size
    lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, np.float64), (n,)))
    hi = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, np.float64), (n,)))
    Qa = None if Q is None else np.ascontiguousarray(Q, dtype=np.float64)
    f = np.zeros(1)
    it = np.zeros(1, np.int32)
    t, rows = _table(table)
    rc = lib().sao_nelder_mead(cid, n, _p(lo), _p(hi), _p(Qa), _p(t), rows, _p(x), step_frac, max_iter, ftol, xtol,
                               1 if adaptive else 0, _p(f), _p(it))
    if rc != 0:
        raise ValueError("sao_nelder_mead failed")
    return x, float(f[0]), int(it[0])
