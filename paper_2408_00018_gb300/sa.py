"""Thin Python binding of the C ABI in include/sa.h (argument marshalling only).

Every step of the annealing runs in the CUDA library ``libsa103.so``; this module
only converts Python arguments to the C structs and back.  PyTorch supplies the
CUDA stream (the current stream of the current device) and, for the
kernel-level calls, device memory.  There is no CPU fallback: if the library is
missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

SA_OK, SA_EINVAL, SA_ENOMEM, SA_ECUDA, SA_ETIMEOUT, SA_ENUMERIC, SA_ESTATE = range(7)
COSTS = {"schwefel": 0, "rastrigin": 1, "ackley": 2, "rosenbrock": 3, "rot_rastrigin": 4, "rot_schwefel": 5,
         "branin": 6, "cosine_mixture": 7, "dekkers_aarts": 8, "easom": 9, "exponential": 10,
         "goldstein_price": 11, "griewank": 12, "himmelblau": 13, "levy_montalvo": 14, "langerman": 15,
         "michalewicz": 16, "salomon": 17, "six_hump_camel": 18, "shubert": 19, "shekel": 20, "foxholes": 21}
BOUNDARY = {"reflect": 0, "clip": 1}
PRECISION = {"fp64": 0, "fp32": 1, "mixed_bf16": 2}
POLISH = {"pgd": 0, "nelder_mead": 1, "nelder_mead_adaptive": 2}
PROPOSAL = {"gaussian": 0, "uniform": 1}


class SAError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {_strerror(status)} (status {status})")


class _Problem(ctypes.Structure):
    _fields_ = [("cost", ctypes.c_int32), ("Q", ctypes.c_void_p), ("table", ctypes.c_void_p),
                ("table_rows", ctypes.c_int32)]


def _table(table):
    """(contiguous FP64 array, rows) of a table of rows (a_i1 .. a_in, c_i), or (None, 0)."""
    if table is None:
        return None, 0
    t = np.ascontiguousarray(np.atleast_2d(np.asarray(table, np.float64)))
    return t, t.shape[0]


def _problem(cost, Qa, tab, rows):
    return _Problem(COSTS[cost] if isinstance(cost, str) else int(cost), None if Qa is None else Qa.ctypes.data,
                    None if tab is None else tab.ctypes.data, rows)


class _Box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p)]


class _Schedule(ctypes.Structure):
    _fields_ = [("T0", ctypes.c_double), ("rho", ctypes.c_double), ("T_min", ctypes.c_double),
                ("levels", ctypes.c_int32), ("sigma_frac", ctypes.c_double), ("boundary", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("surrogate", ctypes.c_int32), ("polish_k", ctypes.c_int32),
                ("trace_levels", ctypes.c_int32), ("cost_repeat", ctypes.c_int32), ("independent", ctypes.c_int32),
                ("exchange_every", ctypes.c_int32), ("polish_method", ctypes.c_int32), ("proposal", ctypes.c_int32),
                ("crossover", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("accepts", ctypes.c_int64), ("levels_done", ctypes.c_int32),
                ("levels_total", ctypes.c_int32), ("f_level", ctypes.c_double), ("argmin", ctypes.c_int64),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64), ("t_start_ns", ctypes.c_int64),
                ("rechecks", ctypes.c_int64), ("true_evals", ctypes.c_int64)]


_lib = None

# symbol -> (restype, argtypes)
_V, _I32, _I64, _U32, _U64, _SZ, _D = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.c_uint64, ctypes.c_size_t, ctypes.c_double)
SIGNATURES = {
    "sa_default_schedule": (None, [_V]),
    "sa_levels_for": (_I32, [_D, _D, _D]),
    "sa_create": (ctypes.c_int, [_V, _V, _I32, _I64, _I32, _V, _U64, _V, _V]),
    "sa_create_batch": (ctypes.c_int, [_V, _V, _V, _V, _I32, _I32, _V, _U64, _V, _V]),
    "sa_autotune": (ctypes.c_int, [_V, _V]),
    "sa_describe": (_I32, [_V, _V, _SZ]),
    "sa_run": (ctypes.c_int, [_V, _I32]),
    "sa_reset": (ctypes.c_int, [_V]),
    "sa_profile": (ctypes.c_int, [_V, _I32, _V, _V]),
    "sa_best": (ctypes.c_int, [_V, _I32, _V, _V, _V]),
    "sa_level_log": (ctypes.c_int, [_V, _I32, _V, _V, _V, _V, _I32, _V]),
    "sa_trace": (ctypes.c_int, [_V, _I32, _V, _SZ]),
    "sa_trace_states": (ctypes.c_int, [_V, _I32, _V, _V]),
    "sa_checkpoint": (ctypes.c_int, [_V, _V, _V]),
    "sa_restore": (ctypes.c_int, [_V, _V, _SZ]),
    "sa_destroy": (None, [_V]),
    "sa_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sa_philox_fill": (ctypes.c_int, [_U32, _U32, _U32, _U32, _U32, _U32, _I64, _V, _V]),
    "sa_polish": (ctypes.c_int, [_I32, _I32, _V, _V, _V, _I32, _V, _I32, _D, _V, _V, _V, _V]),
    "sa_nelder_mead": (ctypes.c_int, [_I32, _I32, _V, _V, _V, _V, _I32, _I32, _V, _D, _I32, _D, _D, _I32, _V, _V, _V,
                                      _V]),
    "sa_gemm_bf16": (ctypes.c_int, [_V, _I32, _V, _I32, _V, _I32, _I32, _I32, _I32, _V, _V]),
    "sa_argmin_scratch_bytes": (_SZ, [_I64]),
    "sa_argmin_f64": (ctypes.c_int, [_V, _I64, _V, _V, _V, _V]),
    "sa_argmin_f64_static": (ctypes.c_int, [_V, _I64, _V, _V, _V]),
    "sa_pipe_rate": (ctypes.c_int, [_I32, _I32, _V, _V, _V]),
    "sa_rotate_rows": (ctypes.c_int, [_V, _I64, _I32, _V, _V, _V, _V]),
    "sa_da_trace": (ctypes.c_int, [_V, _I32, _V, _V]),
    "sa_da_network": (ctypes.c_int, [_V, _V, _V, _V, _V]),
    "sa_set_chain_offset": (ctypes.c_int, [_V, _I64]),
    "sa_restart_point": (ctypes.c_int, [_V, _I32, _V, _V]),
    "sa_set_restart": (ctypes.c_int, [_V, _I32, _V, _D, _I64]),
    "sa_mlp_param_count": (_I64, [_I32]),
    "sa_mlp_init": (ctypes.c_int, [_V, _I32, _U64, _V]),
    "sa_mlp_forward": (ctypes.c_int, [_V, _I32, _V, _I32, _V, _V]),
    "sa_mlp_loss_grad": (ctypes.c_int, [_V, _I32, _V, _V, _I32, _V, _V, _V]),
    "sa_mlp_adam": (ctypes.c_int, [_V, _V, _V, _V, _I64, _I32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, _V]),
}

# Largest input of sa_argmin_f64_static (SA_ARGMIN_STATIC_MAX_COUNT in include/sa.h).
ARGMIN_STATIC_MAX_COUNT = 1 << 27


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libsa103.so (raises if it is missing and build_if_missing is False)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library {_build.LIB} is not built; run __graft_entry__.build()")
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _strerror(status: int) -> str:
    try:
        return load().sa_strerror(status).decode()
    except Exception:  # the library itself failed to load
        return "unknown"


def _check(status: int, where: str):
    if status != SA_OK:
        raise SAError(status, where)


def _current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass
class Schedule:
    T0: float = 100.0
    rho: float = 0.9
    T_min: float = 0.0
    levels: int = 50
    sigma_frac: float = 0.1
    boundary: str = "reflect"
    precision: str = "fp64"
    trace_levels: int = 0
    polish_k: int = 0
    surrogate: int = 0
    cost_repeat: int = 1
    independent: int = 0
    exchange_every: int = 1
    polish_method: str = "pgd"
    proposal: str = "gaussian"
    crossover: int = 0

    def _c(self) -> _Schedule:
        return _Schedule(self.T0, self.rho, self.T_min, self.levels, self.sigma_frac, BOUNDARY[self.boundary],
                         PRECISION[self.precision], self.surrogate, self.polish_k, self.trace_levels,
                         self.cost_repeat, self.independent, self.exchange_every, POLISH[self.polish_method],
                         PROPOSAL[self.proposal], self.crossover)


def levels_for(T0: float, rho: float, T_min: float) -> int:
    return load().sa_levels_for(T0, rho, T_min)


class Handle:
    """One solver (sa_create ... sa_destroy)."""

    def __init__(self, ptr, n, chains, L, schedule):
        self._ptr = ptr
        self.n, self.chains, self.L, self.schedule = n, chains, L, schedule

    def run(self, levels: int = -1):
        _check(load().sa_run(self._ptr, levels), "sa_run")

    def reset(self):
        _check(load().sa_reset(self._ptr), "sa_reset")

    def autotune(self) -> float:
        """Pick launch shapes per dimension group by timing level-0 sweeps; returns the summed ms."""
        ms = ctypes.c_double()
        _check(load().sa_autotune(self._ptr, ctypes.byref(ms)), "sa_autotune")
        return ms.value

    def describe(self):
        """The handle's launch groups (kind, problems, n_max, block, smem, unroll, items)."""
        import json
        lib = load()
        m = lib.sa_describe(self._ptr, None, 0)
        buf = ctypes.create_string_buffer(m + 1)
        lib.sa_describe(self._ptr, buf, m + 1)
        return json.loads(buf.value.decode())

    def profile(self, levels: int = -1):
        """Eager run with CUDA events: per-level (sweep_ms, level_ms)."""
        n_levels = self.schedule.levels if self.schedule.levels > 0 else levels_for(
            self.schedule.T0, self.schedule.rho, self.schedule.T_min)
        m = n_levels if levels == -1 else levels
        sw = np.zeros(m)
        lv = np.zeros(m)
        _check(load().sa_profile(self._ptr, levels, sw.ctypes.data, lv.ctypes.data), "sa_profile")
        return sw, lv

    def best(self, problem: int = 0):
        x = np.zeros(self.n)
        f = ctypes.c_double()
        st = _Stats()
        _check(load().sa_best(self._ptr, problem, x.ctypes.data, ctypes.byref(f), ctypes.byref(st)), "sa_best")
        stats = {k: getattr(st, k) for k, _ in _Stats._fields_}
        return x, f.value, stats

    def level_log(self, problem: int = 0, cap: int = 1 << 20):
        cap = min(cap, 1 << 20)
        st = _Stats()
        lib = load()
        n_levels = self.schedule.levels if self.schedule.levels > 0 else levels_for(
            self.schedule.T0, self.schedule.rho, self.schedule.T_min)
        cap = min(cap, n_levels)
        am = np.zeros(cap, np.int64)
        fl = np.zeros(cap)
        fi = np.zeros(cap)
        tn = np.zeros(cap, np.int64)
        cnt = ctypes.c_int32()
        _check(lib.sa_level_log(self._ptr, problem, am.ctypes.data, fl.ctypes.data, fi.ctypes.data, tn.ctypes.data,
                                cap, ctypes.byref(cnt)), "sa_level_log")
        m = cnt.value
        del st
        return {"argmin": am[:m], "f_level": fl[:m], "f_inc": fi[:m], "t_ns": tn[:m]}

    def trace(self, level: int, total_chains: int | None = None):
        C = self.chains if total_chains is None else total_chains
        words = (self.L + 31) // 32
        bits = np.zeros((C, words), np.uint32)
        _check(load().sa_trace(self._ptr, level, bits.ctypes.data, bits.size), "sa_trace")
        return bits

    def trace_states(self, level: int):
        X = np.zeros((self.chains, self.n))
        F = np.zeros(self.chains)
        _check(load().sa_trace_states(self._ptr, level, X.ctypes.data, F.ctypes.data), "sa_trace_states")
        return X, F

    def set_chain_offset(self, offset: int) -> None:
        """sa_set_chain_offset: this handle's chains are global chains offset .. offset + chains - 1."""
        _check(load().sa_set_chain_offset(self._ptr, offset), "sa_set_chain_offset")

    def restart_point(self, problem: int = 0):
        """sa_restart_point: (x, f) of this handle's restart point after the last level."""
        x = np.zeros(self.n)
        f = ctypes.c_double()
        _check(load().sa_restart_point(self._ptr, problem, x.ctypes.data, ctypes.byref(f)), "sa_restart_point")
        return x, f.value

    def set_restart(self, x, f: float, argmin: int, problem: int = 0) -> None:
        """sa_set_restart: the exchanged restart point of the next level."""
        x = np.ascontiguousarray(x, np.float64)
        _check(load().sa_set_restart(self._ptr, problem, x.ctypes.data, float(f), int(argmin)), "sa_set_restart")

    def da_trace(self, level: int):
        """Surrogate values of a traced delayed-acceptance level: (ft0 [chains], ftp [L, chains])."""
        ft0 = np.zeros(self.chains, np.float32)
        ftp = np.zeros((self.L, self.chains), np.float32)
        _check(load().sa_da_trace(self._ptr, level, ft0.ctypes.data, ftp.ctypes.data), "sa_da_trace")
        return ft0, ftp

    def da_network(self):
        """The surrogate network of the last completed level (sa_da_network):
        (params [sa_mlp_param_count(n)], (mu, sigma), mid [n], inv_half [n]), FP32."""
        lib = load()
        P = int(lib.sa_mlp_param_count(self.n))
        p = np.zeros(P, np.float32)
        ms = np.zeros(2, np.float32)
        mid = np.zeros(self.n, np.float32)
        ih = np.zeros(self.n, np.float32)
        _check(lib.sa_da_network(self._ptr, p.ctypes.data, ms.ctypes.data, mid.ctypes.data, ih.ctypes.data),
               "sa_da_network")
        return p, (float(ms[0]), float(ms[1])), mid, ih

    def checkpoint(self) -> bytes:
        lib = load()
        ln = ctypes.c_size_t()
        _check(lib.sa_checkpoint(self._ptr, None, ctypes.byref(ln)), "sa_checkpoint")
        buf = ctypes.create_string_buffer(ln.value)
        _check(lib.sa_checkpoint(self._ptr, buf, ctypes.byref(ln)), "sa_checkpoint")
        return buf.raw[:ln.value]

    def restore(self, blob: bytes):
        _check(load().sa_restore(self._ptr, blob, len(blob)), "sa_restore")

    def destroy(self):
        if self._ptr:
            load().sa_destroy(self._ptr)
            self._ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def create(cost, lo, hi, n, chains, L, schedule: Schedule | None = None, seed: int = 0, Q=None, stream=None,
           table=None) -> Handle:
    """sa_create: one box-constrained problem (Eq. 1) with `chains` chains of L steps per level.
    Rotated costs take Q (n x n); Tests 11, 18 and 19 take table (rows of (a_i1 .. a_in, c_i))."""
    lib = load()
    schedule = schedule or Schedule()
    lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, np.float64), (n,)))
    hi = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, np.float64), (n,)))
    Qa = None if Q is None else np.ascontiguousarray(Q, dtype=np.float64)
    tab, rows = _table(table)
    prob = _problem(cost, Qa, tab, rows)
    box = _Box(lo.ctypes.data, hi.ctypes.data)
    sch = schedule._c()
    out = ctypes.c_void_p()
    s = _current_stream() if stream is None else ctypes.c_void_p(stream)
    _check(lib.sa_create(ctypes.byref(prob), ctypes.byref(box), n, chains, L, ctypes.byref(sch), seed, s,
                         ctypes.byref(out)), "sa_create")
    return Handle(out, n, chains, L, schedule)


class BatchHandle(Handle):
    """sa_create_batch: several independent problems in one solver."""

    def __init__(self, ptr, ns, chains, L, schedule):
        super().__init__(ptr, max(ns), sum(chains), L, schedule)
        self.ns, self.chains_per = list(ns), list(chains)

    def best(self, problem: int = 0):
        x = np.zeros(self.ns[problem])
        f = ctypes.c_double()
        st = _Stats()
        _check(load().sa_best(self._ptr, problem, x.ctypes.data, ctypes.byref(f), ctypes.byref(st)), "sa_best")
        return x, f.value, {k: getattr(st, k) for k, _ in _Stats._fields_}

    def trace_states(self, level: int):
        """Final states of a traced level: list over problems of (X [chains_p, n_p], F [chains_p])."""
        total = sum(n * c for n, c in zip(self.ns, self.chains_per))
        X = np.zeros(total)
        F = np.zeros(sum(self.chains_per))
        _check(load().sa_trace_states(self._ptr, level, X.ctypes.data, F.ctypes.data), "sa_trace_states")
        out, xo, co = [], 0, 0
        for n, c in zip(self.ns, self.chains_per):
            out.append((X[xo:xo + n * c].reshape(c, n), F[co:co + c]))
            xo += n * c
            co += c
        return out

    def trace(self, level: int):
        """Accept bits of a traced level: list over problems of [chains_p, words]."""
        words = (self.L + 31) // 32
        bits = np.zeros((sum(self.chains_per), words), np.uint32)
        _check(load().sa_trace(self._ptr, level, bits.ctypes.data, bits.size), "sa_trace")
        out, co = [], 0
        for c in self.chains_per:
            out.append(bits[co:co + c])
            co += c
        return out


def create_batch(problems, L, schedule: Schedule | None = None, seed: int = 0, stream=None) -> BatchHandle:
    """sa_create_batch: problems is a list of dicts with cost, n, chains, lo, hi (and Q for rotated costs,
    table for Tests 11, 18, 19)."""
    lib = load()
    schedule = schedule or Schedule()
    P = len(problems)
    los = [np.ascontiguousarray(np.broadcast_to(np.asarray(p["lo"], np.float64), (p["n"],))) for p in problems]
    his = [np.ascontiguousarray(np.broadcast_to(np.asarray(p["hi"], np.float64), (p["n"],))) for p in problems]
    Qs = [None if p.get("Q") is None else np.ascontiguousarray(p["Q"], dtype=np.float64) for p in problems]
    tabs = [_table(p.get("table")) for p in problems]
    probs = (_Problem * P)(*[_problem(p["cost"], q, t, r) for p, q, (t, r) in zip(problems, Qs, tabs)])
    boxes = (_Box * P)(*[_Box(lo.ctypes.data, hi.ctypes.data) for lo, hi in zip(los, his)])
    ns = np.array([p["n"] for p in problems], np.int32)
    cs = np.array([p["chains"] for p in problems], np.int64)
    sch = schedule._c()
    out = ctypes.c_void_p()
    s = _current_stream() if stream is None else ctypes.c_void_p(stream)
    _check(lib.sa_create_batch(probs, boxes, ns.ctypes.data, cs.ctypes.data, P, L, ctypes.byref(sch), seed, s,
                               ctypes.byref(out)), "sa_create_batch")
    return BatchHandle(out, ns.tolist(), cs.tolist(), L, schedule)


def polish(cost, x0, lo, hi, max_iter: int = 1000, tol: float = 1e-10, Q=None, stream=None):
    """sa_polish: box-projected gradient descent from each row of x0 (k x n); returns (x, f, iters).
    Rotated costs take Q (n x n)."""
    x0 = np.ascontiguousarray(np.atleast_2d(np.asarray(x0, np.float64)))
    k, n = x0.shape
    lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, np.float64), (n,)))
    hi = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, np.float64), (n,)))
    x = np.zeros_like(x0)
    f = np.zeros(k)
    it = np.zeros(k, np.int32)
    s = _current_stream() if stream is None else ctypes.c_void_p(stream)
    Qa = None if Q is None else np.ascontiguousarray(Q, dtype=np.float64)
    _check(load().sa_polish(COSTS[cost] if isinstance(cost, str) else int(cost), n, lo.ctypes.data, hi.ctypes.data,
                            None if Qa is None else Qa.ctypes.data, k, x0.ctypes.data, max_iter, tol, x.ctypes.data,
                            f.ctypes.data, it.ctypes.data, s),
           "sa_polish")
    return x, f, it


def nelder_mead(cost, x0, lo, hi, step_frac: float = 0.05, max_iter: int = 20000, ftol: float = 1e-12,
                xtol: float = 1e-10, Q=None, stream=None, table=None, adaptive: bool = False):
    """sa_nelder_mead: Nelder-Mead with box clipping from each row of x0 (k x n); returns (x, f, iters).
    Rotated costs take Q (n x n); Tests 11, 18 and 19 take table."""
    x0 = np.ascontiguousarray(np.atleast_2d(np.asarray(x0, np.float64)))
    k, n = x0.shape
    lo = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, np.float64), (n,)))
    hi = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, np.float64), (n,)))
    x = np.zeros_like(x0)
    f = np.zeros(k)
    it = np.zeros(k, np.int32)
    s = _current_stream() if stream is None else ctypes.c_void_p(stream)
    Qa = None if Q is None else np.ascontiguousarray(Q, dtype=np.float64)
    tab, rows = _table(table)
    _check(load().sa_nelder_mead(COSTS[cost] if isinstance(cost, str) else int(cost), n, lo.ctypes.data,
                                 hi.ctypes.data, None if Qa is None else Qa.ctypes.data,
                                 None if tab is None else tab.ctypes.data, rows, k, x0.ctypes.data, step_frac,
                                 max_iter, ftol, xtol, 1 if adaptive else 0, x.ctypes.data, f.ctypes.data,
                                 it.ctypes.data, s),
           "sa_nelder_mead")
    return x, f, it


def philox_fill(ctr, key, out) -> None:
    """Philox4x32-10 blocks for counters (ctr0 + i, ctr1, ctr2, ctr3) into a uint32/int32 CUDA tensor of 4*count."""
    count = out.numel() // 4
    _check(load().sa_philox_fill(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1], count,
                                 ctypes.c_void_p(out.data_ptr()), _current_stream()), "sa_philox_fill")


def argmin_f64(F):
    """Lowest-index argmin of a float64 CUDA tensor; returns (index, value) as 0-d CUDA tensors."""
    import torch
    lib = load()
    count = F.numel()
    scratch = torch.empty(max(1, lib.sa_argmin_scratch_bytes(count)), dtype=torch.uint8, device=F.device)
    idx = torch.empty((), dtype=torch.int64, device=F.device)
    val = torch.empty((), dtype=torch.float64, device=F.device)
    _check(lib.sa_argmin_f64(ctypes.c_void_p(F.data_ptr()), count, ctypes.c_void_p(idx.data_ptr()),
                             ctypes.c_void_p(val.data_ptr()), ctypes.c_void_p(scratch.data_ptr()),
                             _current_stream()), "sa_argmin_f64")
    return idx, val


def argmin_f64_static(F):
    """Like argmin_f64 but without any scratch allocation: the library's fixed
    1 MiB scratch is used instead (inputs up to ARGMIN_STATIC_MAX_COUNT values;
    calls overlapping on the GPU race on that scratch)."""
    import torch
    idx = torch.empty((), dtype=torch.int64, device=F.device)
    val = torch.empty((), dtype=torch.float64, device=F.device)
    _check(load().sa_argmin_f64_static(ctypes.c_void_p(F.data_ptr()), F.numel(), ctypes.c_void_p(idx.data_ptr()),
                                       ctypes.c_void_p(val.data_ptr()), _current_stream()), "sa_argmin_f64_static")
    return idx, val


def rotate_rows(X, Q):
    """sa_rotate_rows: Y = X Q^T on the tensor cores as double-float pairs, for a float32 CUDA
    tensor X [rows x n] and a float64 CUDA tensor Q [n x n]; returns Y [rows x n x 2] (hi, lo)
    and the GEMMs' status word."""
    import torch
    Y = torch.empty((X.shape[0], X.shape[1], 2), dtype=torch.float32, device=X.device)
    st = torch.zeros(1, dtype=torch.int32, device=X.device)
    _check(load().sa_rotate_rows(_ptr(X), X.shape[0], X.shape[1], _ptr(Q), _ptr(Y), _ptr(st), _current_stream()),
           "sa_rotate_rows")
    return Y, st


# ---------------------------------------------------------------- pipe rates (roofline)
PIPE_OPS = {"sin": 0, "cos": 1, "lg2": 2, "ex2": 3, "sqrt": 4, "rsqrt": 5, "imad_wide": 6, "imad_hi": 7,
            "imad_lo": 8, "lop3": 9, "ffma": 10, "dfma": 11, "philox": 12}


def pipe_rate(op: str, iters: int = 4096):
    """sa_pipe_rate: measured (operations per clock per SM, operations per second)
    of one pipe of the current GPU (Philox: whole blocks)."""
    per_clk = ctypes.c_double()
    per_s = ctypes.c_double()
    _check(load().sa_pipe_rate(PIPE_OPS[op], iters, _current_stream(), ctypes.byref(per_clk), ctypes.byref(per_s)),
           "sa_pipe_rate")
    return per_clk.value, per_s.value


# ---------------------------------------------------------------- surrogate network
def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def mlp_param_count(n: int) -> int:
    """Parameters of the surrogate for inputs of dimension n (sa_mlp_param_count)."""
    return int(load().sa_mlp_param_count(n))


def mlp_init(params, n: int, seed: int = 0) -> None:
    """sa_mlp_init on a float32 CUDA tensor of mlp_param_count(n) elements."""
    _check(load().sa_mlp_init(_ptr(params), n, seed, _current_stream()), "sa_mlp_init")


def mlp_forward(params, n: int, X):
    """sa_mlp_forward: surrogate values of the rows of a float32 CUDA tensor X [B x n]."""
    import torch
    y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    _check(load().sa_mlp_forward(_ptr(params), n, _ptr(X), X.shape[0], _ptr(y), _current_stream()), "sa_mlp_forward")
    return y


def mlp_loss_grad(params, n: int, X, t):
    """sa_mlp_loss_grad: (loss, gradient) of the mean squared error on rows X [B x n], targets t [B]."""
    import torch
    g = torch.empty_like(params)
    loss = torch.empty((), dtype=torch.float32, device=X.device)
    _check(load().sa_mlp_loss_grad(_ptr(params), n, _ptr(X), _ptr(t), X.shape[0], _ptr(g), _ptr(loss),
                                   _current_stream()), "sa_mlp_loss_grad")
    return loss, g


def mlp_adam(params, grad, m, v, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8) -> None:
    """sa_mlp_adam: one in-place Adam step of float32 CUDA tensors."""
    _check(load().sa_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(), step, lr, beta1, beta2, eps,
                              _current_stream()), "sa_mlp_adam")
