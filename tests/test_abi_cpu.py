"""The C ABI library loads, exports every symbol include/sa.h declares, and
validates arguments on the host (no GPU call is made by these tests)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "sa.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sa_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def sa():
    import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)
    from paper_2408_00018_gb300 import _build, sa as sa_mod
    _build.build()
    return sa_mod


def test_library_exports_every_declared_symbol(sa):
    lib = sa.load()
    syms = _declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
    # the binding wraps every declared entry point
    assert set(syms) <= set(sa.SIGNATURES)


def test_host_only_calls(sa):
    lib = sa.load()
    assert lib.sa_levels_for(1000.0, 0.99, 0.01) == 1146
    assert lib.sa_levels_for(1.0, 1.5, 0.1) == -1
    assert lib.sa_strerror(0).decode() == "ok"
    assert "invalid" in lib.sa_strerror(1).decode()
    s = sa._Schedule()
    lib.sa_default_schedule(ctypes.byref(s))
    assert (s.T0, s.rho, s.levels, s.sigma_frac, s.boundary, s.precision) == (100.0, 0.9, 50, 0.1, 0, 0)


@pytest.mark.parametrize("bad", ["n0", "chains0", "L0", "rho", "T0", "lohi", "nan", "sigma", "rot_noQ", "cost", "prec",
                                 "levels_tmin"])
def test_create_rejects_bad_arguments_before_any_device_work(sa, bad):
    lib = sa.load()
    n, chains, L = 3, 64, 10
    lo, hi = np.full(n, -1.0), np.full(n, 1.0)
    cost = 0
    sch = sa.Schedule(levels=5)._c()
    if bad == "n0": n = 0
    if bad == "chains0": chains = 0
    if bad == "L0": L = 0
    if bad == "rho": sch.rho = 1.0
    if bad == "T0": sch.T0 = -1.0
    if bad == "lohi": lo[1] = 2.0
    if bad == "nan": hi[2] = np.nan
    if bad == "sigma": sch.sigma_frac = 0.0
    if bad == "rot_noQ": cost = 4
    if bad == "cost": cost = 17
    if bad == "prec": sch.precision = 9
    if bad == "levels_tmin": sch.levels, sch.T_min = 0, 200.0
    prob = sa._Problem(cost, None)
    box = sa._Box(lo.ctypes.data, hi.ctypes.data)
    out = ctypes.c_void_p(123)
    rc = lib.sa_create(ctypes.byref(prob), ctypes.byref(box), n, chains, L, ctypes.byref(sch), 0, None, ctypes.byref(out))
    assert rc == sa.SA_EINVAL
    assert not out.value


def test_null_and_range_checks(sa):
    lib = sa.load()
    assert lib.sa_run(None, 1) == sa.SA_EINVAL
    assert lib.sa_best(None, 0, None, None, None) == sa.SA_EINVAL
    assert lib.sa_philox_fill(0, 0, 0, 0, 0, 0, -1, None, None) == sa.SA_EINVAL
    assert lib.sa_philox_fill(0, 0, 0, 0, 0, 0, 5, None, None) == sa.SA_EINVAL
    assert lib.sa_argmin_f64(None, 0, None, None, None, None) == sa.SA_EINVAL
    assert lib.sa_argmin_scratch_bytes(0) == 0
    assert lib.sa_argmin_scratch_bytes(2048) == 16 and lib.sa_argmin_scratch_bytes(2049) == 32
    lib.sa_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2408_00018_gb300 import _build, sa as sa_mod
    monkeypatch.setattr(sa_mod, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError):
        sa_mod.load()
