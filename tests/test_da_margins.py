"""The delayed-acceptance step takes both stages' decisions in FP32 outside margins and in
FP64 inside them; this pins the margins' derivation on the host.  The FP32 formulas of the
step are restated with exact IEEE single-precision arithmetic (round to nearest; an FMA
rounded once, through exact rationals), and on cases placed at the margins' edges every
FP32 decision must be one the FP64 tests would also take directly, for each way the
compiler may contract the FP64 margins' products and sums into FMAs.  A stage-1 margin
narrower than the FP64 one (3% suffices) or a stage-2 margin without the term for the FP32
threshold's rounding fails here, where a GPU parity test could not tell the wrong decisions
from near-ties."""
from fractions import Fraction
import itertools

import numpy as np

f32 = np.float32


def fma32(a, b, c):
    """fmaf: a b + c exactly, rounded once to FP32 (round to nearest even)."""
    exact = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    return _round32(exact)


def fma64(a, b, c):
    """fma: a b + c exactly, rounded once to FP64."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))  # Fraction -> float rounds to nearest even


def _round32(q):
    # the FP64 nearest of q, then FP32: exact unless q sits within 2^-53 of an FP32 tie, so
    # break such ties from the rational itself
    d = float(q)
    r = f32(d)
    if Fraction(float(r)) == q:
        return r
    lo = r if Fraction(float(r)) < q else np.nextafter(r, f32(-np.inf))
    hi = np.nextafter(lo, f32(np.inf))
    dlo, dhi = q - Fraction(float(lo)), Fraction(float(hi)) - q
    if dlo < dhi:
        return lo
    if dhi < dlo:
        return hi
    return lo if (int(lo.view(np.uint32)) & 1) == 0 else hi


def _sum64_variants(terms):
    """Every FP64 value of t0 + c1 x1 + c2 x2 + ... (left to right, t0 not a product) with
    each product either rounded on its own or fused into the running sum."""
    base, rest = terms[0], terms[1:]
    out = []
    for fuse in itertools.product((False, True), repeat=len(rest)):
        acc = base
        for (c, x), fz in zip(rest, fuse):
            acc = fma64(c, x, acc) if fz else acc + c * x
        out.append(acc)
    return out


def stage1_fast(ftp, ftc, t1, Tf):
    """The step's FP32 stage-1 test: True (pass), False (fail) or None (FP64 decides)."""
    if ftp <= ftc:
        return True
    d32 = f32(ftp - ftc)
    M1 = fma32(f32(1.1e-6), t1, fma32(f32(4.4e-7), Tf, f32(f32(2.4e-7) * d32)))
    if d32 < f32(t1 - M1):
        return True
    if d32 > f32(t1 + M1):
        return False
    return None


def stage2_fast(ftp, ftc, tau, dF, B, Tf):
    d32 = f32(ftp - ftc)
    thr32 = f32(d32 + tau)
    inner = f32(f32(4.0e-7) * f32(abs(d32) + abs(thr32)))
    Bt32 = fma32(f32(1.00001), B, fma32(f32(1.2e-6), abs(tau), fma32(f32(4.8e-7), Tf, inner)))
    if dF < f32(thr32 - Bt32):
        return True
    if dF > f32(thr32 + Bt32):
        return False
    return None


def _cases(rng, count):
    """Temperatures over six decades, with f~(x) at 0 (the differences then exact on the
    finest grid), of the order of T, or large (a coarse grid)."""
    for i in range(count):
        T = float(10.0 ** rng.uniform(-3, 3))
        ftc = (f32(0.0), f32(rng.uniform(-1.0, 1.0) * T), f32(rng.uniform(-500.0, 500.0)))[i % 3]
        yield T, f32(T), ftc


def test_stage1_fp32_decisions_are_the_fp64_ones():
    rng = np.random.default_rng(11)
    decided = 0
    for T, Tf, ftc in _cases(rng, 4000):
        t1 = f32(T * 10.0 ** rng.uniform(-4, 1.1))  # -T ln u for u in (3e-6, 0.9999)
        # ftp such that d32 sits a few ulps around the edges t1 -/+ M1
        for edge in (-1, 1):
            M1 = fma32(f32(1.1e-6), t1, fma32(f32(4.4e-7), Tf, f32(f32(2.4e-7) * t1)))
            target = f32(t1 + edge * M1)
            for k in range(-6, 7):
                ftp = f32(ftc + np.float32(target))
                for _ in range(abs(k)):
                    ftp = np.nextafter(ftp, f32(np.inf) if k > 0 else f32(-np.inf))
                fast = stage1_fast(ftp, ftc, t1, Tf)
                if fast is None:
                    continue
                decided += 1
                dFs = float(ftp) - float(ftc)
                tau1 = float(t1)
                # 1e-6 tau1 + 4e-7 T: either product may be fused into the sum, or neither
                for m1 in (1.0e-6 * tau1 + 4.0e-7 * T, fma64(1.0e-6, tau1, 4.0e-7 * T),
                           fma64(4.0e-7, T, 1.0e-6 * tau1)):
                    if fast:
                        assert dFs <= 0.0 or dFs < tau1 - m1, (ftp, ftc, t1, T)
                    else:
                        assert dFs > tau1 + m1, (ftp, ftc, t1, T)
    assert decided > 10000


def test_stage2_fp32_decisions_are_the_fp64_ones():
    rng = np.random.default_rng(12)
    decided = 0
    for T, Tf, ftc in _cases(rng, 6000):
        tau = f32(T * 10.0 ** rng.uniform(-4, 1.1))
        ftp = f32(ftc + f32(T * rng.uniform(-5.0, 5.0)))
        B = f32(float(tau) * 10.0 ** rng.uniform(-9, -2))
        d32 = f32(ftp - ftc)
        thr32 = f32(d32 + tau)
        inner = f32(f32(4.0e-7) * f32(abs(d32) + abs(thr32)))
        Bt32 = fma32(f32(1.00001), B, fma32(f32(1.2e-6), abs(tau), fma32(f32(4.8e-7), Tf, inner)))
        for edge in (-1, 1):
            target = f32(thr32 + edge * Bt32)
            for k in range(-6, 7):
                dF = target
                for _ in range(abs(k)):
                    dF = np.nextafter(dF, f32(np.inf) if k > 0 else f32(-np.inf))
                fast = stage2_fast(ftp, ftc, tau, dF, B, Tf)
                if fast is None:
                    continue
                decided += 1
                dFs = float(ftp) - float(ftc)
                thr = dFs + float(tau)
                for Bt in _sum64_variants([float(B), (1.0e-6, abs(float(tau))), (4.0e-7, T), (1e-12, abs(dFs))]):
                    if fast:
                        assert float(dF) < thr - Bt, (ftp, ftc, tau, dF, B, T)
                    else:
                        assert float(dF) > thr + Bt, (ftp, ftc, tau, dF, B, T)
    assert decided > 10000


def test_margins_are_not_loose_by_orders_of_magnitude():
    """The FP32 paths leave to FP64 only a band of a few of its own margins: a point just
    outside 2 margins is decided in FP32."""
    T, Tf = 3.0, f32(3.0)
    t1 = f32(2.5)
    ftc = f32(-120.0)
    M1 = 1.1e-6 * 2.5 + 4.4e-7 * 3.0 + 2.4e-7 * 2.5
    assert stage1_fast(f32(ftc + f32(2.5 - 2 * M1)), ftc, t1, Tf) is True
    assert stage1_fast(f32(ftc + f32(2.5 + 2 * M1)), ftc, t1, Tf) is False
