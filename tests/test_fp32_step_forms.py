"""Two branch-free forms the FP32 sweeps use in place of the written-out step of Sec. 2.1
must give the same bits as the forms they replace, since the FP32 parity tests compare
decisions taken on those bits.  Both are checked here on the host in IEEE single precision:

- the box handling of a proposal, "reflect once at the face it crossed, then clip", as
  min(min(max(xp, 2 lo - xp), max(2 hi - xp, lo)), hi) against the case-by-case form, on
  random and edge cases including steps several box widths long;
- the FP32 uniform's bit pattern 0x3F800000 | (w >> 9), built by one funnel shift of the
  pair (0x7F, w) right by 9, against the shift-and-or form, on random words and the ends.
"""
import numpy as np

f32 = np.float32


def reflect_clip_cases(xp, lo, hi):
    """Reflect once at the crossed face, then clip: the case-by-case form."""
    if xp < lo:
        r = f32(f32(2.0) * lo - xp)
    elif xp > hi:
        r = f32(f32(2.0) * hi - xp)
    else:
        r = xp
    return min(max(r, lo), hi)


def reflect_clip_minmax(xp, lo, hi):
    """The form of the sweeps: four minima and maxima, a and b rounded once."""
    a = f32(f32(2.0) * lo - xp)
    b = f32(f32(2.0) * hi - xp)
    return min(min(max(xp, a), max(b, lo)), hi)


def test_reflect_clip_minmax_equals_case_form():
    rng = np.random.default_rng(20241204)
    checked = 0
    for _ in range(60000):
        lo = f32(rng.uniform(-600.0, 100.0))
        hi = f32(lo + f32(rng.uniform(1e-3, 1200.0)))
        if not hi > lo:
            continue
        w = float(hi) - float(lo)
        # steps up to three box widths past either face, plus the faces and their neighbours
        pick = rng.integers(0, 4)
        if pick == 0:
            xp = f32(float(lo) + rng.uniform(-3.0, 4.0) * w)
        elif pick == 1:
            xp = f32(rng.choice([lo, hi]))
        elif pick == 2:
            xp = np.nextafter(lo, f32(-np.inf)) if rng.integers(0, 2) else np.nextafter(hi, f32(np.inf))
        else:
            xp = f32(float(lo) + rng.uniform(-1e-6, 1e-6) * w)
        assert reflect_clip_minmax(xp, lo, hi) == reflect_clip_cases(xp, lo, hi), (xp, lo, hi)
        checked += 1
    assert checked > 50000


def test_reflect_clip_result_stays_in_box():
    rng = np.random.default_rng(7)
    for _ in range(20000):
        lo = f32(rng.uniform(-5.12, 0.0))
        hi = f32(rng.uniform(0.0, 5.12))
        xp = f32(rng.normal(0.0, 20.0))
        r = reflect_clip_minmax(xp, lo, hi)
        assert lo <= r <= hi


def funnelshift_r(lo, hi, shift):
    """The low 32 bits of the 64-bit pair (hi, lo) shifted right (the funnel shift)."""
    return ((int(hi) << 32) | int(lo)) >> shift & 0xFFFFFFFF


def test_uniform_bits_by_funnel_shift():
    rng = np.random.default_rng(3)
    words = list(rng.integers(0, 2**32, size=100000, dtype=np.uint64)) + [0, 1, 511, 512, 2**31, 2**32 - 1]
    for w in words:
        w = int(w)
        assert funnelshift_r(w, 0x7F, 9) == (0x3F800000 | (w >> 9))
    # and the uniform it gives is (k + 1/2) 2^-23 in (0, 1), k the top 23 bits
    for w in (0, 2**32 - 1, 0x80000000):
        u = np.frombuffer(np.uint32(funnelshift_r(w, 0x7F, 9)).tobytes(), dtype=np.float32)[0] - f32(0.999999940395355225)
        k = w >> 9
        assert float(u) == (k + 0.5) * 2.0**-23
