"""The GEMM epilogues' erf (Hastings' rational approximation, Abramowitz and Stegun 7.1.26):
the constants as written in the kernel source, evaluated in FP64, stay within the formula's
published error bound (1.5e-7) of the exact erf over the whole line; a mistyped constant
breaks the bound."""
import math
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2408_00018_gb300", "csrc", "gelu.cuh")


def _kernel_constants():
    src = open(SRC).read()
    body = re.search(r"float erf_hastings\(float x\) \{(.*?)\n\}", src, re.S).group(1)
    # t = 1 / fmaf(p, |x|, 1); poly = t * (a1 + t (a2 + ...)) written innermost first: a5 .. a1
    p = float(re.search(r"fmaf\((-?\d+\.\d+)f, ax, 1\.0f\)", body).group(1))
    poly = re.search(r"const float poly =(.*?);", body, re.S).group(1)
    a5, a4, a3, a2, a1 = [float(v) for v in re.findall(r"(-?\d+\.\d+)f", poly)]
    return p, (a1, a2, a3, a4, a5)


def _erf(x, p, a):
    ax = abs(x)
    t = 1.0 / (1.0 + p * ax)
    poly = t * (a[0] + t * (a[1] + t * (a[2] + t * (a[3] + t * a[4]))))
    return math.copysign(1.0 - poly * math.exp(-ax * ax), x)


def test_kernel_constants_meet_the_published_bound():
    p, a = _kernel_constants()
    xs = np.concatenate([np.linspace(-6.0, 6.0, 120001), [0.0, 1e-6, -1e-6, 10.0, -10.0]])
    err = max(abs(_erf(float(x), p, a) - math.erf(float(x))) for x in xs)
    assert err <= 1.5e-7, err


def test_a_mistyped_constant_breaks_the_bound():
    p, a = _kernel_constants()
    xs = np.linspace(0.0, 4.0, 4001)
    for i in range(5):
        b = list(a)
        b[i] *= 1.0 + 1e-5
        err = max(abs(_erf(float(x), p, b) - math.erf(float(x))) for x in xs)
        assert err > 1.5e-7, (i, err)


def _forward_constants():
    """The forward pass's GELU constants as the kernel source writes them: products of
    Hastings' literals with a scale, parsed back (scale, literal) so each is checked."""
    src = open(SRC).read()
    p = re.search(r"kGeluP = (-?\d+\.\d+)f \* (-?\d+\.\d+)f;", src).groups()
    b = dict((k, (float(s), float(v))) for k, s, v in
             re.findall(r"(kGeluB\d) = (-?\d+\.\d+)f \* (-?\d+\.\d+)f", src))
    c = float(re.search(r"kGeluC = (-?\d+\.\d+)f;", src).group(1))
    return (float(p[0]), float(p[1])), b, c


def test_forward_gelu_constants_are_hastings_scaled():
    """z Phi(z) = max(z, 0) - |z| poly(t)/2 e^(-z^2/2), t = 1/(1 + p |z|/sqrt 2): the
    forward constants are p/sqrt 2, -a_i/2 and -log2(e)/2 of the pinned erf constants."""
    p, a = _kernel_constants()
    (pp, inv_sqrt2), b, c = _forward_constants()
    assert pp == p and abs(inv_sqrt2 - 1 / math.sqrt(2)) < 1e-15
    for i in range(5):
        scale, lit = b["kGeluB%d" % (i + 1)]
        assert scale == -0.5 and lit == a[i]
    assert abs(c + 0.5 / math.log(2)) < 1e-15


def _gelu_forward(z, pp, b, c):
    az = abs(z)
    t = 1.0 / (1.0 + pp * az)
    q = t * (b[0] + t * (b[1] + t * (b[2] + t * (b[3] + t * b[4]))))
    return max(z, 0.0) + az * q * 2.0 ** (c * z * z)


def test_forward_gelu_matches_exact_gelu_within_hastings_bound():
    (pp, s), bd, c = _forward_constants()
    b = [bd["kGeluB%d" % (i + 1)][0] * bd["kGeluB%d" % (i + 1)][1] for i in range(5)]
    zs = np.linspace(-8.0, 8.0, 40001)
    for z in zs:
        exact = 0.5 * z * (1.0 + math.erf(z / math.sqrt(2.0)))
        assert abs(_gelu_forward(float(z), pp * s, b, c) - exact) <= 0.5 * abs(z) * 1.5e-7 + 1e-15, z
    # a flipped sign of the correction term is far outside the bound
    z = 0.7
    exact = 0.5 * z * (1.0 + math.erf(z / math.sqrt(2.0)))
    assert abs(_gelu_forward(z, pp * s, [-x for x in b], c) - exact) > 0.1
