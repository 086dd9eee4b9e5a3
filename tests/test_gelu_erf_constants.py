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
