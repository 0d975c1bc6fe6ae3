"""Pin of the geometry kernels' own arcsine polynomial (no GPU needed).

The cylinder's clamped inverse Phi-hat = 2 arcsin(sqrt(S)) (Sec. 4.2.1, in
the half-angle form the kernels use) is evaluated on the device as
sqrt(s) p(s), with p a degree-8 polynomial for 2 arcsin(sqrt(s)) / sqrt(s) on
[0, 1/2].  This test reads the coefficients of `asin_sqrt_ratio2` from the
CUDA source, evaluates them in FP32 Horner order with fused multiply-adds
(each step formed exactly in FP64, then rounded once to FP32), and checks the
relative error bound the source states, 6.4e-8, against math.asin on a dense
grid (and the polynomial's own 3.9e-9 in FP64).  The scalar and the packed (two-lane) copies of the polynomial must
carry the same coefficients.
"""
import math
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2609_29253_gb300", "csrc",
                   "pat_geom.cuh")


def _coeffs(name):
    text = open(SRC).read()
    m = re.search(r"__device__ __forceinline__ \w+ " + name + r"\([^)]*\)\s*\{(.*?)\n\}", text, re.S)
    assert m, name
    nums = [float(v) for v in re.findall(r"(-?\d+\.\d*(?:e-?\d+)?)f", m.group(1))]
    return nums


def _horner_fp32(c, s):
    """c[0] s^8 + ... + c[8] by FP32 fused multiply-adds."""
    s = np.float32(s)
    p = np.float32(c[0])
    for ci in c[1:]:
        p = np.float32(np.float64(p) * np.float64(s) + np.float64(np.float32(ci)))
    return p


def test_scalar_and_packed_coefficients_agree():
    a = _coeffs("asin_sqrt_ratio2")
    b = _coeffs("asin_sqrt_ratio2_x2")
    assert len(a) == 9 and a == b


def test_polynomial_within_stated_bound():
    c = _coeffs("asin_sqrt_ratio2")
    s = np.concatenate([np.linspace(0.0, 0.5, 200001)[1:], np.geomspace(1e-12, 1e-3, 2000)])
    worst = 0.0
    for sv in s.astype(np.float32):
        x = float(sv)
        if x <= 0.0:
            continue
        exact = 2.0 * math.asin(math.sqrt(x)) / math.sqrt(x)
        got = float(_horner_fp32(c, sv))
        worst = max(worst, abs(got - exact) / exact)
    assert worst <= 6.4e-8, worst
    # the polynomial itself, evaluated in FP64
    c64 = np.array(c)
    xs = s[s > 0].astype(np.float64)
    rel = np.abs(np.polyval(c64, xs) / (2.0 * np.arcsin(np.sqrt(xs)) / np.sqrt(xs)) - 1.0)
    assert rel.max() <= 3.9e-9, rel.max()
    # s = 0: the limit 2 arcsin(sqrt(s)) / sqrt(s) -> 2 exactly
    assert float(_horner_fp32(c, np.float32(0.0))) == 2.0
