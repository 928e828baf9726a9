"""Error bounds of the closed forms the kernels use in place of library calls.

The FP32-mixed viscous kernels take log(1 + x) of the perturbation ratios p'/p0 and rho'/rho0
from log(1 + x) = 2 atanh(z), z = x / (2 + x), summing the Taylor series of atanh through z^7
(|x| <= 1/32; the library's log1pf elsewhere).  These checks bound that evaluation: the truncated
series in FP64 against log1p, and the FP32 evaluation in the kernel's order (division, then the
fused multiply-adds of the Horner form, with a correctly rounded division; the kernels' approximate
division adds at most about two units of z) within four units in the last place of FP32."""
import math

import numpy as np


def _series_f64(x):
    z = x / (2.0 + x)
    z2 = z * z
    return 2.0 * z * (1.0 + z2 * (1.0 / 3.0 + z2 * (0.2 + z2 / 7.0)))


def _fma32(a, b, c):
    # the exact a b + c rounded once to FP32 (the product of two FP32 values is exact in FP64)
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _series_f32(x):
    x = np.float32(x)
    z = np.float32(x / np.float32(np.float32(2.0) + x))
    z2 = np.float32(z * z)
    s = _fma32(z2, _fma32(z2, _fma32(z2, np.float32(1.0 / 7.0), np.float32(0.2)), np.float32(1.0 / 3.0)),
               np.float32(1.0))
    return np.float32(np.float32(np.float32(2.0) * z) * s)


def test_truncated_atanh_series_is_exact_to_fp64_on_its_range():
    xs = np.concatenate([np.linspace(-1 / 32, 1 / 32, 4001), np.geomspace(1e-12, 1 / 32, 200),
                         -np.geomspace(1e-12, 1 / 32, 200)])
    rel = [abs(_series_f64(x) - math.log1p(x)) / abs(math.log1p(x)) for x in xs if x != 0.0]
    assert max(rel) < 1e-14


def test_fp32_evaluation_within_a_few_ulp():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(-1 / 32, 1 / 32, 20000), rng.uniform(-1e-4, 1e-4, 5000),
                         np.float32([1 / 32, -1 / 32, 1e-7, -1e-7])]).astype(np.float32)
    worst = 0.0
    for x in xs:
        if x == 0.0:
            continue
        exact = math.log1p(float(x))
        got = float(_series_f32(x))
        ulp = float(np.spacing(np.float32(abs(exact))))
        worst = max(worst, abs(got - exact) / ulp)
    assert worst <= 4.0, worst
