"""Pins of the oracle's smoothing kernels (Eqs. 8 and 9) against the kernel
conditions of Sect. 2.2 (compact support, unit normalisation) and calculus
(continuity of the spline pieces, the derivative of W_p)."""
import math

import numpy as np
import pytest
from scipy import integrate


@pytest.mark.parametrize("h", [0.3, 1.0, 2.7])
def test_spline_normalisation(orc, h):
    # int W d^3r = 1 (normalisation condition of Sect. 2.2), in 3-D spherical shells
    val, _ = integrate.quad(lambda r: 4 * math.pi * r * r * orc.W(r / h, h), 0, 2 * h,
                            points=[h], epsabs=1e-13, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-10


@pytest.mark.parametrize("h", [0.3, 1.0, 2.7])
def test_pressure_kernel_normalisation(orc, h):
    val, _ = integrate.quad(lambda r: 4 * math.pi * r * r * orc.Wp(r / h, h), 0, 2 * h,
                            epsabs=1e-13, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-10


def test_compact_support(orc):
    for xi in [2.0, 2.0 + 1e-12, 2.5, 10.0]:
        assert orc.W(xi, 1.3) == 0.0
        assert orc.Wp(xi, 1.3) == 0.0
        assert orc.dWp_dxi(xi, 1.3) == 0.0
    assert orc.W(2.0 - 1e-6, 1.0) > 0.0


def test_spline_is_c2_at_the_joint(orc):
    # both pieces of Eq. 8 meet at xi = 1 with equal value, slope and curvature
    h = 1.0
    d = 1e-4
    left = [orc.W(1 - k * d, h) for k in (0, 1, 2)]
    right = [orc.W(1 + k * d, h) for k in (0, 1, 2)]
    assert abs(orc.W(1 - 1e-12, h) - orc.W(1 + 1e-12, h)) < 1e-9
    s_left = (3 * left[0] - 4 * left[1] + left[2]) / (2 * d)
    s_right = -(3 * right[0] - 4 * right[1] + right[2]) / (2 * d)
    assert abs(s_left - s_right) < 1e-6
    c_left = (left[0] - 2 * left[1] + left[2]) / d ** 2
    c_right = (right[0] - 2 * right[1] + right[2]) / d ** 2
    assert abs(c_left - c_right) < 1e-3 * abs(c_left)
    # value at the centre: W(0, h) = 1 / (pi h^3)
    assert abs(orc.W(0.0, 0.5) - 1.0 / (math.pi * 0.125)) < 1e-12


@pytest.mark.parametrize("xi", [0.05, 0.5, 1.0, 1.5, 1.9])
def test_pressure_kernel_derivative(orc, xi):
    h = 0.8
    d = 1e-6
    fd = (orc.Wp(xi + d, h) - orc.Wp(xi - d, h)) / (2 * d)
    assert abs(orc.dWp_dxi(xi, h) - fd) < 1e-7 * max(1.0, abs(fd))


def test_pressure_kernel_slope_at_centre(orc):
    # The derivative at xi -> 0 follows from Eq. 9 as -45/(16 pi h^3); the limit
    # printed after Eq. 9 (-45/(64 pi h^4)) drops the (2 - xi)^2 = 4 factor.
    for h in (0.5, 1.0, 2.0):
        assert abs(orc.dWp_dxi(0.0, h) + 45.0 / (16.0 * math.pi * h ** 3)) < 1e-12


def test_delta_limit(orc):
    # As h -> 0 the smoothed value of a smooth field tends to the field value
    # (third kernel condition of Sect. 2.2): for f(r) = 1 + r^2 the smoothed
    # value at the origin is 1 + h^2 * const, so the error falls as h^2.
    errs = []
    for h in (0.4, 0.2, 0.1):
        val, _ = integrate.quad(lambda r: 4 * math.pi * r * r * orc.W(r / h, h) * (1 + r * r),
                                0, 2 * h, points=[h], epsabs=1e-14, epsrel=1e-13)
        errs.append(val - 1.0)
    assert errs[0] > errs[1] > errs[2] > 0
    assert abs(errs[0] / errs[1] - 4.0) < 1e-6
    assert abs(errs[1] / errs[2] - 4.0) < 1e-6
