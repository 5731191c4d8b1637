"""Pins for the fundamental solution and its normal derivatives."""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle.kernels import kernel_values


def _G(x, y, k):
    r = np.hypot(*(x - y))
    return 0.25j * sp.hankel1(0, k * r)


@pytest.mark.parametrize("k", [2 * math.pi, 15.7, 4 * math.pi * (1 + 0.05j)])
def test_kernels_against_finite_differences(k):
    x = np.array([0.3, -0.2]); y = np.array([-0.55, 0.4])
    nx = np.array([math.cos(0.4), math.sin(0.4)]); ny = np.array([math.cos(2.1), math.sin(2.1)])
    S, D, Ds, N = kernel_values(x, nx, y, ny, k)
    h = 1e-5
    assert abs(S - _G(x, y, k)) < 1e-14
    dGy = (_G(x, y + h * ny, k) - _G(x, y - h * ny, k)) / (2 * h)
    dGx = (_G(x + h * nx, y, k) - _G(x - h * nx, y, k)) / (2 * h)
    assert abs(D - dGy) < 1e-8 * abs(dGy) + 1e-9
    assert abs(Ds - dGx) < 1e-8 * abs(dGx) + 1e-9
    Dp = kernel_values(x + h * nx, nx, y, ny, k)[1]
    Dm = kernel_values(x - h * nx, nx, y, ny, k)[1]
    assert abs(N - (Dp - Dm) / (2 * h)) < 1e-7 * abs(N) + 1e-8


def test_real_and_complex_branches_agree():
    x = np.array([[0.1, 0.2]]); y = np.array([[1.0, -0.3]]); n = np.array([[1.0, 0.0]])
    a = kernel_values(x, n, y, n, 7.5)
    b = kernel_values(x, n, y, n, 7.5 + 1e-300j)
    for u, v in zip(a, b):
        assert np.allclose(u, v, rtol=1e-14)
