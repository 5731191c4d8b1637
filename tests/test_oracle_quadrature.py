"""Pins for the Kress weights and the trigonometric differentiation matrix."""
import math

import numpy as np
import pytest

from oracle import quadrature as q


@pytest.mark.parametrize("n", [16, 64, 128])
def test_kress_weights_integrate_log_kernel(n):
    # Fourier coefficients of ln(4 sin^2(s/2)) = -2 sum_{m>=1} cos(m s)/m:
    # int_0^{2pi} ln(4 sin^2((t - tau)/2)) e^{i m tau} dtau = -2 pi/|m| e^{i m t}, 0 for m = 0.
    R = q.kress_matrix(n)
    t = 2 * math.pi * np.arange(n) / n
    for m in range(-(n // 2) + 1, n // 2):
        f = np.exp(1j * m * t)
        expect = 0.0 if m == 0 else -2 * math.pi / abs(m)
        assert np.allclose(R @ f, expect * f, atol=1e-12, rtol=0)


def test_kress_weights_against_brute_force_integral():
    # Integrate ln(4 sin^2(tau/2)) * cos(tau)^2 (a trig polynomial of degree 2) with
    # an adaptive library quadrature and compare with the product rule at t = 0.
    from scipy.integrate import quad as squad
    n = 32
    t = 2 * math.pi * np.arange(n) / n
    f = np.cos(t) ** 2
    val, _ = squad(lambda s: math.log(4 * math.sin(s / 2) ** 2) * math.cos(s) ** 2, 0, 2 * math.pi,
                   points=[0.0, 2 * math.pi], limit=200)
    assert abs(q.kress_matrix(n)[0] @ f - val) < 1e-10


@pytest.mark.parametrize("n", [16, 64])
def test_diff_matrix_exact_on_trig_polynomials(n):
    t = 2 * math.pi * np.arange(n) / n
    f = np.sin(3 * t) + 0.5 * np.cos(5 * t) + 0.25 * np.sin((n // 2 - 1) * t)
    df = 3 * np.cos(3 * t) - 2.5 * np.sin(5 * t) + 0.25 * (n // 2 - 1) * np.cos((n // 2 - 1) * t)
    assert np.allclose(q.diff_matrix(n) @ f, df, atol=1e-11)


def test_odd_n_rejected():
    with pytest.raises(ValueError):
        q.kress_weights(15)
