"""Pins for the disk series of oracle/mie.py: Graf's addition theorem, the
Jacobi-Anger expansion of the plane wave, and flux conservation of the
single-disk coefficients."""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import mie


def test_graf_addition_theorem():
    k = 2 * math.pi
    ci, cj = np.array([1.0, 0.3]), np.array([-0.2, 0.1])
    M = 40
    W = mie.translation_matrix(ci, cj, k, M)
    ms = np.arange(-M, M + 1)
    x = ci + 0.35 * np.array([math.cos(2.0), math.sin(2.0)])
    dj, di = x - cj, x - ci
    for m in [0, 1, -3, 7]:
        lhs = sp.hankel1(m, k * np.hypot(*dj)) * np.exp(1j * m * math.atan2(dj[1], dj[0]))
        rhs = np.sum(W[:, m + M] * sp.jv(ms, k * np.hypot(*di)) * np.exp(1j * ms * math.atan2(di[1], di[0])))
        assert abs(lhs - rhs) < 1e-12


def test_incident_coefficients_reproduce_the_plane_wave():
    """Jacobi-Anger about a centre c: e^{i k d.x} = sum_m e_m J_m(k r) e^{i m theta}."""
    k, ang, c = 7.0, 0.9, np.array([1.3, -0.4])
    M = 60
    e = mie.incident_coeffs(c, k, ang, M)
    ms = np.arange(-M, M + 1)
    for r, th in [(0.3, 0.2), (0.8, 2.9), (1.5, -1.7)]:
        x = c + r * np.array([math.cos(th), math.sin(th)])
        exact = np.exp(1j * k * (math.cos(ang) * x[0] + math.sin(ang) * x[1]))
        assert abs(np.sum(e * sp.jv(ms, k * r) * np.exp(1j * ms * th)) - exact) < 1e-13


@pytest.mark.parametrize("k1", [4 * math.pi, 3.3, 4 * math.pi * (1 + 0.05j)])
def test_single_disk_coefficients_conserve_flux(k1):
    """Outside the disk each mode is e_m [ (1 + 2 T_m)/2 H^(1)_m + H^(2)_m / 2 ]:
    a lossless disk sends out what comes in, |1 + 2 T_m| = 1; an absorbing one
    no more, |1 + 2 T_m| <= 1 (high orders barely reach the interior, so
    there it tends to 1).  Modes of order -m and m scatter alike."""
    a, k0 = 0.4, 2 * math.pi
    M = 30
    T = mie.t_matrix(a, k0, k1, (k1 / k0) ** 2, M)
    S = np.abs(1 + 2 * T)
    if np.imag(k1) == 0:
        assert np.max(np.abs(S - 1)) < 1e-12
    else:
        assert np.all(S <= 1 + 1e-12) and np.min(S) < 0.99
    assert np.allclose(T, T[::-1], rtol=1e-12, atol=1e-300)
