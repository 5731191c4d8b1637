"""Quadrature tables for the self blocks.

* Kress's product rule for log-singular periodic kernels (R. Kress, "Boundary
  integral equations in time-harmonic acoustic scattering", Math. Comput.
  Modelling 15 (1991); Colton & Kress, Inverse Acoustic and Electromagnetic
  Scattering Theory, Sec. 3.6): on n = 2M equispaced nodes,
      int_0^{2pi} ln(4 sin^2((t - tau)/2)) f(tau) dtau  ~  sum_j R_j(t) f(t_j),
      R_j(t) = -(2 pi / M) sum_{m=1}^{M-1} cos(m (t - t_j)) / m
               - (pi / M^2) cos(M (t - t_j)).
  The paper uses a zeta-corrected rule instead (Sec. 2.2); the log-split rule
  serves both the oracle and the CUDA path.
* The trigonometric (Fourier) differentiation matrix on n equispaced nodes
  (n even): D_ij = 1/2 (-1)^(i-j) cot((t_i - t_j)/2), D_ii = 0 (Trefethen,
  Spectral Methods in MATLAB, ch. 3); used by Maue's form of N.

Parity pinned by tests/test_oracle_quadrature.py: exact integration of
e^{i m tau} against the log kernel (closed form -2 pi/|m|, 0 for m = 0) and
exact differentiation of trigonometric polynomials.
"""
import math

import numpy as np


def kress_weights(n):
    """R[d] = R_j(t_i) for d = (i - j) mod n."""
    if n % 2:
        raise ValueError("n must be even")
    M = n // 2
    s = 2 * math.pi * np.arange(n) / n
    R = np.zeros(n)
    for m in range(1, M):
        R += np.cos(m * s) / m
    R *= -2 * math.pi / M
    R -= (math.pi / M ** 2) * np.cos(M * s)
    return R


def kress_matrix(n):
    R = kress_weights(n)
    i = np.arange(n)
    return R[(i[:, None] - i[None, :]) % n]


def diff_matrix(n):
    if n % 2:
        raise ValueError("n must be even")
    t = 2 * math.pi * np.arange(n) / n
    i = np.arange(n)
    d = i[:, None] - i[None, :]
    D = np.zeros((n, n))
    off = d != 0
    D[off] = 0.5 * ((-1.0) ** d[off]) / np.tan((t[:, None] - t[None, :])[off] / 2)
    return D
