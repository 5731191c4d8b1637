"""Fundamental solution of the 2-D Helmholtz equation and its normal
derivatives (paper Sec. 2.1, eqs. slp, dlp, d_slp, d_dlp).

The paper writes G = H_0^(1)(k|x-y|); the jump terms +-1/2 of its Burton-Miller
system only hold for the standard normalisation, so the oracle uses
G(x, y) = (i/4) H_0^(1)(k |x - y|).  With d = x - y,
r = |d|, z = k r:

  G             = (i/4) H0(z)
  dG/dn(y)      = (i k/4) H1(z) (n_y . d) / r                       (D kernel)
  dG/dn(x)      = -(i k/4) H1(z) (n_x . d) / r                      (D* kernel)
  d2G/dn(x)dn(y)= (i k/4) [ k H0(z) (n_x.d)(n_y.d)/r^2
                            + H1(z)/r (n_x.n_y - 2 (n_x.d)(n_y.d)/r^2) ]  (N kernel)

Bessel/Hankel values come from scipy.special (library routines).
Parity pinned by tests/test_oracle_kernels.py: the derivative kernels against
centred finite differences of G, and G against scipy.special.hankel1.
"""
import numpy as np
import scipy.special as sp


def bessel_parts(z):
    """H0, H1 (first kind) and J0, J1 at z (real > 0 or complex)."""
    z = np.asarray(z)
    if np.iscomplexobj(z) and np.any(np.imag(z) != 0):
        J0, J1 = sp.jv(0, z), sp.jv(1, z)
        return sp.hankel1(0, z), sp.hankel1(1, z), J0, J1
    zr = np.real(z).astype(np.float64)
    J0, J1, Y0, Y1 = sp.j0(zr), sp.j1(zr), sp.y0(zr), sp.y1(zr)
    return J0 + 1j * Y0, J1 + 1j * Y1, J0 + 0j, J1 + 0j


def kernel_values(xt, nt, xs, ns, k):
    """S, D, D*, N kernel values (no quadrature weight) for broadcastable point sets.

    xt, nt: (..., 2) target points / unit normals; xs, ns: (..., 2) sources.
    """
    d = xt - xs
    r = np.hypot(d[..., 0], d[..., 1])
    H0, H1, _, _ = bessel_parts(k * r)
    ndx = np.sum(nt * d, -1)
    ndy = np.sum(ns * d, -1)
    nxny = np.sum(nt * ns, -1)
    S = 0.25j * H0
    D = 0.25j * k * H1 * ndy / r
    Ds = -0.25j * k * H1 * ndx / r
    N = 0.25j * k * (k * H0 * ndx * ndy / r ** 2 + H1 / r * (nxny - 2 * ndx * ndy / r ** 2))
    return S, D, Ds, N
