"""Nystrom blocks of the PMCHWT systems (paper Sec. 2.2).

Unknowns per inclusion: phi_i = [q_i; u_i]; equation rows per inclusion:
[u-equation rows (first n); q-equation rows (next n)]; right-hand side
f_i = [-u^I_i; -q^I_i].

Off-diagonal blocks (i != j) use the trapezoid rule, entry = kernel * w_j:
  Omit : [[-eps+ S+,  D+], [-D*+,  N+/eps+]]                 (eq. pmchwt_omit_bie)
  All  : [[-(eps+ S+ + eps- S-), D+ + D-],
          [-(D*+ + D*-), N+/eps+ + N-/eps-]]                 (eq. pmchwt_all_bie)
Self blocks (i = j), both formulations:
  [[-(eps+ S+ + eps- S-), D+ + D-], [-(D*+ + D*-), N+/eps+ + N-/eps-]]
with S, D, D* by Kress's log-split rule and N by Maue's identity
  N phi = (1/|x'(t)|) d/dt S0[dphi/dtau] + k^2 n_x . S[n_y phi],
discretised as  N = diag(1/|x'|) Dt S0 Dt + k^2 (S o n n^T)
(S0: the single layer without the speed factor |x'(tau)|, Dt: trigonometric
differentiation).  These quadratures replace the paper's zeta-corrected
rule, identically on both sides of every parity check.

Log split (Colton & Kress Sec. 3.6), t != tau, d = x(t) - x(tau), r = |d|:
  S-kernel * |x'(tau)| = M1 ln(4 sin^2((t-tau)/2)) + M2,
      M1 = -(1/4pi) J0(kr) |x'(tau)|,
      M2(t,t) = [i/4 - C/(2pi) - (1/2pi) ln(k |x'(t)|/2)] |x'(t)|  (C = Euler's constant)
  D-kernel * |x'(tau)| = L1 ln(...) + L2,
      L1 = -(k/4pi) J1(kr) (n_y.d)/r |x'(tau)|,  L2(t,t) = (1/4pi) (n.x'')/|x'|
  D*-kernel * |x'(tau)| = L1* ln(...) + L2*,
      L1* = (k/4pi) J1(kr) (n_x.d)/r |x'(tau)|,  L2*(t,t) = (1/4pi) (n.x'')/|x'|
  matrix entry = R(t_i - t_j) * (log coefficient) + (2 pi/n) * (smooth part).

Burton-Miller (eq. bm_bie), unknowns per inclusion [u_i; q_i], rows
[exterior equation; interior equation], alpha = i / k+, I the identity:
  self:  [[D+ - I/2 + alpha N+,  -eps+ S+ - alpha eps+ (D*+ + I/2)],
          [D- + I/2,             -eps- S-]]
  i != j: [[D+ + alpha N+,  -eps+ (S+ + alpha D*+)],
           [D-,              -eps- S-]]   (interior kernel of the source inclusion)
  right-hand side [-(u^I + alpha q^I); 0].
The simplified Burton-Miller system drops the interior terms of the
off-diagonal blocks (their lower blocks are zero), the case Sec. 3 shows to
make R A^{-1} L singular.

Parity pinned by tests/test_oracle_blocks.py (circle eigenvalues, Calderon
identities on stars / ellipses, Green's formula between two curves) and, for
the Burton-Miller blocks, by the disk series of tests/test_oracle_dense.py.
"""
import math

import numpy as np

from . import quadrature as quad
from .kernels import bessel_parts, kernel_values

EULER_C = 0.57721566490153286061


def self_operators(nd, k):
    """Kress/Maue matrices S, D, D*, N (n x n) on one curve for wavenumber k."""
    n = nd["n"]
    x, nrm, speed = nd["x"], nd["nrm"], nd["speed"]
    t = nd["t"]
    d = x[:, None, :] - x[None, :, :]
    r = np.hypot(d[..., 0], d[..., 1])
    off = ~np.eye(n, dtype=bool)
    rs = np.where(off, r, 1.0)
    H0, H1, J0, J1 = bessel_parts(k * rs)
    sp_j = speed[None, :]
    ndy = np.sum(nrm[None, :, :] * d, -1)
    ndx = np.sum(nrm[:, None, :] * d, -1)
    logsin = np.log(4 * np.sin((t[:, None] - t[None, :]) / 2) ** 2 + np.where(off, 0.0, 1.0))
    Rm = quad.kress_matrix(n)
    h = 2 * math.pi / n

    # single layer
    M = 0.25j * H0 * sp_j
    M1 = -(1 / (4 * math.pi)) * J0 * sp_j
    M2 = M - M1 * logsin
    diag_M2 = (0.25j - EULER_C / (2 * math.pi) - np.log(k * speed / 2) / (2 * math.pi)) * speed
    M1 = np.where(off, M1, -(1 / (4 * math.pi)) * speed[None, :])
    M2 = np.where(off, M2, np.diag(diag_M2))
    S = Rm * M1 + h * M2

    # double layer and its adjoint
    diag_L = nd["curv_term"] / (4 * math.pi)
    L = 0.25j * k * H1 * ndy / rs * sp_j
    L1 = -(k / (4 * math.pi)) * J1 * ndy / rs * sp_j
    L2 = np.where(off, L - L1 * logsin, np.diag(diag_L))
    L1 = np.where(off, L1, 0.0)
    D = Rm * L1 + h * L2
    Ls = -0.25j * k * H1 * ndx / rs * sp_j
    Ls1 = (k / (4 * math.pi)) * J1 * ndx / rs * sp_j
    Ls2 = np.where(off, Ls - Ls1 * logsin, np.diag(diag_L))
    Ls1 = np.where(off, Ls1, 0.0)
    Ds = Rm * Ls1 + h * Ls2

    # hypersingular operator via Maue
    Dt = quad.diff_matrix(n)
    S0 = S / sp_j
    nn = nrm @ nrm.T
    N = (Dt @ S0 @ Dt) / speed[:, None] + k * k * S * nn
    return S, D, Ds, N


def self_block(nd, k_out, k_in, eps_out, eps_in):
    """A_ii (2n x 2n) of PMCHWT: [[-(e+S+ + e-S-), D+ + D-], [-(D*+ + D*-), N+/e+ + N-/e-]]."""
    Sp, Dp, Dsp, Np = self_operators(nd, k_out)
    Sm, Dm, Dsm, Nm = self_operators(nd, k_in)
    return np.block([[-(eps_out * Sp + eps_in * Sm), Dp + Dm],
                     [-(Dsp + Dsm), Np / eps_out + Nm / eps_in]])


def offdiag_operators(nt, ns, k):
    """Trapezoid-rule S, D, D*, N (n_t x n_s) from curve ns to curve nt (disjoint)."""
    S, D, Ds, N = kernel_values(nt["x"][:, None, :], nt["nrm"][:, None, :],
                                ns["x"][None, :, :], ns["nrm"][None, :, :], k)
    w = ns["w"][None, :]
    return S * w, D * w, Ds * w, N * w


def omit_block(nt, ns, k_out, eps_out=1.0):
    """A_ij (i != j) of PMCHWT (Omit): exterior potentials only."""
    S, D, Ds, N = offdiag_operators(nt, ns, k_out)
    return np.block([[-eps_out * S, D], [-Ds, N / eps_out]])


def all_block(nt, ns, k_out, k_in_src, eps_out, eps_in_src):
    """A_ij (i != j) of PMCHWT (All): exterior plus the source inclusion's interior potentials."""
    Sp, Dp, Dsp, Np = offdiag_operators(nt, ns, k_out)
    Sm, Dm, Dsm, Nm = offdiag_operators(nt, ns, k_in_src)
    return np.block([[-(eps_out * Sp + eps_in_src * Sm), Dp + Dm],
                     [-(Dsp + Dsm), Np / eps_out + Nm / eps_in_src]])


def bm_self_block(nd, k_out, k_in, eps_out, eps_in):
    """A_ii (2n x 2n) of the Burton-Miller system, unknowns [u; q]."""
    Sp, Dp, Dsp, Np = self_operators(nd, k_out)
    Sm, Dm, Dsm, Nm = self_operators(nd, k_in)
    n = nd["n"]
    eye = np.eye(n)
    a = 1j / k_out
    return np.block([[Dp - eye / 2 + a * Np, -eps_out * Sp - a * eps_out * (Dsp + eye / 2)],
                     [Dm + eye / 2, -eps_in * Sm]])


def bm_block(nt, ns, k_out, k_in_src, eps_out, eps_in_src, simplified=False):
    """A_ij (i != j) of the Burton-Miller system (unknowns [u; q]); with
    simplified=True the interior (lower) blocks are dropped."""
    Sp, Dp, Dsp, Np = offdiag_operators(nt, ns, k_out)
    a = 1j / k_out
    upper = [Dp + a * Np, -eps_out * (Sp + a * Dsp)]
    if simplified:
        z = np.zeros_like(Sp)
        return np.block([upper, [z, z]])
    Sm, Dm, Dsm, Nm = offdiag_operators(nt, ns, k_in_src)
    return np.block([upper, [Dm, -eps_in_src * Sm]])
