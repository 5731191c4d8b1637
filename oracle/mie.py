"""Exact solutions for circular inclusions (independent pins; not in the paper).

Single disk (Mie series): with the incident wave expanded about the disk
centre c, u^I = e^{i k0 d.c} sum_m i^m e^{-i m a} J_m(k0 r) e^{i m theta},
the scattered field sum_m a_m H_m(k0 r) e^{i m theta} and the interior field
sum_m b_m J_m(k1 r) e^{i m theta} satisfy, per m, the transmission conditions
of eqs. (pressure) and (flux):
    e_m J_m(k0 a) + a_m H_m(k0 a) = b_m J_m(k1 a)
    (k0/eps+) [e_m J'_m(k0 a) + a_m H'_m(k0 a)] = (k1/eps-) b_m J'_m(k1 a).
Several disks (Foldy-Lax multipole method): a_m^i = T_m^i e_m^i with
    T_m = [(k1/eps-) J_m(k0a) J'_m(k1a) - (k0/eps+) J'_m(k0a) J_m(k1a)]
        / [(k0/eps+) H'_m(k0a) J_m(k1a) - (k1/eps-) H_m(k0a) J'_m(k1a)],
and e^i = (incident coefficients about c_i) + (Graf translation of the other
disks' outgoing fields):  H_m(k r_j) e^{i m th_j}
    = sum_n H_{m-n}(k R) e^{i (m-n) Th} J_n(k r_i) e^{i n th_i},
(R, Th) the polar coordinates of c_i - c_j, valid for r_i < R (Graf's
addition theorem, DLMF 10.23.7).  The translation formula is itself checked
numerically in tests/test_oracle_mie.py.

Boundary values: u = sum (e_m J_m(k0a) + a_m H_m(k0a)) e^{i m th},
q = (k0/eps+) sum (e_m J'_m(k0a) + a_m H'_m(k0a)) e^{i m th}.
High orders are kept in range by solving for a_m H_m(k0 a) instead of a_m.
"""
import math

import numpy as np
import scipy.special as sp

EPS_OUT = 1.0


def _H(m, z):
    return sp.hankel1(m, z)


def _Hp(m, z):
    return sp.h1vp(m, z)


def _J(m, z):
    return sp.jv(m, z)


def _Jp(m, z):
    return sp.jvp(m, z)


def t_matrix(a, k0, k1, eps_in, M):
    m = np.arange(-M, M + 1)
    num = (k1 / eps_in) * _J(m, k0 * a) * _Jp(m, k1 * a) - (k0 / EPS_OUT) * _Jp(m, k0 * a) * _J(m, k1 * a)
    den = (k0 / EPS_OUT) * _Hp(m, k0 * a) * _J(m, k1 * a) - (k1 / eps_in) * _H(m, k0 * a) * _Jp(m, k1 * a)
    return num / den


def incident_coeffs(center, k0, angle, M):
    m = np.arange(-M, M + 1)
    phase = np.exp(1j * k0 * (math.cos(angle) * center[0] + math.sin(angle) * center[1]))
    return phase * (1j ** m) * np.exp(-1j * m * angle)


def translation_matrix(ci, cj, k0, M):
    """W[n, m]: coefficient of J_n(k r_i) e^{i n th_i} in H_m(k r_j) e^{i m th_j}."""
    dx, dy = ci[0] - cj[0], ci[1] - cj[1]
    R, Th = math.hypot(dx, dy), math.atan2(dy, dx)
    m = np.arange(-M, M + 1)
    diff = m[None, :] - m[:, None]
    return _H(diff, k0 * R) * np.exp(1j * diff * Th)


def disks_solution(centers, a, k0, k1, eps_in, angle, M=None):
    """Boundary mode coefficients of every disk (equal radius a).

    Unknowns are scaled to stay in floating-point range at high orders:
    alpha_m = a_m H_m(k0 a) (the outgoing field's boundary amplitude).  The
    translated excitation is applied in the form
    J_n(k0 a) e_n = J_n(k0 a) [inc_n + sum_j sum_m W_nm alpha^j_m / H_m(k0 a)].
    Returns (U, Q, M): per disk the coefficients of e^{i m theta} of u and q.
    """
    if M is None:
        M = int(math.ceil(max(abs(k0), abs(k1)) * a)) + 30
    nd = len(centers)
    m = np.arange(-M, M + 1)
    size = 2 * M + 1
    T = t_matrix(a, k0, k1, eps_in, M)
    Hm, Hpm = _H(m, k0 * a), _Hp(m, k0 * a)
    Jm, Jpm = _J(m, k0 * a), _Jp(m, k0 * a)
    TH = T * Hm
    Asys = np.eye(nd * size, dtype=np.complex128)
    rhs = np.zeros(nd * size, dtype=np.complex128)
    Wsc = {}
    for i in range(nd):
        rhs[i * size:(i + 1) * size] = TH * incident_coeffs(centers[i], k0, angle, M)
        for j in range(nd):
            if i != j:
                Wsc[i, j] = translation_matrix(centers[i], centers[j], k0, M) / Hm[None, :]
                Asys[i * size:(i + 1) * size, j * size:(j + 1) * size] = -TH[:, None] * Wsc[i, j]
    alpha = np.linalg.solve(Asys, rhs).reshape(nd, size)
    U = np.zeros_like(alpha)
    Q = np.zeros_like(alpha)
    for i in range(nd):
        inc = incident_coeffs(centers[i], k0, angle, M)
        eJ, eJp = Jm * inc, Jpm * inc
        for j in range(nd):
            if i != j:
                eJ = eJ + Jm * (Wsc[i, j] @ alpha[j])
                eJp = eJp + Jpm * (Wsc[i, j] @ alpha[j])
        U[i] = eJ + alpha[i]
        Q[i] = (k0 / EPS_OUT) * (eJp + alpha[i] * Hpm / Hm)
    return U, Q, M


def boundary_values(U, Q, theta, M):
    """(u, q) on a disk boundary at polar angles theta from mode coefficients."""
    m = np.arange(-M, M + 1)
    E = np.exp(1j * np.outer(theta, m))
    return E @ U, E @ Q
