"""Scattered field off the boundaries and its far-field pattern (paper Sec. 1:
the fields the boundary solution represents; Sec. 4.3's frequency study uses
the same solutions).

With the boundary values u and q = (1/eps+) du/dn on every Gamma_j (the
solution phi = [q_j; u_j]), the exterior (radiating) scattered field is
Green's representation over all boundaries, the incident wave contributing
nothing outside the inclusions:
    u^s(x) = sum_j int_{Gamma_j} [ dG(x,y)/dn(y) u(y) - G(x,y) eps+ q(y) ] ds(y),
G = (i/4) H0(k+ |x - y|), evaluated with the trapezoid rule (accurate for x a
few node spacings away from every boundary).  Its far-field pattern, defined
by u^s(x) = e^{i k r} / sqrt(r) (u_inf(xhat) + O(1/r)), r = |x|:
    u_inf(xhat) = gamma sum_l w_l e^{-i k xhat.y_l} [ -i k (xhat.n_l) u_l - eps+ q_l ],
    gamma = (i/4) sqrt(2/(pi k)) e^{-i pi/4}
(from H0(z) ~ sqrt(2/(pi z)) e^{i(z - pi/4)} and |x - y| ~ r - xhat.y).

Pinned by tests/test_oracle_field.py: the single disk's Mie far field and
near field, and the optical theorem for lossless inclusions (any number):
    int_0^{2 pi} |u_inf|^2 dtheta = -sqrt(8 pi / k) Re(e^{i pi/4} u_inf(d)),
d the incidence direction.
"""
import math

import numpy as np

from .dense import EPS_OUT, split
from .geometry import all_nodes
from .kernels import bessel_parts


def _boundary(prob, phi):
    nds = all_nodes(prob)
    y = np.concatenate([nd["x"] for nd in nds])
    n = np.concatenate([nd["nrm"] for nd in nds])
    w = np.concatenate([nd["w"] for nd in nds])
    parts = split(prob, phi)
    q = np.concatenate([p[0] for p in parts])
    u = np.concatenate([p[1] for p in parts])
    return y, n, w, q, u


def far_field(prob, phi, angles):
    """u_inf at directions (cos a, sin a) for one solution vector phi (2N)."""
    k = float(prob["k_out"])
    y, n, w, q, u = _boundary(prob, np.asarray(phi))
    xh = np.stack([np.cos(angles), np.sin(angles)], -1)
    gamma = 0.25j * math.sqrt(2 / (math.pi * k)) * np.exp(-0.25j * math.pi)
    pw = np.exp(-1j * k * (xh @ y.T)) * w[None, :]
    return gamma * ((pw * (-1j * k * (xh @ n.T))) @ u - EPS_OUT * pw @ q)


def scattered_field(prob, phi, points):
    """u^s at points (P x 2) outside every inclusion for one solution vector phi."""
    k = float(prob["k_out"])
    y, n, w, q, u = _boundary(prob, np.asarray(phi))
    pts = np.asarray(points, dtype=np.float64)
    d = pts[:, None, :] - y[None, :, :]
    r = np.hypot(d[..., 0], d[..., 1])
    H0, H1, _, _ = bessel_parts(k * r)
    G = 0.25j * H0
    # dG/dn(y) = (i k / 4) H1(k r) (n_y . (x - y)) / r
    dGdn = 0.25j * k * H1 * np.sum(n[None, :, :] * d, -1) / r
    return (dGdn * w[None, :]) @ u - EPS_OUT * (G * w[None, :]) @ q
