"""Boundary curves and Nystrom nodes (paper Sec. 2.2: n quadrature points per
boundary Gamma_j, equispaced in the parameter t).

Each curve is x(t) = c + Rot(rot) rho(t), t in [0, 2 pi), counter-clockwise,
so the unit normal n = (x2', -x1') / |x'| points out of the inclusion, into
Omega^+ (Sec. 2.1).  Node l sits at t_l = 2 pi l / n with trapezoid weight
w_l = (2 pi / n) |x'(t_l)|.

Parity pinned by tests/test_oracle_geometry.py (perimeter and enclosed area
against closed forms; normals against finite differences).
"""
import math

import numpy as np

SHAPE_CIRCLE, SHAPE_ELLIPSE, SHAPE_STAR, SHAPE_FOURIER = 0, 1, 2, 3


def _polar_radius(shape, prm, t):
    """r(t), r'(t), r''(t) for the polar shapes."""
    if shape == SHAPE_CIRCLE:
        a = prm[0]
        return a + 0 * t, 0 * t, 0 * t
    if shape == SHAPE_STAR:
        r0, e, p = prm[0], prm[1], prm[2]
        return (r0 * (1 + e * np.cos(p * t)), -r0 * e * p * np.sin(p * t),
                -r0 * e * p * p * np.cos(p * t))
    if shape == SHAPE_FOURIER:
        r0 = prm[0]
        r, dr, ddr = np.ones_like(t), np.zeros_like(t), np.zeros_like(t)
        for i, m in enumerate(range(2, 7)):
            a, ph = prm[1 + i], prm[6 + i]
            r = r + a * np.cos(m * t + ph)
            dr = dr - a * m * np.sin(m * t + ph)
            ddr = ddr - a * m * m * np.cos(m * t + ph)
        return r0 * r, r0 * dr, r0 * ddr
    raise ValueError(f"not a polar shape: {shape}")


def curve(inc, t):
    """Return x, x', x'' at parameters t, each of shape (len(t), 2)."""
    t = np.asarray(t, dtype=np.float64)
    shape, prm = inc["shape"], inc["prm"]
    c, s = np.cos(t), np.sin(t)
    if shape == SHAPE_ELLIPSE:
        a, b = prm[0], prm[1]
        loc = np.stack([a * c, b * s], -1)
        dloc = np.stack([-a * s, b * c], -1)
        ddloc = np.stack([-a * c, -b * s], -1)
    else:
        r, dr, ddr = _polar_radius(shape, prm, t)
        loc = np.stack([r * c, r * s], -1)
        dloc = np.stack([dr * c - r * s, dr * s + r * c], -1)
        ddloc = np.stack([ddr * c - 2 * dr * s - r * c, ddr * s + 2 * dr * c - r * s], -1)
    cr, sr = math.cos(inc["rot"]), math.sin(inc["rot"])
    rot = np.array([[cr, -sr], [sr, cr]])
    x = loc @ rot.T + np.array([inc["cx"], inc["cy"]])
    return x, dloc @ rot.T, ddloc @ rot.T


def nodes(inc):
    """Nystrom nodes of one inclusion: dict of t, x, dx, ddx, speed, nrm, w, curv_term.

    curv_term = (n . x'') / |x'|, the quantity in the diagonal limit of the
    double-layer kernels.
    """
    n = inc["n"]
    t = 2 * math.pi * np.arange(n) / n
    x, dx, ddx = curve(inc, t)
    speed = np.hypot(dx[:, 0], dx[:, 1])
    nrm = np.stack([dx[:, 1], -dx[:, 0]], -1) / speed[:, None]
    w = (2 * math.pi / n) * speed
    curv_term = np.sum(nrm * ddx, -1) / speed
    return {"t": t, "x": x, "dx": dx, "ddx": ddx, "speed": speed, "nrm": nrm, "w": w,
            "curv_term": curv_term, "n": n}


def all_nodes(prob):
    return [nodes(inc) for inc in prob["inclusions"]]


def eps_in(prob, j):
    """Interior material constant eps^- = (k^- / k^+)^2 with eps^+ = 1 (Sec. 2.1, k = omega sqrt(eps))."""
    return (prob["inclusions"][j]["k_in"] / prob["k_out"]) ** 2
