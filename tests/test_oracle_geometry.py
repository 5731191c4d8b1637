"""Pins for boundary curves and Nystrom nodes."""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import geometry as g
from paper_2603_09381_gb300 import workloads as wl


def _inc(shape, prm, n=128, rot=0.3, cx=1.5, cy=-0.5):
    return wl._inclusion(shape, cx, cy, rot, prm, n, 4.0)


def test_circle_perimeter_and_normals():
    nd = g.nodes(_inc(wl.SHAPE_CIRCLE, [0.4]))
    assert abs(nd["w"].sum() - 2 * math.pi * 0.4) < 1e-13
    radial = (nd["x"] - np.array([1.5, -0.5])) / 0.4
    assert np.allclose(nd["nrm"], radial, atol=1e-14)
    assert np.allclose(nd["curv_term"], -1.0, atol=1e-13)  # n . x'' / |x'| = -1 on a circle


def test_ellipse_perimeter_closed_form():
    a, b = 0.45, 0.2
    nd = g.nodes(_inc(wl.SHAPE_ELLIPSE, [a, b], n=256))
    exact = 4 * a * sp.ellipe(1 - (b / a) ** 2)
    assert abs(nd["w"].sum() - exact) < 1e-12


def test_star_area_closed_form():
    r0, e, p = 0.4, 0.2, 5
    nd = g.nodes(_inc(wl.SHAPE_STAR, [r0, e, p]))
    x = nd["x"] - np.array([1.5, -0.5])
    area = 0.5 * np.sum((x[:, 0] * nd["dx"][:, 1] - x[:, 1] * nd["dx"][:, 0])) * 2 * math.pi / nd["n"]
    assert abs(area - math.pi * r0 ** 2 * (1 + e ** 2 / 2)) < 1e-13
    # outward normal: area > 0 with counter-clockwise orientation; normals unit and orthogonal to x'
    assert np.allclose(np.hypot(*nd["nrm"].T), 1.0)
    assert np.allclose(np.sum(nd["nrm"] * nd["dx"], -1), 0.0, atol=1e-14)


@pytest.mark.parametrize("shape,prm", [(wl.SHAPE_STAR, [0.4, 0.2, 5]),
                                       (wl.SHAPE_FOURIER, [0.4, 0.01, 0.03, 0.02, 0.04, 0.0, 1, 2, 3, 4, 5]),
                                       (wl.SHAPE_ELLIPSE, [0.3, 0.2])])
def test_derivatives_against_finite_differences(shape, prm):
    inc = _inc(shape, prm)
    t = np.linspace(0, 2 * math.pi, 17)
    h = 1e-5
    x0, d0, dd0 = g.curve(inc, t)
    xp, dp, _ = g.curve(inc, t + h)
    xm, dm, _ = g.curve(inc, t - h)
    assert np.allclose((xp - xm) / (2 * h), d0, atol=1e-8)
    assert np.allclose((dp - dm) / (2 * h), dd0, atol=1e-8)
