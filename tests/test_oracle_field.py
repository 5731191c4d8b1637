"""Pins for the scattered field and its far-field pattern (oracle/field.py)."""
import math

import numpy as np
import pytest

from oracle import dense, field, mie
from paper_2603_09381_gb300 import workloads as wl


def _single_disk_series(prob, angle):
    """a_m of the scattered field sum_m a_m H_m(k r) e^{i m theta} of one disk at the origin."""
    inc = prob["inclusions"][0]
    k0, k1, a = prob["k_out"], inc["k_in"], inc["prm"][0]
    M = int(math.ceil(max(abs(k0), abs(k1)) * a)) + 30
    T = mie.t_matrix(a, k0, k1, (k1 / k0) ** 2, M)
    return T * mie.incident_coeffs((0.0, 0.0), k0, angle, M), M


def test_far_field_of_a_disk_matches_the_mie_series():
    prob = wl.circle_grid(1, 1, n=64)
    angle = 0.7
    phi = dense.solve(prob, [angle])[:, 0]
    am, M = _single_disk_series(prob, angle)
    k = prob["k_out"]
    th = np.linspace(0, 2 * np.pi, 37)
    m = np.arange(-M, M + 1)
    exact = math.sqrt(2 / (math.pi * k)) * np.exp(-0.25j * math.pi) * (
        np.exp(1j * np.outer(th, m)) @ (am * (-1j) ** m))
    got = field.far_field(prob, phi, th)
    assert np.max(np.abs(got - exact)) < 1e-11 * np.max(np.abs(exact))


def test_near_field_of_a_disk_matches_the_mie_series():
    prob = wl.circle_grid(1, 1, n=64)
    angle = 2.0
    phi = dense.solve(prob, [angle])[:, 0]
    am, M = _single_disk_series(prob, angle)
    k = prob["k_out"]
    rng = np.random.default_rng(3)
    r = rng.uniform(0.7, 3.0, 20)
    t = rng.uniform(0, 2 * np.pi, 20)
    pts = np.stack([r * np.cos(t), r * np.sin(t)], -1)
    m = np.arange(-M, M + 1)
    from scipy.special import hankel1
    exact = np.array([np.sum(am * hankel1(m, k * ri) * np.exp(1j * m * ti)) for ri, ti in zip(r, t)])
    got = field.scattered_field(prob, phi, pts)
    assert np.max(np.abs(got - exact)) < 1e-10 * np.max(np.abs(exact))


@pytest.mark.parametrize("grid", ["disks", "stars"])
def test_optical_theorem_for_lossless_inclusions(grid):
    """Energy balance of a lossless configuration: the power scattered into all
    directions equals the extinction given by the forward far field."""
    prob = wl.circle_grid(2, 2, n=96) if grid == "disks" else wl.star_grid(2, 2, n=128, seed=5, spacing=1.6)
    angle = 0.4
    phi = dense.solve(prob, [angle])[:, 0]
    k = prob["k_out"]
    th = 2 * np.pi * np.arange(512) / 512
    uf = field.far_field(prob, phi, th)
    scattered = np.sum(np.abs(uf) ** 2) * 2 * np.pi / 512
    forward = field.far_field(prob, phi, np.array([angle]))[0]
    extinction = -math.sqrt(8 * math.pi / k) * (np.exp(0.25j * math.pi) * forward).real
    assert abs(scattered - extinction) < 1e-8 * scattered
    # an absorbing interior breaks the balance: extinction exceeds scattering
    lossy = wl.circle_grid(2, 2, n=96, k_in=4 * math.pi * (1 + 0.05j))
    phil = dense.solve(lossy, [angle])[:, 0]
    ufl = field.far_field(lossy, phil, th)
    sc = np.sum(np.abs(ufl) ** 2) * 2 * np.pi / 512
    ext = -math.sqrt(8 * math.pi / k) * (np.exp(0.25j * math.pi) * field.far_field(lossy, phil, np.array([angle]))[0]).real
    assert ext > sc * (1 + 1e-3)
