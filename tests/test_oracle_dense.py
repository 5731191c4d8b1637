"""Pins for the conventional (dense) BIEM: exact disk solutions and energy balance."""
import math

import numpy as np
import pytest

from oracle import dense, geometry, mie
from paper_2603_09381_gb300 import workloads as wl

ANG = math.radians(30.0)


def _mie_error(prob, angle=ANG, formulation="omit"):
    phi = dense.solve(prob, [angle], formulation)[:, 0]
    k0 = prob["k_out"]
    inc0 = prob["inclusions"][0]
    k1, a = inc0["k_in"], inc0["prm"][0]
    cents = [(i["cx"], i["cy"]) for i in prob["inclusions"]]
    U, Q, M = mie.disks_solution(cents, a, k0, k1, (k1 / k0) ** 2, angle)
    err, ref = [], []
    for j, (q, u) in enumerate(dense.split(prob, phi)):
        theta = geometry.nodes(prob["inclusions"][j])["t"]
        ue, qe = mie.boundary_values(U[j], Q[j], theta, M)
        err.append(np.concatenate([q - qe, u - ue]))
        ref.append(np.concatenate([qe, ue]))
    return np.linalg.norm(np.concatenate(err)) / np.linalg.norm(np.concatenate(ref))


def test_single_disk_mie():
    assert _mie_error(wl.circle_grid(1, 1, n=64)) < 1e-12


def test_single_lossy_disk_mie():
    assert _mie_error(wl.circle_grid(1, 1, n=64, k_in=4 * math.pi * (1 + 0.05j))) < 1e-12


def test_two_disks_multipole():
    # the plain trapezoid rule of the off-diagonal blocks (gap 0.2) limits n = 64 to ~2e-10
    assert _mie_error(wl.circle_grid(2, 1, n=64)) < 3e-10
    assert _mie_error(wl.circle_grid(2, 1, n=80)) < 1e-10


def test_two_by_two_grid_multipole():
    assert _mie_error(wl.circle_grid(2, 2, n=64)) < 6e-10
    assert _mie_error(wl.circle_grid(2, 2, n=96), angle=1.1) < 1e-10


@pytest.mark.parametrize("lossy", [False, True])
def test_energy_balance(lossy):
    k_in = 15.707963267948966 * ((1 + 0.05j) if lossy else 1)
    # spacing 1.6: the off-diagonal trapezoid rule is then accurate, so the discrete
    # solution satisfies the exact identity to near machine precision
    prob = wl.star_grid(2, 2, n=128, seed=5, spacing=1.6)
    for inc in prob["inclusions"]:
        inc["k_in"] = k_in
    phi = dense.solve(prob, [0.4])[:, 0]
    eps = (k_in / prob["k_out"]) ** 2
    for j, (q, u) in enumerate(dense.split(prob, phi)):
        w = geometry.nodes(prob["inclusions"][j])["w"]
        flux = np.sum(w * np.conj(u) * q) * eps
        scale = np.sum(w * np.abs(u) * np.abs(q)) * abs(eps)
        if lossy:
            assert flux.imag < -1e-3 * scale
        else:
            assert abs(flux.imag) < 1e-9 * scale


def test_omit_and_all_agree_to_discretisation_error():
    prob = wl.circle_grid(2, 2, n=96)
    a = dense.solve(prob, [ANG], "omit")[:, 0]
    b = dense.solve(prob, [ANG], "all")[:, 0]
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-9
    # and the interior off-diagonal potentials applied to the solution nearly vanish
    A_all = dense.assemble(prob, "all")
    A_omit = dense.assemble(prob, "omit")
    assert np.linalg.norm((A_all - A_omit) @ a) < 1e-9 * np.linalg.norm(A_omit @ a)


def test_uneven_node_counts_multipole():
    """Each inclusion has its own n (its own offsets, weights and self block)."""
    prob = wl.circle_grid(2, 2, n=96)
    for inc, n in zip(prob["inclusions"], (80, 96, 112, 128)):
        inc["n"] = n
    assert dense.offsets(prob)[-1] == 2 * (80 + 96 + 112 + 128)
    assert _mie_error(prob, angle=1.1) < 1e-10


@pytest.mark.parametrize("n,bound", [(64, 6e-10), (96, 1e-10)])
def test_burton_miller_matches_the_multipole_solution(n, bound):
    """The Burton-Miller system (eq. bm_bie: alpha = i/k+, the +-1/2 jump terms
    of G = (i/4) H0, unknowns [u; q], right-hand side [-(u^I + alpha q^I); 0])
    solves the same 2 x 2 disk problem: a wrong sign of a jump term or of
    alpha would miss the Foldy-Lax solution by O(1)."""
    assert _mie_error(wl.circle_grid(2, 2, n=n), formulation="bm") < bound
    assert _mie_error(wl.circle_grid(1, 1, n=64), formulation="bm") < 1e-12


def test_burton_miller_rhs_map_and_unknown_order():
    prob = wl.circle_grid(2, 1, n=16)
    f = np.arange(64) + 1j * np.arange(64)[::-1]
    b = dense.bm_rhs(prob, f)
    a = 1j / prob["k_out"]
    assert np.allclose(b[:16], f[:16] + a * f[16:32]) and not b[16:32].any()
    assert np.allclose(b[32:48], f[32:48] + a * f[48:64]) and not b[48:].any()
    x = np.arange(64.0)
    y = dense.bm_to_pmchwt_order(prob, x)
    assert np.array_equal(y[:16], x[16:32]) and np.array_equal(y[16:32], x[:16])
