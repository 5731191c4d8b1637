"""Pins for the proxy/ID fast direct solver: agreement with the dense solve."""
import math

import numpy as np
import pytest

from oracle import dense, proxy
from paper_2603_09381_gb300 import workloads as wl


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_small_circle_grid_matches_dense():
    prob, opts, angs = wl.config_fp64_small()
    fac = proxy.factor(prob, opts)
    F = np.stack([dense.plane_wave(prob, a) for a in angs], 1)
    assert _rel(proxy.solve(fac, F), dense.solve(prob, angs)) < 1e-11
    # 64 nodes per circle at 1e-12 keep every index: this case checks the
    # algebra of eq. compressed and the recovery formula, not compression
    assert fac["L"] == 1 and fac["stats"]["K"] == 512


def test_single_level_compression_matches_dense():
    """2 x 2 stars with 128 nodes at 1e-10: one compressed level that drops
    almost a third of the unknowns and still solves to the threshold."""
    prob = wl.star_grid(2, 2, n=128, seed=1)
    fac = proxy.factor(prob, {"tol": 1e-10, "proxy_factor": 1.5})
    assert fac["L"] == 1 and fac["stats"]["K"] < 0.75 * fac["N"]
    angs = [0.3, 1.9]
    F = np.stack([dense.plane_wave(prob, a) for a in angs], 1)
    assert _rel(proxy.solve(fac, F), dense.solve(prob, angs)) < 30 * 1e-10


def test_single_inclusion_degenerates_to_dense():
    prob = wl.star_grid(1, 1, n=64)
    fac = proxy.factor(prob, {"tol": 1e-10})
    assert fac["L"] == 0
    f = dense.plane_wave(prob, 0.7)
    assert _rel(proxy.solve(fac, f), dense.solve(prob, [0.7])[:, 0]) < 1e-13


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_star_grid_matches_dense_within_tolerance(tol):
    prob = wl.star_grid(4, 4, n=64, seed=1)
    fac = proxy.factor(prob, {"tol": tol, "proxy_factor": 1.5})
    phi = proxy.solve(fac, dense.plane_wave(prob, 0.3))
    ref = dense.solve(prob, [0.3])[:, 0]
    assert _rel(phi, ref) < 30 * tol
    assert fac["stats"]["K"] < fac["N"]


def test_ranks_shrink_with_looser_tolerance():
    prob = wl.star_grid(4, 4, n=64, seed=1)
    k_tight = proxy.factor(prob, {"tol": 1e-10})["stats"]["K"]
    k_loose = proxy.factor(prob, {"tol": 1e-4})["stats"]["K"]
    assert k_loose < k_tight


def test_ragged_grid_and_multi_rhs():
    prob = wl.circle_grid(3, 2, n=48)
    fac = proxy.factor(prob, {"tol": 1e-10})
    angs = [0.1, 2.0, 4.0]
    F = np.stack([dense.plane_wave(prob, a) for a in angs], 1)
    assert _rel(proxy.solve(fac, F), dense.solve(prob, angs)) < 1e-8


def test_uneven_node_counts_match_dense():
    prob = wl.star_grid(3, 3, n=64, seed=6)
    for j, inc in enumerate(prob["inclusions"]):
        inc["n"] = 48 + 16 * (j % 4)
    fac = proxy.factor(prob, {"tol": 1e-10})
    F = np.stack([dense.plane_wave(prob, a) for a in (0.2, 2.5)], 1)
    assert _rel(proxy.solve(fac, F), dense.solve(prob, [0.2, 2.5])) < 3e-9


def test_full_rank_degenerates_to_the_dense_solve():
    """With a threshold below rounding every ID keeps all of its indices: the
    compressed system is the whole matrix and the solve is exact up to rounding."""
    prob = wl.circle_grid(2, 2, n=32)
    fac = proxy.factor(prob, {"tol": 1e-16, "proxy_points": 64})
    assert fac["stats"]["K"] == fac["N"] == 256
    x = proxy.solve(fac, dense.plane_wave(prob, 0.3))
    assert _rel(x, dense.solve(prob, [0.3])[:, 0]) < 1e-13


def test_loose_threshold_keeps_a_nonsingular_factorization():
    prob = wl.circle_grid(2, 2, n=32)
    fac = proxy.factor(prob, {"tol": 0.5, "proxy_points": 64})
    assert 8 <= fac["stats"]["K"] < 64
    x = proxy.solve(fac, dense.plane_wave(prob, 0.3))
    assert np.all(np.isfinite(x)) and _rel(x, dense.solve(prob, [0.3])[:, 0]) < 1.0


@pytest.mark.parametrize("form", ["all", "bm"])
def test_other_formulations_match_their_dense_solve(form):
    """PMCHWT (All) and Burton-Miller through the proxy solver: the proxies
    carry the interior kernel too (All: a second density family; BM: its own
    entries on the proxy circle), so the compressed solve reproduces the
    formulation's dense solve: exactly with every index kept, within the
    threshold when it compresses."""
    prob, opts, angs = wl.config_fp64_small()
    F = np.stack([dense.plane_wave(prob, a) for a in angs], 1)
    fac = proxy.factor(prob, dict(opts, formulation=form))
    assert _rel(proxy.solve(fac, F), dense.solve(prob, angs, form)) < 1e-12
    stars = wl.star_grid(2, 2, n=128, seed=1, k_out=5.0, k_ratio=5 ** 0.5)
    fac = proxy.factor(stars, {"tol": 1e-10, "formulation": form})
    assert fac["stats"]["K"] < fac["N"]
    F = np.stack([dense.plane_wave(stars, a) for a in angs], 1)
    assert _rel(proxy.solve(fac, F), dense.solve(stars, angs, form)) < 30 * 1e-10


def test_simplified_burton_miller_compressed_block_is_singular():
    """Sec. 3: without the off-diagonal interior terms the interior rows see no
    far field, their interpolation vanishes and R A^{-1} L is singular."""
    with pytest.raises(proxy.SingularError):
        proxy.factor(wl.circle_grid(2, 2), {"tol": 1e-10, "formulation": "bm_simplified"})


def test_arbitrary_arrangement_matches_dense():
    """Inclusions placed at random, not on a grid (Sec. 4.4): the automatic
    quadtree with containment-based near lists solves to the threshold."""
    prob = wl.random_arrangement(20, seed=6)
    fac = proxy.factor(prob, {"tol": 1e-10})
    assert fac["L"] >= 2 and fac["stats"]["K"] < fac["N"]
    F = np.stack([dense.plane_wave(prob, a) for a in (0.3, 2.2)], 1)
    assert _rel(proxy.solve(fac, F), dense.solve(prob, [0.3, 2.2])) < 30 * 1e-10
