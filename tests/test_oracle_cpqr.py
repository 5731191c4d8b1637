"""Pins for column-pivoted QR and the interpolative decomposition."""
import numpy as np
import pytest

from oracle import cpqr as cp


def _greedy_brute_force(Z, steps):
    """Pick, at every step, the column with the largest residual after projecting
    out the already chosen columns (least squares), lowest index on exact ties."""
    chosen, res_norms = [], []
    for _ in range(steps):
        if chosen:
            B = Z[:, chosen]
            coef, *_ = np.linalg.lstsq(B, Z, rcond=None)
            resid = Z - B @ coef
        else:
            resid = Z
        nrm = np.linalg.norm(resid, axis=0)
        nrm[chosen] = -1
        j = int(np.argmax(nrm))
        chosen.append(j)
        res_norms.append(nrm[j])
    return chosen, np.array(res_norms)


@pytest.mark.parametrize("shape", [(9, 6), (6, 9), (30, 12)])
def test_pivots_and_rdiag_match_greedy_projection(shape):
    rng = np.random.default_rng(11)
    Z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    Z *= np.logspace(0, -3, shape[1])[None, :]
    steps = min(shape)
    perm, R, rdiag, _ = cp.cpqr(Z, 0.0)
    chosen, res = _greedy_brute_force(Z, steps)
    assert list(perm[:steps]) == chosen
    assert np.allclose(rdiag, res, rtol=1e-10)
    # R reproduces the pivoted matrix up to a unitary factor: R^H R = (Z P)^H (Z P)
    ZP = Z[:, perm]
    assert np.allclose(R.conj().T @ R, ZP.conj().T @ ZP, atol=1e-12)


def test_tie_rule_prefers_lowest_index():
    Z = np.zeros((4, 3), dtype=complex)
    Z[0, 2] = 1.0
    Z[1, 1] = 1.0
    Z[2, 0] = 1.0 + 1e-14  # within the 1e-12 tie band of the others
    perm, _, _, _ = cp.cpqr(Z, 0.0)
    assert list(perm) == [0, 1, 2]


@pytest.mark.parametrize("tol", [1e-6, 1e-10, 1e-12])
def test_interpolative_decomposition_of_low_rank_matrix(tol):
    rng = np.random.default_rng(3)
    W, n, r = 200, 60, 25
    U = rng.standard_normal((W, r)) + 1j * rng.standard_normal((W, r))
    V = rng.standard_normal((r, n)) + 1j * rng.standard_normal((r, n))
    s = np.logspace(0, -16, r)
    Z = (U * s) @ V
    perm, rank, T = cp.column_id(Z, tol)
    err = np.linalg.norm(Z[:, perm[rank:]] - Z[:, perm[:rank]] @ T)
    assert err <= 50 * tol * np.linalg.norm(Z)
    sv = np.linalg.svd(Z, compute_uv=False)
    # the rank is near the numerical rank at tol
    assert abs(rank - np.sum(sv > tol * sv[0])) <= 3


def test_rank_zero_matrix_and_stateful_extension():
    f = cp.CPQR(np.zeros((5, 4), dtype=complex), 1e-10)
    assert f.find_rank() == 0
    rng = np.random.default_rng(0)
    Z = rng.standard_normal((40, 10)) @ rng.standard_normal((10, 20)) + 0j
    f = cp.CPQR(Z, 1e-8)
    k = f.find_rank()
    assert k == 10
    f.extend(14)
    perm, R, _, _ = cp.cpqr(Z, 1e-8, max_steps=14)
    assert list(f.perm[:14]) == list(perm[:14])
    assert np.allclose(np.abs(np.diag(f.R[:, :14])), np.abs(np.diag(R[:, :14])), atol=1e-12)


def test_decision_margins_flag_near_ties_only():
    """The margins (bookkeeping for parity tests) are large for well separated
    column norms and shrink to rounding size when a candidate sits at the tie
    band's edge or a diagonal entry sits at the rank threshold."""
    rng = np.random.default_rng(5)
    Z = rng.standard_normal((40, 12)) + 1j * rng.standard_normal((40, 12))
    Z *= np.logspace(0, -6, 12)[None, :]
    f = cp.CPQR(Z, 1e-9)
    f.find_rank()
    assert f.margin_pivot > 1e6 and f.margin_rank > 1e6
    # two orthogonal columns whose norms differ by exactly the tie band
    Y = np.zeros((4, 2), dtype=complex)
    Y[0, 0] = 1.0
    Y[1, 1] = np.sqrt(1.0 - cp.TIE)
    g = cp.CPQR(Y, 0.0)
    g.find_rank()
    assert g.margin_pivot < 10
    # a column whose trailing norm equals tol |R_11|
    X = np.diag([1.0, 1e-3, 1e-8]).astype(complex)
    h = cp.CPQR(X, 1e-3)
    assert h.find_rank() == 1 and h.margin_rank < 10
