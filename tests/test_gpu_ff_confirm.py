"""GPU parity of the refinement ended by the folded float-float product (the
default) and by the FP64 product (PM_FLAG_FP64_CONFIRM)."""
import numpy as np
import pytest

from oracle import dense
from paper_2603_09381_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_09381_gb300 import pmchwt
    return pmchwt


@pytest.mark.parametrize("ff_confirm", [True, False])
def test_confirming_residual_matches_the_oracle(pm, ff_confirm):
    prob = wl.star_grid(4, 4, n=64, seed=1)
    angs = [0.3, 1.9, 4.4]
    g = pm.Geometry(prob)
    F = g.plane_wave(angs)
    f = pm.Factor(g, 1e-10, precision=pm.PM_MIXED, ff_confirm=ff_confirm)
    phi = f.solve(F)
    info = f.last_info
    assert 1 <= info["iterations"] <= 6 and info["residual"] <= 1e-10
    A = dense.assemble(prob)
    ref = np.linalg.solve(A, F)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-8
    # the residual the library stopped on is the true one, recomputed with the oracle's matrix
    res = max(np.linalg.norm(F[:, r] - A @ phi[:, r]) / np.linalg.norm(F[:, r]) for r in range(len(angs)))
    assert res <= 2e-10
    assert abs(res - info["residual"]) <= 5e-12


@pytest.mark.parametrize("top_fp64", [False, True])
def test_top_level_precision_matches_the_oracle(pm, top_fp64):
    """The mixed preconditioner's top-level system factored in complex64 with
    one FP64-residual correction per solve (default) or in complex128
    (PM_FLAG_TOP_FP64): the refined solution agrees with the dense oracle
    either way, and the complex64 top takes no more refinement steps than
    the complex128 one plus one."""
    prob = wl.star_grid(4, 4, n=64, seed=1)
    angs = [0.3, 1.9, 4.4]
    g = pm.Geometry(prob)
    F = g.plane_wave(angs)
    f = pm.Factor(g, 1e-10, precision=pm.PM_MIXED, top_fp64=top_fp64)
    phi = f.solve(F)
    info = f.last_info
    assert info["residual"] <= 1e-10
    A = dense.assemble(prob)
    ref = np.linalg.solve(A, F)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-8
    if not top_fp64:
        f64 = pm.Factor(g, 1e-10, precision=pm.PM_MIXED, top_fp64=True)
        f64.solve(F)
        assert info["iterations"] <= f64.last_info["iterations"] + 1


def test_operator_assembled_beside_or_after_the_factorization(pm):
    """The dense FP64 operator assembled beside the complex64 factorization
    (persistent kernel on a low-priority stream, the default) or after it
    (PM_FLAG_OPERATOR_AFTER, the tiled kernel): the same refined solution,
    in agreement with the dense oracle."""
    prob = wl.star_grid(4, 4, n=64, seed=1)
    angs = [0.3, 1.9, 4.4]
    g = pm.Geometry(prob)
    F = g.plane_wave(angs)
    A = dense.assemble(prob)
    ref = np.linalg.solve(A, F)
    out = {}
    for after in (False, True):
        f = pm.Factor(g, 1e-10, precision=pm.PM_MIXED, operator_after=after)
        out[after] = f.solve(F)
        assert f.last_info["residual"] <= 1e-10
        assert np.linalg.norm(out[after] - ref) / np.linalg.norm(ref) < 1e-8
    assert np.linalg.norm(out[False] - out[True]) / np.linalg.norm(out[True]) < 1e-9
