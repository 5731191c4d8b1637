"""Independent problems factored and solved concurrently (one stream per worker)."""
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


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("mixed", [False, True])
def test_batch_matches_dense_and_single(pm, mixed):
    probs = wl.ellipse_batch(count=6, seed=3, m_lo=2, m_hi=12, n_lo=64, n_hi=128)
    geoms = [pm.Geometry(p) for p in probs]
    prec = pm.PM_MIXED if mixed else pm.PM_FP64
    facs = pm.factor_batch(geoms, 1e-10, precision=prec, workers=4)
    angs = [0.3, 1.7]
    rhs = [g.plane_wave(angs) for g in geoms]
    sols = pm.solve_batch(facs, rhs, workers=4)
    for p, g, f, r, x in zip(probs, geoms, facs, rhs, sols):
        ref = dense.solve(p, angs)
        assert _rel(x, ref) < (1e-8 if mixed else 1e-9)
        if not mixed:   # the same factorization as a single-problem call, bit for bit
            one = pm.Factor(g, 1e-10)
            assert np.array_equal(one.solve(r), x)
