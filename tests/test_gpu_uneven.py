"""GPU parity with a different node count, shape and interior wavenumber per
inclusion within one problem (FP64 and mixed paths) against the dense oracle."""
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


def _uneven_problem():
    prob = wl.star_grid(3, 3, n=64, seed=6)
    for j, inc in enumerate(prob["inclusions"]):
        inc["n"] = 48 + 16 * (j % 4)
        inc["k_in"] = prob["k_out"] * (1.5 + 0.25 * (j % 3))
    prob["inclusions"][4] = wl._inclusion(wl.SHAPE_ELLIPSE, 1.0, 1.0, 0.4, [0.42, 0.25], 96, 12.0)
    prob["inclusions"][8]["k_in"] *= 1 + 0.05j   # one lossy interior
    return prob


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_uneven_inclusions_fp64_and_mixed(pm):
    prob = _uneven_problem()
    angs = [0.2, 2.5]
    g = pm.Geometry(prob)
    assert g.N == dense.offsets(prob)[-1]
    F = g.plane_wave(angs)
    ref = dense.solve(prob, angs)
    f = pm.Factor(g, 1e-12)
    assert _rel(f.solve(F), ref) < 1e-9
    fm = pm.Factor(g, 1e-10, precision=pm.PM_MIXED)
    phi = fm.solve(F)
    assert fm.last_info["residual"] <= 1e-10
    assert _rel(phi, ref) < 1e-8
