"""The QR-first update's C -= V Y on the tensor cores (the default) against
the same update on the CUDA cores: both are FP32-accurate, so the complex64
factorizations agree in size to within rounding-level rank decisions, both
refined solutions match the dense oracle, and the tensor-core kernel is the
one that ran."""
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


@pytest.mark.parametrize("n,grid", [(64, 4), (128, 4)])
def test_tensor_core_update_matches_cuda_cores(pm, n, grid):
    prob = wl.star_grid(grid, grid, n=n, seed=3)
    g = pm.Geometry(prob)
    angs = [0.4, 2.2]
    F = g.plane_wave(angs)
    ref = dense.solve(prob, angs)
    f_tc = pm.Factor(g, 1e-10, precision=pm.PM_MIXED, profile=True)
    f_cc = pm.Factor(g, 1e-10, precision=pm.PM_MIXED, profile=True, qr_tensor_cores=False)
    prof_tc, prof_cc = f_tc.profile(), f_cc.profile()
    assert "qr_update_tc32" in prof_tc and "qr_update32" not in prof_tc
    assert "qr_update32" in prof_cc and "qr_update_tc32" not in prof_cc
    k_tc, k_cc = f_tc.stats()["K"], f_cc.stats()["K"]
    print(f"n={n}: K tensor cores {k_tc}, CUDA cores {k_cc}")
    assert abs(k_tc - k_cc) <= max(2, 0.01 * k_cc)
    for f in (f_tc, f_cc):
        assert _rel(f.solve(F), ref) < 1e-8
