"""The library's cache of freed device blocks: a factorization that reuses the
blocks of a freed one gives the same bits, the cache gives its memory back on
request, and a request larger than what is cached still succeeds."""
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


def test_reused_blocks_give_identical_results(pm):
    import torch
    prob = wl.star_grid(4, 4, n=64, seed=3)
    g = pm.Geometry(prob)
    F = g.plane_wave([0.3, 1.1])
    pm.release_cached_memory()
    f1 = pm.Factor(g, 1e-10)
    x1 = f1.solve(F)
    del f1
    free_cached, _ = torch.cuda.mem_get_info()
    f2 = pm.Factor(g, 1e-10)        # draws on the blocks f1 gave back
    x2 = f2.solve(F)
    assert np.array_equal(x1, x2)   # FP64 factorizations are bitwise reproducible
    assert _rel(x2, dense.solve(prob, [0.3, 1.1])) < 1e-9
    del f2
    released = pm.release_cached_memory()
    assert released > 0
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after >= free_cached + released // 2
    assert pm.release_cached_memory() == 0


def test_mixed_factorizations_reuse_the_dense_operator(pm):
    prob = wl.star_grid(4, 4, n=64, seed=3)
    g = pm.Geometry(prob)
    F = g.plane_wave([0.7])
    ref = dense.solve(prob, [0.7])
    for _ in range(3):   # the operator block of one factor serves the next
        f = pm.Factor(g, 1e-10, precision=pm.PM_MIXED)
        assert _rel(f.solve(F), ref) < 1e-8
        del f
    # a larger problem than anything cached still gets its memory
    big = wl.star_grid(8, 8, n=64, seed=3)
    gb = pm.Geometry(big)
    fb = pm.Factor(gb, 1e-10, precision=pm.PM_MIXED)
    xb = fb.solve(gb.plane_wave([0.7]))
    assert np.all(np.isfinite(xb))
    del fb
    pm.release_cached_memory()
