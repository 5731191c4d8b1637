"""Solve graphs: the second application of a factor's compressed inverse (or
of the mixed preconditioner) for a right-hand-side count is captured into a
CUDA graph, later ones replay it, and the results equal eager launches: bit
for bit in FP64; in the mixed mode to 1e-11, since the refinement's dense
products add column-split partial sums with FP64 atomics (mixed solves
reproduce to ~1e-13 from run to run)."""
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


def test_fp64_solves_replay_a_captured_graph(pm):
    prob = wl.star_grid(4, 4, n=64, seed=2)
    g = pm.Geometry(prob)
    F = g.plane_wave([0.2, 2.9, 4.1])
    eager = pm.Factor(g, 1e-10, graphs=False)
    ref = eager.solve(F)
    f = pm.Factor(g, 1e-10)
    outs = [f.solve(F) for _ in range(4)]
    st = f.stats()
    assert st["graph_captures"] == 1 and st["graph_launches"] == 3
    for x in outs:
        assert np.array_equal(x, ref)
    # another right-hand-side count gets its own plan
    x1 = f.solve(F[:, :1])
    assert np.array_equal(x1[:, 0], ref[:, 0]) or np.allclose(x1[:, 0], ref[:, 0], rtol=0, atol=1e-13)
    assert eager.stats()["graph_captures"] == 0
    assert np.linalg.norm(ref - dense.solve(prob, [0.2, 2.9, 4.1])) < 1e-8 * np.linalg.norm(ref)


def test_mixed_refinement_replays_the_preconditioner_graph(pm):
    prob = wl.star_grid(4, 4, n=64, seed=3)
    g = pm.Geometry(prob)
    F = g.plane_wave([0.7, 3.3])
    eager = pm.Factor(g, 1e-10, precision=pm.PM_MIXED, graphs=False)
    ref = eager.solve(F)
    f = pm.Factor(g, 1e-10, precision=pm.PM_MIXED)
    x = f.solve(F)
    it = f.last_info["iterations"]
    st = f.stats()
    assert it >= 3 and it == eager.last_info["iterations"]
    assert st["graph_captures"] == 1 and st["graph_launches"] == it - 1
    assert np.linalg.norm(x - ref) < 1e-11 * np.linalg.norm(ref)
    x2 = f.solve(F)    # a second solve replays from its first application
    it2 = f.last_info["iterations"]
    assert np.linalg.norm(x2 - ref) < 1e-11 * np.linalg.norm(ref)
    assert f.stats()["graph_launches"] == it - 1 + it2
    assert np.linalg.norm(ref - dense.solve(prob, [0.7, 3.3])) < 1e-8 * np.linalg.norm(ref)
