"""Oracle pins against values the paper prints (fixtures in tests/golden/)."""
import math
import os

from oracle import dense, geometry
from paper_2603_09381_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [tuple(int(v) for v in line.split()) for line in f
                if line.strip() and not line.startswith("#")]


def test_degrees_of_freedom_of_the_star_grids():
    """Sec. 4's star grids with n = 200: the oracle's system size equals the
    printed degrees of freedom (u and q at every quadrature point)."""
    rows = _rows("dof_star_grid_n200.txt")
    assert [m for m, _ in rows] == [16, 64, 256, 1024, 4096]
    for m, dof in rows:
        side = math.isqrt(m)
        prob = wl.star_grid(side, side, n=200, seed=1)
        assert len(prob["inclusions"]) == m
        assert dense.offsets(prob)[-1] == dof
        if m <= 64:   # the node sets themselves, not only the declared counts
            assert 2 * sum(len(nd["w"]) for nd in geometry.all_nodes(prob)) == dof
