"""Full-size parity (16 x 16 stars, N = 65,536, the bench's workload and launch
configuration): the oracle evaluates sampled rows of the FP64 Nystrom matrix one
by one and checks the GPU solution's residual on them."""
import numpy as np
import pytest

from oracle import blocks, geometry, proxy
from paper_2603_09381_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_09381_gb300 import pmchwt as pm
    prob, opts, angs = wl.config_star16()
    g = pm.Geometry(prob)
    return pm, prob, opts, angs, g


def _sampled_rows(prob, rows):
    """Rows of A (oracle): self-block part from the Kress/Maue block of the row's
    inclusion, off-diagonal part from the exterior kernels to every other node."""
    nds = geometry.all_nodes(prob)
    ix = proxy._Index(prob, nds)
    N = ix.off[-1]
    out = np.zeros((len(rows), N), dtype=np.complex128)
    cols = np.arange(N)
    for a, r in enumerate(rows):
        j = int(np.searchsorted(ix.off, r, side="right") - 1)
        other = (cols < ix.off[j]) | (cols >= ix.off[j + 1])
        out[a, other] = proxy.entries(ix, prob["k_out"], np.array([r]), cols[other])[0]
        S = blocks.self_block(nds[j], prob["k_out"], prob["inclusions"][j]["k_in"], 1.0, geometry.eps_in(prob, j))
        out[a, ix.off[j]:ix.off[j + 1]] = S[r - ix.off[j]]
    return out


@pytest.mark.parametrize("mixed", [True, False])
def test_fullsize_sampled_residual(setup, mixed):
    pm, prob, opts, angs, g = setup
    prec = pm.PM_MIXED if mixed else pm.PM_FP64
    f = pm.Factor(g, opts["tol"], opts["proxy_factor"], opts["proxy_points"], precision=prec)
    F = g.plane_wave(angs[:2])
    phi = f.solve(F)
    rng = np.random.default_rng(7)
    rows = np.sort(rng.choice(g.N, 24, replace=False))
    A = _sampled_rows(prob, rows)
    res = A @ phi - F[rows]
    rel = np.linalg.norm(res, axis=0) / np.linalg.norm(F[rows], axis=0)
    # mixed: refined to a relative residual of 1e-10 on the whole vector; FP64: the
    # compressed solver at tol 1e-10
    assert np.max(rel) < (2e-9 if mixed else 1e-8), rel
    if mixed:
        assert f.last_info["residual"] <= 1e-10
