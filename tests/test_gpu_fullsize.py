"""Full-size parity (16 x 16 stars, N = 65,536, the bench's workload and launch
configuration): the oracle evaluates sampled rows of the FP64 Nystrom matrix one
by one and checks the GPU solution's residual on them; the complex128 path is
also compared box by box and solution by solution with the proxy oracle's
factorization of the same problem (tests/golden/star16_fp64_oracle.npz,
written by tests/golden/make_star16_oracle.py from oracle/ alone)."""
import os

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


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "star16_fp64_oracle.npz")


def test_fullsize_fp64_matches_the_proxy_oracle(setup):
    """The complex128 path against the proxy oracle at full size (paper Sec. 3,
    eq. compressed and the recovery formula): skeletons box by box, the
    compressed size K and the solution on the oracle's 4,096 stored sample
    unknowns for all eight right-hand sides.  Boxes whose own ID decisions all
    lie more than 100 rounding units from their thresholds (and whose children
    agree) must choose the oracle's skeletons; with every box agreeing the
    solutions agree to 1e-10, and in any case to the solver's tolerance."""
    pm, prob, opts, angs, g = setup
    z = np.load(GOLDEN)
    f = pm.Factor(g, opts["tol"], opts["proxy_factor"], opts["proxy_points"])
    phi = f.solve(g.plane_wave(list(z["angles"])))
    ref = z["phi"]
    err = np.linalg.norm(phi[z["idx"]] - ref) / np.linalg.norm(ref)
    lev, box, off = z["skel_level"], z["skel_box"], z["skel_off"]
    L = int(lev.max())
    agree = {}
    robust_mismatch = []
    for i in np.argsort(-lev, kind="stable"):    # leaves first, so children are known before parents
        l, b = int(lev[i]), int(box[i])
        r, c = f.skeleton(l, b)
        ok = set(r) == set(z["skel_rows"][off[i]:off[i + 1]]) and set(c) == set(z["skel_cols"][off[i]:off[i + 1]])
        agree[l, b] = ok
        # the 16 x 16 grid fills its quadtree: box b's children are boxes 4b..4b+3 of the level below
        kids_ok = l == L or all(agree.get((l + 1, cb), False) for cb in range(4 * b, 4 * b + 4)
                                if (l + 1, cb) in agree)
        if not ok and kids_ok and z["margin"][i] > 100:
            robust_mismatch.append((l, b, float(z["margin"][i])))
    same = sum(agree.values())
    print(f"16x16 FP64: skeletons {same}/{len(agree)} boxes agree, K={f.stats()['K']} (oracle {int(z['K'])}), "
          f"rel diff on sampled unknowns {err:.3e}, min margin {float(z['margin'].min()):.3g}")
    assert not robust_mismatch, robust_mismatch
    if same == len(agree):
        assert f.stats()["K"] == int(z["K"])
        assert err < 1e-10
    assert err < 1e-8
