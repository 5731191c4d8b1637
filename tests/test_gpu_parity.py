"""GPU parity: the CUDA path through the C ABI against the CPU oracle."""
import math

import numpy as np
import pytest

from oracle import blocks, dense, geometry, mie, proxy
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


def _mixed_problem():
    prob = wl.star_grid(2, 2, n=64, seed=7)
    prob["inclusions"][1] = wl._inclusion(wl.SHAPE_ELLIPSE, 1.0, 0.0, 0.4, [0.42, 0.25], 96, 12.0)
    prob["inclusions"][2] = wl._inclusion(wl.SHAPE_FOURIER, 0.0, 1.0, 0.0,
                                          [0.4, .04, .01, .03, .02, .04, 1, 2, 3, 4, 5], 80, 20.0)
    prob["inclusions"][3] = wl._inclusion(wl.SHAPE_CIRCLE, 1.0, 1.0, 0.3, [0.35], 32, 9.0)
    prob["inclusions"][0]["k_in"] = 15.7 * (1 + 0.05j)   # a lossy interior
    return prob


def test_nodes_match_oracle(pm):
    prob = _mixed_problem()
    g = pm.Geometry(prob)
    xy, nrm, w = g.nodes()
    nds = geometry.all_nodes(prob)
    assert np.allclose(xy, np.concatenate([d["x"] for d in nds]), atol=1e-14, rtol=0)
    assert np.allclose(nrm, np.concatenate([d["nrm"] for d in nds]), atol=1e-14, rtol=0)
    assert np.allclose(w, np.concatenate([d["w"] for d in nds]), atol=1e-15, rtol=1e-14)


def test_self_blocks_match_oracle(pm):
    prob = _mixed_problem()
    g = pm.Geometry(prob)
    nds = geometry.all_nodes(prob)
    for j, inc in enumerate(prob["inclusions"]):
        A = g.self_block(j, inc["n"])
        ref = blocks.self_block(nds[j], prob["k_out"], inc["k_in"], 1.0, geometry.eps_in(prob, j))
        assert _rel(A, ref) < 1e-12, j


def test_offdiagonal_entries_match_oracle(pm):
    prob = wl.star_grid(4, 4, n=64, seed=3)
    g = pm.Geometry(prob)
    rng = np.random.default_rng(0)
    N = g.N
    rows = rng.integers(0, N, 300)
    cols = rng.integers(0, N, 257)
    got = g.matrix_entries(rows, cols)
    nds = geometry.all_nodes(prob)
    ix = proxy._Index(prob, nds)
    ref = proxy.entries(ix, prob["k_out"], rows, cols)
    same = (rows[:, None] // 128) == (cols[None, :] // 128)
    ref[same] = 0
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))


def test_plane_wave_rhs(pm):
    prob = _mixed_problem()
    g = pm.Geometry(prob)
    angs = [0.3, 2.5]
    got = g.plane_wave(angs)
    ref = np.stack([dense.plane_wave(prob, a) for a in angs], 1)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_small_circle_grid_solution(pm):
    prob, opts, angs = wl.config_fp64_small()
    g = pm.Geometry(prob)
    f = pm.Factor(g, opts["tol"], opts["proxy_factor"], opts["proxy_points"])
    phi = f.solve(g.plane_wave(angs))
    assert _rel(phi, dense.solve(prob, angs)) < 1e-10
    fo = proxy.factor(prob, opts)
    assert _rel(phi, proxy.solve(fo, dense.plane_wave(prob, angs[0]))[:, None]) < 1e-10
    # and the exact multipole solution of the 2 x 2 disks
    U, Q, M = mie.disks_solution([(i["cx"], i["cy"]) for i in prob["inclusions"]], 0.4, prob["k_out"],
                                 prob["inclusions"][0]["k_in"], 4.0, angs[0])
    th = geometry.nodes(prob["inclusions"][0])["t"]
    exact = np.concatenate([np.concatenate(mie.boundary_values(U[j], Q[j], th, M)[::-1]) for j in range(4)])
    assert _rel(phi[:, 0], exact) < 1e-9


def test_single_inclusion_is_dense(pm):
    prob = wl.star_grid(1, 1, n=128)
    g = pm.Geometry(prob)
    f = pm.Factor(g, 1e-10)
    assert f.stats()["levels"] == 0
    phi = f.solve(g.plane_wave([0.7]))
    assert _rel(phi, dense.solve(prob, [0.7])) < 1e-12


def _skeletons_agree(f, fo):
    """Boxes (all levels) whose selected row and column index sets equal the oracle's."""
    same = total = 0
    for lev in range(1, fo["L"] + 1):
        for b in range(len(fo["tree"]["levels"][lev])):
            r, c = f.skeleton(lev, b)
            d = fo["data"][lev, b]
            total += 1
            same += set(r) == set(d["srows"]) and set(c) == set(d["scols"])
    return same, total


# (grid side, nodes per star, ID threshold): one compressed level (2 x 2 stars,
# K 709 of 1024), two levels at a loose and at the 16 x 16 workload's threshold
@pytest.mark.parametrize("nx,n,tol", [(2, 128, 1e-10), (4, 64, 1e-6), (4, 64, 1e-10)])
def test_compressed_fp64_matches_proxy_oracle(pm, nx, n, tol):
    """The FP64 path and the proxy oracle choose the same skeletons box by box
    and give the same solution to 1e-10 (paper Sec. 3: eq. compressed and the
    recovery formula), on inputs that really compress (K < N).  The oracle's
    decision margins show that no pivot or rank decision lies within 100
    rounding units of its threshold, so the skeletons are unique under
    rounding and must agree exactly."""
    prob = wl.star_grid(nx, nx, n=n, seed=1)
    opts = {"tol": tol, "proxy_factor": 1.5, "proxy_points": 0}
    fo = proxy.factor(prob, opts)
    margin = min(d["margin"] for d in fo["data"].values())
    assert margin > 100, margin
    g = pm.Geometry(prob)
    f = pm.Factor(g, tol)
    angs = [0.3, 1.9, 4.4]
    phi = f.solve(g.plane_wave(angs))
    F = np.stack([dense.plane_wave(prob, a) for a in angs], 1)
    ref = proxy.solve(fo, F)
    dref = dense.solve(prob, angs)
    same, total = _skeletons_agree(f, fo)
    print(f"{nx}x{nx} n={n} tol={tol:g}: skeletons {same}/{total} boxes agree, K={f.stats()['K']} "
          f"(oracle {fo['stats']['K']}, N={g.N}), min margin {margin:.3g}")
    assert fo["stats"]["K"] < g.N
    assert same == total
    assert f.stats()["K"] == fo["stats"]["K"]
    assert _rel(phi, ref) < 1e-10
    assert _rel(phi, dref) < 30 * tol


def test_ragged_grid_device_buffers(pm):
    import torch
    prob = wl.circle_grid(3, 2, n=48)
    g = pm.Geometry(prob)
    f = pm.Factor(g, 1e-10)
    angs = [0.1, 2.0, 4.0, 5.5]
    F = torch.zeros((len(angs), g.N), dtype=torch.complex128, device="cuda")
    g.plane_wave_device(angs, F.data_ptr())
    out = torch.zeros_like(F)
    f.solve_device(F.data_ptr(), len(angs), out.data_ptr())
    torch.cuda.synchronize()
    phi = out.cpu().numpy().T
    assert _rel(phi, dense.solve(prob, angs)) < 1e-8
    # in-place (aliased) solve gives the same
    f.solve_device(F.data_ptr(), len(angs), F.data_ptr())
    torch.cuda.synchronize()
    assert _rel(F.cpu().numpy().T, phi) < 1e-14


# ---- mixed precision: FP32 factorization + FP64 refinement -------------------------

def test_mixed_small_circles(pm):
    prob, opts, angs = wl.config_fp64_small()
    g = pm.Geometry(prob)
    f = pm.Factor(g, opts["tol"], opts["proxy_factor"], opts["proxy_points"], precision=pm.PM_MIXED)
    phi = f.solve(g.plane_wave(angs))
    assert f.last_info["residual"] <= 1e-10
    assert _rel(phi, dense.solve(prob, angs)) < 1e-8


@pytest.mark.parametrize("nx,n,qr_first,tensor_cores", [(4, 64, True, False), (2, 128, True, False),
                                                        (4, 64, False, False), (4, 64, True, True)])
def test_mixed_star_grid_matches_dense(pm, nx, n, qr_first, tensor_cores):
    """Every complex64 ID variant: pivoting on the full input, on its
    triangle after an unpivoted blocked QR, that QR's updates on the tensor
    cores."""
    prob = wl.star_grid(nx, nx, n=n, seed=1)
    angs = [0.3, 1.9, 4.4]
    g = pm.Geometry(prob)
    f = pm.Factor(g, 1e-10, precision=pm.PM_MIXED, qr_first=qr_first, tensor_cores=tensor_cores)
    F = g.plane_wave(angs)
    phi = f.solve(F)
    info = f.last_info
    assert 1 <= info["iterations"] <= 6 and info["residual"] <= 1e-10
    A = dense.assemble(prob)
    ref = np.linalg.solve(A, F)
    assert _rel(phi, ref) < 1e-8
    # the refinement residual is the FP64 operator's: recompute it with the oracle's matrix
    res = max(np.linalg.norm(F[:, r] - A @ phi[:, r]) / np.linalg.norm(F[:, r]) for r in range(len(angs)))
    assert res <= 2e-10


def test_mixed_refinement_reports_non_convergence(pm):
    prob = wl.star_grid(2, 2, n=64, seed=1)
    g = pm.Geometry(prob)
    f = pm.Factor(g, 1e-10, precision=pm.PM_MIXED, max_refine=1, refine_tol=1e-15)
    with pytest.raises(pm.PmError) as e:
        f.solve(g.plane_wave([0.5]))
    assert e.value.status == 5


def test_offdiagonal_entries_large_arguments(pm):
    # 16 x 16 stars, k0 = 7.85: k r spans ~0.3 .. 170 (both Hankel branches)
    prob, _, _ = wl.config_star16()
    g = pm.Geometry(prob)
    rng = np.random.default_rng(5)
    rows = rng.integers(0, g.N, 200)
    cols = rng.integers(0, g.N, 300)
    got = g.matrix_entries(rows, cols)
    nds = geometry.all_nodes(prob)
    ix = proxy._Index(prob, nds)
    ref = proxy.entries(ix, prob["k_out"], rows, cols)
    same = (rows[:, None] // 256) == (cols[None, :] // 256)
    ref[same] = 0
    got[same] = 0
    err = np.abs(got - ref)
    assert np.max(err) < 1e-13 * np.max(np.abs(ref))
    assert np.max(err / np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))) < 1e-11


@pytest.mark.parametrize("k_out", [3.0, 6.0, 12.0, 20.0])
def test_offdiagonal_entries_across_the_hankel_intervals(pm, k_out):
    # two disks 3 apart: k r spans [2.2 k, 3.8 k], across z = 8, 12, 20, 30 and
    # 60, where the GPU's H0 / H1 change from CUDA's Bessel functions to the
    # four polynomial fits and to the asymptotic expansion
    prob = wl.circle_grid(2, 1, radius=0.4, spacing=3.0, k_out=k_out, k_in=2 * k_out, n=96)
    g = pm.Geometry(prob)
    n = 96
    rows = np.arange(0, 2 * n)                 # both equation groups of disk 0
    cols = np.arange(2 * n, 4 * n)             # both density groups of disk 1
    got = g.matrix_entries(rows, cols)
    nds = geometry.all_nodes(prob)
    ix = proxy._Index(prob, nds)
    ref = proxy.entries(ix, prob["k_out"], rows, cols)
    err = np.abs(got - ref)
    assert np.max(err) < 2e-14 * np.max(np.abs(ref))
    assert np.max(err / np.maximum(np.abs(ref), 1e-6 * np.max(np.abs(ref)))) < 1e-12


# ---- lossy interiors (complex k-), FP64 and mixed ---------------------------------

def test_lossy_small_circles_fp64_and_mixed(pm):
    prob, opts, angs = wl.config_lossy_small()
    g = pm.Geometry(prob)
    ref = dense.solve(prob, angs)
    f = pm.Factor(g, opts["tol"], opts["proxy_factor"], opts["proxy_points"])
    assert _rel(f.solve(g.plane_wave(angs)), ref) < 1e-10
    fm = pm.Factor(g, opts["tol"], opts["proxy_factor"], opts["proxy_points"], precision=pm.PM_MIXED)
    phi = fm.solve(g.plane_wave(angs))
    assert fm.last_info["residual"] <= 1e-10
    assert _rel(phi, ref) < 1e-8
    # the lossy Mie / multipole solution as an independent check
    k1 = prob["inclusions"][0]["k_in"]
    U, Q, M = mie.disks_solution([(i["cx"], i["cy"]) for i in prob["inclusions"]], 0.4, prob["k_out"], k1,
                                 (k1 / prob["k_out"]) ** 2, angs[0])
    th = geometry.nodes(prob["inclusions"][0])["t"]
    exact = np.concatenate([np.concatenate(mie.boundary_values(U[j], Q[j], th, M)[::-1]) for j in range(4)])
    assert _rel(phi[:, 0], exact) < 1e-9


def test_mixed_dense_and_on_the_fly_operators_agree(pm):
    prob = wl.star_grid(4, 4, n=64, seed=2)
    g = pm.Geometry(prob)
    F = g.plane_wave([0.9, 3.1])
    a = pm.Factor(g, 1e-10, precision=pm.PM_MIXED, dense_operator=True)
    b = pm.Factor(g, 1e-10, precision=pm.PM_MIXED, dense_operator=False)
    xa, xb = a.solve(F), b.solve(F)
    # the dense path forms residuals above 1e-5 with compensated FP32 sums (~1e-7
    # absolute), so its early corrections differ slightly; both converge to 1e-10
    assert abs(a.last_info["iterations"] - b.last_info["iterations"]) <= 1
    assert a.last_info["residual"] <= 1e-10 and b.last_info["residual"] <= 1e-10
    assert a.last_info["history"][0] == pytest.approx(b.last_info["history"][0], rel=5e-2)
    assert _rel(xa, xb) < 1e-9
    ref = dense.solve(prob, [0.9, 3.1])
    assert _rel(xa, ref) < 1e-8


def test_levels_in_chunks_reproduce_the_unchunked_factorization(pm):
    """A scratch budget too small for one box per launch makes every level run
    box by box (the way the 64 x 64 grid's upper levels fit in memory); the
    complex128 factorization is the same bit for bit."""
    prob = wl.star_grid(4, 4, n=64, seed=1)
    g = pm.Geometry(prob)
    F = g.plane_wave([0.3, 2.9])
    whole = pm.Factor(g, 1e-10)
    chunked = pm.Factor(g, 1e-10, scratch_gb=1e-6)
    sw, sc = whole.stats(), chunked.stats()
    assert sw["level_chunks"] == sw["levels"]
    assert sc["level_chunks"] == 16 + 4          # one chunk per box at both levels
    assert (sw["K"], sw["skeleton"]) == (sc["K"], sc["skeleton"])
    assert np.array_equal(whole.solve(F), chunked.solve(F))
    for lev in (1, 2):
        for b in range(4 if lev == 1 else 16):
            assert all(np.array_equal(x, y) for x, y in zip(whole.skeleton(lev, b), chunked.skeleton(lev, b)))
    # mixed mode: the chunked complex64 levels still precondition the refinement to 1e-10
    m = pm.Factor(g, 1e-10, precision=pm.PM_MIXED, scratch_gb=1e-6)
    x = m.solve(F)
    assert m.last_info["residual"] <= 1e-10
    assert _rel(x, dense.solve(prob, [0.3, 2.9])) < 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_arbitrary_arrangement_matches_the_oracle(pm, precision):
    """20 ellipses at random positions (spacing 0, Sec. 4.4's general
    arrangements): the same automatic quadtree as the oracle (same depth,
    boxes and compressed size in FP64) and the solution within the
    threshold of the dense solve."""
    prob = wl.random_arrangement(20, seed=6)
    g = pm.Geometry(prob)
    prec = pm.PM_MIXED if precision == "mixed" else pm.PM_FP64
    f = pm.Factor(g, 1e-10, precision=prec)
    angs = [0.3, 2.2]
    phi = f.solve(g.plane_wave(angs))
    ref = dense.solve(prob, angs)
    fo = proxy.factor(prob, {"tol": 1e-10})
    assert f.stats()["levels"] == fo["L"]
    if precision == "fp64":
        assert _rel(phi, ref) < 30 * 1e-10
        F = np.stack([dense.plane_wave(prob, a) for a in angs], 1)
        assert _rel(phi, proxy.solve(fo, F)) < 30 * 1e-10
        print(f"random arrangement: K={f.stats()['K']} (oracle {fo['stats']['K']})")
    else:
        assert f.last_info["residual"] <= 1e-10 and _rel(phi, ref) < 1e-8
