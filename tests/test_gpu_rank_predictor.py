"""The learned rank predictor: GPU kernels against the CPU reference MLP,
training, and what the trained network changes in a factorization."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2603_09381_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_09381_gb300 import pmchwt
    return pmchwt


def _dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a.astype(dtype))).cuda()


def test_gradient_matches_cpu_reference_fp64(pm):
    import torch
    rng = np.random.default_rng(2)
    theta = omlp.init_params(4) + 0.05 * rng.standard_normal(omlp.NPARAM)
    X = rng.standard_normal((150, 8))
    T = rng.standard_normal((150, 2))
    L, g = omlp.loss_grad(theta, X, T, 4.0)
    dth, dX, dT = _dev(theta, np.float64), _dev(X, np.float64), _dev(T, np.float64)
    grad = torch.zeros(omlp.NPARAM, dtype=torch.float64, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    pm.mlp_loss_grad(1, dth.data_ptr(), 150, dX.data_ptr(), dT.data_ptr(), 4.0, grad.data_ptr(), loss.data_ptr())
    assert abs(loss.item() - L) < 1e-12 * L
    assert np.max(np.abs(grad.cpu().numpy() - g)) < 1e-12 * np.max(np.abs(g))


def test_forward_fp32_and_adam_match_reference(pm):
    import torch
    rng = np.random.default_rng(3)
    theta = omlp.init_params(5)
    X = rng.standard_normal((77, 8))
    Y, _ = omlp.forward(theta, X)
    dth, dX = _dev(theta, np.float32), _dev(X, np.float32)
    dY = torch.zeros((77, 2), dtype=torch.float32, device="cuda")
    pm.mlp_forward(0, dth.data_ptr(), 77, dX.data_ptr(), dY.data_ptr())
    assert np.max(np.abs(dY.cpu().numpy() - Y)) < 1e-5
    g = rng.standard_normal(omlp.NPARAM)
    m, v = rng.standard_normal(omlp.NPARAM) * 0.1, np.abs(rng.standard_normal(omlp.NPARAM)) * 0.1
    ref, mr, vr = omlp.adam_step(theta, g, m, v, 7, lr=0.01)
    d = [_dev(a, np.float64) for a in (theta, g, m, v)]
    pm.mlp_adam_step(1, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), d[3].data_ptr(), 7, 0.01)
    assert np.allclose(d[0].cpu().numpy(), ref, rtol=0, atol=1e-14)
    assert np.allclose(d[2].cpu().numpy(), mr, atol=1e-15) and np.allclose(d[3].cpu().numpy(), vr, atol=1e-15)


def test_training_fits_a_smooth_map(pm):
    import torch
    from paper_2603_09381_gb300 import rank_predictor as rp
    rng = np.random.default_rng(0)
    X = rng.standard_normal((2000, 8)).astype(np.float32)
    T = np.stack([0.5 + 0.3 * np.tanh(X[:, 0] - 0.5 * X[:, 3]), 0.4 + 0.2 * np.sin(X[:, 1])], 1).astype(np.float32)
    model, hist = rp.train(X, T, epochs=60, batch=64, lr=3e-3, lam=1.0)
    assert hist[-1] < 0.05 * hist[0]
    dX = _dev((X - model[4866:4874]) / model[4874:4882], np.float32)
    dY = torch.zeros((2000, 2), dtype=torch.float32, device="cuda")
    dth = _dev(model[:4866], np.float32)
    pm.mlp_forward(0, dth.data_ptr(), 2000, dX.data_ptr(), dY.data_ptr())
    assert np.sqrt(np.mean((dY.cpu().numpy() - T) ** 2)) < 0.03


def test_predictor_presizes_ranks_and_proxy_counts(pm):
    """Trained on the solver's own ranks and held-out proxy-check outcomes, the
    network presizes a held-out problem's factorization.  With a fixed proxy
    count the ranks and the solution are those of the run without it and the
    host rank checks drop; with learned proxy counts the ID inputs shrink, the
    compressed system is no larger, and the solution stays within the
    solver's tolerance of the rule's (PM_FP64: every lowered box judged by
    the held-out check, failures redone with the rule's count)."""
    from paper_2603_09381_gb300 import rank_predictor as rp
    from oracle import dense
    train_probs = [(wl.star_grid(4, 4, n=64, seed=s), tol) for s in (1, 2) for tol in (1e-10, 1e-6)] + \
                  [(wl.fourier_grid(4, 4, n=128, seed=5), 1e-10), (wl.star_grid(8, 8, n=64, seed=4), 1e-10)]
    X, T = rp.harvest(train_probs, ladder=(1.0, 0.6, 0.35))
    assert X.shape[1] == 8 and np.all((T[:, 1] > 0) & (T[:, 1] <= 1))
    model, _ = rp.train(X, T, epochs=300, batch=32, lr=2e-3, lam=4.0)
    dm = rp.to_device(model)
    held = wl.fourier_grid(4, 4, n=128, seed=21)
    g = pm.Geometry(held)
    F = g.plane_wave([0.4, 2.2])
    # 1. ranks only (fixed proxy count): the same factorization, fewer host syncs
    f0 = pm.Factor(g, 1e-10, proxy_points=96)
    f1 = pm.Factor(g, 1e-10, proxy_points=96, rank_model=dm.data_ptr())
    s0, s1 = f0.stats(), f1.stats()
    assert s0["skeleton"] == s1["skeleton"] and s0["K"] == s1["K"]
    assert np.array_equal(f0.solve(F), f1.solve(F))
    assert s1["rank_checks"] < s0["rank_checks"]
    # 2. learned proxy counts
    ref = dense.solve(held, [0.4, 2.2])
    res = {}
    for prec in (pm.PM_FP64, pm.PM_MIXED):
        rule = pm.Factor(g, 1e-10, precision=prec)
        lrn = pm.Factor(g, 1e-10, precision=prec, rank_model=dm.data_ptr())
        sr, sl = rule.stats(), lrn.stats()
        xr, xl = rule.solve(F), lrn.solve(F)
        assert np.linalg.norm(xl - ref) <= 30 * 1e-10 * np.linalg.norm(ref) + np.linalg.norm(xr - ref)
        assert sl["K"] <= sr["K"]
        if sl["proxy_fallbacks"] == 0:
            assert sl["id_rows"] < sr["id_rows"]
        if prec == pm.PM_FP64:
            assert sl["proxy_checked"] > 0
        res[prec] = (sr, sl)
        print(f"precision {prec}: id_rows {sr['id_rows']} -> {sl['id_rows']}, K {sr['K']} -> {sl['K']}, "
              f"proxy checks {sl['proxy_checked']}, fallbacks {sl['proxy_fallbacks']}, "
              f"factor ms {sr['ms_total']:.1f} -> {sl['ms_total']:.1f}, rank checks {sr['rank_checks']} -> "
              f"{sl['rank_checks']}")
