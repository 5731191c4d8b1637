"""Learned ID-rank and proxy-count predictor: harvest (features, targets) from
factorizations, train the MLP with the library's own kernels, save / load the
model.  Targets per box and index group: the adaptive ID rank / n_g, and the
smallest fraction of the closed-form proxy count that passes the library's
held-out proxy check.

Marshalling only: factorizations, training steps and inference run in the
CUDA library (pm_factorize records the samples; pm_mlp_train trains).
Model file: float32 array of PM_MLP_NPARAM weights, 8 feature means, 8
feature scales (the scaling statistics are computed from the harvested data).
"""
import os

import numpy as np

from . import pmchwt as pm
from . import workloads as wl

NPARAM = 4866
MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "rank_mlp.npy")


def init_params(seed=0):
    """Scaled-normal weights, zero biases (same layout as the kernels)."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape in [(64, 8), (64,), (64, 64), (64,), (2, 64), (2,)]:
        parts.append(rng.standard_normal(shape).ravel() * np.sqrt(1.0 / shape[1]) if len(shape) == 2
                     else np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)


def training_problems():
    """Workloads the solver learns ranks from: circle grids (the 2x2 checks), star
    grids of the 16x16 recipe, random smooth shapes and ellipses."""
    out = []
    for tol in (1e-12, 1e-10, 1e-5):
        out.append((wl.circle_grid(2, 2), tol))
        out.append((wl.circle_grid(4, 4, n=64), tol))
    for nx in (4, 8, 16):
        for tol in (1e-10, 1e-5):
            out.append((wl.star_grid(nx, nx, n=128, seed=1), tol))
    out.append((wl.star_grid(8, 8, n=64, seed=9), 1e-8))
    for tol in (1e-10, 1e-6):
        out.append((wl.fourier_grid(8, 8, n=128, seed=11), tol))
    for prob in wl.ellipse_batch(count=6, seed=13, m_lo=4, m_hi=64):
        out.append((prob, 1e-10))
    return out


def harvest(problems, precision=pm.PM_FP64, ladder=(1.0, 0.7, 0.5, 0.35, 0.25), bound=200.0):
    """(X, T) of every box and index group of the problems' factorizations.

    T[:, 0]: max(row rank, column rank) / n_g at the rule's proxy count.
    T[:, 1]: the smallest fraction s of the rule's proxy count on the ladder
    such that the box passes the held-out proxy check (ratio <= bound) at s
    and at every larger fraction of the ladder, from one factorization per
    fraction with the check on.  Features come from the rule's run (they use
    the rule's input sizes in every run)."""
    X, T = [], []
    for prob, tol in problems:
        g = pm.Geometry(prob)
        x = t = None
        ok = None
        label = None
        for s in sorted(ladder, reverse=True):
            f = pm.Factor(g, tol, precision=precision, proxy_scale=s, proxy_check=True)
            xs, ts = f.rank_data()
            ratio, _ = f.proxy_data()
            if x is None:
                x, t = xs, ts.copy()
                ok = np.ones(len(xs), dtype=bool)
                label = np.full(len(xs), float(s), dtype=np.float32)
            if len(xs) == len(x):
                ok &= (ratio >= 0) & (ratio <= bound)
                label[ok] = s
            del f
        t[:, 1] = label
        X.append(x)
        T.append(t)
        del g
    return np.concatenate(X), np.concatenate(T)


def train(X, T, epochs=400, batch=64, lr=2e-3, lam=4.0, seed=0):
    """Returns (model array, loss history).  Device memory through torch."""
    import torch
    mu = X.mean(0)
    sd = X.std(0)
    sd[sd == 0] = 1.0
    Xn = ((X - mu) / sd).astype(np.float32)
    theta = torch.from_numpy(init_params(seed)).cuda()
    dX = torch.from_numpy(np.ascontiguousarray(Xn)).cuda()
    dT = torch.from_numpy(np.ascontiguousarray(T.astype(np.float32))).cuda()
    hist = pm.mlp_train(theta.data_ptr(), len(X), dX.data_ptr(), dT.data_ptr(), epochs, batch, lr, lam, seed)
    model = np.concatenate([theta.cpu().numpy(), mu.astype(np.float32), sd.astype(np.float32)])
    return model, hist


def save(model, path=MODEL_PATH):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.save(path, model.astype(np.float32))


def load_model(path=MODEL_PATH):
    return np.load(path) if os.path.exists(path) else None


def to_device(model):
    """A device copy of the model (keep the returned tensor alive while factoring)."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(model.astype(np.float32))).cuda()


if __name__ == "__main__":
    # python -m paper_2603_09381_gb300.rank_predictor [output.npy]: harvest the
    # training problems' ranks and proxy-check outcomes, train, save
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import __graft_entry__
    __graft_entry__.build()
    out = sys.argv[1] if len(sys.argv) > 1 else MODEL_PATH
    X, T = harvest(training_problems(), ladder=(1.0, 0.6, 0.35))
    model, hist = train(X, T)
    save(model, out)
    print(f"samples {len(X)}  proxy label mean {T[:, 1].mean():.3f}  loss first {hist[0]:.4f} "
          f"last {hist[-1]:.5f}  -> {out}")
