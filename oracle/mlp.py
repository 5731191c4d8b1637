"""Reference MLP for the learned ID-rank predictor (not in the paper; it
presizes the interpolative decompositions of Sec. 3).

Network: x (8) -> tanh(W1 x + b1) (64) -> tanh(W2 h1 + b2) (64) -> W3 h2 + b3 (2).
Loss over a batch of B samples (asymmetric squared error: under-prediction,
which forces the adaptive fallback, costs 1 + lam times more):
    L = (1/B) sum_i sum_o (1 + lam [y_io < t_io]) (y_io - t_io)^2.
Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Flat parameter layout (row-major): W1 (64x8), b1 (64), W2 (64x64), b2 (64),
W3 (2x64), b3 (2): 4866 numbers.

Pinned by tests/test_oracle_mlp.py: backward pass against central finite
differences of the loss; Adam against its closed form for one step.
"""
import numpy as np

SIZES = [(64, 8), (64,), (64, 64), (64,), (2, 64), (2,)]
NPARAM = sum(int(np.prod(s)) for s in SIZES)


def unpack(theta):
    out, o = [], 0
    for s in SIZES:
        k = int(np.prod(s))
        out.append(theta[o:o + k].reshape(s))
        o += k
    return out


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    parts = []
    for s in SIZES:
        if len(s) == 2:
            parts.append(rng.standard_normal(s).ravel() * np.sqrt(1.0 / s[1]))
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)


def forward(theta, X):
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3.T + b3, (h1, h2)


def loss_grad(theta, X, T, lam):
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    B = X.shape[0]
    Y, (h1, h2) = forward(theta, X)
    w = 1.0 + lam * (Y < T)
    L = np.sum(w * (Y - T) ** 2) / B
    dY = 2.0 * w * (Y - T) / B
    gW3 = dY.T @ h2
    gb3 = dY.sum(0)
    dz2 = (dY @ W3) * (1 - h2 ** 2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (1 - h1 ** 2)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    return L, np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def adam_step(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
