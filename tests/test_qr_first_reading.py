"""Pivoting on the triangle of a tall ID input, checked on the CPU.

Column-pivoted QR of a tall ID input Z (W x n, W > n) and of the n x n
triangle R of its unpivoted QR choose the same pivots (Q^H keeps every
trailing column norm), which is what lets the complex64 GPU path pivot on
R.  The blocked algorithm the GPU uses for that QR (panels of 32 reflectors
in the zlarfg phase convention, one fused pass per reflector that applies
reflector j and sums the norm and dot products defining reflector j+1,
compact-WY trailing update C - V T^H V^H C) is restated here in NumPy and
checked against LAPACK's R.
"""
import numpy as np
import scipy.linalg as sla

NB = 32


def _panel_fused(Z, j0, jb):
    W = Z.shape[0]
    taus, sc, f = [], 0.0, np.zeros(NB, complex)
    for ja in range(-1, jb):
        jn, ca, cn = ja + 1, j0 + ja, j0 + ja + 1
        N, S, row = 0.0, np.zeros(NB, complex), np.zeros(NB, complex)
        for r in range(ca if ja >= 0 else cn, W):
            v = Z[r, j0:j0 + jb].copy()
            if ja >= 0:
                vr = 1.0 if r == ca else v[ja] * sc
                if r > ca:
                    Z[r, j0 + ja] = vr
                for k in range(ja + 1, jb):
                    v[k] -= f[k] * vr
                    Z[r, j0 + k] = v[k]
            if jn < jb and r >= cn:
                y = v[jn]
                N += abs(y) ** 2
                if r == cn:
                    row[jn:jb] = v[jn:jb]
                else:
                    S[jn + 1:jb] += np.conj(y) * v[jn + 1:jb]
        if jn >= jb:
            break
        alpha, xn = row[jn], np.sqrt(N)
        if xn > 0:
            beta = -np.copysign(xn, alpha.real)
            tau, scn = (beta - alpha) / beta, 1.0 / (alpha - beta)
        else:
            beta, tau, scn = 0.0, 0.0, 0.0
        Z[cn, cn] = beta
        taus.append(tau)
        f[jn + 1:jb] = np.conj(tau) * (row[jn + 1:jb] + np.conj(scn) * S[jn + 1:jb])
        sc = scn
    return taus


def blocked_qr_r(Z):
    Z = np.array(Z, dtype=np.complex128)
    W, n = Z.shape
    for j0 in range(0, n, NB):
        jb = min(NB, n - j0)
        taus = _panel_fused(Z, j0, jb)
        V = np.zeros((W - j0, jb), complex)
        for j in range(jb):
            V[j, j] = 1.0
            V[j + 1:, j] = Z[j0 + j + 1:, j0 + j]
        G = V.conj().T @ V
        T = np.zeros((jb, jb), complex)
        for j in range(jb):
            T[j, j] = taus[j]
            if j:
                T[:j, j] = -taus[j] * (T[:j, :j] @ G[:j, j])
        C = Z[j0:, j0 + jb:]
        Z[j0:, j0 + jb:] = C - V @ (T.conj().T @ (V.conj().T @ C))
    return np.triu(Z[:n, :n])


def _greedy_pivots(A, k):
    """Column pivots by brute force: at each step the column with the largest
    residual norm after projecting out the chosen columns (lowest index on ties)."""
    A = np.array(A, dtype=np.complex128)
    chosen = []
    for _ in range(k):
        if chosen:
            Q, _ = np.linalg.qr(A[:, chosen])
            Rm = A - Q @ (Q.conj().T @ A)
        else:
            Rm = A
        nr = np.linalg.norm(Rm, axis=0)
        nr[chosen] = -1
        chosen.append(int(np.argmax(nr)))
    return chosen


def test_blocked_fused_qr_reproduces_lapack_r():
    rng = np.random.default_rng(7)
    for W, n in [(150, 70), (200, 33), (97, 45)]:
        Z = rng.standard_normal((W, n)) + 1j * rng.standard_normal((W, n))
        R = blocked_qr_r(Z)
        R0 = sla.qr(Z, mode="r")[0][:n]
        d = np.diag(R) / np.diag(R0)
        assert np.max(np.abs(np.abs(d) - 1)) < 1e-13          # same R up to unit phases per row
        assert np.max(np.abs(R - d[:, None] * R0)) < 1e-13 * np.abs(R0).max()
        assert np.allclose(np.linalg.norm(R, axis=0), np.linalg.norm(Z, axis=0), rtol=1e-13)


def test_pivots_of_the_triangle_are_those_of_the_tall_input():
    rng = np.random.default_rng(8)
    W, n, rank = 120, 24, 9
    # numerically low rank with distinct column scales (no ties)
    Z = (rng.standard_normal((W, rank)) + 1j * rng.standard_normal((W, rank))) @ \
        (rng.standard_normal((rank, n)) + 1j * rng.standard_normal((rank, n)))
    Z = Z * np.linspace(1.0, 2.0, n) + 1e-9 * rng.standard_normal((W, n))
    R = blocked_qr_r(Z)
    assert _greedy_pivots(R, rank) == _greedy_pivots(Z, rank)
