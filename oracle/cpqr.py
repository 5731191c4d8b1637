"""Column-pivoted QR and the interpolative decomposition (paper Sec. 3: the
ID of Cheng et al. 2005 computed by column-pivoted QR; the rank is decided
adaptively from the diagonal of R against the threshold epsilon).

Where the paper is silent: the threshold is relative, a column is kept
while |R_jj| > tol |R_11|; trailing column norms are recomputed from scratch
at every step (no downdating); a column whose squared trailing norm is at
least (1 - 1e-12) times the largest counts as tied, and among tied columns
the lowest original index wins.

Householder step (LAPACK zlarfg convention): for x = trailing part of the
pivot column, alpha = x_0, beta = -sign(Re alpha) ||x||, tau = (beta - alpha)/beta,
v = x / (alpha - beta) with v_0 = 1; H = I - tau v v^H satisfies
H^H x = beta e_1, so the trailing columns are updated with H^H (conj(tau)).
The ID T = R11^{-1} R12 does not depend on this phase convention.

Decision margins (bookkeeping only, no effect on the arithmetic): every
pivot choice and the rank decision compare floating-point norms against a
threshold, so a second implementation that rounds differently can only
disagree where a compared quantity lies within its rounding error of the
threshold.  ``margin_pivot`` records, over all steps, the smallest distance
|norm2_c - (1 - TIE) max| of any non-maximal candidate from the tie band's
edge, measured in norms (|sqrt(norm2_c) - sqrt((1 - TIE) max)|), and
``margin_rank`` the smallest |norm - tol |R_11|| over the kept steps and the
stopping test; both in units of eps |R_11| (eps = 2^-52), the size of the
rounding error a backward-stable QR leaves in a trailing column norm.

Parity pinned by tests/test_oracle_cpqr.py: pivots equal brute-force greedy
selection on tiny matrices; ID error on random low-rank matrices.
"""
import numpy as np
import scipy.linalg as sla

TIE = 1e-12
EPS = 2.0 ** -52


class CPQR:
    """Column-pivoted Householder QR of Z (W x n), advanced step by step.

    ``find_rank()`` runs steps while the next pivot's trailing norm |R_jj|
    exceeds tol |R_11| and records the rank; ``extend(k)`` continues to k
    steps.  After j steps, perm[:j] are the chosen columns and the first j
    rows of ``A`` (in pivoted column order) are final rows of R.
    """

    def __init__(self, Z, tol):
        Z = np.asarray(Z, dtype=np.complex128)
        W, n = Z.shape
        self.maxsteps = min(W, n)
        if W > n:
            # Column norms and R are invariant under Z -> Q0^H Z, so the pivoted
            # factorization of Z equals that of its unpivoted triangular factor
            # (a library QR step); this only shortens the loop below.
            Z = np.linalg.qr(Z, mode="r")
        self.A = np.array(Z, dtype=np.complex128, copy=True)
        self.W, self.n = self.A.shape
        self.perm = np.arange(self.n)
        self.tol = tol
        self.j = 0
        self.ref = None
        self.rank = None
        self.rdiag = []
        self.margin_pivot = np.inf
        self.margin_rank = np.inf

    def _norms2(self):
        B = self.A[self.j:, self.j:]
        return np.sum(B.real ** 2 + B.imag ** 2, axis=0)

    def _step(self, norms2):
        j, A = self.j, self.A
        mx = norms2.max()
        if self.ref and len(norms2) > 1:
            others = np.delete(norms2, int(np.argmax(norms2)))
            gap = np.min(np.abs(np.sqrt(others) - np.sqrt((1.0 - TIE) * mx))) / (EPS * self.ref)
            self.margin_pivot = min(self.margin_pivot, gap)
        tied = np.nonzero(norms2 >= (1.0 - TIE) * mx)[0]
        p = j + tied[np.argmin(self.perm[j + tied])]
        if p != j:
            A[:, [j, p]] = A[:, [p, j]]
            self.perm[[j, p]] = self.perm[[p, j]]
        x = A[j:, j]
        xnorm = np.sqrt(np.sum(x.real ** 2 + x.imag ** 2))
        self.rdiag.append(xnorm)
        if xnorm > 0.0:
            alpha = x[0]
            beta = -np.copysign(xnorm, alpha.real)
            tau = (beta - alpha) / beta
            v = x / (alpha - beta)
            v[0] = 1.0
            A[j:, j + 1:] -= np.conj(tau) * np.outer(v, v.conj() @ A[j:, j + 1:])
            A[j, j] = beta
            A[j + 1:, j] = 0.0
        self.j += 1

    def find_rank(self):
        while self.j < self.maxsteps:
            norms2 = self._norms2()
            if self.ref is None:
                self.ref = np.sqrt(norms2.max())
            if self.ref > 0:
                self.margin_rank = min(self.margin_rank, abs(np.sqrt(norms2.max()) - self.tol * self.ref)
                                       / (EPS * self.ref))
            if not np.sqrt(norms2.max()) > self.tol * self.ref:
                break
            self._step(norms2)
        self.rank = self.j
        return self.rank

    def extend(self, k):
        while self.j < min(k, self.maxsteps):
            self._step(self._norms2())

    @property
    def R(self):
        return self.A[:self.j, :]


def cpqr(Z, tol, max_steps=None):
    """Convenience wrapper: (perm, R, rdiag, rank) after ``max_steps`` steps
    (default min(W, n)); rank as decided by ``CPQR.find_rank``."""
    f = CPQR(Z, tol)
    rank = f.find_rank()
    f.extend(f.maxsteps if max_steps is None else max_steps)
    return f.perm, f.R, np.array(f.rdiag), rank


def interp_matrix(R, k):
    """T = R11^{-1} R12 for the first k pivots (k x (n - k))."""
    if k == 0:
        return np.zeros((0, R.shape[1]), dtype=np.complex128)
    return sla.solve_triangular(R[:k, :k], R[:k, k:], lower=False)


def column_id(Z, tol):
    """Column ID: Z[:, perm[k:]] ~ Z[:, perm[:k]] @ T."""
    perm, R, _, rank = cpqr(Z, tol)
    return perm, rank, interp_matrix(R, rank)
