"""Multilevel proxy / ID fast direct solver for PMCHWT (Omit) (paper Sec. 3).

Factor (upward, levels L..1):
  * a box's current diagonal block D_b: at the leaf the self block A_ii; at a
    parent the children's compressed blocks A~_c on the diagonal and the
    original matrix entries A(skeleton rows of c, skeleton cols of c') off
    the diagonal (the multilevel merge, Sec. 3 last paragraphs);
  * four IDs per box (block-diagonal L_i = diag(L^1, L^2), R_i = diag(R^1, R^2),
    Sec. 3): row IDs of the u-equation and q-equation rows, column IDs of the
    q and u columns.  Each ID is computed on [near block | proxy block]: the
    near block holds the original (exterior-only, Omit) entries between the
    box's active indices and its near boxes' active indices, the proxy block
    the same exterior kernels between the box and a virtual boundary (the
    proxy circle, treated like an inclusion with p nodes, outward normals and
    weights 2 pi R_p / p).  Only the exterior wavenumber enters: the paper's
    point for the Omit formulation;
  * ranks: each ID is decided by its own CPQR (cpqr.py); row group g and
    column group g (u-eq rows with q cols, q-eq rows with u cols) then share
    k_g = max(row rank, column rank) so that A~ is square (the paper does not
    say how unequal row and column ranks are reconciled);
  * A~_b = (R_b D_b^{-1} L_b)^{-1}  (Sec. 3, definition of A~_i); singular -> error.
Top: D_root assembled like a parent from the level-1 boxes, partial-pivot LU.

Solve (eq. compressed and the recovery formula of Sec. 3):
  up:   g_b = D_b^{-1} f_b,  f~_b = A~_b R_b g_b  (f of a parent = children's f~)
  top:  psi = D_root^{-1} f_root
  down: x_b = g_b - (D_b^{-1} L_b)(f~_b - A~_b y_b), y_b = the box's slice of
        its parent's x (of psi at level 1); x at the leaves is phi.

Parity pinned by tests/test_oracle_proxy.py against dense.py.
"""
import numpy as np
import scipy.linalg as sla

from . import cpqr as cp
from . import tree as tr
from .dense import EPS_OUT, offsets
from .geometry import all_nodes, eps_in
from .kernels import kernel_values
from .blocks import self_block


class SingularError(RuntimeError):
    pass


class _Index:
    """Global row/column index -> (node, group) for the stacked system."""

    def __init__(self, prob, nds):
        self.off = np.array(offsets(prob))
        ns = np.array([inc["n"] for inc in prob["inclusions"]])
        self.n = ns
        self.node_off = np.concatenate([[0], np.cumsum(ns)])
        self.X = np.concatenate([nd["x"] for nd in nds])
        self.NRM = np.concatenate([nd["nrm"] for nd in nds])
        self.W = np.concatenate([nd["w"] for nd in nds])

    def decode(self, g):
        g = np.asarray(g)
        j = np.searchsorted(self.off, g, side="right") - 1
        loc = g - self.off[j]
        grp = loc // self.n[j]
        node = self.node_off[j] + loc % self.n[j]
        return node, grp


def _combine(S, D, Ds, N, rg, cg, w):
    """Omit off-diagonal entry for row group rg (0: u-eq, 1: q-eq) and column group cg (0: q, 1: u)."""
    val = np.where(rg == 0, np.where(cg == 0, -EPS_OUT * S, D),
                   np.where(cg == 0, -Ds, N / EPS_OUT))
    return val * w


def entries(ix, k0, rows, cols):
    """A(rows, cols) for rows and cols on different inclusions (exterior kernel only)."""
    rn, rg = ix.decode(rows)
    cn, cg = ix.decode(cols)
    S, D, Ds, N = kernel_values(ix.X[rn][:, None, :], ix.NRM[rn][:, None, :],
                                ix.X[cn][None, :, :], ix.NRM[cn][None, :, :], k0)
    return _combine(S, D, Ds, N, rg[:, None], cg[None, :], ix.W[cn][None, :])


def proxy_row_block(ix, k0, rows, box):
    """Rows of the box against the proxy boundary's 2p densities (q then u)."""
    px, pn, pw = tr.proxy_points(box)
    p = len(pw)
    rn, rg = ix.decode(rows)
    S, D, Ds, N = kernel_values(ix.X[rn][:, None, :], ix.NRM[rn][:, None, :],
                                px[None, :, :], pn[None, :, :], k0)
    S, D, Ds, N = (np.concatenate([a, a], 1) for a in (S, D, Ds, N))
    cg = np.repeat([0, 1], p)[None, :]
    return _combine(S, D, Ds, N, rg[:, None], cg, np.concatenate([pw, pw])[None, :])


def proxy_col_block(ix, k0, box, cols):
    """The proxy boundary's 2p equations (u-eq then q-eq) against the box's columns."""
    px, pn, _ = tr.proxy_points(box)
    p = len(px)
    cn, cg = ix.decode(cols)
    S, D, Ds, N = kernel_values(px[:, None, :], pn[:, None, :],
                                ix.X[cn][None, :, :], ix.NRM[cn][None, :, :], k0)
    S, D, Ds, N = (np.concatenate([a, a], 0) for a in (S, D, Ds, N))
    rg = np.repeat([0, 1], p)[:, None]
    return _combine(S, D, Ds, N, rg, cg[None, :], ix.W[cn][None, :])


def factor(prob, opts):
    nds = all_nodes(prob)
    ix = _Index(prob, nds)
    k0 = float(prob["k_out"])
    tol = float(opts["tol"])
    tree = tr.build(prob, nds, opts)
    L = tree["L"]
    levels = tree["levels"]
    off = ix.off
    stats = {"ranks": {}, "K": None}
    data = {}

    def leaf_init(box):
        j = box["leaves"][0]
        rows = off[j] + np.arange(2 * ix.n[j])
        grp = np.repeat([0, 1], ix.n[j])
        D = self_block(nds[j], k0, prob["inclusions"][j]["k_in"], EPS_OUT, eps_in(prob, j))
        return rows, grp, rows.copy(), grp.copy(), D

    def merge(lev, box):
        kids = [data[lev + 1, c] for c in box["children"]]
        rows = np.concatenate([d["srows"] for d in kids])
        rgrp = np.concatenate([d["srgrp"] for d in kids])
        cols = np.concatenate([d["scols"] for d in kids])
        cgrp = np.concatenate([d["scgrp"] for d in kids])
        nr = [len(d["srows"]) for d in kids]
        ro = np.concatenate([[0], np.cumsum(nr)])
        D = np.zeros((ro[-1], ro[-1]), dtype=np.complex128)
        for a, da in enumerate(kids):
            for b, db in enumerate(kids):
                if a == b:
                    D[ro[a]:ro[a + 1], ro[b]:ro[b + 1]] = da["At"]
                else:
                    D[ro[a]:ro[a + 1], ro[b]:ro[b + 1]] = entries(ix, k0, da["srows"], db["scols"])
        return rows, rgrp, cols, cgrp, D

    for lev in range(L, 0, -1):
        boxes = levels[lev]
        active = {}
        for bi, box in enumerate(boxes):
            active[bi] = leaf_init(box) if lev == L else merge(lev, box)
        ranks_lev = []
        for bi, box in enumerate(boxes):
            rows, rgrp, cols, cgrp, D = active[bi]
            near_cols = np.concatenate([active[o][2] for o in box["near"]]) if box["near"] else np.zeros(0, np.int64)
            near_rows = np.concatenate([active[o][0] for o in box["near"]]) if box["near"] else np.zeros(0, np.int64)
            ids = {}
            for g in (0, 1):
                rpos = np.nonzero(rgrp == g)[0]
                Mr = np.concatenate([entries(ix, k0, rows[rpos], near_cols),
                                     proxy_row_block(ix, k0, rows[rpos], box)], 1)
                ids["r", g] = (rpos, cp.CPQR(Mr.T, tol))
                cpos = np.nonzero(cgrp == g)[0]
                Mc = np.concatenate([entries(ix, k0, near_rows, cols[cpos]),
                                     proxy_col_block(ix, k0, box, cols[cpos])], 0)
                ids["c", g] = (cpos, cp.CPQR(Mc, tol))
            kg = []
            for g in (0, 1):
                fr, fc = ids["r", g][1], ids["c", g][1]
                k = min(max(fr.find_rank(), fc.find_rank()), fr.maxsteps, fc.maxsteps)
                fr.extend(k)
                fc.extend(k)
                kg.append(k)
            kb = sum(kg)
            Lm = np.zeros((len(rows), kb), dtype=np.complex128)
            Rm = np.zeros((kb, len(cols)), dtype=np.complex128)
            srows, srgrp, scols, scgrp = [], [], [], []
            o = 0
            for g in (0, 1):
                k = kg[g]
                rpos, f = ids["r", g]
                perm, T = f.perm, cp.interp_matrix(f.R, k)
                Lm[rpos[perm[:k]], o + np.arange(k)] = 1.0
                Lm[np.ix_(rpos[perm[k:]], o + np.arange(k))] = T.T
                srows.append(rows[rpos[perm[:k]]])
                srgrp.append(np.full(k, g))
                cpos, f = ids["c", g]
                perm, T = f.perm, cp.interp_matrix(f.R, k)
                Rm[o + np.arange(k), cpos[perm[:k]]] = 1.0
                Rm[np.ix_(o + np.arange(k), cpos[perm[k:]])] = T
                scols.append(cols[cpos[perm[:k]]])
                scgrp.append(np.full(k, g))
                o += k
            lu = sla.lu_factor(D)
            X = sla.lu_solve(lu, Lm)
            Y = Rm @ X
            if kb > 0 and np.linalg.cond(Y) > 1e15:
                raise SingularError(f"R D^-1 L singular at level {lev} box {bi}")
            At = np.linalg.inv(Y) if kb > 0 else np.zeros((0, 0), dtype=np.complex128)
            data[lev, bi] = {"rows": rows, "cols": cols, "lu": lu, "X": X, "R": Rm, "At": At,
                             "srows": np.concatenate(srows), "srgrp": np.concatenate(srgrp),
                             "scols": np.concatenate(scols), "scgrp": np.concatenate(scgrp),
                             "kg": kg, "skel": {key: (v[0], v[1].perm[:v[1].j].copy(), v[1].rank)
                                                 for key, v in ids.items()},
                             "margin": min(min(v[1].margin_pivot, v[1].margin_rank) for v in ids.values())}
            ranks_lev.append(kg)
        stats["ranks"][lev] = ranks_lev
    root = levels[0][0]
    if L == 0:
        rows, _, cols, _, Droot = leaf_init(root)
    else:
        rows, _, cols, _, Droot = merge(0, root)
    stats["K"] = Droot.shape[0]
    return {"L": L, "tree": tree, "data": data, "root_lu": sla.lu_factor(Droot),
            "root_rows": rows, "root_cols": cols, "N": int(off[-1]), "stats": stats}


def solve(fac, F):
    """phi = A^{-1} F (F: 2N x nrhs) through the compressed factorization."""
    F = np.asarray(F, dtype=np.complex128)
    vec = F.ndim == 1
    if vec:
        F = F[:, None]
    L, data, levels = fac["L"], fac["data"], fac["tree"]["levels"]
    up = {}
    for lev in range(L, 0, -1):
        for bi, box in enumerate(levels[lev]):
            d = data[lev, bi]
            if lev == L:
                f = F[d["rows"]]
            else:
                f = np.concatenate([up[lev + 1, c][1] for c in box["children"]])
            g = sla.lu_solve(d["lu"], f)
            ft = d["At"] @ (d["R"] @ g)
            up[lev, bi] = (g, ft)
    if L == 0:
        return _ret(sla.lu_solve(fac["root_lu"], F[fac["root_rows"]]), vec)
    froot = np.concatenate([up[1, c][1] for c in levels[0][0]["children"]])
    x = {(0, 0): sla.lu_solve(fac["root_lu"], froot)}
    phi = np.zeros((fac["N"], F.shape[1]), dtype=np.complex128)
    for lev in range(1, L + 1):
        parents = levels[lev - 1]
        for pi, pbox in enumerate(parents):
            xp = x[lev - 1, pi]
            o = 0
            for c in pbox["children"]:
                d = data[lev, c]
                kb = d["At"].shape[0]
                y = xp[o:o + kb]
                o += kb
                g, ft = up[lev, c]
                xc = g - d["X"] @ (ft - d["At"] @ y)
                x[lev, c] = xc
                if lev == L:
                    phi[d["cols"]] = xc
    return _ret(phi, vec)


def _ret(a, vec):
    return a[:, 0] if vec else a
