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
from .dense import EPS_OUT, bm_rhs, bm_to_pmchwt_order, offsets
from .geometry import all_nodes, eps_in
from .kernels import kernel_values
from .blocks import bm_self_block, self_block

FORMS = ("omit", "all", "bm", "bm_simplified")


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
        self.k_in = [inc["k_in"] for inc in prob["inclusions"]]
        self.eps_in = [eps_in(prob, j) for j in range(len(prob["inclusions"]))]

    def incl_of_node(self, node):
        return np.searchsorted(self.node_off, np.asarray(node), side="right") - 1

    def decode(self, g):
        g = np.asarray(g)
        j = np.searchsorted(self.off, g, side="right") - 1
        loc = g - self.off[j]
        grp = loc // self.n[j]
        node = self.node_off[j] + loc % self.n[j]
        return node, grp


def _combine(S, D, Ds, N, rg, cg, w, eps=EPS_OUT):
    """Omit off-diagonal entry for row group rg (0: u-eq, 1: q-eq) and column group cg (0: q, 1: u)
    (with eps = eps- and interior kernel values: the interior terms of PMCHWT (All))."""
    val = np.where(rg == 0, np.where(cg == 0, -eps * S, D),
                   np.where(cg == 0, -Ds, N / eps))
    return val * w


def _combine_bm(Sp, Dp, Dsp, Np, Sm, Dm, rg, cg, w, k0, eps_in, simplified=False):
    """Burton-Miller off-diagonal entry: row group rg (0: exterior eq., 1: interior
    eq.), column group cg (0: u, 1: q); exterior kernel values Sp..Np, interior Sm, Dm."""
    a = 1j / k0
    ext = np.where(cg == 0, Dp + a * Np, -EPS_OUT * (Sp + a * Dsp))
    inner = 0.0 if simplified else np.where(cg == 0, Dm, -eps_in * Sm)
    return np.where(rg == 0, ext, inner) * w


def _kvals(xt, nt, xs, ns, k):
    return kernel_values(xt, nt, xs, ns, k)


def entries(ix, k0, rows, cols, form="omit"):
    """A(rows, cols) for rows and cols on different inclusions: PMCHWT (Omit,
    exterior kernel only), PMCHWT (All) or Burton-Miller (plain or simplified),
    interior terms with the source inclusion's k- and eps-."""
    rn, rg = ix.decode(rows)
    cn, cg = ix.decode(cols)
    xt, nt = ix.X[rn][:, None, :], ix.NRM[rn][:, None, :]
    xs, ns = ix.X[cn][None, :, :], ix.NRM[cn][None, :, :]
    w = ix.W[cn][None, :]
    Sp, Dp, Dsp, Np = _kvals(xt, nt, xs, ns, k0)
    if form == "omit":
        return _combine(Sp, Dp, Dsp, Np, rg[:, None], cg[None, :], w)
    jin = ix.incl_of_node(cn)
    out = np.zeros((len(rn), len(cn)), dtype=np.complex128)
    for j in np.unique(jin):          # interior terms: the source inclusion's k- and eps-
        sel = jin == j
        kin, ein = ix.k_in[j], ix.eps_in[j]
        if form == "all":
            Sm, Dm, Dsm, Nm = _kvals(xt, nt, xs[:, sel], ns[:, sel], kin)
            out[:, sel] = (_combine(Sp[:, sel], Dp[:, sel], Dsp[:, sel], Np[:, sel], rg[:, None], cg[None, sel],
                                    w[:, sel])
                           + _combine(Sm, Dm, Dsm, Nm, rg[:, None], cg[None, sel], w[:, sel], ein))
        elif form in ("bm", "bm_simplified"):
            Sm, Dm, _, _ = _kvals(xt, nt, xs[:, sel], ns[:, sel], kin)
            out[:, sel] = _combine_bm(Sp[:, sel], Dp[:, sel], Dsp[:, sel], Np[:, sel], Sm, Dm, rg[:, None],
                                      cg[None, sel], w[:, sel], k0, ein, form == "bm_simplified")
        else:
            raise ValueError(form)
    return out


def _box_interior(ix, box):
    """k- and eps- of the box's inclusions (the interior proxy family of PMCHWT
    (All) and Burton-Miller assumes one interior medium per box)."""
    j = box["leaves"][0]
    return ix.k_in[j], ix.eps_in[j]


def proxy_row_block(ix, k0, rows, box, form="omit"):
    """Rows of the box against the proxy boundary's densities: Omit 2p (q then
    u, exterior kernel); All 4p (the exterior family, then the same with the
    interior kernel); Burton-Miller 2p (u then q, the proxy circle treated as an
    inclusion of the box's interior medium)."""
    px, pn, pw = tr.proxy_points(box)
    p = len(pw)
    rn, rg = ix.decode(rows)
    xt, nt = ix.X[rn][:, None, :], ix.NRM[rn][:, None, :]
    w = np.concatenate([pw, pw])[None, :]
    cg = np.repeat([0, 1], p)[None, :]
    two = lambda vals: [np.concatenate([a, a], 1) for a in vals]
    Sp, Dp, Dsp, Np = two(kernel_values(xt, nt, px[None, :, :], pn[None, :, :], k0))
    if form == "omit":
        return _combine(Sp, Dp, Dsp, Np, rg[:, None], cg, w)
    kin, ein = _box_interior(ix, box)
    Sm, Dm, Dsm, Nm = two(kernel_values(xt, nt, px[None, :, :], pn[None, :, :], kin))
    if form == "all":
        return np.concatenate([_combine(Sp, Dp, Dsp, Np, rg[:, None], cg, w),
                               _combine(Sm, Dm, Dsm, Nm, rg[:, None], cg, w, ein)], 1)
    return _combine_bm(Sp, Dp, Dsp, Np, Sm, Dm, rg[:, None], cg, w, k0, ein, form == "bm_simplified")


def proxy_col_block(ix, k0, box, cols, form="omit"):
    """The proxy boundary's equations against the box's columns (the same
    families as proxy_row_block, the proxy circle as the target inclusion)."""
    px, pn, _ = tr.proxy_points(box)
    p = len(px)
    cn, cg = ix.decode(cols)
    xs, ns = ix.X[cn][None, :, :], ix.NRM[cn][None, :, :]
    w = ix.W[cn][None, :]
    rg = np.repeat([0, 1], p)[:, None]
    two = lambda vals: [np.concatenate([a, a], 0) for a in vals]
    Sp, Dp, Dsp, Np = two(kernel_values(px[:, None, :], pn[:, None, :], xs, ns, k0))
    if form == "omit":
        return _combine(Sp, Dp, Dsp, Np, rg, cg[None, :], w)
    jin = ix.incl_of_node(cn)
    if form == "all":
        parts = []
        out_m = np.zeros((2 * p, len(cn)), dtype=np.complex128)
        for j in np.unique(jin):
            sel = jin == j
            Sm, Dm, Dsm, Nm = two(kernel_values(px[:, None, :], pn[:, None, :], xs[:, sel], ns[:, sel], ix.k_in[j]))
            out_m[:, sel] = _combine(Sm, Dm, Dsm, Nm, rg, cg[None, sel], w[:, sel], ix.eps_in[j])
        return np.concatenate([_combine(Sp, Dp, Dsp, Np, rg, cg[None, :], w), out_m], 0)
    out = np.zeros((2 * p, len(cn)), dtype=np.complex128)
    for j in np.unique(jin):
        sel = jin == j
        Sm, Dm, _, _ = two(kernel_values(px[:, None, :], pn[:, None, :], xs[:, sel], ns[:, sel], ix.k_in[j]))
        out[:, sel] = _combine_bm(Sp[:, sel], Dp[:, sel], Dsp[:, sel], Np[:, sel], Sm, Dm, rg, cg[None, sel],
                                  w[:, sel], k0, ix.eps_in[j], form == "bm_simplified")
    return out


def heldout_row_block(ix, k0, rows, box):
    """Rows of the box against the held-out ring's densities (q then u)."""
    px, pn, pw = tr.heldout_points(box)
    p = len(pw)
    rn, rg = ix.decode(rows)
    S, D, Ds, N = kernel_values(ix.X[rn][:, None, :], ix.NRM[rn][:, None, :], px[None, :, :], pn[None, :, :], k0)
    S, D, Ds, N = (np.concatenate([a, a], 1) for a in (S, D, Ds, N))
    cg = np.repeat([0, 1], p)[None, :]
    return _combine(S, D, Ds, N, rg[:, None], cg, np.concatenate([pw, pw])[None, :])


def heldout_col_block(ix, k0, box, cols):
    """The held-out ring's equations (u-eq then q-eq) against the box's columns."""
    px, pn, _ = tr.heldout_points(box)
    p = len(px)
    cn, cg = ix.decode(cols)
    S, D, Ds, N = kernel_values(px[:, None, :], pn[:, None, :], ix.X[cn][None, :, :], ix.NRM[cn][None, :, :], k0)
    S, D, Ds, N = (np.concatenate([a, a], 0) for a in (S, D, Ds, N))
    rg = np.repeat([0, 1], p)[:, None]
    return _combine(S, D, Ds, N, rg, cg[None, :], ix.W[cn][None, :])


def id_heldout_error(H, perm, k, T):
    """Relative error ||H[:, J] - H[:, S] T||_F / ||H||_F of an ID (skeleton S =
    perm[:k], the rest J = perm[k:], T = R11^{-1} R12) on a held-out block H
    whose columns are the ID's candidates (no counterpart in the paper: the
    a posteriori check of a proxy count)."""
    E = H[:, perm[k:]] - H[:, perm[:k]] @ T
    return float(np.linalg.norm(E) / max(np.linalg.norm(H), 1e-300))


def factor(prob, opts):
    """opts: tol, proxy_factor, proxy_points, proxy_scale, proxy_check and
    formulation ("omit" (default), "all", "bm", "bm_simplified").  PMCHWT
    (All) and Burton-Miller need the interior kernel in the proxies too: the
    closed-form proxy count then uses the largest wavenumber."""
    form = opts.get("formulation", "omit")
    if form not in FORMS:
        raise ValueError(form)
    nds = all_nodes(prob)
    ix = _Index(prob, nds)
    k0 = float(prob["k_out"])
    tol = float(opts["tol"])
    if form != "omit":
        opts = dict(opts, k_rule=max([k0] + [abs(complex(inc["k_in"]).real) for inc in prob["inclusions"]]))
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
        blk = bm_self_block if form.startswith("bm") else self_block
        D = blk(nds[j], k0, prob["inclusions"][j]["k_in"], EPS_OUT, eps_in(prob, j))
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
                    D[ro[a]:ro[a + 1], ro[b]:ro[b + 1]] = entries(ix, k0, da["srows"], db["scols"], form)
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
                Mr = np.concatenate([entries(ix, k0, rows[rpos], near_cols, form),
                                     proxy_row_block(ix, k0, rows[rpos], box, form)], 1)
                ids["r", g] = (rpos, cp.CPQR(Mr.T, tol))
                cpos = np.nonzero(cgrp == g)[0]
                Mc = np.concatenate([entries(ix, k0, near_rows, cols[cpos], form),
                                     proxy_col_block(ix, k0, box, cols[cpos], form)], 0)
                ids["c", g] = (cpos, cp.CPQR(Mc, tol))
            kg = []
            for g in (0, 1):
                fr, fc = ids["r", g][1], ids["c", g][1]
                k = min(max(fr.find_rank(), fc.find_rank()), fr.maxsteps, fc.maxsteps)
                fr.extend(k)
                fc.extend(k)
                kg.append(k)
            check = None
            if opts.get("proxy_check"):
                # held-out ring check of every ID: rows (resp. columns) of the box
                # against the held-out ring, interpolated through the ID
                check = 0.0
                for g in (0, 1):
                    rpos, f = ids["r", g]
                    H = heldout_row_block(ix, k0, rows[rpos], box).T
                    check = max(check, id_heldout_error(H, f.perm, kg[g], cp.interp_matrix(f.R, kg[g])))
                    cpos, f = ids["c", g]
                    H = heldout_col_block(ix, k0, box, cols[cpos])
                    check = max(check, id_heldout_error(H, f.perm, kg[g], cp.interp_matrix(f.R, kg[g])))
            kb = sum(kg)
            Lm = np.zeros((len(rows), kb), dtype=np.complex128)
            Rm = np.zeros((kb, len(cols)), dtype=np.complex128)
            srows, srgrp, scols, scgrp = [], [], [], []
            o = 0
            for g in (0, 1):
                k = kg[g]
                rpos, f = ids["r", g]
                perm = f.perm
                # an exactly zero ID input (no far field at all, e.g. the interior
                # rows of the simplified Burton-Miller system): zero interpolation
                if f.ref:
                    T = cp.interp_matrix(f.R, k)
                    Lm[rpos[perm[:k]], o + np.arange(k)] = 1.0
                    Lm[np.ix_(rpos[perm[k:]], o + np.arange(k))] = T.T
                srows.append(rows[rpos[perm[:k]]])
                srgrp.append(np.full(k, g))
                cpos, f = ids["c", g]
                perm = f.perm
                if f.ref:
                    T = cp.interp_matrix(f.R, k)
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
                             "margin": min(min(v[1].margin_pivot, v[1].margin_rank) for v in ids.values()),
                             "check": check}
            ranks_lev.append(kg)
        stats["ranks"][lev] = ranks_lev
    root = levels[0][0]
    if L == 0:
        rows, _, cols, _, Droot = leaf_init(root)
    else:
        rows, _, cols, _, Droot = merge(0, root)
    stats["K"] = Droot.shape[0]
    return {"L": L, "tree": tree, "data": data, "root_lu": sla.lu_factor(Droot),
            "root_rows": rows, "root_cols": cols, "N": int(off[-1]), "stats": stats, "form": form, "prob": prob}


def solve(fac, F):
    """phi = A^{-1} F (F: 2N x nrhs) through the compressed factorization.
    F is the PMCHWT right-hand side [-u^I; -q^I] per inclusion and phi is
    returned as [q; u] per inclusion for every formulation (Burton-Miller maps
    F to its own right-hand side and reorders its [u; q] unknowns)."""
    F = np.asarray(F, dtype=np.complex128)
    vec = F.ndim == 1
    if vec:
        F = F[:, None]
    if fac.get("form", "omit").startswith("bm"):
        x = _solve_system(fac, bm_rhs(fac["prob"], F))
        return _ret(bm_to_pmchwt_order(fac["prob"], x), vec)
    return _ret(_solve_system(fac, F), vec)


def _solve_system(fac, F):
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
        return sla.lu_solve(fac["root_lu"], F[fac["root_rows"]])
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
    return phi


def _ret(a, vec):
    return a[:, 0] if vec else a
