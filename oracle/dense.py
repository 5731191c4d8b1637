"""The conventional BIEM (paper Sec. 4): dense Nystrom assembly of the whole
PMCHWT system (eq. block_linear) and a partial-pivot LU solve.

Global ordering: inclusion j (input order) owns 2 n_j consecutive rows and
columns; within it rows are [u-equation rows; q-equation rows] and columns
[q_j; u_j] (Sec. 2.2).

Incident plane wave u^I = exp(i k+ d.x), d = (cos a, sin a);
q^I = (1/eps+) du^I/dn = (1/eps+) i k+ (d.n) u^I  (eq. flux applied to u^I).

Parity pinned by tests/test_oracle_dense.py against the Mie series / multipole
solutions of mie.py and by the energy balance of the interior field.
"""
import numpy as np
import scipy.linalg as sla

from . import blocks
from .geometry import all_nodes, eps_in

EPS_OUT = 1.0


def offsets(prob):
    off = [0]
    for inc in prob["inclusions"]:
        off.append(off[-1] + 2 * inc["n"])
    return off


def assemble(prob, formulation="omit", nds=None):
    nds = nds if nds is not None else all_nodes(prob)
    m = len(nds)
    off = offsets(prob)
    A = np.zeros((off[-1], off[-1]), dtype=np.complex128)
    k0 = prob["k_out"]
    for i in range(m):
        for j in range(m):
            if i == j:
                blk = blocks.self_block(nds[i], k0, prob["inclusions"][i]["k_in"], EPS_OUT,
                                        eps_in(prob, i))
            elif formulation == "omit":
                blk = blocks.omit_block(nds[i], nds[j], k0, EPS_OUT)
            elif formulation == "all":
                blk = blocks.all_block(nds[i], nds[j], k0, prob["inclusions"][j]["k_in"],
                                       EPS_OUT, eps_in(prob, j))
            else:
                raise ValueError(formulation)
            A[off[i]:off[i + 1], off[j]:off[j + 1]] = blk
    return A


def assemble_bm(prob, nds=None, simplified=False):
    """The Burton-Miller system (eq. bm_bie): unknowns [u_i; q_i] and rows
    [exterior; interior] per inclusion (blocks.bm_self_block / bm_block)."""
    nds = nds if nds is not None else all_nodes(prob)
    m = len(nds)
    off = offsets(prob)
    A = np.zeros((off[-1], off[-1]), dtype=np.complex128)
    k0 = prob["k_out"]
    for i in range(m):
        for j in range(m):
            if i == j:
                blk = blocks.bm_self_block(nds[i], k0, prob["inclusions"][i]["k_in"], EPS_OUT, eps_in(prob, i))
            else:
                blk = blocks.bm_block(nds[i], nds[j], k0, prob["inclusions"][j]["k_in"], EPS_OUT, eps_in(prob, j),
                                      simplified)
            A[off[i]:off[i + 1], off[j]:off[j + 1]] = blk
    return A


def plane_wave(prob, angle, nds=None):
    """Right-hand side f = [-u^I_i; -q^I_i] per inclusion for incidence angle ``angle``."""
    nds = nds if nds is not None else all_nodes(prob)
    k0 = prob["k_out"]
    dvec = np.array([np.cos(angle), np.sin(angle)])
    parts = []
    for nd in nds:
        uI = np.exp(1j * k0 * (nd["x"] @ dvec))
        qI = (1.0 / EPS_OUT) * 1j * k0 * (nd["nrm"] @ dvec) * uI
        parts += [-uI, -qI]
    return np.concatenate(parts)


def bm_rhs(prob, f):
    """The Burton-Miller right-hand side [-(u^I + alpha q^I); 0] per inclusion
    from the PMCHWT one f = [-u^I; -q^I] (alpha = i / k+)."""
    f = np.asarray(f)
    a = 1j / prob["k_out"]
    out = np.zeros_like(f)
    off = offsets(prob)
    for j, inc in enumerate(prob["inclusions"]):
        n = inc["n"]
        out[off[j]:off[j] + n] = f[off[j]:off[j] + n] + a * f[off[j] + n:off[j] + 2 * n]
    return out


def bm_to_pmchwt_order(prob, x):
    """[u_i; q_i] per inclusion -> [q_i; u_i] (the PMCHWT unknown order)."""
    x = np.asarray(x)
    out = np.empty_like(x)
    off = offsets(prob)
    for j, inc in enumerate(prob["inclusions"]):
        n = inc["n"]
        out[off[j]:off[j] + n] = x[off[j] + n:off[j] + 2 * n]
        out[off[j] + n:off[j] + 2 * n] = x[off[j]:off[j] + n]
    return out


def solve(prob, angles, formulation="omit"):
    """phi (2N x nrhs, [q_i; u_i] per inclusion) of the conventional BIEM for
    plane waves at ``angles``; formulation "omit", "all" or "bm"."""
    nds = all_nodes(prob)
    F = np.stack([plane_wave(prob, a, nds) for a in angles], 1)
    if formulation == "bm":
        A = assemble_bm(prob, nds)
        X = sla.lu_solve(sla.lu_factor(A), bm_rhs(prob, F))
        return bm_to_pmchwt_order(prob, X)
    A = assemble(prob, formulation, nds)
    lu = sla.lu_factor(A)
    return sla.lu_solve(lu, F)


def split(prob, phi):
    """Per inclusion (q_i, u_i) from a stacked solution vector."""
    off = offsets(prob)
    out = []
    for j, inc in enumerate(prob["inclusions"]):
        n = inc["n"]
        seg = phi[off[j]:off[j + 1]]
        out.append((seg[:n], seg[n:]))
    return out
