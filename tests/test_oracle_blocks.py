"""Pins for the Nystrom blocks: circle eigenvalues and Calderon / Green identities."""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import blocks, geometry
from oracle.kernels import bessel_parts
from paper_2603_09381_gb300 import workloads as wl

KS = [2 * math.pi, 4 * math.pi, 4 * math.pi * (1 + 0.05j)]


def _circle(n=64, a=0.4):
    return geometry.nodes(wl._inclusion(wl.SHAPE_CIRCLE, 0.7, -1.2, 0.9, [a], n, 1.0))


@pytest.mark.parametrize("k", KS)
def test_circle_eigenvalues(k):
    a = 0.4
    nd = _circle(a=a)
    S, D, Ds, N = blocks.self_operators(nd, k)
    z = k * a
    theta = nd["t"] + 0.9  # polar angle of node l about the centre (rotation 0.9)
    for m in [0, 1, 2, 5, 11, 20]:
        J, Jp = sp.jv(m, z), sp.jvp(m, z)
        H, Hp = sp.hankel1(m, z), sp.h1vp(m, z)
        lam = {"S": 1j * math.pi * a / 2 * J * H,
               "D": 1j * math.pi * z / 4 * (J * Hp + Jp * H),
               "N": 1j * math.pi * a * k * k / 2 * Jp * Hp}
        f = np.exp(1j * m * theta)
        scale = max(1.0, abs(lam["N"]))
        assert np.allclose(S @ f, lam["S"] * f, atol=1e-13)
        assert np.allclose(D @ f, lam["D"] * f, atol=1e-13)
        assert np.allclose(Ds @ f, lam["D"] * f, atol=1e-13)
        assert np.allclose(N @ f, lam["N"] * f, atol=1e-12 * scale)


def _point_field(nd, z, k):
    d = nd["x"] - z
    r = np.hypot(*d.T)
    H0, H1, _, _ = bessel_parts(k * r)
    return 0.25j * H0, -0.25j * k * H1 * np.sum(nd["nrm"] * d, -1) / r


@pytest.mark.parametrize("shape,prm,n", [(wl.SHAPE_STAR, [0.4, 0.2, 5], 128),
                                         (wl.SHAPE_ELLIPSE, [0.45, 0.2], 128),
                                         (wl.SHAPE_FOURIER, [0.4, .04, .03, .02, .01, .04, 1, 2, 3, 4, 5], 96)])
@pytest.mark.parametrize("k", [7.853981633974483, 15.707963267948966, 12 * (1 + 0.05j)])
def test_calderon_identities(shape, prm, n, k):
    nd = geometry.nodes(wl._inclusion(shape, 0.0, 0.0, 0.7, prm, n, 1.0))
    S, D, Ds, N = blocks.self_operators(nd, k)
    # radiating field of a source inside: (D - 1/2) v - S dv = 0, N v - (D* + 1/2) dv = 0
    v, dv = _point_field(nd, np.array([0.05, -0.03]), k)
    sc = np.linalg.norm(v) + np.linalg.norm(dv)
    assert np.linalg.norm(D @ v - 0.5 * v - S @ dv) < 1e-10 * sc
    assert np.linalg.norm(N @ v - Ds @ dv - 0.5 * dv) < 1e-9 * sc * abs(k)
    # field regular inside (source outside): (D + 1/2) w - S dw = 0, N w - (D* - 1/2) dw = 0
    w, dw = _point_field(nd, np.array([1.1, 0.6]), k)
    sc = np.linalg.norm(w) + np.linalg.norm(dw)
    assert np.linalg.norm(D @ w + 0.5 * w - S @ dw) < 1e-10 * sc
    assert np.linalg.norm(N @ w - Ds @ dw + 0.5 * dw) < 1e-9 * sc * abs(k)


@pytest.mark.parametrize("k", [7.853981633974483, 4 * math.pi * (1 + 0.05j)])
def test_offdiagonal_green_formula(k):
    src = geometry.nodes(wl._inclusion(wl.SHAPE_STAR, 0.0, 0.0, 0.3, [0.4, 0.2, 5], 128, 1.0))
    tgt = geometry.nodes(wl._inclusion(wl.SHAPE_STAR, 1.6, 0.4, 1.1, [0.4, 0.2, 5], 128, 1.0))
    S, D, Ds, N = blocks.offdiag_operators(tgt, src, k)
    z = np.array([0.02, 0.05])
    v, dv = _point_field(src, z, k)
    vt, dvt = _point_field(tgt, z, k)
    assert np.linalg.norm(D @ v - S @ dv - vt) < 1e-10 * np.linalg.norm(vt)
    assert np.linalg.norm(N @ v - Ds @ dv - dvt) < 1e-10 * np.linalg.norm(dvt)


def test_self_block_layout():
    nd = _circle()
    k0, k1 = 2 * math.pi, 4 * math.pi
    e1 = (k1 / k0) ** 2
    A = blocks.self_block(nd, k0, k1, 1.0, e1)
    Sp, Dp, Dsp, Np = blocks.self_operators(nd, k0)
    Sm, Dm, Dsm, Nm = blocks.self_operators(nd, k1)
    n = nd["n"]
    assert np.allclose(A[:n, :n], -(Sp + e1 * Sm))
    assert np.allclose(A[:n, n:], Dp + Dm)
    assert np.allclose(A[n:, :n], -(Dsp + Dsm))
    assert np.allclose(A[n:, n:], Np + Nm / e1)
