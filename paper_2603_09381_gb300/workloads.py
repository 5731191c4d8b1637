"""Seeded synthetic workloads: plain problem descriptors, no solver arithmetic.

Both the CUDA path and the CPU oracle consume these descriptors.  The module
only draws shapes, positions, rotations, wavenumbers and incidence angles;
it evaluates no curve, kernel or matrix.

Descriptor layout (mirrors ``pm_inclusion`` / ``pm_problem`` in
``include/pmchwt.h``):

  inclusion = {"shape": SHAPE_*, "cx": float, "cy": float, "rot": float,
               "prm": [16 floats], "n": int, "k_in": complex}
  problem   = {"k_out": float, "inclusions": [...], "grid_nx": int,
               "grid_ny": int, "spacing": float}

Shapes (local polar angle t, rotated by ``rot`` about the centre):
  SHAPE_CIRCLE  prm[0]=a                       r(t) = a
  SHAPE_ELLIPSE prm[0]=a, prm[1]=b             x(t) = (a cos t, b sin t)
  SHAPE_STAR    prm[0]=r0, prm[1]=e, prm[2]=p  r(t) = r0 (1 + e cos(p t))
  SHAPE_FOURIER prm[0]=r0, prm[1..5]=a_2..a_6, prm[6..10]=phi_2..phi_6
                r(t) = r0 (1 + sum_m a_m cos(m t + phi_m))

The workloads stand in for the paper's star-shaped inclusions on a square
grid (Sec. 4, Fig. "star"), whose exact shape, spacing and rotations are
given only as a figure.
"""
import math

import numpy as np

SHAPE_CIRCLE, SHAPE_ELLIPSE, SHAPE_STAR, SHAPE_FOURIER = 0, 1, 2, 3


def _inclusion(shape, cx, cy, rot, prm, n, k_in):
    p = [0.0] * 16
    for i, v in enumerate(prm):
        p[i] = float(v)
    return {"shape": int(shape), "cx": float(cx), "cy": float(cy), "rot": float(rot),
            "prm": p, "n": int(n), "k_in": complex(k_in)}


def circle_grid(nx, ny, radius=0.4, spacing=1.0, k_out=2 * math.pi, k_in=4 * math.pi, n=64):
    """nx x ny grid of circles (the 2x2 case is the 512-unknown FP64 check)."""
    inc = [_inclusion(SHAPE_CIRCLE, ix * spacing, iy * spacing, 0.0, [radius], n, k_in)
           for iy in range(ny) for ix in range(nx)]
    return {"k_out": float(k_out), "inclusions": inc, "grid_nx": nx, "grid_ny": ny,
            "spacing": float(spacing)}


def star_grid(nx, ny, n=128, seed=1, k_out=None, k_ratio=2.0, spacing=1.0,
              r0=0.4, eps=0.2, arms=5, wavelengths=20.0):
    """nx x ny grid of stars r = r0 (1 + eps cos(arms t)), rotations ~ U[0, 2 pi/arms).

    k_out defaults to 2 pi * wavelengths / (16 spacings), i.e. the 16 x 16 box is
    ``wavelengths`` wavelengths wide; k_in = k_ratio * k_out.
    """
    rng = np.random.default_rng(seed)
    rots = rng.uniform(0.0, 2 * math.pi / arms, size=nx * ny)
    if k_out is None:
        k_out = 2 * math.pi * wavelengths / (16 * spacing)
    inc = []
    for iy in range(ny):
        for ix in range(nx):
            j = iy * nx + ix
            inc.append(_inclusion(SHAPE_STAR, ix * spacing, iy * spacing, rots[j],
                                  [r0, eps, arms], n, k_ratio * k_out))
    return {"k_out": float(k_out), "inclusions": inc, "grid_nx": nx, "grid_ny": ny,
            "spacing": float(spacing)}


def fourier_grid(nx, ny, n=128, seed=4, k_out=5.0, spacing=1.0, r0=0.4, amax=0.04,
                 ratio_lo=1.5, ratio_hi=3.0):
    """Random smooth shapes r = r0 (1 + sum_{m=2..6} a_m cos(m t + phi_m)).

    a_m ~ U(0, amax), phi_m ~ U[0, 2 pi), per-inclusion k_in/k_out ~ U(lo, hi).
    """
    rng = np.random.default_rng(seed)
    inc = []
    for iy in range(ny):
        for ix in range(nx):
            a = rng.uniform(0.0, amax, size=5)
            ph = rng.uniform(0.0, 2 * math.pi, size=5)
            ratio = rng.uniform(ratio_lo, ratio_hi)
            inc.append(_inclusion(SHAPE_FOURIER, ix * spacing, iy * spacing, 0.0,
                                  [r0, *a, *ph], n, ratio * k_out))
    return {"k_out": float(k_out), "inclusions": inc, "grid_nx": nx, "grid_ny": ny,
            "spacing": float(spacing)}


def ellipse_batch(count=64, seed=3, m_lo=4, m_hi=400, spacing=1.0, n_lo=64, n_hi=256):
    """Independent problems with uneven sizes: ellipses on square-ish grids,
    m ~ U{m_lo..m_hi}, n ~ U{n_lo, n_lo+32, .., n_hi}, k0 = 2 pi L / (cols spacing)
    with L ~ U(2, 25) wavelengths per grid side, k1/k0 ~ U(1.5, 3)."""
    rng = np.random.default_rng(seed)
    probs = []
    for _ in range(count):
        m = int(rng.integers(m_lo, m_hi + 1))
        cols = int(math.ceil(math.sqrt(m)))
        rows = int(math.ceil(m / cols))
        n = int(rng.choice(np.arange(n_lo, n_hi + 1, 32)))
        lam = rng.uniform(2.0, 25.0)
        k_out = 2 * math.pi * lam / (spacing * cols)
        inc = []
        for j in range(m):
            a, b = rng.uniform(0.2, 0.45, size=2)
            rot = rng.uniform(0.0, math.pi)
            ratio = rng.uniform(1.5, 3.0)
            inc.append(_inclusion(SHAPE_ELLIPSE, (j % cols) * spacing, (j // cols) * spacing,
                                  rot, [a, b], n, ratio * k_out))
        probs.append({"k_out": float(k_out), "inclusions": inc, "grid_nx": cols,
                      "grid_ny": rows, "spacing": float(spacing)})
    return probs


def random_arrangement(m, seed=6, box=4.0, min_gap=0.12, n=96, k_out=2 * math.pi, k_ratio=2.0):
    """m ellipses (semi-axes ~ U(0.2, 0.4), orientation ~ U[0, pi)) at random
    positions in a box x box square, not on a grid (spacing 0): centres drawn
    one by one and kept when the bounding circles stay min_gap apart."""
    rng = np.random.default_rng(seed)
    inc, cs, rs = [], [], []
    tries = 0
    while len(inc) < m:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place the inclusions")
        a, b = rng.uniform(0.2, 0.4, size=2)
        c = rng.uniform(0.0, box, size=2)
        r = max(a, b)
        if any(np.hypot(*(c - c2)) < r + r2 + min_gap for c2, r2 in zip(cs, rs)):
            continue
        cs.append(c)
        rs.append(r)
        inc.append(_inclusion(SHAPE_ELLIPSE, c[0], c[1], rng.uniform(0.0, math.pi), [a, b], n, k_ratio * k_out))
    return {"k_out": float(k_out), "inclusions": inc, "grid_nx": 0, "grid_ny": 0, "spacing": 0.0}


def plane_wave_angles(count, seed=2):
    """Incidence angles ~ U[0, 2 pi) for multi-RHS solves."""
    return np.random.default_rng(seed).uniform(0.0, 2 * math.pi, size=count).tolist()


# Named workloads ----------------------------------------------------------------

def config_fp64_small():
    """2x2 circles r=0.4, k0=2pi, k1=4pi, n=64 (N=512), one level, tol 1e-12, 64 proxies."""
    prob = circle_grid(2, 2)
    opts = {"tol": 1e-12, "proxy_points": 64, "proxy_factor": 1.5}
    return prob, opts, [math.radians(30.0)]


def config_star16(nx=16, ny=16, n=128):
    """16x16 stars, k0 = 2 pi 20/16, k1 = 2 k0, n=128 (N=65,536), tol 1e-10, 8 RHS."""
    prob = star_grid(nx, ny, n=n, seed=1)
    opts = {"tol": 1e-10, "proxy_points": 0, "proxy_factor": 1.5}
    return prob, opts, plane_wave_angles(8, seed=2)


def config_fourier64(nx=64, ny=64, n=128):
    """64x64 random smooth shapes r = 0.4 (1 + sum_{m=2..6} a_m cos(m t + phi_m)),
    a_m ~ U(0, 0.04), per-inclusion k1/k0 ~ U(1.5, 3) (seed 4), k0 = 5,
    n = 128 (N = 1,048,576), tol 1e-9, 8 RHS."""
    prob = fourier_grid(nx, ny, n=n, seed=4, k_out=5.0)
    opts = {"tol": 1e-9, "proxy_points": 0, "proxy_factor": 1.5}
    return prob, opts, plane_wave_angles(8, seed=2)


def config_lossy_small():
    """The 2x2 circle geometry with lossy interior k1 = 4 pi (1 + 0.05 i)."""
    prob = circle_grid(2, 2, k_in=4 * math.pi * (1 + 0.05j))
    opts = {"tol": 1e-12, "proxy_points": 64, "proxy_factor": 1.5}
    return prob, opts, [math.radians(30.0)]


def num_unknowns(prob):
    return sum(2 * inc["n"] for inc in prob["inclusions"])
