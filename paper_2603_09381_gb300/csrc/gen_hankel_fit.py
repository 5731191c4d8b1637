"""Writes hankel_fit.h: polynomial fits of the modulus-phase functions of the
Hankel functions H_0 and H_1 on intervals of z in [8, 60).

For real z > 0 (DLMF 10.17, Abramowitz & Stegun 9.2.5-9.2.6),
    J_nu(z) = sqrt(2/(pi z)) (P_nu(z) cos chi - Q_nu(z) sin chi),
    Y_nu(z) = sqrt(2/(pi z)) (P_nu(z) sin chi + Q_nu(z) cos chi),
    chi = z - (nu/2 + 1/4) pi,
so P_nu = sqrt(pi z/2) (J_nu cos chi + Y_nu sin chi) and
Q_nu = sqrt(pi z/2) (Y_nu cos chi - J_nu sin chi).  P_nu - 1 and z Q_nu are
smooth, even functions of 1/z; on each interval [za, zb) they are fitted as
polynomials in x = (v - vm) / vh, v = 1/z^2, mapped onto [-1, 1]: Chebyshev
interpolation at Chebyshev points from 40-digit values (mpmath), converted to
monomial coefficients for Horner's rule.  Every fit is then checked: its
FP64 Horner evaluation is compared with 40-digit values of P_nu and Q_nu at
161 points of the interval and must stay within 2e-17 absolute.

Run from this directory (needs mpmath and numpy):  python gen_hankel_fit.py
(the header is committed; the build does not run this script).
"""
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 40
INTERVALS = [(8, 12, 8), (12, 20, 7), (20, 30, 5), (30, 60, 5)]   # (za, zb, degree)
NPTS = 64
TOL = 2e-17


def pq(nu, z):
    j, y = mp.besselj(nu, z), mp.bessely(nu, z)
    chi = z - (mp.mpf(nu) / 2 + mp.mpf(1) / 4) * mp.pi
    c, s = mp.cos(chi), mp.sin(chi)
    f = mp.sqrt(mp.pi * z / 2)
    return f * (j * c + y * s), f * (y * c - j * s)


def fit(za, zb, deg):
    va, vb = 1 / mp.mpf(za) ** 2, 1 / mp.mpf(zb) ** 2
    vm, vh = (va + vb) / 2, (va - vb) / 2
    zof = lambda x: 1 / mp.sqrt(vm + vh * x)
    xs = [mp.cos(mp.pi * (k + mp.mpf(1) / 2) / NPTS) for k in range(NPTS)]
    vals = {nu: [pq(nu, zof(x)) for x in xs] for nu in (0, 1)}
    out = {}
    for nu in (0, 1):
        for name, f in (("P", lambda p, q, x: p - 1), ("Q", lambda p, q, x: q * zof(x))):
            F = [f(p, q, x) for (p, q), x in zip(vals[nu], xs)]
            cheb = []
            for j in range(deg + 1):
                s = mp.fsum(F[k] * mp.cos(j * mp.pi * (k + mp.mpf(1) / 2) / NPTS) for k in range(NPTS))
                cheb.append(s * (2 if j else 1) / NPTS)
            mono = np.polynomial.chebyshev.cheb2poly([float(c) for c in cheb])
            worst = 0.0
            for x in np.linspace(-1.0, 1.0, 161):
                acc = 0.0
                for a in mono[::-1]:
                    acc = acc * x + a
                z = zof(mp.mpf(x))
                p, q = pq(nu, z)
                ref = p - 1 if name == "P" else q * z
                err = abs(ref - mp.mpf(acc))
                if name == "Q":
                    err /= z
                worst = max(worst, float(err))
            if worst > TOL:
                raise SystemExit(f"fit [{za}, {zb}) nu={nu} {name}: error {worst:.2e} > {TOL}")
            out[(name, nu)] = (mono, worst)
    return float(vm), float(1 / vh), out


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "// Generated by gen_hankel_fit.py (do not edit): polynomial fits of P_nu - 1",
        "// and z Q_nu (nu = 0, 1; Hankel's modulus-phase functions) in",
        "// x = (1/z^2 - vm) * ivh on [za, zb), as Horner's rule with FMAs; each",
        "// fit's FP64 Horner evaluation is within 2e-17 of 40-digit values of",
        "// P_nu and Q_nu on its interval.",
        "#pragma once",
        "",
    ]

    def horner(mono):
        e = repr(float(mono[-1]))
        for a in mono[-2::-1]:
            e = f"fma({e}, x, {float(a)!r})"
        return e

    for i, (za, zb, deg) in enumerate(INTERVALS):
        vm, ivh, out = fit(za, zb, deg)
        lines.append(f"// [{za}, {zb}): degree {deg}; worst errors " +
                     ", ".join(f"{k[0]}{k[1]} {v[1]:.1e}" for k, v in sorted(out.items())))
        lines.append(f"__device__ __forceinline__ void hankel_fit{i}(double v, double& P0, double& zQ0, "
                     "double& P1, double& zQ1) {")
        lines.append(f"  const double x = (v - {vm!r}) * {ivh!r};")
        lines.append(f"  P0 = 1.0 + {horner(out[('P', 0)][0])};")
        lines.append(f"  zQ0 = {horner(out[('Q', 0)][0])};")
        lines.append(f"  P1 = 1.0 + {horner(out[('P', 1)][0])};")
        lines.append(f"  zQ1 = {horner(out[('Q', 1)][0])};")
        lines.append("}")
        lines.append("")
    with open(os.path.join(here, "hankel_fit.h"), "w") as fh:
        fh.write("\n".join(lines))
    print("wrote hankel_fit.h")


if __name__ == "__main__":
    main()
