"""Write the proxy oracle's complex128 factorization of the 16 x 16 star grid
(n = 128 nodes per star, N = 65,536 unknowns, ID threshold 1e-10, eight
plane waves) to ``star16_fp64_oracle.npz`` beside this script.

Calls only ``oracle/`` and the seeded workload descriptors; nothing comes
from the CUDA path.  Stored (compressed NumPy archive):

  K            size of the top-level dense system
  ranks        per level (1..L): sum of the box ranks
  skel_level, skel_box, skel_off, skel_rows, skel_cols
               the selected global row and column indices of every box
               (box b of level l owns skel_rows[skel_off[i]:skel_off[i+1]]
               for i the position of (l, b) in skel_level / skel_box)
  margin       per box: the smallest decision margin of its four IDs in
               rounding units eps |R_11| (oracle/cpqr.py); a second
               implementation may choose another skeleton only where it
               rounds by that much
  idx, phi     the solution at 4,096 sampled unknowns (seeded), all eight
               right-hand sides, and its full column norms (phi_norm)
  angles       incidence angles of the right-hand sides

Run: python tests/golden/make_star16_oracle.py   (about 10 minutes on 8 cores)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import dense, proxy  # noqa: E402
from paper_2603_09381_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(HERE, "star16_fp64_oracle.npz")


def main():
    prob, opts, angs = wl.config_star16()
    t0 = time.time()
    fo = proxy.factor(prob, opts)
    t1 = time.time()
    F = np.stack([dense.plane_wave(prob, a) for a in angs], 1)
    phi = proxy.solve(fo, F)
    t2 = time.time()
    lv, bx, off, rows, cols, marg = [], [], [0], [], [], []
    for lev in range(1, fo["L"] + 1):
        for b in range(len(fo["tree"]["levels"][lev])):
            d = fo["data"][lev, b]
            lv.append(lev)
            bx.append(b)
            rows.append(np.asarray(d["srows"], np.int32))
            cols.append(np.asarray(d["scols"], np.int32))
            off.append(off[-1] + len(d["srows"]))
            marg.append(d["margin"])
    idx = np.sort(np.random.default_rng(11).choice(fo["N"], 4096, replace=False))
    ranks = [sum(sum(k) for k in fo["stats"]["ranks"][lev]) for lev in range(1, fo["L"] + 1)]
    np.savez_compressed(OUT, K=fo["stats"]["K"], ranks=np.array(ranks), skel_level=np.array(lv, np.int32),
                        skel_box=np.array(bx, np.int32), skel_off=np.array(off, np.int64),
                        skel_rows=np.concatenate(rows), skel_cols=np.concatenate(cols), margin=np.array(marg),
                        idx=idx, phi=phi[idx], phi_norm=np.linalg.norm(phi, axis=0), angles=np.array(angs))
    print(f"K={fo['stats']['K']} ranks={ranks} factor {t1 - t0:.0f} s solve {t2 - t1:.0f} s "
          f"min margin {min(marg):.3g} -> {OUT}")


if __name__ == "__main__":
    main()
