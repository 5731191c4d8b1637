"""The batched-GEMM autotuner: tuning picks the fastest tile shape per batch
class and changes no result.

Runs in a fresh process, so that the process-wide cache of tuned classes
starts empty: a factorization with tuning off (every batch on the 32 x 32
tile), one that tunes every class it meets, and one that reuses the cached
choices.  FP64 solutions must be bit-identical.  In the mixed mode the
factorizations must be identical (K, ranks per level) and the refined
solutions agree to 1e-11: the refinement's dense products add column-split
partial sums with FP64 atomics, so mixed solves reproduce to ~1e-13 from
run to run, not bit for bit.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import __graft_entry__
__graft_entry__.build()
from paper_2603_09381_gb300 import pmchwt as pm
from paper_2603_09381_gb300 import workloads as wl
out = {}
for prec in (pm.PM_FP64, pm.PM_MIXED):
    prob = wl.star_grid(4, 4, n=64, seed=4)
    g = pm.Geometry(prob)
    F = g.plane_wave([0.2, 1.3])
    sols, st = [], []
    for tune in (False, True, True):
        f = pm.Factor(g, 1e-10, precision=prec, autotune=tune)
        sols.append(f.solve(F))
        st.append((f.stats()["K"], f.stats()["skeleton"]))
    out[str(prec)] = {"equal": [bool(np.array_equal(sols[0], s)) for s in sols[1:]],
                      "rel": [float(np.linalg.norm(s - sols[0]) / np.linalg.norm(sols[0])) for s in sols[1:]],
                      "same_factor": [st[0] == t for t in st[1:]]}
out["table"] = pm.autotune_table()
print(json.dumps(out))
"""


def test_tuning_changes_no_result_and_keeps_the_fastest_shape():
    code = "ROOT = " + repr(ROOT) + "\n" + SCRIPT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["0"]["equal"] == [True, True]     # FP64: tuned and cached runs equal the untuned one bit for bit
    assert res["1"]["same_factor"] == [True, True]   # mixed: the same factorization
    assert max(res["1"]["rel"]) < 1e-11                # and the same refined solution up to the atomics' rounding
    table = res["table"]
    assert table, "no batch class was tuned"
    shapes = [(32, 32), (64, 64), (64, 32), (128, 8), (64, 16)]
    for e in table:
        assert tuple(e["tile"]) in shapes
        ms = e["ms"]
        assert all(t > 0 for t in ms)
        assert ms[shapes.index(tuple(e["tile"]))] == min(ms)
        assert e["uses"] >= 1
    print(f"{len(table)} tuned classes; non-default choices: "
          f"{sum(tuple(e['tile']) != (32, 32) for e in table)}")
