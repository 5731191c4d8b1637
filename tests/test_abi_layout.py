"""The ctypes binding mirrors include/pmchwt.h byte for byte.

A small C program, compiled with the host C compiler against the header,
prints every struct's size and every field's offset and the header's
constants; the ctypes classes and constants of the binding must agree.  A
mismatch would hand the library shifted fields without any error.
"""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pmchwt.h")

STRUCTS = ["pm_c64", "pm_inclusion", "pm_problem", "pm_factor_opts", "pm_solve_info", "pm_stats",
           "pm_kernel_stat", "pm_tune_entry"]


def _c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_2603_09381_gb300 import pmchwt as pm
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pmchwt.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("size {s} %zu\\n", sizeof({s}));')
        for f, _ in getattr(pm, s)._fields_:
            lines.append(f'  printf("off {s}.{f} %zu\\n", offsetof({s}, {f}));')
    text = open(HEADER).read()
    consts = re.findall(r"\b(PM_[A-Z0-9_]+)\s*=\s*\d+", text)
    for c in consts:
        lines.append(f'  printf("const {c} %d\\n", (int){c});')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), src, "-o", exe],
                       check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        kind, key, val = line.split()
        res[kind, key] = int(val)
    return res, consts


def test_struct_sizes_and_field_offsets_match_the_header():
    import ctypes as ct
    from paper_2603_09381_gb300 import pmchwt as pm
    c, _ = _c_layout()
    for s in STRUCTS:
        cls = getattr(pm, s)
        assert ct.sizeof(cls) == c["size", s], s
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == c["off", f"{s}.{f}"], f"{s}.{f}"


def test_constants_match_the_header():
    from paper_2603_09381_gb300 import pmchwt as pm
    from paper_2603_09381_gb300 import rank_predictor as rp
    c, consts = _c_layout()
    status = {v: k for k, v in pm.STATUS.items()}
    for name in consts:
        val = c["const", name]
        if name in status:
            assert status[name] == val, name
        elif name == "PM_MLP_NPARAM":
            assert rp.NPARAM == val
        elif name in ("PM_CIRCLE", "PM_ELLIPSE", "PM_STAR", "PM_FOURIER"):
            from paper_2603_09381_gb300 import workloads as wl
            assert getattr(wl, "SHAPE_" + name[3:]) == val, name
        else:
            assert getattr(pm, name) == val, name
    assert set(status) <= set(consts)
