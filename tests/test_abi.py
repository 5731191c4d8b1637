"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pmchwt.h")).read()
    return sorted(set(re.findall(r"\b(pm_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2603_09381_gb300.build import build_library
    import ctypes
    lib = ctypes.CDLL(build_library())
    names = _declared()
    assert "pm_factorize" in names and "pm_solve" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_declares_every_symbol():
    from paper_2603_09381_gb300 import pmchwt
    assert sorted(pmchwt.EXPORTS) == _declared()


def test_calls_fail_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2603_09381_gb300 import pmchwt as pm
    from paper_2603_09381_gb300 import workloads as wl
    with pytest.raises(pm.PmError) as e:
        pm.Geometry(wl.circle_grid(1, 1))
    assert e.value.status == 3  # PM_ERR_CUDA: no CPU fallback


def test_release_cached_memory_without_gpu_is_a_no_op():
    from paper_2603_09381_gb300 import pmchwt as pm
    assert pm.release_cached_memory() == 0


def test_invalid_arguments_rejected_before_device_use():
    from paper_2603_09381_gb300 import pmchwt as pm
    from paper_2603_09381_gb300 import workloads as wl
    prob = wl.circle_grid(1, 1)
    prob["inclusions"][0]["n"] = 15
    with pytest.raises(pm.PmError) as e:
        pm.Geometry(prob)
    assert e.value.status == 1
    prob = wl.circle_grid(1, 1, k_in=3 - 0.1j)   # gain medium: Im k- < 0 is rejected
    with pytest.raises(pm.PmError) as e:
        pm.Geometry(prob)
    assert e.value.status == 1


def test_more_invalid_arguments_rejected_before_device_use():
    """Argument checks at the C boundary come before any CUDA call, so they hold
    on a machine without a GPU: each returns PM_ERR_INVALID_ARG (1) with a message."""
    import ctypes as ct
    from paper_2603_09381_gb300 import pmchwt as pm
    from paper_2603_09381_gb300 import workloads as wl
    lib = pm.load()
    one = (ct.c_float * 2)(1.0, 0.0)
    zero = (ct.c_float * 2)(0.0, 0.0)
    buf = ct.c_void_p(16)   # never dereferenced: every call below fails its checks first
    # tensor-core GEMM: leading dimensions below the matrix sizes, negative sizes, NULL scalars
    assert lib.pm_gemm_c32(8, 8, 8, buf, 4, 0, buf, 8, 0, buf, 8, one, zero, None) == 1
    assert lib.pm_gemm_c32(8, 16, 8, buf, 8, 0, buf, 8, 1, buf, 8, one, zero, None) == 1  # conj_b needs ldb >= n
    assert lib.pm_gemm_c32(-1, 8, 8, buf, 8, 0, buf, 8, 0, buf, 8, one, zero, None) == 1
    assert lib.pm_gemm_c32(8, 8, 8, buf, 8, 0, buf, 8, 0, buf, 8, None, zero, None) == 1
    assert b"pm_gemm_c32" in lib.pm_last_error()
    # NULL arguments and a non-positive inclusion count
    out = ct.c_void_p()
    assert lib.pm_build_geometry(None, ct.byref(out)) == 1
    p, arr = pm.make_problem(wl.circle_grid(1, 1))
    p.m = 0
    assert lib.pm_build_geometry(ct.byref(p), ct.byref(out)) == 1
    assert lib.pm_factorize(None, None, ct.byref(out)) == 1
    assert lib.pm_solve(None, None, 1, None, 0) == 1
    assert lib.pm_factor_stats(None, None) == 1
    # allocation-free self block: NULL geometry or output
    assert lib.pm_self_block_noalloc(None, 0, buf) == 1
    assert lib.pm_self_block_noalloc(None, 0, None) == 1
    assert b"pm_self_block_noalloc" in lib.pm_last_error()
    # peak measurement: unknown pipe, non-positive or excessive duration, NULL output
    v = ct.c_double()
    assert lib.pm_measure_peak(2, 10.0, ct.byref(v), None) == 1
    assert lib.pm_measure_peak(0, 0.0, ct.byref(v), None) == 1
    assert lib.pm_measure_peak(0, 1e6, ct.byref(v), None) == 1
    assert lib.pm_measure_peak(1, 10.0, None, None) == 1


def _bad(field, value):
    def edit(prob):
        inc = prob["inclusions"][0]
        if field in ("k_out", "spacing"):
            prob[field] = value
        elif field == "prm0":
            inc["prm"][0] = value
        elif field == "prm5":
            inc["prm"][5] = value
        else:
            inc[field] = value
    return edit


@pytest.mark.parametrize("field,value,word", [
    ("shape", 4, "shape"), ("shape", -1, "shape"), ("n", 8, "n_nodes"), ("n", 4098, "n_nodes"),
    ("n", 65, "n_nodes"), ("cx", float("nan"), "centre"), ("rot", float("inf"), "centre"),
    ("prm0", 0.0, "size"), ("prm5", float("nan"), "shape parameter"), ("k_in", -2.0 + 0j, "positive real"),
    ("k_in", 0.0 + 1j, "positive real"), ("k_in", 3.0 - 1e-3j, "Im"), ("k_out", 0.0, "k_out"),
    ("k_out", float("nan"), "k_out"), ("spacing", -1.0, "spacing")])
def test_each_invalid_descriptor_field_is_named(field, value, word):
    """Every descriptor check of pm_build_geometry runs before the first CUDA
    call: PM_ERR_INVALID_ARG and a message naming the field, with or without a GPU."""
    from paper_2603_09381_gb300 import pmchwt as pm
    from paper_2603_09381_gb300 import workloads as wl
    prob = wl.circle_grid(2, 1)
    _bad(field, value)(prob)
    with pytest.raises(pm.PmError) as e:
        pm.Geometry(prob)
    assert e.value.status == 1
    assert word in str(e.value)


def test_predictor_and_batch_entry_points_check_arguments_first():
    """Sizes, counts, dtypes and NULL pointers are checked before any CUDA call."""
    import ctypes as ct
    from paper_2603_09381_gb300 import pmchwt as pm
    lib = pm.load()
    p = ct.c_void_p(16)          # never dereferenced: each call fails its checks first
    assert lib.pm_mlp_forward(2, p, 4, p, p, None) == 1                     # dtype
    assert lib.pm_mlp_forward(0, p, -1, p, p, None) == 1                    # batch size
    assert lib.pm_mlp_forward(0, None, 4, p, p, None) == 1
    assert lib.pm_mlp_loss_grad(0, p, 0, p, p, 1e-3, p, p, None) == 1        # empty batch
    assert lib.pm_mlp_adam_step(1, p, p, p, p, 0, 1e-3, 0.9, 0.999, 1e-8, None) == 1   # step count from 1
    assert lib.pm_mlp_train(p, 16, p, p, 0, 8, 1e-3, 0.0, 1, None, None) == 1          # no epochs
    assert lib.pm_mlp_train(p, 16, p, p, 4, 0, 1e-3, 0.0, 1, None, None) == 1          # no batch
    arr = (ct.c_void_p * 1)(16)
    opts = pm.pm_factor_opts()
    assert lib.pm_factor_batch(arr, 0, ct.byref(opts), arr, 1) == 1                      # empty batch
    assert lib.pm_factor_batch(arr, 1, None, arr, 1) == 1
    assert lib.pm_solve_batch(arr, 1, arr, 0, arr, 0, 1) == 1                            # no right-hand sides
    assert b"pm_solve_batch" in lib.pm_last_error()


def test_factor_options_marshalling(monkeypatch):
    """The binding's keyword options land in pm_factor_opts as the header
    defines them (checked with a stand-in for the library)."""
    import ctypes as ct
    from paper_2603_09381_gb300 import pmchwt as pm
    seen = {}

    class FakeLib:
        def pm_factorize(self, gh, optp, outp):
            o = ct.cast(optp, ct.POINTER(pm.pm_factor_opts)).contents
            seen.update({f: getattr(o, f) for f, _ in pm.pm_factor_opts._fields_})
            return 0

        def pm_factor_free(self, h):
            pass

    monkeypatch.setattr(pm, "load", lambda path=None: FakeLib())

    class G:
        h = ct.c_void_p(16)

    cases = [({}, 0), ({"profile": True}, pm.PM_FLAG_PROFILE), ({"dense_operator": False}, pm.PM_FLAG_NO_DENSE_OPERATOR),
             ({"qr_first": False}, pm.PM_FLAG_NO_QR_FIRST), ({"tensor_cores": True}, pm.PM_FLAG_TENSOR_CORES),
             ({"ff_confirm": False}, pm.PM_FLAG_FP64_CONFIRM),
             ({"ff_confirm": False, "qr_first": False, "profile": True},
              pm.PM_FLAG_FP64_CONFIRM | pm.PM_FLAG_NO_QR_FIRST | pm.PM_FLAG_PROFILE)]
    for kw, flags in cases:
        seen.clear()
        f = pm.Factor(G(), 1e-9, 1.7, 48, precision=pm.PM_MIXED, refine_tol=1e-11, max_refine=7, low_tol=4e-6, **kw)
        f.h = None
        assert seen["flags"] == flags, kw
        assert (seen["tol"], seen["proxy_factor"], seen["proxy_points"], seen["precision"]) == (1e-9, 1.7, 48, 1)
        assert (seen["refine_tol"], seen["max_refine"], seen["low_tol"]) == (1e-11, 7, 4e-6)
        assert not seen["stream"] and not seen["rank_model"]
