"""ctypes binding of libpmchwt.so: the same entry points as include/pmchwt.h.

Argument marshalling only; every step of the solver runs in the CUDA
library.  Loading fails loudly if the library has not been built (there is
no CPU fallback).
"""
import ctypes as ct
import os

import numpy as np

from .build import LIB

PM_OK = 0
STATUS = {0: "PM_OK", 1: "PM_ERR_INVALID_ARG", 2: "PM_ERR_OOM", 3: "PM_ERR_CUDA", 4: "PM_ERR_SINGULAR",
          5: "PM_ERR_NOT_CONVERGED", 6: "PM_ERR_TIMEOUT", 7: "PM_ERR_GEOMETRY", 8: "PM_ERR_UNSUPPORTED"}
PM_FP64 = 0
PM_MIXED = 1
PM_FORM_OMIT = 0
PM_FORM_ALL = 1
PM_FORM_BM = 2
PM_FORM_BM_SIMPLIFIED = 3


class PmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class pm_c64(ct.Structure):
    _fields_ = [("re", ct.c_double), ("im", ct.c_double)]


class pm_inclusion(ct.Structure):
    _fields_ = [("shape", ct.c_int32), ("cx", ct.c_double), ("cy", ct.c_double), ("rot", ct.c_double),
                ("prm", ct.c_double * 16), ("n_nodes", ct.c_int32), ("k_in", pm_c64)]


class pm_problem(ct.Structure):
    _fields_ = [("m", ct.c_int32), ("inc", ct.POINTER(pm_inclusion)), ("k_out", ct.c_double),
                ("grid_nx", ct.c_int32), ("grid_ny", ct.c_int32), ("spacing", ct.c_double)]


class pm_factor_opts(ct.Structure):
    _fields_ = [("tol", ct.c_double), ("proxy_factor", ct.c_double), ("proxy_points", ct.c_int32),
                ("precision", ct.c_int32), ("stream", ct.c_void_p), ("flags", ct.c_uint32),
                ("refine_tol", ct.c_double), ("max_refine", ct.c_int32), ("low_tol", ct.c_double),
                ("rank_model", ct.c_void_p), ("debug_flags", ct.c_uint32), ("proxy_scale", ct.c_double),
                ("formulation", ct.c_int32), ("scratch_gb", ct.c_double)]


class pm_solve_info(ct.Structure):
    _fields_ = [("iterations", ct.c_int32), ("residual", ct.c_double), ("history", ct.c_double * 16)]


class pm_stats(ct.Structure):
    _fields_ = [("levels", ct.c_int32), ("N", ct.c_int32), ("K", ct.c_int32), ("skeleton", ct.c_int32 * 16),
                ("ms_assemble", ct.c_double), ("ms_id", ct.c_double), ("ms_schur", ct.c_double),
                ("ms_top", ct.c_double), ("ms_total", ct.c_double), ("cpqr_launches", ct.c_int32),
                ("rank_checks", ct.c_int32), ("predictor_fallbacks", ct.c_int32), ("ms_level", ct.c_double * 16),
                ("graph_captures", ct.c_int32), ("graph_launches", ct.c_int32), ("proxy_checked", ct.c_int32),
                ("proxy_fallbacks", ct.c_int32), ("id_rows", ct.c_int64), ("level_chunks", ct.c_int32)]


class pm_tune_entry(ct.Structure):
    _fields_ = [("device", ct.c_int32), ("complex_bytes", ct.c_int32), ("log2_m", ct.c_int32),
                ("log2_n", ct.c_int32), ("log2_k", ct.c_int32), ("log2_count", ct.c_int32), ("tm", ct.c_int32),
                ("tn", ct.c_int32), ("ms", ct.c_float * 8), ("uses", ct.c_int64)]


class pm_kernel_stat(ct.Structure):
    _fields_ = [("name", ct.c_char * 32), ("launches", ct.c_int32), ("ms", ct.c_double), ("work", ct.c_double)]


PM_FLAG_PROFILE = 1
PM_FLAG_NO_DENSE_OPERATOR = 2
PM_FLAG_NO_QR_FIRST = 4
PM_FLAG_TENSOR_CORES = 8
PM_FLAG_FF_CONFIRM = 16
PM_FLAG_FP64_CONFIRM = 32
PM_FLAG_NO_AUTOTUNE = 64
PM_FLAG_NO_GRAPHS = 128
PM_FLAG_PROXY_CHECK = 256
PM_FLAG_QR_CUDA_CORES = 512
PM_FLAG_TOP_FP64 = 1024
PM_FLAG_OPERATOR_AFTER = 2048
PM_DEBUG_SINGULAR_BLOCK = 1
PM_DEBUG_SINGULAR_COMPRESSED = 2
PM_DEBUG_UNDERPREDICT = 4
PM_DEBUG_TC_NO_ARRIVE = 8
PM_DEBUG_SOLVE_NO_FLAG = 16
_lib = None

EXPORTS = {
    "pm_build_geometry": (ct.c_int, [ct.POINTER(pm_problem), ct.POINTER(ct.c_void_p)]),
    "pm_geometry_size": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32)]),
    "pm_geometry_nodes": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "pm_plane_wave_rhs": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_int32]),
    "pm_factorize": (ct.c_int, [ct.c_void_p, ct.POINTER(pm_factor_opts), ct.POINTER(ct.c_void_p)]),
    "pm_solve": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_int32]),
    "pm_solve_ex": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_int32,
                               ct.POINTER(pm_solve_info)]),
    "pm_factor_stats": (ct.c_int, [ct.c_void_p, ct.POINTER(pm_stats)]),
    "pm_factor_batch": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.POINTER(pm_factor_opts), ct.c_void_p, ct.c_int32]),
    "pm_solve_batch": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_int32,
                                  ct.c_int32]),
    "pm_factor_skeleton": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_int32,
                                      ct.POINTER(ct.c_int32)]),
    "pm_matrix_entries": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_int32, ct.c_void_p]),
    "pm_self_block": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p]),
    "pm_far_field": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_int32,
                                ct.c_void_p]),
    "pm_scattered_field": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_int32,
                                      ct.c_void_p]),
    "pm_factor_profile": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int32, ct.POINTER(ct.c_int32)]),
    "pm_launch_counter": (ct.c_int, [ct.POINTER(ct.c_uint64)]),
    "pm_autotune_table": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.POINTER(ct.c_int32)]),
    "pm_factor_rank_data": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int32, ct.POINTER(ct.c_int32)]),
    "pm_factor_proxy_data": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int32, ct.POINTER(ct.c_int32)]),
    "pm_mlp_forward": (ct.c_int, [ct.c_int32, ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "pm_mlp_loss_grad": (ct.c_int, [ct.c_int32, ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_double,
                                    ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "pm_mlp_adam_step": (ct.c_int, [ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int32,
                                    ct.c_double, ct.c_double, ct.c_double, ct.c_double, ct.c_void_p]),
    "pm_mlp_train": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_int32,
                                ct.c_double, ct.c_double, ct.c_uint64, ct.c_void_p, ct.c_void_p]),
    "pm_self_block_noalloc": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p]),
    "pm_gemm_c32": (ct.c_int, [ct.c_int32, ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_void_p,
                               ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_int32, ct.POINTER(ct.c_float),
                               ct.POINTER(ct.c_float), ct.c_void_p]),
    "pm_measure_peak": (ct.c_int, [ct.c_int32, ct.c_double, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]),
    "pm_release_cached_memory": (ct.c_int, [ct.POINTER(ct.c_int64)]),
    "pm_factor_free": (None, [ct.c_void_p]),
    "pm_geometry_free": (None, [ct.c_void_p]),
    "pm_last_error": (ct.c_char_p, []),
}


def load(path=None):
    """Load libpmchwt.so (built by __graft_entry__.build()); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} not built: run __graft_entry__.build() (no CPU fallback)")
    lib = ct.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st):
    if st != PM_OK:
        raise PmError(st, load().pm_last_error().decode())


def make_problem(prob):
    """pm_problem (and the inclusion array it points to) from a workload descriptor dict."""
    m = len(prob["inclusions"])
    arr = (pm_inclusion * m)()
    for j, inc in enumerate(prob["inclusions"]):
        a = arr[j]
        a.shape = inc["shape"]; a.cx = inc["cx"]; a.cy = inc["cy"]; a.rot = inc["rot"]
        for i, v in enumerate(inc["prm"]):
            a.prm[i] = v
        a.n_nodes = inc["n"]
        a.k_in = pm_c64(complex(inc["k_in"]).real, complex(inc["k_in"]).imag)
    p = pm_problem(m, arr, float(prob["k_out"]), int(prob.get("grid_nx", 0)), int(prob.get("grid_ny", 0)),
                   float(prob["spacing"]))
    return p, arr


def gemm_c32(m, n, k, A_ptr, lda, conj_a, B_ptr, ldb, conj_b, C_ptr, ldc, alpha=1.0, beta=0.0, stream=None):
    """C = alpha op(A) op(B) + beta C on the tensor cores (device pointers, complex64, column-major)."""
    al = (ct.c_float * 2)(complex(alpha).real, complex(alpha).imag)
    be = (ct.c_float * 2)(complex(beta).real, complex(beta).imag)
    _check(load().pm_gemm_c32(m, n, k, A_ptr, lda, int(conj_a), B_ptr, ldb, int(conj_b), C_ptr, ldc, al, be,
                              ct.c_void_p(stream) if stream else None))


def measure_peak(which, ms_target=200.0):
    """(TFLOP/s, SM MHz during the loop) of the library's FMA loop on the current
    device: which 0 = FP64, 1 = FP32."""
    v, mhz = ct.c_double(), ct.c_double()
    _check(load().pm_measure_peak(int(which), float(ms_target), ct.byref(v), ct.byref(mhz)))
    return v.value, mhz.value


def release_cached_memory():
    """Free the device blocks the library keeps for reuse; returns the bytes freed."""
    n = ct.c_int64()
    _check(load().pm_release_cached_memory(ct.byref(n)))
    return n.value


def autotune_table():
    """The batched-GEMM autotuner's cached choices: one dict per batch class."""
    cnt = ct.c_int32()
    _check(load().pm_autotune_table(None, 0, ct.byref(cnt)))
    arr = (pm_tune_entry * max(cnt.value, 1))()
    _check(load().pm_autotune_table(arr, cnt.value, ct.byref(cnt)))
    return [{"device": e.device, "complex_bytes": e.complex_bytes, "log2_m": e.log2_m, "log2_n": e.log2_n,
             "log2_k": e.log2_k, "log2_count": e.log2_count, "tile": (e.tm, e.tn), "ms": list(e.ms)[:5],
             "uses": e.uses} for e in arr[: cnt.value]]


def launch_counter():
    v = ct.c_uint64()
    _check(load().pm_launch_counter(ct.byref(v)))
    return v.value


class Geometry:
    def __init__(self, prob):
        lib = load()
        p, self._arr = make_problem(prob)
        h = ct.c_void_p()
        _check(lib.pm_build_geometry(ct.byref(p), ct.byref(h)))
        self.h = h
        N, T = ct.c_int32(), ct.c_int32()
        _check(lib.pm_geometry_size(h, ct.byref(N), ct.byref(T)))
        self.N, self.total_nodes = N.value, T.value

    def nodes(self):
        xy = np.zeros((self.total_nodes, 2)); nrm = np.zeros((self.total_nodes, 2)); w = np.zeros(self.total_nodes)
        _check(load().pm_geometry_nodes(self.h, xy.ctypes.data, nrm.ctypes.data, w.ctypes.data))
        return xy, nrm, w

    def plane_wave(self, angles):
        angles = np.ascontiguousarray(angles, dtype=np.float64)
        out = np.zeros((len(angles), self.N), dtype=np.complex128)  # column-major N x nrhs
        _check(load().pm_plane_wave_rhs(self.h, angles.ctypes.data, len(angles), out.ctypes.data, 0))
        return out.T

    def plane_wave_device(self, angles, out_ptr):
        angles = np.ascontiguousarray(angles, dtype=np.float64)
        _check(load().pm_plane_wave_rhs(self.h, angles.ctypes.data, len(angles), out_ptr, 1))

    def matrix_entries(self, rows, cols):
        rows = np.ascontiguousarray(rows, dtype=np.int32); cols = np.ascontiguousarray(cols, dtype=np.int32)
        out = np.zeros((len(cols), len(rows)), dtype=np.complex128)
        _check(load().pm_matrix_entries(self.h, rows.ctypes.data, len(rows), cols.ctypes.data, len(cols),
                                        out.ctypes.data))
        return out.T

    def self_block(self, j, n):
        out = np.zeros((2 * n, 2 * n), dtype=np.complex128)
        _check(load().pm_self_block(self.h, j, out.ctypes.data))
        return out.T  # column-major -> row-major view

    def far_field(self, phi, angles):
        """u_inf at directions angles for host solutions phi (N,) or (N, nrhs)."""
        phi = np.asarray(phi, dtype=np.complex128)
        vec = phi.ndim == 1
        P = np.ascontiguousarray((phi[:, None] if vec else phi).T)
        ang = np.ascontiguousarray(angles, dtype=np.float64)
        out = np.zeros((P.shape[0], len(ang)), dtype=np.complex128)
        _check(load().pm_far_field(self.h, P.ctypes.data, P.shape[0], 0, ang.ctypes.data, len(ang), out.ctypes.data))
        return out[0] if vec else out.T

    def scattered_field(self, phi, points):
        """u^s at points (P x 2) for host solutions phi (N,) or (N, nrhs)."""
        phi = np.asarray(phi, dtype=np.complex128)
        vec = phi.ndim == 1
        P = np.ascontiguousarray((phi[:, None] if vec else phi).T)
        pts = np.ascontiguousarray(points, dtype=np.float64)
        out = np.zeros((P.shape[0], len(pts)), dtype=np.complex128)
        _check(load().pm_scattered_field(self.h, P.ctypes.data, P.shape[0], 0, pts.ctypes.data, len(pts),
                                         out.ctypes.data))
        return out[0] if vec else out.T

    def self_block_noalloc(self, j, out_ptr):
        """A_jj into a caller-owned device buffer, with no device allocation."""
        _check(load().pm_self_block_noalloc(self.h, j, out_ptr))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.pm_geometry_free(self.h)
            self.h = None


class Factor:
    def __init__(self, geom, tol, proxy_factor=1.5, proxy_points=0, precision=PM_FP64, stream=None,
                 profile=False, refine_tol=0.0, max_refine=0, low_tol=0.0, rank_model=None, dense_operator=True,
                 qr_first=True, tensor_cores=False, ff_confirm=True, debug_flags=0, autotune=True, graphs=True,
                 proxy_scale=0.0, proxy_check=False, formulation=PM_FORM_OMIT, scratch_gb=0.0,
                 qr_tensor_cores=True, top_fp64=False, operator_after=False):
        """rank_model: device pointer (int) of a trained predictor, or None;
        qr_tensor_cores: the QR-first update's C -= V Y on the tensor cores (default) or,
        with False, on the CUDA cores (PM_FLAG_QR_CUDA_CORES);
        top_fp64: PM_MIXED factors the top-level system in complex128 (PM_FLAG_TOP_FP64)
        instead of complex64;
        operator_after: PM_MIXED assembles the dense operator after the factorization
        (PM_FLAG_OPERATOR_AFTER) instead of beside it;
        ff_confirm: the refinement ends on the folded float-float product (default) or,
        with False, on the FP64 product (PM_FLAG_FP64_CONFIRM);
        debug_flags: PM_DEBUG_* fault injection for failure-path tests (0 in normal use)."""
        lib = load()
        self.geom = geom
        self.last_info = None
        o = pm_factor_opts(float(tol), float(proxy_factor), int(proxy_points), int(precision),
                           ct.c_void_p(stream) if stream else None,
                           (PM_FLAG_PROFILE if profile else 0) | (0 if dense_operator else PM_FLAG_NO_DENSE_OPERATOR)
                           | (0 if qr_first else PM_FLAG_NO_QR_FIRST) | (PM_FLAG_TENSOR_CORES if tensor_cores else 0)
                           | (0 if ff_confirm else PM_FLAG_FP64_CONFIRM) | (0 if autotune else PM_FLAG_NO_AUTOTUNE)
                           | (0 if graphs else PM_FLAG_NO_GRAPHS) | (PM_FLAG_PROXY_CHECK if proxy_check else 0)
                           | (0 if qr_tensor_cores else PM_FLAG_QR_CUDA_CORES)
                           | (PM_FLAG_TOP_FP64 if top_fp64 else 0)
                           | (PM_FLAG_OPERATOR_AFTER if operator_after else 0),
                           float(refine_tol), int(max_refine), float(low_tol),
                           ct.c_void_p(rank_model) if rank_model else None, int(debug_flags), float(proxy_scale),
                           int(formulation), float(scratch_gb))
        h = ct.c_void_p()
        _check(lib.pm_factorize(geom.h, ct.byref(o), ct.byref(h)))
        self.h = h

    def stats(self):
        s = pm_stats()
        _check(load().pm_factor_stats(self.h, ct.byref(s)))
        return {"levels": s.levels, "N": s.N, "K": s.K, "skeleton": list(s.skeleton)[: s.levels + 1],
                "ms_assemble": s.ms_assemble, "ms_id": s.ms_id, "ms_schur": s.ms_schur, "ms_top": s.ms_top,
                "ms_total": s.ms_total, "cpqr_launches": s.cpqr_launches, "rank_checks": s.rank_checks,
                "predictor_fallbacks": s.predictor_fallbacks, "ms_level": list(s.ms_level)[: s.levels + 1],
                "graph_captures": s.graph_captures, "graph_launches": s.graph_launches,
                "proxy_checked": s.proxy_checked, "proxy_fallbacks": s.proxy_fallbacks, "id_rows": s.id_rows,
                "level_chunks": s.level_chunks}

    def rank_data(self):
        """(X, T): features (n x 8) and, per box and group, (max(row rank, column rank) / n_g,
        proxy count used / the rule's count) (n x 2)."""
        cnt = ct.c_int32()
        _check(load().pm_factor_rank_data(self.h, None, None, 0, ct.byref(cnt)))
        X = np.zeros((cnt.value, 8), dtype=np.float32)
        T = np.zeros((cnt.value, 2), dtype=np.float32)
        _check(load().pm_factor_rank_data(self.h, X.ctypes.data, T.ctypes.data, cnt.value, ct.byref(cnt)))
        return X, T

    def proxy_data(self):
        """(ratio, redone) per sample of rank_data(): the held-out proxy check's
        ||H_J - H_S T|| / (tol ||H||) of the box (-1: not run) and whether the
        box was redone with the rule's proxy count."""
        cnt = ct.c_int32()
        _check(load().pm_factor_proxy_data(self.h, None, None, 0, ct.byref(cnt)))
        r = np.zeros(cnt.value, dtype=np.float32)
        d = np.zeros(cnt.value, dtype=np.int32)
        _check(load().pm_factor_proxy_data(self.h, r.ctypes.data, d.ctypes.data, cnt.value, ct.byref(cnt)))
        return r, d

    def profile(self):
        cnt = ct.c_int32()
        _check(load().pm_factor_profile(self.h, None, 0, ct.byref(cnt)))
        arr = (pm_kernel_stat * max(cnt.value, 1))()
        _check(load().pm_factor_profile(self.h, arr, cnt.value, ct.byref(cnt)))
        return {a.name.decode(): {"launches": a.launches, "ms": a.ms, "work": a.work} for a in arr[: cnt.value]}

    def solve(self, rhs):
        """Host solve: rhs (N,) or (N, nrhs) complex128 -> phi of the same shape."""
        rhs = np.asarray(rhs, dtype=np.complex128)
        vec = rhs.ndim == 1
        R = rhs[:, None] if vec else rhs
        nrhs = R.shape[1]
        buf = np.ascontiguousarray(R.T)  # column-major N x nrhs
        out = np.zeros_like(buf)
        info = pm_solve_info()
        _check(load().pm_solve_ex(self.h, buf.ctypes.data, nrhs, out.ctypes.data, 0, ct.byref(info)))
        self.last_info = {"iterations": info.iterations, "residual": info.residual,
                          "history": list(info.history)[: info.iterations]}
        phi = out.T
        return phi[:, 0] if vec else phi

    def solve_device(self, rhs_ptr, nrhs, phi_ptr):
        info = pm_solve_info()
        _check(load().pm_solve_ex(self.h, rhs_ptr, nrhs, phi_ptr, 1, ct.byref(info)))
        self.last_info = {"iterations": info.iterations, "residual": info.residual,
                          "history": list(info.history)[: info.iterations]}
        return self.last_info

    def skeleton(self, level, box, cap=100000):
        rows = np.zeros(cap, dtype=np.int32); cols = np.zeros(cap, dtype=np.int32); k = ct.c_int32()
        _check(load().pm_factor_skeleton(self.h, level, box, rows.ctypes.data, cols.ctypes.data, cap, ct.byref(k)))
        return rows[: k.value].copy(), cols[: k.value].copy()

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.pm_factor_free(self.h)
            self.h = None


def mlp_forward(dtype, theta_ptr, B, x_ptr, y_ptr, stream=None):
    _check(load().pm_mlp_forward(dtype, theta_ptr, B, x_ptr, y_ptr, stream))


def mlp_loss_grad(dtype, theta_ptr, B, x_ptr, t_ptr, lam, grad_ptr, loss_ptr, stream=None):
    _check(load().pm_mlp_loss_grad(dtype, theta_ptr, B, x_ptr, t_ptr, lam, grad_ptr, loss_ptr, stream))


def mlp_adam_step(dtype, theta_ptr, grad_ptr, m_ptr, v_ptr, t, lr, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    _check(load().pm_mlp_adam_step(dtype, theta_ptr, grad_ptr, m_ptr, v_ptr, t, lr, b1, b2, eps, stream))


def mlp_train(theta_ptr, nsamples, x_ptr, t_ptr, epochs, batch, lr, lam, seed, stream=None):
    hist = np.zeros(epochs)
    _check(load().pm_mlp_train(theta_ptr, nsamples, x_ptr, t_ptr, epochs, batch, lr, lam, seed,
                               hist.ctypes.data, stream))
    return hist


class _Handle:
    """A factor handle produced by factor_batch (same interface as Factor)."""

    def __init__(self, geom, h):
        self.geom, self.h, self.last_info = geom, h, None

    stats = Factor.stats
    proxy_data = Factor.proxy_data
    solve = Factor.solve
    solve_device = Factor.solve_device
    skeleton = Factor.skeleton
    profile = Factor.profile
    __del__ = Factor.__del__


def factor_batch(geoms, tol, precision=PM_FP64, workers=8, rank_model=None, **kw):
    """Factor independent problems concurrently (one stream per worker thread)."""
    n = len(geoms)
    o = pm_factor_opts(float(tol), float(kw.get("proxy_factor", 1.5)), int(kw.get("proxy_points", 0)),
                       int(precision), None, 0, float(kw.get("refine_tol", 0.0)), int(kw.get("max_refine", 0)),
                       float(kw.get("low_tol", 0.0)), ct.c_void_p(rank_model) if rank_model else None,
                       int(kw.get("debug_flags", 0)), float(kw.get("proxy_scale", 0.0)),
                       int(kw.get("formulation", PM_FORM_OMIT)), float(kw.get("scratch_gb", 0.0)))
    gh = (ct.c_void_p * n)(*[g.h.value for g in geoms])
    out = (ct.c_void_p * n)()
    _check(load().pm_factor_batch(gh, n, ct.byref(o), out, workers))
    return [_Handle(g, ct.c_void_p(out[i])) for i, g in enumerate(geoms)]


def solve_batch(factors, rhs_list, workers=8):
    """Host right-hand sides (N_i x nrhs complex128 each) -> solutions, solved concurrently."""
    n = len(factors)
    nrhs = rhs_list[0].shape[1]
    bufs = [np.ascontiguousarray(r.T) for r in rhs_list]
    outs = [np.zeros_like(b) for b in bufs]
    fh = (ct.c_void_p * n)(*[f.h.value for f in factors])
    rp = (ct.c_void_p * n)(*[b.ctypes.data for b in bufs])
    op = (ct.c_void_p * n)(*[o.ctypes.data for o in outs])
    _check(load().pm_solve_batch(fh, n, rp, nrhs, op, 0, workers))
    return [o.T for o in outs]
