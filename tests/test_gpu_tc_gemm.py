"""Tensor-core complex64 GEMM (tcgen05, kind::tf32 with a three-term split)
against the complex128 product of the same float32 inputs.

The three-term split keeps FP32 accuracy: a wrong operand layout gives O(1)
errors and a tf32-only product ~1e-3, both far outside the bound used here
(FP32 rounding of a k-term sum, relative to |alpha| |op(A)| |op(B)| + |beta| |C|).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_09381_gb300 import pmchwt as pm
    return pm


def _rand(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def _dev(a):
    # column-major device copy: a torch tensor of the transpose is contiguous
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda()


def _run(pm, m, n, k, conj_a, conj_b, alpha, beta, seed):
    rng = np.random.default_rng(seed)
    A = _rand(rng, (k, m) if conj_a else (m, k))
    B = _rand(rng, (n, k) if conj_b else (k, n))
    C0 = _rand(rng, (m, n))
    dA, dB, dC = _dev(A), _dev(B), _dev(C0)
    pm.gemm_c32(m, n, k, dA.data_ptr(), max(A.shape[0], 1), conj_a, dB.data_ptr(), max(B.shape[0], 1), conj_b,
                dC.data_ptr(), m, alpha, beta)
    torch.cuda.synchronize()
    got = dC.cpu().numpy().T
    opA = A.astype(np.complex128).conj().T if conj_a else A.astype(np.complex128)
    opB = B.astype(np.complex128).conj().T if conj_b else B.astype(np.complex128)
    ref = alpha * (opA @ opB) + beta * C0.astype(np.complex128)
    scale = abs(alpha) * (np.abs(opA) @ np.abs(opB)) + abs(beta) * np.abs(C0) + 1e-30
    return np.max(np.abs(got - ref) / scale), k


@pytest.mark.parametrize("m,n,k", [(64, 32, 16), (100, 45, 37), (200, 97, 300), (5, 3, 1), (130, 70, 1000)])
@pytest.mark.parametrize("conj_a,conj_b", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_tc_gemm_matches_complex128(m, n, k, conj_a, conj_b):
    pm = _lib()
    err, kk = _run(pm, m, n, k, conj_a, conj_b, 0.75 - 0.5j, 0.25 + 1.0j, seed=m * 7 + n + k + 3 * conj_a + conj_b)
    assert err < (kk + 4) * 2.0 ** -22, err


def test_tc_gemm_empty_k_scales_c():
    pm = _lib()
    err, _ = _run(pm, 40, 20, 0, 0, 0, 1.0, -2.0 + 0.5j, seed=11)
    assert err < 1e-6


def test_tc_gemm_identity_reproduces_b():
    """op(A) = I: every output entry is one input entry (layout check)."""
    pm = _lib()
    rng = np.random.default_rng(5)
    m, n = 96, 40
    A = np.eye(m, dtype=np.complex64)
    B = _rand(rng, (m, n))
    dA, dB, dC = _dev(A), _dev(B), _dev(np.zeros((m, n), np.complex64))
    pm.gemm_c32(m, n, m, dA.data_ptr(), m, 0, dB.data_ptr(), m, 0, dC.data_ptr(), m)
    got = dC.cpu().numpy().T
    assert np.max(np.abs(got - B) / np.abs(B).max()) < 2.0 ** -21
