// Batched complex64 GEMM on the fifth-generation tensor cores (tcgen05,
// kind::tf32 with a three-term split for FP32 accuracy).
#pragma once
#include <cuda_runtime.h>
#include "pm_common.cuh"

// C = alpha * op(A) op(B) + beta * C, all complex64, column-major.
// op(A) is m x k: A itself (lda >= m) or, with conj_a, the conjugate
// transpose of a stored k x m matrix (lda >= k).  op(B) is k x n: B (ldb >= k)
// or, with conj_b, the conjugate transpose of a stored n x k matrix.
struct TcGemmProb {
  const float2* A; int lda; int conj_a;
  const float2* B; int ldb; int conj_b;
  float2* C; int ldc;
  int m, n, k;
  float2 alpha, beta;
};

constexpr int TC_TM = 64;   // complex rows per tile (128 real rows of the MMA)
constexpr int TC_TN = 32;   // complex columns per tile

inline int tc_tiles(int m, int n) { return ((m + TC_TM - 1) / TC_TM) * ((n + TC_TN - 1) / TC_TN); }

// d_tile_off[i] = first tile of problem i (prefix sums of tc_tiles, which may
// start at tile_base: then d_tile_off[0] == tile_base), total_tiles = the
// tiles of the nprob problems; d_err: an int the kernel sets nonzero when a
// wait on the tensor cores runs out (the launch's results are then invalid).
// no_arrive (tests of the timeout path): every CTA first waits, with a bound
// of about a millisecond, on a barrier that nothing arrives at, then skips
// its tile, frees its tensor memory and sets *d_err, having issued no copy
// and no MMA.
void tc_gemm_batched(const TcGemmProb* d_prob, const int* d_tile_off, int nprob, int total_tiles, int* d_err,
                     cudaStream_t st, int tile_base = 0, bool no_arrive = false);
