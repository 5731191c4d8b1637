// Batched complex dense linear algebra used by the factorization: GEMM,
// partial-pivot LU and LU solves for many variable-size matrices at once.
// All matrices are column-major with interleaved complex entries.
#pragma once
#include <cuda_runtime.h>
#include "pm_common.cuh"

template <typename C>
struct GemmDesc {      // Cm = alpha * A(m x k) * B(k x n) + beta * Cm
  int m, n, k;
  const C* A; int lda;
  const C* B; int ldb;
  C* Cm; int ldc;
  C alpha, beta;
  int beta_zero;       // 1: Cm is write-only (beta ignored)
};

template <typename C>
struct LuProb {        // in-place LU of the leading m x m block of A
  C* A; int m; int ld;
  int* ipiv;           // m entries, 0-based row interchanged with row i at step i
  int* info;           // set to (first zero-pivot column + 1); 0 if none
};

template <typename C>
struct SolveProb {     // B (m x nrhs) <- A^{-1} B using the LU of A
  const C* A; int m; int ld;
  const int* ipiv;
  C* B; int ldb; int nrhs;
};

// Host launchers (dense_la.cu).  Descriptors live in device memory.
template <typename C>
void la_gemm_batched(const GemmDesc<C>* d_desc, const int* d_tile_off, int nprob, int total_tiles,
                     cudaStream_t st);
// h_m: host copy of the matrix sizes (flop accounting for the optional profiler)
template <typename C>
void la_getrf_batched(const LuProb<C>* d_prob, int nprob, int maxm, const int* h_m, cudaStream_t st);
// d_sync / d_err (optional, device): for one matrix with at most 8
// right-hand sides each triangle runs as one chained launch (k_trsv_chain);
// d_sync holds la_getrs_sync_ints(maxm) ints (zeroed by the call) and
// *d_err is set to 1 if one of its bounded waits runs out (results invalid).
// debug_no_flag (failure-path tests): the chained launches first wait, with
// a 1 ms bound, on a flag that nothing sets.
int la_getrs_sync_ints(int maxm);
template <typename C>
void la_getrs_batched(const SolveProb<C>* d_prob, int nprob, int maxm, int maxrhs, const int* h_m,
                      const int* h_rhs, cudaStream_t st, int* d_sync = nullptr, int* d_err = nullptr,
                      int debug_no_flag = 0);

// tiles of a GEMM problem for the 32 x 32 output tiling
inline int gemm_tiles(int m, int n) { return ((m + 31) / 32) * ((n + 31) / 32); }

// Output tile shapes of the batched GEMM (shape 0 is la_gemm_batched's 32 x 32).
// All shapes sum over k in the same order, so they give bit-identical results.
struct GemmShape { int tm, tn; };
constexpr int GEMM_NSHAPES = 5;
extern const GemmShape kGemmShapes[GEMM_NSHAPES];
inline int gemm_tiles_shape(int shape, int m, int n) {
  const GemmShape s = kGemmShapes[shape];
  return ((m + s.tm - 1) / s.tm) * ((n + s.tn - 1) / s.tn);
}
// d_tile_off: prefix sums of gemm_tiles_shape(shape, m, n) over the problems.
template <typename C>
void la_gemm_batched_shape(int shape, const GemmDesc<C>* d_desc, const int* d_tile_off, int nprob, int total_tiles,
                           cudaStream_t st);
