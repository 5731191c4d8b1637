// Batched complex dense linear algebra used by the factorization: GEMM,
// partial-pivot LU and LU solves for many variable-size matrices at once.
// All matrices are column-major with interleaved complex entries.
#pragma once
#include <cuda_runtime.h>
#include <vector>
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
// Chained triangular solves (k_trsv_chain): with at most 8 right-hand sides
// per matrix, each triangle of every matrix of the batch runs in ONE launch
// whose blocks wait on one another through flags (bounded waits).
// la_chain_items fills the 2 x total ticket items (lower, then upper) for the
// matrix sizes h_m and `groups` groups of right-hand sides, and returns total
// = the number of (RS_NB-row block, group) pairs; a group holds rhs_per_cta
// columns (groups * rhs_per_cta >= the most right-hand sides of a matrix);
// the sync buffer holds la_chain_sync_ints(total) ints (zeroed by the call);
// *err is set to 1 if a wait runs out (the results are then invalid).
// no_flag (failure-path tests): every block first waits, with a 1 ms bound,
// on a flag that nothing sets.
struct ChainArgs {
  const int4* items;
  int total_blocks;   // items per triangle
  int* sync;
  int* err;
  int no_flag;
  int rhs_per_cta;    // 1 .. 8; at most 4 splits each product's two sums over two threads
};
int la_chain_items(const int* h_m, int nprob, int groups, std::vector<int4>& items);
int la_chain_sync_ints(int total);
template <typename C>
void la_getrs_batched(const SolveProb<C>* d_prob, int nprob, int maxm, int maxrhs, const int* h_m,
                      const int* h_rhs, cudaStream_t st, const ChainArgs* chain = nullptr);

// B (m x nrhs) <- U^{-1} B for the upper triangle U (diagonal included) of A,
// blocked (diagonal blocks of 32, then GEMM updates of the rows above);
// `name` and `flops` label the launches for the optional profiler.
template <typename C>
void la_trsm_upper_batched(const SolveProb<C>* d_prob, int nprob, int maxm, int maxrhs, const char* name,
                           double flops, cudaStream_t st);

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
