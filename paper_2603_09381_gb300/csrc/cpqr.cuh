// Batched column-pivoted QR with fresh column norms and the interpolative
// decomposition built from it (paper Sec. 3: ID via CPQR, adaptive rank).
#pragma once
#include <cuda_runtime.h>
#include "pm_common.cuh"

enum { CPQR_FIND_RANK = 0, CPQR_EXTEND = 1 };

template <typename C>
struct CpqrProb {
  C* Z; int ld; int W; int n;    // W x n, factored in place (columns never move)
  double tol;
  int mode;                      // CPQR_FIND_RANK or CPQR_EXTEND
  int base;                      // steps already done when this phase starts
  int target;                    // stop before step `target`
  double* norm2;                 // 2 * n: squared trailing norms, ping-pong by step parity (-1: pivoted)
  int* perm;                     // perm[s] = column chosen at step s
  C* rdiag;                      // rdiag[s] = R_ss
  int* rank;                     // -1 until the rank criterion stops the factorization
  double* ref;                   // |R_11|
};

struct CpqrChunk { int id; int c0; int c1; int first; };

template <typename C>
struct InterpProb {              // T (k x (n-k)) = R11^{-1} R12 in pivot order
  const C* Z; int ld; int n; int k;
  const int* perm; const C* rdiag;
  C* T; int ldt;
};

template <typename C>
struct ScatterProb {             // dense L (rows = box positions) or R (columns = box positions)
  C* out; int ld; int off; int isL;
  const int* pos; const int* perm; int k; int ng;
  const C* T; int ldt;
};

template <typename S, typename D = S>
struct CopyProb { const S* src; int lds; D* dst; int ldd; int m; int n; };

struct PermFill { int* perm; int n; int done; };   // perm[done..n) <- unchosen columns, ascending

void complete_perm(const PermFill* d_prob, int nprob, cudaStream_t st);
template <typename C>
void cpqr_init_norms(const CpqrProb<C>* d_prob, const CpqrChunk* d_chunk, int nchunk, cudaStream_t st);
// One elimination step (launch index t) of every active matrix; d_counter:
// a zeroed int, distinct for every launch (chunk dispenser).
template <typename C>
void cpqr_step(const CpqrProb<C>* d_prob, const CpqrChunk* d_chunk, int nchunk, int t, int* d_counter,
               cudaStream_t st);
template <typename C>
void interp_solve(const InterpProb<C>* d_prob, int nprob, int max_cols, cudaStream_t st);
template <typename C>
void scatter_interp(const ScatterProb<C>* d_prob, int nprob, int max_elems, cudaStream_t st);
template <typename S, typename D>
void copy_batched(const CopyProb<S, D>* d_prob, int nprob, int max_elems, cudaStream_t st);

constexpr int CPQR_CB = 16;      // columns per chunk
