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
  C* R11;                        // k x k workspace (leading dimension k): R11 in pivot order
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

// Unpivoted blocked Householder QR of a tall Z (W x n, W > n) in place: the
// n x n triangle R ends in the top rows with zeros below its diagonal.  Column
// norms of every trailing block are those of Z, so the column-pivoted QR of R
// picks the pivots and R factor of Z's (exact arithmetic).
constexpr int QR_NB = 32;        // panel width
constexpr int QR_RB = 256;       // rows per block of the trailing update
template <typename C>
struct QrProb {
  C* Z; int ld; int W; int n;
  C* T;                          // QR_NB x QR_NB: compact-WY factor of the current panel
  C* V;                          // W x QR_NB (leading dimension W), or NULL: the panel's V
                                 // (rows j0.. at rows 0..) written out with its unit diagonal
  C* Yp;                         // update workspace: ceil(n/32) x mrb blocks of 32 x 32
  int mrb;                       // row blocks of QR_RB rows covering W
};
// Panels [j0, j0 + QR_NB) of every matrix with j0 < n; max_tiles = the most
// 32-column tiles right of a panel in any matrix.
template <typename C>
void qr_panel(const QrProb<C>* d_prob, int nprob, int j0, cudaStream_t st);
// max_rb: the most QR_RB-row blocks of rows j0..W-1 in any matrix.  With
// tc_err (complex64 only) the last step, C -= V Y, runs on the tensor cores
// (k_qr_apply_tc; max_w = the largest W), which set *tc_err if a bounded wait
// runs out; without it, on the CUDA cores.  no_arrive: see k_qr_apply_tc
// (tests of the timeout path).
template <typename C>
void qr_update(const QrProb<C>* d_prob, int nprob, int j0, int max_tiles, int max_rb, cudaStream_t st,
               int* tc_err = nullptr, int max_w = 0, bool no_arrive = false);
template <typename C>
void qr_zero_lower(const QrProb<C>* d_prob, int nprob, int max_n, cudaStream_t st);

void complete_perm(const PermFill* d_prob, int nprob, cudaStream_t st);
template <typename C>
void cpqr_init_norms(const CpqrProb<C>* d_prob, const CpqrChunk* d_chunk, int nchunk, cudaStream_t st);
// One elimination step (launch index t) of every active matrix; d_counter:
// a zeroed int, distinct for every launch (chunk dispenser).  tall: some
// complex64 matrix has W >= 2048 rows (selects the kernel instance with the
// register-resident column path).
template <typename C>
void cpqr_step(const CpqrProb<C>* d_prob, const CpqrChunk* d_chunk, int nchunk, int t, int* d_counter,
               cudaStream_t st, bool tall);
// R11 (upper triangular, diagonal from rdiag) and R12 of every problem gathered
// in pivot order into R11 and T (ldt = k), for a blocked triangular solve
// T <- R11^{-1} T; max_elems = the largest k * n.
template <typename C>
void interp_gather(const InterpProb<C>* d_prob, int nprob, size_t max_elems, cudaStream_t st);
template <typename C>
void scatter_interp(const ScatterProb<C>* d_prob, int nprob, int max_elems, cudaStream_t st);
template <typename S, typename D>
void copy_batched(const CopyProb<S, D>* d_prob, int nprob, int max_elems, cudaStream_t st);

constexpr int CPQR_CB = 16;      // columns per chunk
