// FP64 application of the PMCHWT (Omit) operator on the fly, used as the
// residual of iterative refinement in the mixed-precision mode, and small
// vector kernels for the refinement loop.
#pragma once
#include <cuda_runtime.h>
#include "pm_common.cuh"

struct OpNodes {
  const double *x, *y, *nx, *ny, *w;
  const int* incl;   // owning inclusion
  const int* iu;     // row of the node's u-equation = column of its q density
  const int* iq;     // row of the node's q-equation = column of its u density
};

// Y[:, 0:nrhs] += A_offdiag X[:, 0:nrhs]  (trapezoid-rule exterior kernels between
// different inclusions; same-inclusion pairs are skipped).
void apply_offdiag64(OpNodes nd, int total_nodes, double k0, const double2* X, int ldx, double2* Y, int ldy,
                     int nrhs, cudaStream_t st);
// The dense operator is stored split, in two planes of float2 with the same
// column-major layout: each complex entry a as hi = a truncated to 24
// significant bits (per part) and lo = the next 24 bits, so hi + lo is exact
// in FP64 and within 2^-47 of the entry, in 16 bytes; a product that needs
// only the hi parts reads half of them.
struct SplitOp {
  float2* hi;
  float2* lo;
  size_t ld;
  __host__ __device__ SplitOp at(size_t row, size_t col) const {
    return SplitOp{hi + row + col * ld, lo + row + col * ld, ld};
  }
};
// The stored operator is column-scaled: As = A diag(1 / cs) with cs[u index]
// = w/4 and cs[q index] = k0 w/4 (dense_colscale), so that A X = As (cs X):
// every product below takes cs X (scale_rows) as its right-hand operand.
// Off-diagonal part written out densely; same-inclusion pairs untouched (the
// caller copies the self blocks in).  One Hankel evaluation per node pair
// fills the pair's 2 x 2 entries.
void assemble_dense_offdiag64(OpNodes nd, int total_nodes, double k0, SplitOp A, cudaStream_t st);
// The same entries from one persistent CTA of 128 threads per SM taking rows
// from *counter (zeroed here), so that the assembly can run beside other
// kernels on a low-priority stream.
void assemble_dense_offdiag64_rows(OpNodes nd, int total_nodes, double k0, SplitOp A, int* counter,
                                   cudaStream_t st);
void dense_colscale(const double* w, const int* iu, const int* iq, int total_nodes, double k0, double* cs,
                    cudaStream_t st);
// Xs = diag(cs) X, N x nrhs.
void scale_rows(const double* cs, const double2* X, int ldx, double2* Xs, int ldxs, int N, int nrhs,
                cudaStream_t st);
// dst (split) <- src diag(1 / cs) (FP64) for an m x n block (cs: its n column
// scales, or nullptr for none).
void split_copy(const double2* src, int lds, SplitOp dst, int m, int n, const double* cs, cudaStream_t st);
// Y (N x nrhs) = A X in FP64 arithmetic (entries hi + lo); Y overwritten.
void dense_matvec64(SplitOp A, int N, const double2* X, int ldx, double2* Y, int ldy, int nrhs,
                    cudaStream_t st);
// The same product in float-float arithmetic on the FP32 pipes: error-free
// FP32 products of the hi parts (FMA), first-order cross terms, compensated
// sums; ~1e-13 relative, for refinement residuals.
void dense_matvec_ff(SplitOp A, int N, const double2* X, int ldx, double2* Y, int ldy, int nrhs,
                     cudaStream_t st);
// The float-float product with its sums folded into FP64 every 16 columns:
// worst-case error ~9e-13 of sum_j |a_ij||x_j| per row, so it may decide the
// convergence of the refinement (PM_FLAG_FF_CONFIRM).
void dense_matvec_ffc(SplitOp A, int N, const double2* X, int ldx, double2* Y, int ldy, int nrhs,
                      cudaStream_t st);
// The same product with the hi parts in FP32 arithmetic (~1e-7 relative to
// |A| |X|): the first refinement residual only.
void dense_matvec32(SplitOp A, int N, const double2* X, int ldx, double2* Y, int ldy, int nrhs,
                    cudaStream_t st);
// R = B - Y, and norms2[2 r] += |R[:, r]|^2, norms2[2 r + 1] += |B[:, r]|^2 (norms2 zeroed by caller)
void residual64(const double2* B, const double2* Y, double2* R, int N, int nrhs, double* norms2, cudaStream_t st);
// dst[:, r] = scale[r] * src[:, r] (FP64 -> FP32)
void scale_to32(const double2* src, float2* dst, int N, int nrhs, const double* scale, cudaStream_t st);
// X += D (FP64, N x nrhs, contiguous columns)
void axpy64(double2* X, const double2* D, int N, int nrhs, cudaStream_t st);
// x[:, r] += scale[r] * d[:, r] (FP32 -> FP64)
void axpy_from32(double2* x, const float2* d, int N, int nrhs, const double* scale, cudaStream_t st);
