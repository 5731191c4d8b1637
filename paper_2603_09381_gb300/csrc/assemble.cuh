// Geometry, right-hand side and matrix-entry assembly for the PMCHWT (Omit)
// system (paper Sec. 2.2).
#pragma once
#include <cuda_runtime.h>
#include "pm_common.cuh"

struct InclDev {           // one inclusion, as uploaded by the host
  int shape;               // 0 circle, 1 ellipse, 2 star, 3 fourier
  int n;                   // nodes on this boundary (even)
  int node_off;            // first node in the global node arrays
  int row_off;             // first global row / column (= 2 * node_off)
  double cx, cy, rot;
  double prm[16];
  double k_in_re, k_in_im; // interior wavenumber k^-
  double eps_in_re, eps_in_im;  // eps^- = (k^- / k^+)^2
};

struct NodesDev {          // structure-of-arrays node data, length = total nodes
  double *x, *y, *nx, *ny, *speed, *w, *curv, *kress;
  int* incl;               // owning inclusion of every node
};

struct PointsDev {         // points addressable by the gather assembly (nodes + proxies)
  double *x, *y, *nx, *ny, *w;
};

template <typename C>
struct GatherProb {        // out[i + j ld] = A(t, s): t = tgt[trans ? j : i], s = src[trans ? i : j]
  C* out; int ld; int M, N;
  const int* tgt;          // packed point*2 + row group (0 u-eq, 1 q-eq)
  const int* src;          // packed point*2 + column group (0 q, 1 u)
  int trans;
  double k;                // exterior wavenumber of this problem's kernels (0: the launch's k0);
                           // lets problems of different frequencies share one launch
  int mode;                // entries (complex128 only beyond GATHER_OMIT): see GatherMode
  double k_in, eps_in;     // interior wavenumber and eps- (real) of the interior terms
};

// Entry formulas of the gather, packed codes point*2 + group:
//  GATHER_OMIT   PMCHWT (Omit), rows (0 u-eq, 1 q-eq) x columns (0 q, 1 u):
//                [[-eps+ S+, D+], [-D*+, N+/eps+]]
//  GATHER_ALL    PMCHWT (All): Omit plus [[-eps- S-, D-], [-D*-, N-/eps-]]
//  GATHER_BM     Burton-Miller, rows (0 exterior, 1 interior eq.) x columns (0 u, 1 q):
//                [[D+ + alpha N+, -eps+ (S+ + alpha D*+)], [D-, -eps- S-]], alpha = i/k+
//  GATHER_BM_SIMPLIFIED  the same without the interior row (zeros)
//  GATHER_INTERIOR  the Omit layout with the interior kernel and eps-: the
//                interior proxy family of PMCHWT (All)
enum GatherMode { GATHER_OMIT = 0, GATHER_ALL = 1, GATHER_BM = 2, GATHER_BM_SIMPLIFIED = 3, GATHER_INTERIOR = 4 };

// p points at angles 2 pi (s + phase) / p (phase 0: the proxy circle; 0.5: the
// held-out ring of the proxy check)
struct ProxyBoxDev { double cx, cy, R; int p; int point_off; double phase; };

void geom_nodes(const InclDev* d_inc, NodesDev nodes, int total_nodes, const InclDev* h_inc, cudaStream_t st);
void geom_points_from_nodes(NodesDev nodes, PointsDev pts, int total_nodes, cudaStream_t st);
void geom_proxy_points(const ProxyBoxDev* d_box, int nbox, PointsDev pts, int total_proxy, int proxy_off,
                       cudaStream_t st);
template <typename C>
void plane_wave_rhs(const InclDev* d_inc, NodesDev nodes, int total_nodes, double k0, const double* d_angles,
                    int nrhs, C* F, int ldf, cudaStream_t st);
// Self blocks, pointwise part: writes the S, D, D* blocks and the k^2 S o nn term
// of A_jj (2n x 2n, leading dim lda), and the Maue middle factor Cm (n x n).
// bm != 0: the Burton-Miller self block (unknowns [u; q], rows [exterior;
// interior]); the Maue middle factor is then alpha S0+ and its product goes to
// the (exterior, u) block.  Otherwise the PMCHWT self block.
template <typename C>
void self_pointwise(const InclDev* d_inc, int m, int maxn, NodesDev nodes, double k0, C* const* d_A,
                    const int* d_lda, C* const* d_Cm, cudaStream_t st, int bm = 0);
// Trigonometric differentiation matrix Dt (n x n) and diag(1/|x'|) Dt for an inclusion.
template <typename C>
void diff_matrices(int n, C* Dt, cudaStream_t st);
// dst[b] = src[b] rounded to complex64, for nblk square blocks of order n[b]
// (leading dimension n[b] on both sides); maxn: the largest order.
void round_blocks(const double2* const* d_src, float2* const* d_dst, const int* d_n, int nblk, int maxn,
                  cudaStream_t st);
template <typename C>
void scaled_diff(const InclDev* d_inc, int m, int maxn, NodesDev nodes, C* const* d_DtS, cudaStream_t st);
template <typename C>
void gather_assemble(const GatherProb<C>* d_prob, const int* d_tile_off, int nprob, int total_tiles,
                     PointsDev pts, double k0, cudaStream_t st);
inline int gather_tiles(int M, int N) { return ((M + 31) / 32) * ((N + 7) / 8); }
