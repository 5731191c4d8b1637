// Batched complex GEMM / LU / LU-solve kernels.
//
// On GB300 the FP64 pipe (about 1.2 TFLOP/s) is the bound for all of these:
// even a rank-1 update streamed from HBM needs only ~0.25 flop/byte, above
// the chip's FP64:HBM balance (~0.18).  The kernels therefore favour simple
// shared-memory tiling with enough resident warps to keep the DFMA pipe busy.
#include "dense_la.cuh"
#include "prof.cuh"
#include <algorithm>
#include <vector>
#include <cooperative_groups.h>

namespace {

constexpr int TB = 32;   // output tile
constexpr int TK = 16;   // k step
constexpr int MAXNB = 16;   // panel width bound of the LU kernels

// One 32 x 32 output tile of  Cm = alpha * A * B + beta * Cm  (256 threads).
// SUB: the caller's alpha = -1 and beta = 1, applied as Cm - A * B (the same
// bits: multiplying by (-1, 0) and (1, 0) is exact), which spares the
// epilogue's complex multiplications (an eighth of an update's FP64 work at
// k = 16).
template <typename C, bool SUB = false>
__device__ __forceinline__ void gemm_tile(int m, int n, int k, const C* __restrict__ A, int lda,
                                          const C* __restrict__ B, int ldb, C* Cm, int ldc,
                                          C alpha, C beta, int beta_zero, int tm, int tn) {
  __shared__ C As[TK][TB + 1];
  __shared__ C Bs[TK][TB + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int r0 = tm * TB, c0 = tn * TB;
  C acc00 = czero<C>(), acc01 = czero<C>(), acc10 = czero<C>(), acc11 = czero<C>();
  for (int l0 = 0; l0 < k; l0 += TK) {
    for (int e = tid; e < TB * TK; e += 256) {
      int i = e % TB, l = e / TB;
      int gi = r0 + i, gl = l0 + l;
      As[l][i] = (gi < m && gl < k) ? A[gi + (size_t)gl * lda] : czero<C>();
    }
    for (int e = tid; e < TB * TK; e += 256) {
      int l = e % TK, j = e / TK;
      int gl = l0 + l, gj = c0 + j;
      Bs[l][j] = (gl < k && gj < n) ? B[gl + (size_t)gj * ldb] : czero<C>();
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < TK; ++l) {
      C a0 = As[l][tx], a1 = As[l][tx + 16];
      C b0 = Bs[l][ty], b1 = Bs[l][ty + 16];
      cfma(acc00, a0, b0); cfma(acc01, a0, b1);
      cfma(acc10, a1, b0); cfma(acc11, a1, b1);
    }
    __syncthreads();
  }
  C accs[2][2] = {{acc00, acc01}, {acc10, acc11}};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int gi = r0 + tx + 16 * a, gj = c0 + ty + 16 * b;
      if (gi < m && gj < n) {
        C* p = Cm + gi + (size_t)gj * ldc;
        if (SUB) {
          *p = *p - accs[a][b];
        } else {
          C v = alpha * accs[a][b];
          if (!beta_zero) v = v + beta * (*p);
          *p = v;
        }
      }
    }
}

template <typename C>
__global__ void __launch_bounds__(256) k_gemm_batched(const GemmDesc<C>* __restrict__ d,
                                                      const int* __restrict__ tile_off, int nprob) {
  int t = blockIdx.x;
  int lo = 0, hi = nprob;  // find prob with tile_off[prob] <= t < tile_off[prob+1]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (tile_off[mid] <= t) lo = mid; else hi = mid;
  }
  const GemmDesc<C> g = d[lo];
  int local = t - tile_off[lo];
  int tiles_m = (g.m + TB - 1) / TB;
  if (g.m <= 0 || g.n <= 0) return;
  gemm_tile<C>(g.m, g.n, g.k, g.A, g.lda, g.B, g.ldb, g.Cm, g.ldc, g.alpha, g.beta, g.beta_zero,
               local % tiles_m, local / tiles_m);
}

// The same product with a TM x TN output tile, each of the 256 threads
// holding MR x NR outputs (TM / MR by TN / NR threads).  Every output
// accumulates over k in the same order as gemm_tile (chunks of TK, each in
// order), so all tile shapes give bit-identical results; the autotuner picks
// among them by speed alone.
template <typename C, int TM, int TN, int MR, int NR>
__device__ __forceinline__ void gemm_tile_t(int m, int n, int k, const C* __restrict__ A, int lda,
                                            const C* __restrict__ B, int ldb, C* Cm, int ldc, C alpha, C beta,
                                            int beta_zero, int r0, int c0) {
  constexpr int TX = TM / MR, TY = TN / NR;
  static_assert(TX * TY == 256, "256 threads per tile");
  __shared__ C As[TK][TM + 1];
  __shared__ C Bs[TK][TN + 1];
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  C acc[MR][NR];
#pragma unroll
  for (int a = 0; a < MR; ++a)
#pragma unroll
    for (int b = 0; b < NR; ++b) acc[a][b] = czero<C>();
  for (int l0 = 0; l0 < k; l0 += TK) {
    for (int e = tid; e < TM * TK; e += 256) {
      const int i = e % TM, l = e / TM;
      const int gi = r0 + i, gl = l0 + l;
      As[l][i] = (gi < m && gl < k) ? A[gi + (size_t)gl * lda] : czero<C>();
    }
    for (int e = tid; e < TN * TK; e += 256) {
      const int l = e % TK, j = e / TK;
      const int gl = l0 + l, gj = c0 + j;
      Bs[l][j] = (gl < k && gj < n) ? B[gl + (size_t)gj * ldb] : czero<C>();
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < TK; ++l) {
      C av[MR], bv[NR];
#pragma unroll
      for (int a = 0; a < MR; ++a) av[a] = As[l][tx + TX * a];
#pragma unroll
      for (int b = 0; b < NR; ++b) bv[b] = Bs[l][ty + TY * b];
#pragma unroll
      for (int a = 0; a < MR; ++a)
#pragma unroll
        for (int b = 0; b < NR; ++b) cfma(acc[a][b], av[a], bv[b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < MR; ++a)
#pragma unroll
    for (int b = 0; b < NR; ++b) {
      const int gi = r0 + tx + TX * a, gj = c0 + ty + TY * b;
      if (gi < m && gj < n) {
        C* p = Cm + gi + (size_t)gj * ldc;
        C v = alpha * acc[a][b];
        if (!beta_zero) v = v + beta * (*p);
        *p = v;
      }
    }
}

template <typename C, int TM, int TN, int MR, int NR>
__global__ void __launch_bounds__(256) k_gemm_batched_t(const GemmDesc<C>* __restrict__ d,
                                                        const int* __restrict__ tile_off, int nprob) {
  const int t = blockIdx.x;
  int lo = 0, hi = nprob;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tile_off[mid] <= t) lo = mid; else hi = mid;
  }
  const GemmDesc<C> g = d[lo];
  if (g.m <= 0 || g.n <= 0) return;
  const int local = t - tile_off[lo];
  const int tiles_m = (g.m + TM - 1) / TM;
  gemm_tile_t<C, TM, TN, MR, NR>(g.m, g.n, g.k, g.A, g.lda, g.B, g.ldb, g.Cm, g.ldc, g.alpha, g.beta, g.beta_zero,
                                 (local % tiles_m) * TM, (local / tiles_m) * TN);
}

// ---- LU with partial pivoting (blocked, right-looking) ---------------------------------

__device__ __forceinline__ double2 shfl_c(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ float2 shfl_c(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Panel: columns [p, p+jb) of rows [p, m), one CTA per matrix, left-looking
// (Crout): column c is brought up to date only when it is reached, from the
// final L entries of the panel's earlier columns, so every entry is stored
// once per column step and the update is fused with the pivot search.
// Pivot = the largest |a|^2 in the column, lowest row index on ties (the
// same choice as the right-looking order, up to rounding).
template <typename C, int NT>
__global__ void __launch_bounds__(NT) k_lu_panel(const LuProb<C>* __restrict__ P, int p, int nb) {
  typedef typename real_of<C>::type R;
  const LuProb<C> pr = P[blockIdx.x];
  const int m = pr.m;
  if (p >= m) return;
  const int jb = min(nb, m - p);
  C* A = pr.A;
  const size_t ld = pr.ld;
  __shared__ R sval[NT / 32];
  __shared__ int sidx[NT / 32];
  __shared__ C s_l[MAXNB][MAXNB + 1];
  __shared__ C s_u[MAXNB];
  __shared__ int s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int jj = 0; jj < jb; ++jj) {
    const int c = p + jj;
    C* colc = A + (size_t)c * ld;
    if (jj > 0) {
      // U[0:jj, jj] = L11^{-1} A[p:c, c] (unit lower L11 of the current rows)
      for (int e = tid; e < jj * jj; e += NT) s_l[e % jj][e / jj] = A[p + e % jj + (size_t)(p + e / jj) * ld];
      __syncthreads();
      if (warp == 0) {
        C x = lane < jj ? colc[p + lane] : czero<C>();
        for (int l = 0; l < jj - 1; ++l) {
          const C xl = shfl_c(x, l);
          if (lane > l && lane < jj) cfms(x, s_l[lane][l], xl);
        }
        if (lane < jj) {
          s_u[lane] = x;
          colc[p + lane] = x;
        }
      }
      __syncthreads();
    }
    // rows c..m-1: a -= L[r, p:c] u, then the pivot search on the result
    R best = -1;
    int bi = m;
    for (int r = c + tid; r < m; r += NT) {
      C lr[MAXNB];   // the row's L entries, loaded together
#pragma unroll
      for (int l = 0; l < MAXNB; ++l) if (l < jj) lr[l] = A[r + (size_t)(p + l) * ld];
      // four partial sums: short dependent chains (FP64 latency)
      C a0 = colc[r], a1 = czero<C>(), a2 = czero<C>(), a3 = czero<C>();
#pragma unroll
      for (int l = 0; l < MAXNB; l += 4) {
        if (l < jj) cfms(a0, lr[l], s_u[l]);
        if (l + 1 < jj) cfms(a1, lr[l + 1], s_u[l + 1]);
        if (l + 2 < jj) cfms(a2, lr[l + 2], s_u[l + 2]);
        if (l + 3 < jj) cfms(a3, lr[l + 3], s_u[l + 3]);
      }
      const C a = (a0 + a1) + (a2 + a3);
      if (jj > 0) colc[r] = a;
      const R v = abs2(a);
      if (v > best) { best = v; bi = r; }   // rows ascend: the first of equal values stays
    }
    for (int o = 16; o > 0; o >>= 1) {
      const R v2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
    }
    if (lane == 0) { sval[warp] = best; sidx[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      R bv = sval[0];
      int piv = sidx[0];
      for (int w = 1; w < NT / 32; ++w)
        if (sval[w] > bv || (sval[w] == bv && sidx[w] < piv)) { bv = sval[w]; piv = sidx[w]; }
      if (!(bv > 0)) { piv = c; if (*pr.info == 0) *pr.info = c + 1; }
      s_piv = piv;
      pr.ipiv[c] = piv;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != c && tid < jb) {
      C* a = A + c + (size_t)(p + tid) * ld;
      C* b = A + piv + (size_t)(p + tid) * ld;
      const C t = *a; *a = *b; *b = t;
    }
    __syncthreads();
    const C d = colc[c];
    if (abs2(d) > 0) {
      const C inv = cdiv(mk((R)1, (R)0), d);
      int r = c + 1 + tid;
      for (; r + NT < m; r += 2 * NT) {   // two rows per pass: both loads in flight
        const C a0 = colc[r], a1 = colc[r + NT];
        colc[r] = a0 * inv;
        colc[r + NT] = a1 * inv;
      }
      if (r < m) colc[r] = colc[r] * inv;
    }
    __syncthreads();
  }
}

// The same panel with its rows p..m-1 held in shared memory for the whole
// panel (dynamic, (m - p) x jb, leading dimension m - p): loaded once,
// factored there (the lazy updates read the L entries from shared memory
// instead of L2), stored once; the same operations in the same order as
// k_lu_panel, so the same bits.
template <typename C, int NT>
__global__ void __launch_bounds__(NT) k_lu_panel_smem(const LuProb<C>* __restrict__ P, int p, int nb) {
  typedef typename real_of<C>::type R;
  extern __shared__ __align__(16) unsigned char lu_sm[];
  C* pan = reinterpret_cast<C*>(lu_sm);
  const LuProb<C> pr = P[blockIdx.x];
  const int m = pr.m;
  if (p >= m) return;
  const int jb = min(nb, m - p);
  const int mr = m - p;
  C* A = pr.A;
  const size_t ld = pr.ld;
  __shared__ R sval[NT / 32];
  __shared__ int sidx[NT / 32];
  __shared__ C s_l[MAXNB][MAXNB + 1];
  __shared__ C s_u[MAXNB];
  __shared__ int s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < mr * jb; e += NT) pan[e] = A[p + e % mr + (size_t)(p + e / mr) * ld];
  __syncthreads();
  for (int jj = 0; jj < jb; ++jj) {
    C* colc = pan + (size_t)jj * mr;   // local row i = global row p + i
    if (jj > 0) {
      for (int e = tid; e < jj * jj; e += NT) s_l[e % jj][e / jj] = pan[e % jj + (size_t)(e / jj) * mr];
      __syncthreads();
      if (warp == 0) {
        C x = lane < jj ? colc[lane] : czero<C>();
        for (int l = 0; l < jj - 1; ++l) {
          const C xl = shfl_c(x, l);
          if (lane > l && lane < jj) cfms(x, s_l[lane][l], xl);
        }
        if (lane < jj) {
          s_u[lane] = x;
          colc[lane] = x;
        }
      }
      __syncthreads();
    }
    R best = -1;
    int bi = m;
    for (int r = jj + tid; r < mr; r += NT) {
      C lr[MAXNB];
#pragma unroll
      for (int l = 0; l < MAXNB; ++l) if (l < jj) lr[l] = pan[r + (size_t)l * mr];
      C a0 = colc[r], a1 = czero<C>(), a2 = czero<C>(), a3 = czero<C>();
#pragma unroll
      for (int l = 0; l < MAXNB; l += 4) {
        if (l < jj) cfms(a0, lr[l], s_u[l]);
        if (l + 1 < jj) cfms(a1, lr[l + 1], s_u[l + 1]);
        if (l + 2 < jj) cfms(a2, lr[l + 2], s_u[l + 2]);
        if (l + 3 < jj) cfms(a3, lr[l + 3], s_u[l + 3]);
      }
      const C a = (a0 + a1) + (a2 + a3);
      if (jj > 0) colc[r] = a;
      const R v = abs2(a);
      if (v > best) { best = v; bi = p + r; }   // rows ascend: the first of equal values stays
    }
    for (int o = 16; o > 0; o >>= 1) {
      const R v2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
    }
    if (lane == 0) { sval[warp] = best; sidx[warp] = bi; }
    __syncthreads();
    const int c = p + jj;
    if (tid == 0) {
      R bv = sval[0];
      int piv = sidx[0];
      for (int w = 1; w < NT / 32; ++w)
        if (sval[w] > bv || (sval[w] == bv && sidx[w] < piv)) { bv = sval[w]; piv = sidx[w]; }
      if (!(bv > 0)) { piv = c; if (*pr.info == 0) *pr.info = c + 1; }
      s_piv = piv;
      pr.ipiv[c] = piv;
    }
    __syncthreads();
    const int piv = s_piv - p;
    if (piv != jj && tid < jb) {
      C* a = pan + jj + (size_t)tid * mr;
      C* b = pan + piv + (size_t)tid * mr;
      const C t = *a; *a = *b; *b = t;
    }
    __syncthreads();
    const C d = colc[jj];
    if (abs2(d) > 0) {
      const C inv = cdiv(mk((R)1, (R)0), d);
      for (int r = jj + 1 + tid; r < mr; r += NT) colc[r] = colc[r] * inv;
    }
    __syncthreads();
  }
  for (int e = tid; e < mr * jb; e += NT) A[p + e % mr + (size_t)(p + e / mr) * ld] = pan[e];
}

// The same left-looking panel for one large matrix on a cluster of CTAs
// (the top-level LU): the CTAs split the rows, so the lazy column updates
// (FP64-bound on one SM) spread over the cluster's SMs.  Per column: every
// CTA solves the small triangular system for U[0:jj] itself, updates its
// rows and proposes a pivot; the proposals meet through distributed shared
// memory (largest |a|^2, lowest row on ties, as in k_lu_panel); rank 0 swaps
// the two rows; every CTA scales its rows.  Two cluster barriers per column
// order these steps: a row's scaled L entry is next read by the thread that
// wrote it (rows keep their thread from column to column), and the next
// column's triangular solve reads only rows at or above the diagonal.
template <typename C, int NT>
__global__ void __launch_bounds__(NT) k_lu_panel_cluster(const LuProb<C>* __restrict__ P, int p, int nb) {
  typedef typename real_of<C>::type R;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int csize = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const LuProb<C> pr = P[blockIdx.x / csize];
  const int m = pr.m;
  if (p >= m) return;   // the whole cluster leaves
  const int jb = min(nb, m - p);
  C* A = pr.A;
  const size_t ld = pr.ld;
  __shared__ R sval[NT / 32];
  __shared__ int sidx[NT / 32];
  __shared__ R c_val;   // this CTA's proposal, read by the cluster
  __shared__ int c_idx;
  __shared__ C s_l[MAXNB][MAXNB + 1];
  __shared__ C s_u[MAXNB];
  __shared__ int s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int stride = NT * csize;
  for (int jj = 0; jj < jb; ++jj) {
    const int c = p + jj;
    C* colc = A + (size_t)c * ld;
    if (jj > 0) {
      for (int e = tid; e < jj * jj; e += NT) s_l[e % jj][e / jj] = A[p + e % jj + (size_t)(p + e / jj) * ld];
      __syncthreads();
      if (warp == 0) {
        C x = lane < jj ? colc[p + lane] : czero<C>();
        for (int l = 0; l < jj - 1; ++l) {
          const C xl = shfl_c(x, l);
          if (lane > l && lane < jj) cfms(x, s_l[lane][l], xl);
        }
        if (lane < jj) s_u[lane] = x;
      }
      __syncthreads();
    }
    R best = -1;
    int bi = m;
    for (int r = c + rank * NT + tid; r < m; r += stride) {
      C lr[MAXNB];
#pragma unroll
      for (int l = 0; l < MAXNB; ++l) if (l < jj) lr[l] = A[r + (size_t)(p + l) * ld];
      C a0 = colc[r], a1 = czero<C>(), a2 = czero<C>(), a3 = czero<C>();
#pragma unroll
      for (int l = 0; l < MAXNB; l += 4) {
        if (l < jj) cfms(a0, lr[l], s_u[l]);
        if (l + 1 < jj) cfms(a1, lr[l + 1], s_u[l + 1]);
        if (l + 2 < jj) cfms(a2, lr[l + 2], s_u[l + 2]);
        if (l + 3 < jj) cfms(a3, lr[l + 3], s_u[l + 3]);
      }
      const C a = (a0 + a1) + (a2 + a3);
      if (jj > 0) colc[r] = a;
      const R v = abs2(a);
      if (v > best || (v == best && r < bi)) { best = v; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const R v2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
    }
    if (lane == 0) { sval[warp] = best; sidx[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      R bv = sval[0];
      int bix = sidx[0];
      for (int w = 1; w < NT / 32; ++w)
        if (sval[w] > bv || (sval[w] == bv && sidx[w] < bix)) { bv = sval[w]; bix = sidx[w]; }
      c_val = bv;
      c_idx = bix;
    }
    cluster.sync();   // proposals and updated column entries are visible
    if (tid == 0) {
      R bv = -1;
      int piv = m;
      for (int q = 0; q < csize; ++q) {
        const R v = *cluster.map_shared_rank(&c_val, q);
        const int i = *cluster.map_shared_rank(&c_idx, q);
        if (v > bv || (v == bv && i < piv)) { bv = v; piv = i; }
      }
      if (!(bv > 0)) { piv = c; if (rank == 0 && *pr.info == 0) *pr.info = c + 1; }
      s_piv = piv;
      if (rank == 0) pr.ipiv[c] = piv;
    }
    __syncthreads();
    const int piv = s_piv;
    if (rank == 0) {
      if (jj > 0 && tid < jj) colc[p + tid] = s_u[tid];   // U entries of this column
      if (piv != c && tid < jb) {
        C* a = A + c + (size_t)(p + tid) * ld;
        C* b = A + piv + (size_t)(p + tid) * ld;
        const C t = *a; *a = *b; *b = t;
      }
    }
    cluster.sync();   // the swap is visible; every CTA has read its proposal slots
    const C d = colc[c];
    if (abs2(d) > 0) {
      const C inv = cdiv(mk((R)1, (R)0), d);
      for (int r = c + 1 + rank * NT + tid; r < m; r += stride) colc[r] = colc[r] * inv;
    }
    __syncthreads();
  }
  cluster.sync();   // no CTA leaves while another may still read its proposal slots
}

// Row interchanges of the panel applied to every other column, then the unit
// lower triangular solve U12 = L11^{-1} A12 on the columns right of the panel.
// Thread 0 of each CTA composes the panel's jb interchanges into one map over
// the rows they touch (the jb panel rows first, then at most jb rows below).
// One warp per column: lane i gathers the column's entry for position i (the
// panel rows are contiguous, so the first half of the warp reads one
// coalesced segment), the swapped-in rows below are written back, and the
// triangular solve runs across the lanes, each lane's row taking its
// subtractions in the same (ascending) order as a row-by-row substitution.
template <typename C>
__global__ void __launch_bounds__(256) k_lu_swap_trsm(const LuProb<C>* __restrict__ P, int p, int nb) {
  constexpr int MB = MAXNB;
  static_assert(2 * MB <= 32, "one lane per touched row");
  const LuProb<C> pr = P[blockIdx.y];
  const int m = pr.m;
  if (p >= m) return;
  const int jb = min(nb, m - p);
  __shared__ int s_row[2 * MB], s_org[2 * MB];
  __shared__ int s_cnt;
  __shared__ C s_l[MB][MB + 1];
  C* A = pr.A;
  const size_t ld = pr.ld;
  if (threadIdx.x == 0) {
    int cnt = jb;
    for (int i = 0; i < jb; ++i) { s_row[i] = p + i; s_org[i] = p + i; }
    for (int c = 0; c < jb; ++c) {
      const int r = pr.ipiv[p + c];
      int ir = r - p;
      if (ir >= jb) {
        ir = -1;
        for (int i = jb; i < cnt; ++i) if (s_row[i] == r) ir = i;
        if (ir < 0) { ir = cnt++; s_row[ir] = r; s_org[ir] = r; }
      }
      const int t = s_org[c]; s_org[c] = s_org[ir]; s_org[ir] = t;
    }
    s_cnt = cnt;
  }
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) s_l[e % jb][e / jb] = A[p + e % jb + (size_t)(p + e / jb) * ld];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= m || (j >= p && j < p + jb)) return;   // whole warps leave together
  C* col = A + (size_t)j * ld;
  const int cnt = s_cnt;
  C v = lane < cnt ? col[s_org[lane]] : czero<C>();
  __syncwarp();                                    // every read before any write
  if (lane >= jb && lane < cnt) col[s_row[lane]] = v;   // rows below the panel
  if (j >= p + jb) {
    for (int q = 0; q < jb - 1; ++q) {
      const C vq = shfl_c(v, q);
      if (lane > q && lane < jb) cfms(v, s_l[lane][q], vq);
    }
  }
  if (lane < jb) col[p + lane] = v;
}

// Trailing update A22 -= L21 * U12 on the trailing columns [p+jb+lo, p+jb+hi)
// (all of them: lo = 0, hi >= m).  Every entry is the same sum whatever the
// column range, so a split update gives the same bits as the whole one.
template <typename C>
__global__ void __launch_bounds__(256) k_lu_update(const LuProb<C>* __restrict__ P, int p, int nb, int lo, int hi) {
  const LuProb<C> pr = P[blockIdx.y];
  const int m = pr.m;
  if (p >= m) return;
  const int jb = min(nb, m - p);
  const int mt = m - p - jb;
  if (mt <= 0) return;
  const int c0 = p + jb + lo, c1 = p + jb + min(hi, mt);
  if (c1 <= c0) return;
  const int tiles_m = (mt + TB - 1) / TB, tiles_n = (c1 - c0 + TB - 1) / TB;
  const int t = blockIdx.x;
  if (t >= tiles_m * tiles_n) return;
  C* A = pr.A;
  const size_t ld = pr.ld;
  C mone = mk((typename real_of<C>::type)-1, (typename real_of<C>::type)0);
  gemm_tile<C, true>(mt, c1 - c0, jb, A + (p + jb) + p * ld, pr.ld, A + p + c0 * ld, pr.ld,
               A + (p + jb) + c0 * ld, pr.ld, mone, mk((typename real_of<C>::type)1, (typename real_of<C>::type)0),
               0, t % tiles_m, t / tiles_m);
}

// ---- LU solve ----------------------------------------------------------------------

template <typename C>
__global__ void k_getrs_swap(const SolveProb<C>* __restrict__ P) {
  const SolveProb<C> pr = P[blockIdx.y];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= pr.nrhs) return;
  C* col = pr.B + (size_t)j * pr.ldb;
  for (int c = 0; c < pr.m; ++c) {
    int r = pr.ipiv[c];
    if (r != c) { C t = col[c]; col[c] = col[r]; col[r] = t; }
  }
}

// Row interchanges: thread 0 composes the m interchanges into one map in
// shared memory (position i receives original row src[i]); the CTA then
// gathers each of its right-hand sides through a shared-memory stage.
constexpr int SW_RHS = 32;   // right-hand sides per CTA
template <typename C>
__global__ void __launch_bounds__(256) k_getrs_swap_smem(const SolveProb<C>* __restrict__ P) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const SolveProb<C> pr = P[blockIdx.y];
  const int j0 = blockIdx.x * SW_RHS;
  if (j0 >= pr.nrhs) return;
  C* stage = reinterpret_cast<C*>(sm_raw);
  int* src = reinterpret_cast<int*>(stage + pr.m);
  for (int i = threadIdx.x; i < pr.m; i += blockDim.x) src[i] = i;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int c = 0; c < pr.m; ++c) {
      const int r = pr.ipiv[c];
      if (r != c) { const int t = src[c]; src[c] = src[r]; src[r] = t; }
    }
  __syncthreads();
  const int j1 = min(pr.nrhs, j0 + SW_RHS);
  for (int j = j0; j < j1; ++j) {
    C* col = pr.B + (size_t)j * pr.ldb;
    for (int i = threadIdx.x; i < pr.m; i += blockDim.x) stage[i] = col[src[i]];
    __syncthreads();
    for (int i = threadIdx.x; i < pr.m; i += blockDim.x) col[i] = stage[i];
    __syncthreads();
  }
}

// Diagonal block solve on rows [p, p+jb), jb <= 32: unit lower (lower=1) or
// upper.  The block is staged in shared memory; one warp per right-hand side,
// lane r holding row p+r, each solved entry broadcast by a shuffle.
constexpr int DG_RHS = 32;   // right-hand sides per CTA (8 warps)
template <typename C>
__global__ void __launch_bounds__(256) k_getrs_diag(const SolveProb<C>* __restrict__ P, int p, int nb, int lower) {
  typedef typename real_of<C>::type R;
  __shared__ C sa[32][33];
  const SolveProb<C> pr = P[blockIdx.y];
  if (p >= pr.m) return;
  const int jb = min(nb, pr.m - p);
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    const int r = e % jb, c = e / jb;
    sa[r][c] = pr.A[p + r + (size_t)(p + c) * pr.ld];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  // reciprocals of the diagonal, all lanes at once (the solve chain below
  // then multiplies instead of dividing: FP64 division is a long sequence)
  const C dinv = (!lower && lane < jb) ? cdiv(mk((R)1, (R)0), sa[lane][lane]) : czero<C>();
  const int j1 = min(pr.nrhs, (int)(blockIdx.x + 1) * DG_RHS);
  for (int j = blockIdx.x * DG_RHS + (threadIdx.x >> 5); j < j1; j += blockDim.x >> 5) {
    C* col = pr.B + (size_t)j * pr.ldb + p;
    C x = lane < jb ? col[lane] : czero<C>();
    if (lower) {
      for (int c = 0; c < jb - 1; ++c) {
        const C xc = shfl_c(x, c);
        if (lane > c && lane < jb) cfms(x, sa[lane][c], xc);
      }
    } else {
      for (int c = jb - 1; c >= 0; --c) {
        if (lane == c) x = x * dinv;
        const C xc = shfl_c(x, c);
        if (lane < c) cfms(x, sa[lane][c], xc);
      }
    }
    if (lane < jb) col[lane] = x;
  }
}

// Off-diagonal update: lower -> B[p+jb:m) -= L[p+jb:m, p:p+jb] B[p:p+jb);
//                      upper -> B[0:p)    -= U[0:p, p:p+jb]    B[p:p+jb).
template <typename C>
__global__ void __launch_bounds__(256) k_getrs_update(const SolveProb<C>* __restrict__ P, int p, int nb, int lower) {
  typedef typename real_of<C>::type R;
  const SolveProb<C> pr = P[blockIdx.y];
  if (p >= pr.m) return;
  const int jb = min(nb, pr.m - p);
  const int r0 = lower ? p + jb : 0;
  const int mt = lower ? pr.m - p - jb : p;
  if (mt <= 0 || pr.nrhs <= 0) return;
  const int tiles_m = (mt + TB - 1) / TB, tiles_n = (pr.nrhs + TB - 1) / TB;
  const int t = blockIdx.x;
  if (t >= tiles_m * tiles_n) return;
  const size_t ld = pr.ld;
  gemm_tile<C, true>(mt, pr.nrhs, jb, pr.A + r0 + p * ld, pr.ld, pr.B + p, pr.ldb, pr.B + r0, pr.ldb,
               mk((R)-1, (R)0), mk((R)1, (R)0), 0, t % tiles_m, t / tiles_m);
}

// The same update for at most 8 right-hand sides: one thread per (row,
// right-hand side), the block's B rows staged in shared memory (the 32 x 32
// tile of the general kernel would spend 3/4 of its FP64 work on padding).
constexpr int TH_ROWS = 16;
template <typename C>
__global__ void __launch_bounds__(128) k_getrs_update_thin(const SolveProb<C>* __restrict__ P, int p, int nb, int lower) {
  __shared__ C sb[32][8];
  const SolveProb<C> pr = P[blockIdx.y];
  if (p >= pr.m) return;
  const int jb = min(nb, pr.m - p);
  const int r0 = lower ? p + jb : 0;
  const int mt = lower ? pr.m - p - jb : p;
  if (mt <= 0 || blockIdx.x * TH_ROWS >= mt) return;
  for (int e = threadIdx.x; e < jb * pr.nrhs; e += blockDim.x) {
    const int l = e % jb, q = e / jb;
    sb[l][q] = pr.B[p + l + (size_t)q * pr.ldb];
  }
  __syncthreads();
  const int i = blockIdx.x * TH_ROWS + (threadIdx.x & (TH_ROWS - 1)), q = threadIdx.x / TH_ROWS;
  if (i >= mt || q >= pr.nrhs) return;
  const C* a = pr.A + r0 + i + (size_t)p * pr.ld;
  C acc0 = czero<C>(), acc1 = czero<C>();   // two chains (FP64 latency)
  int l = 0;
  for (; l + 1 < jb; l += 2) {
    cfma(acc0, a[(size_t)l * pr.ld], sb[l][q]);
    cfma(acc1, a[(size_t)(l + 1) * pr.ld], sb[l + 1][q]);
  }
  if (l < jb) cfma(acc0, a[(size_t)l * pr.ld], sb[l][q]);
  C* out = pr.B + r0 + i + (size_t)q * pr.ldb;
  *out = *out - (acc0 + acc1);
}

// One triangle of the LU solves of a batch of matrices, each with at most 8
// right-hand sides, as ONE launch: every matrix is a chain of RS_NB-row
// blocks, one CTA per block and group of rg right-hand sides (the columns
// are independent chains; in FP64 a CTA's products and diagonal solve are
// bound by its SM's FP64 rate, so fewer columns per CTA shorten every link
// of the chain).  Each CTA takes a ticket from a counter and
// reads its (matrix, block) from items[ticket]; the items are ordered so that
// every block comes after the blocks it depends on (lower: by block index
// from the top, upper: by distance from the bottom), hence a CTA only ever
// waits on CTAs that took a smaller ticket and are already running: no
// co-residency is assumed.  A CTA subtracts the products of the blocks it
// depends on in the same order and with the same two-chain sums as
// k_getrs_update_thin, each as soon as that block's flag is up, then solves
// its diagonal block as k_getrs_diag does, stores the result and raises its
// own flag.  In FP64 the results are bit-identical to the launch-per-block
// sequence, without ~4 launches per block on the critical path.  With rg <= 4
// the two sums of a product (even and odd terms) are taken by two threads
// and joined in the same order, so the bits do not depend on rg.  Every wait
// is bounded (TS_WAIT_NS); a wait that runs out sets *err and the shared
// abort word, and every CTA then leaves without writing.
// items[t] = (matrix, block, flag base of the matrix and group, group);
// sync: [0] ticket, [1] abort, [2, 2 + items) flags; zeroed before the launch.
// no_flag (failure-path tests): every CTA first waits, with a 1 ms bound, on
// `never`, which nothing sets.
constexpr long long TS_WAIT_NS = 2000000000ll;   // 2 s per wait
__device__ __forceinline__ unsigned long long ts_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ts_load_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void ts_store_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// G: dependencies taken per round.  A round loads the coefficient blocks of
// the next G dependencies together, waits for the first one's flag, adds
// the later ones whose flags are already up, loads their solved rows
// together and subtracts their products one by one in dependency order: a
// block that is behind the chain's front catches up with one pair of
// memory round trips per round instead of per dependency.
template <typename C, int G>
__global__ void __launch_bounds__(256) k_trsv_chain(const SolveProb<C>* __restrict__ P, const int4* __restrict__ items,
                                                    int nitems, int lower, int rg, int* sync, int* err,
                                                    const int* never, int no_flag) {
  typedef typename real_of<C>::type R;
  constexpr int NB = 32;
  __shared__ C sl[G][NB][NB + 1];   // the off-diagonal blocks of this round's dependencies, [col][row]
  __shared__ C sx[G][NB][8];        // their solved rows (this CTA's right-hand sides)
  __shared__ C sa[NB][NB + 1];      // the diagonal block
  __shared__ C s_odd[G][4][NB];     // rg <= 4: the odd-term sums
  __shared__ int s_t, s_stop, s_cnt;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_t = atomicAdd(&sync[0], 1);
    s_stop = 0;
    if (no_flag) {
      const unsigned long long t0 = ts_now();
      while (ts_load_acquire(never) == 0) {
        if (ts_load_acquire(&sync[1]) != 0) break;
        if ((long long)(ts_now() - t0) > 1000000ll) { atomicExch(err, 1); atomicExch(&sync[1], 1); break; }
        __nanosleep(64);
      }
      s_stop = 1;
    }
  }
  __syncthreads();
  if (s_stop) return;
  const int t = s_t;
  if (t >= nitems) return;
  const int4 it = items[t];
  const SolveProb<C> pr = P[it.x];
  const int m = pr.m;
  const int q0 = it.w * rg, nrhs = min(rg, pr.nrhs - q0);   // this CTA's columns q0 .. q0 + nrhs - 1
  if (nrhs <= 0) return;   // the whole (matrix, group) is empty: nobody waits on its flags
  const int nblk = (m + NB - 1) / NB;
  const int b = it.y;
  const int r0 = b * NB, jb = min(NB, m - r0);
  const size_t ld = pr.ld;
  int* flags = sync + 2 + it.z;
  for (int e = tid; e < jb * jb; e += 256) {
    const int r = e % jb, c = e / jb;
    sa[r][c] = pr.A[r0 + r + (size_t)(r0 + c) * ld];
  }
  // this thread's entry (row i, right-hand side q) of the block being solved;
  // with rg <= 4 thread h = 1 of (i, q) takes the odd-term sums for h = 0
  const bool split = rg <= 4;
  const int i = tid & 31, q = split ? (tid >> 5) % rg : tid >> 5, h = split ? (tid >> 5) / rg : 0;
  const bool mine = i < jb && q < nrhs && h == 0;
  const bool odd = split && i < jb && q < nrhs && h == 1;
  C x = mine ? pr.B[r0 + i + (size_t)(q0 + q) * pr.ldb] : czero<C>();
  const int ndep = lower ? b : nblk - 1 - b;
  auto dep = [&](int d) { return lower ? d : nblk - 1 - d; };   // the d-th block this one depends on
  for (int d0 = 0; d0 < ndep;) {
    const int gmax = min(G, ndep - d0);
    // the coefficients do not depend on the flags: load them first
    for (int g = 0; g < gmax; ++g) {
      const int c0 = dep(d0 + g) * NB, jbj = min(NB, m - c0);
      for (int e = tid; e < jb * jbj; e += 256) {
        const int r = e % jb, c = e / jb;
        sl[g][c][r] = pr.A[r0 + r + (size_t)(c0 + c) * ld];
      }
    }
    if (tid == 0) {
      const unsigned long long t0 = ts_now();
      while (ts_load_acquire(&flags[dep(d0)]) == 0) {
        if (ts_load_acquire(&sync[1]) != 0) { s_stop = 1; break; }
        if ((long long)(ts_now() - t0) > TS_WAIT_NS) {
          atomicExch(err, 1);
          atomicExch(&sync[1], 1);
          s_stop = 1;
          break;
        }
        __nanosleep(64);
      }
      int cnt = 1;
      while (cnt < gmax && ts_load_acquire(&flags[dep(d0 + cnt)]) != 0) ++cnt;
      s_cnt = cnt;
    }
    __syncthreads();
    if (s_stop) return;
    const int cnt = s_cnt;
    for (int g = 0; g < cnt; ++g) {
      const int c0 = dep(d0 + g) * NB, jbj = min(NB, m - c0);
      for (int e = tid; e < jbj * nrhs; e += 256) {
        const int l = e % jbj, qq = e / jbj;
        sx[g][l][qq] = __ldcg(pr.B + c0 + l + (size_t)(q0 + qq) * pr.ldb);
      }
    }
    __syncthreads();
    for (int g = 0; g < cnt; ++g) {
      const int jbj = min(NB, m - dep(d0 + g) * NB);
      if (split) {
        // acc0 over the even terms, acc1 over the odd ones, each in order
        C acc = czero<C>();
        if (mine || odd)
          for (int l = h; l < jbj; l += 2) cfma(acc, sl[g][l][i], sx[g][l][q]);
        if (odd) s_odd[g][q][i] = acc;
        __syncthreads();
        if (mine) x = x - (acc + s_odd[g][q][i]);
      } else if (mine) {
        C acc0 = czero<C>(), acc1 = czero<C>();
        int l = 0;
        for (; l + 1 < jbj; l += 2) {
          cfma(acc0, sl[g][l][i], sx[g][l][q]);
          cfma(acc1, sl[g][l + 1][i], sx[g][l + 1][q]);
        }
        if (l < jbj) cfma(acc0, sl[g][l][i], sx[g][l][q]);
        x = x - (acc0 + acc1);
      }
    }
    __syncthreads();   // sl, sx and s_odd are refilled next
    d0 += cnt;
  }
  // the diagonal block: warp q solves right-hand side q, lane r holds row r
  if (mine) sx[0][i][q] = x;
  __syncthreads();
  if (warp < nrhs) {
    const C dinv = (!lower && lane < jb) ? cdiv(mk((R)1, (R)0), sa[lane][lane]) : czero<C>();
    C y = lane < jb ? sx[0][lane][warp] : czero<C>();
    if (lower) {
      for (int c = 0; c < jb - 1; ++c) {
        const C yc = shfl_c(y, c);
        if (lane > c && lane < jb) cfms(y, sa[lane][c], yc);
      }
    } else {
      for (int c = jb - 1; c >= 0; --c) {
        if (lane == c) y = y * dinv;
        const C yc = shfl_c(y, c);
        if (lane < c) cfms(y, sa[lane][c], yc);
      }
    }
    if (lane < jb) pr.B[r0 + lane + (size_t)(q0 + warp) * pr.ldb] = y;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) ts_store_release(&flags[b], 1);
}

}  // namespace

template <typename C>
void la_gemm_batched(const GemmDesc<C>* d_desc, const int* d_tile_off, int nprob, int total_tiles,
                     cudaStream_t st) {
  if (nprob <= 0 || total_tiles <= 0) return;
  KPROF_BEGIN(st);
  k_gemm_batched<C><<<total_tiles, 256, 0, st>>>(d_desc, d_tile_off, nprob);
  pm_launch_count_add(1);
  KPROF_END(st, kname<C>("gemm_batched", "gemm_batched32"), 0.0);
}

const GemmShape kGemmShapes[GEMM_NSHAPES] = {{32, 32}, {64, 64}, {64, 32}, {128, 8}, {64, 16}};

template <typename C>
void la_gemm_batched_shape(int shape, const GemmDesc<C>* d_desc, const int* d_tile_off, int nprob, int total_tiles,
                           cudaStream_t st) {
  if (nprob <= 0 || total_tiles <= 0) return;
  KPROF_BEGIN(st);
  switch (shape) {
    case 1: k_gemm_batched_t<C, 64, 64, 4, 4><<<total_tiles, 256, 0, st>>>(d_desc, d_tile_off, nprob); break;
    case 2: k_gemm_batched_t<C, 64, 32, 4, 2><<<total_tiles, 256, 0, st>>>(d_desc, d_tile_off, nprob); break;
    case 3: k_gemm_batched_t<C, 128, 8, 4, 1><<<total_tiles, 256, 0, st>>>(d_desc, d_tile_off, nprob); break;
    case 4: k_gemm_batched_t<C, 64, 16, 2, 2><<<total_tiles, 256, 0, st>>>(d_desc, d_tile_off, nprob); break;
    default: k_gemm_batched<C><<<total_tiles, 256, 0, st>>>(d_desc, d_tile_off, nprob); break;
  }
  pm_launch_count_add(1);
  KPROF_END(st, kname<C>("gemm_batched", "gemm_batched32"), 0.0);
}

constexpr int LU_NB = 16;
constexpr size_t LU_PANEL_SMEM = 216 * 1024;   // panels up to this size stay in shared memory
static_assert(LU_NB <= MAXNB, "LU panel wider than the kernels' shared tiles");
constexpr int RS_NB = 32;

// Flop counts of step p (panel, unit-lower solve of U12, trailing GEMM) for the profiler.
inline void lu_step_flops(const int* h_m, int nprob, int p, double& fp, double& fs, double& fu) {
  fp = fs = fu = 0;
  for (int i = 0; i < nprob; ++i) {
    const int m = h_m[i];
    if (p >= m) continue;
    const double jb = std::min(LU_NB, m - p), rest = m - p - jb, h = m - p;
    fp += 8.0 * (h * jb * jb / 2);
    fs += 8.0 * rest * jb * jb / 2;
    fu += 8.0 * rest * rest * jb;
  }
}

template <typename C>
void launch_panel_cluster(const LuProb<C>* d_prob, int nprob, int p, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nprob * 8);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 8;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_lu_panel_cluster<C, 256>, d_prob, p, LU_NB);
}

// A few large matrices (the top-level LU) with look-ahead, each panel on a
// cluster of 8 CTAs: step p's update
// of the next panel's LU_NB columns runs first, on a high-priority stream
// with the panels, and the rest of the trailing update on a low-priority
// stream, so that panel p+1 (latency-bound, on one 8-CTA cluster) overlaps
// the bulk of update p instead of leaving the other SMs idle.  Step p+1's
// interchanges wait for that update.  The kernels and their arithmetic are
// those of the plain sequence (identical bits).
template <typename C>
void la_getrf_lookahead(const LuProb<C>* d_prob, int nprob, int maxm, const int* h_m, cudaStream_t st) {
  int pr_lo = 0, pr_hi = 0;
  cudaDeviceGetStreamPriorityRange(&pr_lo, &pr_hi);
  cudaStream_t sp = nullptr, su = nullptr;
  cudaStreamCreateWithPriority(&sp, cudaStreamNonBlocking, pr_hi);
  cudaStreamCreateWithPriority(&su, cudaStreamNonBlocking, pr_lo);
  cudaEvent_t e_fork, e_next, e_rest;
  cudaEventCreateWithFlags(&e_fork, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&e_next, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&e_rest, cudaEventDisableTiming);
  cudaEventRecord(e_fork, st);
  cudaStreamWaitEvent(sp, e_fork, 0);
  cudaStreamWaitEvent(su, e_fork, 0);
  bool rest_pending = false;
  for (int p = 0; p < maxm; p += LU_NB) {
    double fp, fs, fu;
    lu_step_flops(h_m, nprob, p, fp, fs, fu);
    KPROF_BEGIN(sp);
    launch_panel_cluster<C>(d_prob, nprob, p, sp);
    pm_launch_count_add(1);
    KPROF_END(sp, kname<C>("lu_panel", "lu_panel32"), fp);
    if (rest_pending) cudaStreamWaitEvent(sp, e_rest, 0);
    dim3 g1((maxm + 7) / 8, nprob);   // a warp per column
    KPROF_BEGIN(sp);
    k_lu_swap_trsm<C><<<g1, 256, 0, sp>>>(d_prob, p, LU_NB);
    pm_launch_count_add(1);
    KPROF_END(sp, kname<C>("lu_swap_trsm", "lu_swap_trsm32"), fs);
    rest_pending = false;
    const int mt = maxm - p - LU_NB;
    if (mt <= 0) continue;
    const int nrest = mt - LU_NB;
    if (nrest > 0) cudaEventRecord(e_next, sp);   // interchanges and U12 of step p are done
    const int tiles_m = (mt + TB - 1) / TB;
    const double fn = fu * std::min(1.0, (double)LU_NB / mt);
    KPROF_BEGIN(sp);
    k_lu_update<C><<<dim3(tiles_m, nprob), 256, 0, sp>>>(d_prob, p, LU_NB, 0, LU_NB);
    pm_launch_count_add(1);
    KPROF_END(sp, kname<C>("lu_update", "lu_update32"), fn);
    if (nrest > 0) {
      cudaStreamWaitEvent(su, e_next, 0);
      dim3 g2(tiles_m * ((nrest + TB - 1) / TB), nprob);
      KPROF_BEGIN(su);
      k_lu_update<C><<<g2, 256, 0, su>>>(d_prob, p, LU_NB, LU_NB, 1 << 30);
      pm_launch_count_add(1);
      KPROF_END(su, kname<C>("lu_update", "lu_update32"), fu - fn);
      cudaEventRecord(e_rest, su);
      rest_pending = true;
    }
  }
  cudaEventRecord(e_next, sp);
  cudaEventRecord(e_rest, su);
  cudaStreamWaitEvent(st, e_next, 0);
  cudaStreamWaitEvent(st, e_rest, 0);
  cudaEventDestroy(e_fork);
  cudaEventDestroy(e_next);
  cudaEventDestroy(e_rest);
  cudaStreamDestroy(sp);
  cudaStreamDestroy(su);
}

template <typename C>
void la_getrf_batched(const LuProb<C>* d_prob, int nprob, int maxm, const int* h_m, cudaStream_t st) {
  if (nprob <= 0 || maxm <= 0) return;
  if (nprob <= 8 && maxm >= 2048) {
    la_getrf_lookahead<C>(d_prob, nprob, maxm, h_m, st);
    return;
  }
  for (int p = 0; p < maxm; p += LU_NB) {
    double fp = 0, fs = 0, fu = 0;
    if (g_kprof) lu_step_flops(h_m, nprob, p, fp, fs, fu);
    KPROF_BEGIN(st);
    const size_t pan_bytes = (size_t)(maxm - p) * std::min(LU_NB, maxm - p) * sizeof(C);
    if (pan_bytes <= LU_PANEL_SMEM) {
      // the same value every time: idempotent across threads and devices
      cudaFuncSetAttribute(k_lu_panel_smem<C, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LU_PANEL_SMEM);
      k_lu_panel_smem<C, 256><<<nprob, 256, pan_bytes, st>>>(d_prob, p, LU_NB);
    } else {
      k_lu_panel<C, 256><<<nprob, 256, 0, st>>>(d_prob, p, LU_NB);
    }
    pm_launch_count_add(1);
    KPROF_END(st, kname<C>("lu_panel", "lu_panel32"), fp);
    dim3 g1((maxm + 7) / 8, nprob);   // a warp per column
    KPROF_BEGIN(st);
    k_lu_swap_trsm<C><<<g1, 256, 0, st>>>(d_prob, p, LU_NB);
    pm_launch_count_add(1);
    KPROF_END(st, kname<C>("lu_swap_trsm", "lu_swap_trsm32"), fs);
    int mt = maxm - p - LU_NB;
    if (mt > 0) {
      int tiles = ((mt + TB - 1) / TB);
      dim3 g2(tiles * tiles, nprob);
      KPROF_BEGIN(st);
      k_lu_update<C><<<g2, 256, 0, st>>>(d_prob, p, LU_NB, 0, 1 << 30);
      pm_launch_count_add(1);
      KPROF_END(st, kname<C>("lu_update", "lu_update32"), fu);
    }
  }
}

int la_chain_items(const int* h_m, int nprob, int groups, std::vector<int4>& items) {
  std::vector<int> nb(nprob), base(nprob);
  int total = 0, maxb = 0;
  for (int i = 0; i < nprob; ++i) {
    nb[i] = std::max(0, (h_m[i] + RS_NB - 1) / RS_NB);
    base[i] = total;
    total += nb[i];
    maxb = std::max(maxb, nb[i]);
  }
  items.clear();
  items.reserve(2 * (size_t)total * groups);
  // flags of (matrix i, group g): groups * base[i] + g * nb[i] + block
  for (int d = 0; d < maxb; ++d)   // lower: block d of every matrix that has one
    for (int i = 0; i < nprob; ++i)
      for (int g = 0; g < groups; ++g)
        if (d < nb[i]) items.push_back(make_int4(i, d, groups * base[i] + g * nb[i], g));
  for (int d = 0; d < maxb; ++d)   // upper: block d from the bottom
    for (int i = 0; i < nprob; ++i)
      for (int g = 0; g < groups; ++g)
        if (d < nb[i]) items.push_back(make_int4(i, nb[i] - 1 - d, groups * base[i] + g * nb[i], g));
  return total * groups;
}
int la_chain_sync_ints(int total) { return 2 * (2 + total) + 1; }

template <typename C>
void la_getrs_batched(const SolveProb<C>* d_prob, int nprob, int maxm, int maxrhs, const int* h_m,
                      const int* h_rhs, cudaStream_t st, const ChainArgs* chain) {
  if (nprob <= 0 || maxm <= 0 || maxrhs <= 0) return;
  double fl = 0;
  if (g_kprof)
    for (int i = 0; i < nprob; ++i) fl += 8.0 * (double)h_m[i] * h_m[i] * h_rhs[i];
  KPROF_BEGIN(st);
  const size_t swap_smem = (size_t)maxm * (sizeof(C) + sizeof(int));
  if (swap_smem <= 200 * 1024) {
    // the same value every time: idempotent across threads and devices
    if (swap_smem > 48 * 1024)
      cudaFuncSetAttribute(k_getrs_swap_smem<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    k_getrs_swap_smem<C><<<dim3((maxrhs + SW_RHS - 1) / SW_RHS, nprob), 256, swap_smem, st>>>(d_prob);
  } else {
    dim3 gsw((maxrhs + 127) / 128, nprob);
    k_getrs_swap<C><<<gsw, 128, 0, st>>>(d_prob);
  }
  pm_launch_count_add(1);
  if (chain && maxrhs <= 8) {
    // few right-hand sides: each triangle of every matrix in one chained launch
    const int T = chain->total_blocks;
    cudaMemsetAsync(chain->sync, 0, sizeof(int) * la_chain_sync_ints(T), st);
    const int* never = chain->sync + 2 * (2 + T);
    if (T > 0) {
      // complex64: three dependencies per round; FP64: one (its products are
      // bound by the SM's FP64 rate, not by the round trips)
      constexpr int G = sizeof(C) == sizeof(double2) ? 1 : 3;
      k_trsv_chain<C, G><<<T, 256, 0, st>>>(d_prob, chain->items, T, 1, chain->rhs_per_cta, chain->sync, chain->err,
                                            never, chain->no_flag);
      k_trsv_chain<C, G><<<T, 256, 0, st>>>(d_prob, chain->items + T, T, 0, chain->rhs_per_cta, chain->sync + 2 + T,
                                            chain->err, never, chain->no_flag);
      pm_launch_count_add(2);
    }
    KPROF_END(st, kname<C>("getrs", "getrs32"), fl);
    return;
  }
  dim3 gs((maxrhs + DG_RHS - 1) / DG_RHS, nprob);
  const int tiles_n = (maxrhs + TB - 1) / TB;
  for (int p = 0; p < maxm; p += RS_NB) {
    k_getrs_diag<C><<<gs, 256, 0, st>>>(d_prob, p, RS_NB, 1);
    pm_launch_count_add(1);
    int mt = maxm - p - RS_NB;
    if (mt > 0) {
      if (maxrhs <= 8 && sizeof(C) == sizeof(double2)) {   // FP64: padding costs the bounding pipe
        k_getrs_update_thin<C><<<dim3((mt + TH_ROWS - 1) / TH_ROWS, nprob), 128, 0, st>>>(d_prob, p, RS_NB, 1);
      } else {
        dim3 g2(((mt + TB - 1) / TB) * tiles_n, nprob);
        k_getrs_update<C><<<g2, 256, 0, st>>>(d_prob, p, RS_NB, 1);
      }
      pm_launch_count_add(1);
    }
  }
  int last = ((maxm - 1) / RS_NB) * RS_NB;
  for (int p = last; p >= 0; p -= RS_NB) {
    k_getrs_diag<C><<<gs, 256, 0, st>>>(d_prob, p, RS_NB, 0);
    pm_launch_count_add(1);
    if (p > 0) {
      if (maxrhs <= 8 && sizeof(C) == sizeof(double2)) {   // FP64: padding costs the bounding pipe
        k_getrs_update_thin<C><<<dim3((p + TH_ROWS - 1) / TH_ROWS, nprob), 128, 0, st>>>(d_prob, p, RS_NB, 0);
      } else {
        dim3 g2(((p + TB - 1) / TB) * tiles_n, nprob);
        k_getrs_update<C><<<g2, 256, 0, st>>>(d_prob, p, RS_NB, 0);
      }
      pm_launch_count_add(1);
    }
  }
  KPROF_END(st, kname<C>("getrs", "getrs32"), fl);
}

template <typename C>
void la_trsm_upper_batched(const SolveProb<C>* d_prob, int nprob, int maxm, int maxrhs, const char* name,
                           double flops, cudaStream_t st) {
  if (nprob <= 0 || maxm <= 0 || maxrhs <= 0) return;
  KPROF_BEGIN(st);
  dim3 gs((maxrhs + DG_RHS - 1) / DG_RHS, nprob);
  const int tiles_n = (maxrhs + TB - 1) / TB;
  int last = ((maxm - 1) / RS_NB) * RS_NB;
  for (int p = last; p >= 0; p -= RS_NB) {
    k_getrs_diag<C><<<gs, 256, 0, st>>>(d_prob, p, RS_NB, 0);
    pm_launch_count_add(1);
    if (p > 0) {
      dim3 g2(((p + TB - 1) / TB) * tiles_n, nprob);
      k_getrs_update<C><<<g2, 256, 0, st>>>(d_prob, p, RS_NB, 0);
      pm_launch_count_add(1);
    }
  }
  KPROF_END(st, name, flops);
}

template void la_trsm_upper_batched<double2>(const SolveProb<double2>*, int, int, int, const char*, double,
                                             cudaStream_t);
template void la_trsm_upper_batched<float2>(const SolveProb<float2>*, int, int, int, const char*, double,
                                            cudaStream_t);
template void la_gemm_batched_shape<double2>(int, const GemmDesc<double2>*, const int*, int, int, cudaStream_t);
template void la_gemm_batched_shape<float2>(int, const GemmDesc<float2>*, const int*, int, int, cudaStream_t);
template void la_gemm_batched<double2>(const GemmDesc<double2>*, const int*, int, int, cudaStream_t);
template void la_gemm_batched<float2>(const GemmDesc<float2>*, const int*, int, int, cudaStream_t);
template void la_getrf_batched<double2>(const LuProb<double2>*, int, int, const int*, cudaStream_t);
template void la_getrf_batched<float2>(const LuProb<float2>*, int, int, const int*, cudaStream_t);
template void la_getrs_batched<double2>(const SolveProb<double2>*, int, int, int, const int*, const int*, cudaStream_t,
                                        const ChainArgs*);
template void la_getrs_batched<float2>(const SolveProb<float2>*, int, int, int, const int*, const int*, cudaStream_t,
                                       const ChainArgs*);
