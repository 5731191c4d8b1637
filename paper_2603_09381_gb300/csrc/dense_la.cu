// Batched complex GEMM / LU / LU-solve kernels.
//
// On GB300 the FP64 pipe (about 1.2 TFLOP/s) is the bound for all of these:
// even a rank-1 update streamed from HBM needs only ~0.25 flop/byte, above
// the chip's FP64:HBM balance (~0.18).  The kernels therefore favour simple
// shared-memory tiling with enough resident warps to keep the DFMA pipe busy.
#include "dense_la.cuh"
#include "prof.cuh"
#include <algorithm>

namespace {

constexpr int TB = 32;   // output tile
constexpr int TK = 16;   // k step

// One 32 x 32 output tile of  Cm = alpha * A * B + beta * Cm  (256 threads).
template <typename C>
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
        C v = alpha * accs[a][b];
        if (!beta_zero) v = v + beta * (*p);
        *p = v;
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

// ---- LU with partial pivoting (blocked, right-looking) ---------------------------------

// Panel: columns [p, p+jb) of rows [p, m), one CTA per matrix.  Pivot = the
// largest |a|^2 in the column, lowest row index on ties.
template <typename C>
__global__ void __launch_bounds__(256) k_lu_panel(const LuProb<C>* __restrict__ P, int p, int nb) {
  typedef typename real_of<C>::type R;
  const LuProb<C> pr = P[blockIdx.x];
  const int m = pr.m;
  if (p >= m) return;
  const int jb = min(nb, m - p);
  C* A = pr.A;
  const size_t ld = pr.ld;
  __shared__ R sval[256];
  __shared__ int sidx[256];
  __shared__ C rowc[64];
  __shared__ int s_piv;
  const int tid = threadIdx.x;
  for (int jj = 0; jj < jb; ++jj) {
    const int c = p + jj;
    R best = -1; int bi = m;
    for (int r = c + tid; r < m; r += 256) {
      R v = abs2(A[r + c * ld]);
      if (v > best) { best = v; bi = r; }
    }
    sval[tid] = best; sidx[tid] = bi;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (tid < s) {
        R v2 = sval[tid + s]; int i2 = sidx[tid + s];
        if (v2 > sval[tid] || (v2 == sval[tid] && i2 < sidx[tid])) { sval[tid] = v2; sidx[tid] = i2; }
      }
      __syncthreads();
    }
    if (tid == 0) {
      int piv = sidx[0];
      if (!(sval[0] > 0)) { piv = c; if (*pr.info == 0) *pr.info = c + 1; }
      s_piv = piv;
      pr.ipiv[c] = piv;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != c && tid < jb) {
      C* a = A + c + (size_t)(p + tid) * ld;
      C* b = A + piv + (size_t)(p + tid) * ld;
      C t = *a; *a = *b; *b = t;
    }
    __syncthreads();
    if (tid < jb) rowc[tid] = A[c + (size_t)(p + tid) * ld];
    __syncthreads();
    const C d = rowc[jj];
    if (abs2(d) > 0) {
      const C inv = cdiv(mk((R)1, (R)0), d);
      for (int r = c + 1 + tid; r < m; r += 256) {
        C l = A[r + c * ld] * inv;
        A[r + c * ld] = l;
        for (int j = jj + 1; j < jb; ++j) cfms(A[r + (size_t)(p + j) * ld], l, rowc[j]);
      }
    }
    __syncthreads();
  }
}

// Row interchanges of the panel applied to every other column, then the unit
// lower triangular solve U12 = L11^{-1} A12 on the columns right of the panel.
template <typename C>
__global__ void __launch_bounds__(256) k_lu_swap_trsm(const LuProb<C>* __restrict__ P, int p, int nb) {
  const LuProb<C> pr = P[blockIdx.y];
  const int m = pr.m;
  if (p >= m) return;
  const int jb = min(nb, m - p);
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m || (j >= p && j < p + jb)) return;
  C* A = pr.A;
  const size_t ld = pr.ld;
  C* col = A + (size_t)j * ld;
  for (int c = p; c < p + jb; ++c) {
    int r = pr.ipiv[c];
    if (r != c) { C t = col[c]; col[c] = col[r]; col[r] = t; }
  }
  if (j >= p + jb) {
    for (int r = 1; r < jb; ++r) {
      C acc = col[p + r];
      for (int s = 0; s < r; ++s) cfms(acc, A[p + r + (size_t)(p + s) * ld], col[p + s]);
      col[p + r] = acc;
    }
  }
}

// Trailing update A22 -= L21 * U12.
template <typename C>
__global__ void __launch_bounds__(256) k_lu_update(const LuProb<C>* __restrict__ P, int p, int nb) {
  const LuProb<C> pr = P[blockIdx.y];
  const int m = pr.m;
  if (p >= m) return;
  const int jb = min(nb, m - p);
  const int mt = m - p - jb;
  if (mt <= 0) return;
  const int tiles_m = (mt + TB - 1) / TB;
  const int t = blockIdx.x;
  if (t >= tiles_m * tiles_m) return;
  C* A = pr.A;
  const size_t ld = pr.ld;
  C mone = mk((typename real_of<C>::type)-1, (typename real_of<C>::type)0);
  gemm_tile<C>(mt, mt, jb, A + (p + jb) + p * ld, pr.ld, A + p + (p + jb) * ld, pr.ld,
               A + (p + jb) + (p + jb) * ld, pr.ld, mone, mk((typename real_of<C>::type)1, (typename real_of<C>::type)0),
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

// Diagonal block solve on rows [p, p+jb): unit lower (lower=1) or upper.
template <typename C>
__global__ void k_getrs_diag(const SolveProb<C>* __restrict__ P, int p, int nb, int lower) {
  const SolveProb<C> pr = P[blockIdx.y];
  if (p >= pr.m) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= pr.nrhs) return;
  const int jb = min(nb, pr.m - p);
  const C* A = pr.A;
  const size_t ld = pr.ld;
  C* col = pr.B + (size_t)j * pr.ldb;
  if (lower) {
    for (int r = 1; r < jb; ++r) {
      C acc = col[p + r];
      for (int s = 0; s < r; ++s) cfms(acc, A[p + r + (size_t)(p + s) * ld], col[p + s]);
      col[p + r] = acc;
    }
  } else {
    for (int r = jb - 1; r >= 0; --r) {
      C acc = col[p + r];
      for (int s = r + 1; s < jb; ++s) cfms(acc, A[p + r + (size_t)(p + s) * ld], col[p + s]);
      col[p + r] = cdiv(acc, A[p + r + (size_t)(p + r) * ld]);
    }
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
  gemm_tile<C>(mt, pr.nrhs, jb, pr.A + r0 + p * ld, pr.ld, pr.B + p, pr.ldb, pr.B + r0, pr.ldb,
               mk((R)-1, (R)0), mk((R)1, (R)0), 0, t % tiles_m, t / tiles_m);
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

constexpr int LU_NB = 16;
constexpr int RS_NB = 32;

template <typename C>
void la_getrf_batched(const LuProb<C>* d_prob, int nprob, int maxm, const int* h_m, cudaStream_t st) {
  if (nprob <= 0 || maxm <= 0) return;
  for (int p = 0; p < maxm; p += LU_NB) {
    double fp = 0, fs = 0, fu = 0;
    if (g_kprof) {
      for (int i = 0; i < nprob; ++i) {
        int m = h_m[i];
        if (p >= m) continue;
        double jb = std::min(LU_NB, m - p), rest = m - p - jb, h = m - p;
        fp += 8.0 * (h * jb * jb / 2);          // panel: rank-1 updates inside the panel
        fs += 8.0 * rest * jb * jb / 2;          // unit-lower solve of U12
        fu += 8.0 * rest * rest * jb;            // trailing GEMM
      }
    }
    KPROF_BEGIN(st);
    k_lu_panel<C><<<nprob, 256, 0, st>>>(d_prob, p, LU_NB);
    pm_launch_count_add(1);
    KPROF_END(st, kname<C>("lu_panel", "lu_panel32"), fp);
    dim3 g1((maxm + 255) / 256, nprob);
    KPROF_BEGIN(st);
    k_lu_swap_trsm<C><<<g1, 256, 0, st>>>(d_prob, p, LU_NB);
    pm_launch_count_add(1);
    KPROF_END(st, kname<C>("lu_swap_trsm", "lu_swap_trsm32"), fs);
    int mt = maxm - p - LU_NB;
    if (mt > 0) {
      int tiles = ((mt + TB - 1) / TB);
      dim3 g2(tiles * tiles, nprob);
      KPROF_BEGIN(st);
      k_lu_update<C><<<g2, 256, 0, st>>>(d_prob, p, LU_NB);
      pm_launch_count_add(1);
      KPROF_END(st, kname<C>("lu_update", "lu_update32"), fu);
    }
  }
}

template <typename C>
void la_getrs_batched(const SolveProb<C>* d_prob, int nprob, int maxm, int maxrhs, const int* h_m,
                      const int* h_rhs, cudaStream_t st) {
  if (nprob <= 0 || maxm <= 0 || maxrhs <= 0) return;
  double fl = 0;
  if (g_kprof)
    for (int i = 0; i < nprob; ++i) fl += 8.0 * (double)h_m[i] * h_m[i] * h_rhs[i];
  KPROF_BEGIN(st);
  dim3 gs((maxrhs + 127) / 128, nprob);
  k_getrs_swap<C><<<gs, 128, 0, st>>>(d_prob);
  pm_launch_count_add(1);
  const int tiles_n = (maxrhs + TB - 1) / TB;
  for (int p = 0; p < maxm; p += RS_NB) {
    k_getrs_diag<C><<<gs, 128, 0, st>>>(d_prob, p, RS_NB, 1);
    pm_launch_count_add(1);
    int mt = maxm - p - RS_NB;
    if (mt > 0) {
      dim3 g2(((mt + TB - 1) / TB) * tiles_n, nprob);
      k_getrs_update<C><<<g2, 256, 0, st>>>(d_prob, p, RS_NB, 1);
      pm_launch_count_add(1);
    }
  }
  int last = ((maxm - 1) / RS_NB) * RS_NB;
  for (int p = last; p >= 0; p -= RS_NB) {
    k_getrs_diag<C><<<gs, 128, 0, st>>>(d_prob, p, RS_NB, 0);
    pm_launch_count_add(1);
    if (p > 0) {
      dim3 g2(((p + TB - 1) / TB) * tiles_n, nprob);
      k_getrs_update<C><<<g2, 256, 0, st>>>(d_prob, p, RS_NB, 0);
      pm_launch_count_add(1);
    }
  }
  KPROF_END(st, kname<C>("getrs", "getrs32"), fl);
}

template void la_gemm_batched<double2>(const GemmDesc<double2>*, const int*, int, int, cudaStream_t);
template void la_gemm_batched<float2>(const GemmDesc<float2>*, const int*, int, int, cudaStream_t);
template void la_getrf_batched<double2>(const LuProb<double2>*, int, int, const int*, cudaStream_t);
template void la_getrf_batched<float2>(const LuProb<float2>*, int, int, const int*, cudaStream_t);
template void la_getrs_batched<double2>(const SolveProb<double2>*, int, int, int, const int*, const int*, cudaStream_t);
template void la_getrs_batched<float2>(const SolveProb<float2>*, int, int, int, const int*, const int*, cudaStream_t);
