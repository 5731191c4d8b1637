// FP64 operator application for iterative refinement (mixed precision).
//
// Every target node accumulates the exterior-kernel contributions of every
// source node on another inclusion, for all right-hand sides at once:
//   y[u_t] += (-eps+ S w) x[q_s] + (D w) x[u_s]
//   y[q_t] += (-D* w)     x[q_s] + (N/eps+ w) x[u_s]
// (paper Sec. 2.2, off-diagonal blocks of eq. pmchwt_omit_bie).  Sources are
// staged through shared memory in tiles of 64; the grid splits the sources
// into segments whose partial sums meet in FP64 atomics.  One J0/Y0/J1/Y1
// quadruple per node pair (hankel.cuh) serves all four kernels and all right-hand sides,
// so the kernel is bound by the FP64 pipe (Bessel evaluation + 32 complex
// FMAs per pair at 8 right-hand sides).
#include "operator.cuh"
#include "hankel.cuh"
#include "prof.cuh"
#include <algorithm>

namespace {

constexpr int OP_T = 128;   // targets per CTA
constexpr int OP_S = 64;    // sources per shared-memory tile

template <int NR>
__global__ void __launch_bounds__(OP_T) k_apply_offdiag(OpNodes nd, int total, double k, const double2* __restrict__ X,
                                                        int ldx, double2* __restrict__ Y, int ldy, int seg_len) {
  __shared__ double sx[OP_S], sy[OP_S], snx[OP_S], sny[OP_S], sw[OP_S];
  __shared__ int sinc[OP_S];
  __shared__ double2 sxq[NR][OP_S], sxu[NR][OP_S];
  const int t = blockIdx.x * OP_T + threadIdx.x;
  const bool active = t < total;
  const double ik = 1.0 / k;
  double tx = 0, ty = 0, tnx = 0, tny = 0;
  int tinc = -1;
  if (active) { tx = nd.x[t]; ty = nd.y[t]; tnx = nd.nx[t]; tny = nd.ny[t]; tinc = nd.incl[t]; }
  double2 au[NR], aq[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) { au[r] = make_double2(0, 0); aq[r] = make_double2(0, 0); }
  const int s0 = blockIdx.y * seg_len;
  const int s1 = min(total, s0 + seg_len);
  for (int base = s0; base < s1; base += OP_S) {
    __syncthreads();
    const int ls = threadIdx.x;
    if (ls < OP_S) {
      const int s = base + ls;
      if (s < s1) {
        sx[ls] = nd.x[s]; sy[ls] = nd.y[s]; snx[ls] = nd.nx[s]; sny[ls] = nd.ny[s]; sw[ls] = nd.w[s];
        sinc[ls] = nd.incl[s];
        const int iq = nd.iu[s], iu = nd.iq[s];   // q density sits at the u-equation index, u density at the q index
#pragma unroll
        for (int r = 0; r < NR; ++r) { sxq[r][ls] = X[iq + (size_t)r * ldx]; sxu[r][ls] = X[iu + (size_t)r * ldx]; }
      } else {
        sinc[ls] = -2;
      }
    }
    __syncthreads();
    if (!active) continue;
    const int cnt = min(OP_S, s1 - base);
    for (int j = 0; j < cnt; ++j) {
      if (sinc[j] == tinc) continue;
      const double dx = tx - sx[j], dy = ty - sy[j];
      const double ir = rsqrt(dx * dx + dy * dy);       // one reciprocal square root per pair
      const double r = (dx * dx + dy * dy) * ir;
      const double z = k * r;
      double J0, Y0, J1, Y1;
      hankel01_inv(z, ir * ik, J0, Y0, J1, Y1);
      const double w = sw[j];
      const double a = (tnx * dx + tny * dy) * ir, b = (snx[j] * dx + sny[j] * dy) * ir;
      const double nn = tnx * snx[j] + tny * sny[j];
      const double f = 0.25 * k * w;
      const double2 S = make_double2(0.25 * Y0 * w, -0.25 * J0 * w);          // -eps+ S w
      const double2 D = make_double2(-Y1 * b * f, J1 * b * f);                // D w
      const double2 T = make_double2(-Y1 * a * f, J1 * a * f);                // -D* w
      const double c0 = k * a * b, c1 = (nn - 2 * a * b) * ir;
      const double2 Nk = make_double2(-(c0 * Y0 + c1 * Y1) * f, (c0 * J0 + c1 * J1) * f);  // N/eps+ w
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        const double2 xq = sxq[q][j], xu = sxu[q][j];
        cfma(au[q], S, xq); cfma(au[q], D, xu);
        cfma(aq[q], T, xq); cfma(aq[q], Nk, xu);
      }
    }
  }
  if (!active) return;
  const int ru = nd.iu[t], rq = nd.iq[t];
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    double2* yu = Y + ru + (size_t)q * ldy;
    double2* yq = Y + rq + (size_t)q * ldy;
    atomicAdd(&yu->x, au[q].x); atomicAdd(&yu->y, au[q].y);
    atomicAdd(&yq->x, aq[q].x); atomicAdd(&yq->y, aq[q].y);
  }
}

// The dense operator's entries are stored as float pairs d = hi + lo (48
// significant bits).  The kernels that write and read them are bound by the
// FP64 pipe, so the split and the join work on the bit patterns with integer
// instructions: hi = d truncated to 24 significant bits, lo = the next 24 bits
// of the remainder (so lo has hi's sign and |lo| < ulp(hi)); joining adds the
// aligned mantissas exactly.  Values outside the normal float range, and pairs
// not of that form, take the FP64 conversions instead.
__device__ __forceinline__ void split_trunc(double d, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const int ef = e - 1023 + 127;
  if (ef <= 0 || ef >= 255) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
    return;
  }
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  hi = __uint_as_float(sign | ((unsigned int)ef << 23) | (unsigned int)(m >> 29));
  const unsigned int r = (unsigned int)(m & 0x1FFFFFFFu);   // remainder: 29 bits below hi
  if (r == 0) { lo = __uint_as_float(sign); return; }
  const int lz = __clz((int)r);                               // >= 3
  const int el = ef - 52 + (31 - lz);                         // biased float exponent of lo
  if (el <= 0) { lo = __uint_as_float(sign); return; }        // |lo| below 2^-126: dropped
  lo = __uint_as_float(sign | ((unsigned int)el << 23) | (((r << lz) >> 8) & 0x7FFFFFu));
}

__device__ __forceinline__ double join_trunc(float hi, float lo) {
  const unsigned int H = __float_as_uint(hi), L = __float_as_uint(lo);
  const int eh = (int)((H >> 23) & 0xFF), el = (int)((L >> 23) & 0xFF);
  const bool lzero = (L & 0x7FFFFFFFu) == 0;
  if (eh == 0 || eh == 255 || (!lzero && (el == 0 || ((H ^ L) & 0x80000000u)))) return (double)hi + (double)lo;
  unsigned long long M = (unsigned long long)((H & 0x7FFFFFu) | 0x800000u) << 29;   // 53-bit significand of hi
  if (!lzero) {
    const int sh = el - eh + 29;   // lo's significand position in units of the double's last place
    const unsigned long long ml = (L & 0x7FFFFFu) | 0x800000u;
    if (sh >= 0 && sh <= 5) M += ml << sh;
    else if (sh < 0 && sh > -24 && (ml & ((1ull << -sh) - 1)) == 0) M += ml >> -sh;
    else return (double)hi + (double)lo;
    if (M >> 53) return (double)hi + (double)lo;
  }
  return __longlong_as_double((long long)(((unsigned long long)(H & 0x80000000u) << 32) |
                                          ((unsigned long long)(eh - 127 + 1023) << 52) | (M & 0xFFFFFFFFFFFFFull)));
}

// Entry idx of the split operator: hi and lo planes.
__device__ __forceinline__ void store_split(const SplitOp& A, size_t idx, double re, double im) {
  float2 h, l;
  split_trunc(re, h.x, l.x);
  split_trunc(im, h.y, l.y);
  A.hi[idx] = h;
  A.lo[idx] = l;
}

__device__ __forceinline__ float4 split4(double re, double im) {
  const float hr = (float)re, hi = (float)im;
  return make_float4(hr, hi, (float)(re - (double)hr), (float)(im - (double)hi));
}

// Dense off-diagonal operator: thread = (node t, node s) with t < s; a block
// covers 64 t by 4 s (s fastest), so that the writes of both halves fill
// whole 32-byte sectors of each plane: the (t <- s) entries of 8 consecutive
// t per column, the mirrored (s <- t) entries of 4 consecutive s per column.
// One Hankel evaluation fills both 2 x 2 blocks of the pair.  The
// operator is stored column-scaled, A = As diag(cs), with cs = w/4 for a
// u-column (the density of -eps+ S and of the D-type block) and cs = k w/4
// for a q-column, so the quadrature weight and the factors 1/4 and k/4 of
// the kernels leave the per-pair arithmetic (the products scale X by cs
// first).  With d = x_t - x_s, a = n_t.d/r, b = n_s.d/r:
//   (t <- s): u-col (Y0 - i J0, -k a (Y1 - i J1)), q-col (-b (Y1 - i J1), N)
//   (s <- t): u-col (Y0 - i J0, k b (Y1 - i J1)),  q-col (a (Y1 - i J1), N)
// with N = -(c0 Y0 + c1 Y1) + i (c0 J0 + c1 J1), c0 = k a b,
// c1 = (n_t.n_s - 2 a b)/r, symmetric in the pair.
// The pair (t, s), t < s, of different inclusions: both 2 x 2 entry blocks.
__device__ __forceinline__ void offdiag_pair(const OpNodes& nd, int t, int s, double k, double ik, const SplitOp& A) {
  const int ti = nd.incl[t], si = nd.incl[s];
  if (ti == si) return;
  const double dx = nd.x[t] - nd.x[s], dy = nd.y[t] - nd.y[s];
  const double ir = rsqrt(dx * dx + dy * dy);
  const double r = (dx * dx + dy * dy) * ir;
  const double z = k * r;
  double J0, Y0, J1, Y1;
  hankel01_inv(z, ir * ik, J0, Y0, J1, Y1);
  const double tnx = nd.nx[t], tny = nd.ny[t], snx = nd.nx[s], sny = nd.ny[s];
  const double a = (tnx * dx + tny * dy) * ir, b = (snx * dx + sny * dy) * ir;
  const double ab = a * b;
  const double c0 = k * ab, c1 = fma(-2.0, ab, tnx * snx + tny * sny) * ir;
  const double Nre = -fma(c0, Y0, c1 * Y1), Nim = fma(c0, J0, c1 * J1);
  const double ka = k * a, kb = k * b;
  const size_t ut = nd.iu[t], qt = nd.iq[t], us = nd.iu[s], qs = nd.iq[s];
  const size_t lda = A.ld;
  // rows of t, columns of s
  store_split(A, ut + us * lda, Y0, -J0);
  store_split(A, qt + us * lda, -ka * Y1, ka * J1);
  store_split(A, ut + qs * lda, -b * Y1, b * J1);
  store_split(A, qt + qs * lda, Nre, Nim);
  // rows of s, columns of t
  store_split(A, us + ut * lda, Y0, -J0);
  store_split(A, qs + ut * lda, kb * Y1, -kb * J1);
  store_split(A, us + qt * lda, a * Y1, -a * J1);
  store_split(A, qs + qt * lda, Nre, Nim);
}

__global__ void __launch_bounds__(256) k_dense_offdiag(OpNodes nd, int total, double k, double ik, SplitOp A) {
  if (blockIdx.x * 64 >= blockIdx.y * 4 + 3) return;   // whole block on or below the diagonal
  const int s = blockIdx.y * 4 + (threadIdx.x & 3);
  const int t = blockIdx.x * 64 + (threadIdx.x >> 2);
  if (s >= total || t >= s) return;
  offdiag_pair(nd, t, s, k, ik, A);
}

// Persistent form, for a run beside other kernels with a small footprint
// (one CTA of 128 threads per SM): each CTA takes rows of 4 nodes s from a
// counter (longest rows first) and fills their pairs with every t < s in
// passes of 32 t x 4 s (s fastest: whole-sector writes in both halves).
// At most 64 registers: 128 x 64 = 8,192 of the SM's 65,536 (a 512-thread
// CTA of 112 registers still fits beside it).
__global__ void __maxnreg__(64) k_dense_offdiag_rows(OpNodes nd, int total, double k, double ik, SplitOp A,
                                                           int* __restrict__ counter) {
  __shared__ int s_item;
  const int rows = (total + 3) / 4;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();   // s_item is rewritten next round
    if (item >= rows) return;
    const int s0 = (rows - 1 - item) * 4;
    const int s = s0 + (threadIdx.x & 3);
    for (int t = threadIdx.x >> 2; t < s0 + 3; t += 32)
      if (s < total && t < s) offdiag_pair(nd, t, s, k, ik, A);
  }
}

// Column scales of the stored operator: cs[u index] = w/4, cs[q index] = k w/4.
__global__ void k_dense_colscale(const double* __restrict__ w, const int* __restrict__ iu, const int* __restrict__ iq,
                                 int total, double k, double* __restrict__ cs) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  cs[iu[t]] = 0.25 * w[t];
  cs[iq[t]] = 0.25 * k * w[t];
}

// Xs = diag(cs) X (the right-hand operand of a product with the stored operator).
__global__ void k_scale_rows(const double* __restrict__ cs, const double2* __restrict__ X, int ldx,
                             double2* __restrict__ Xs, int ldxs, int N) {
  const int q = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double c = cs[i];
  const double2 v = X[i + (size_t)q * ldx];
  Xs[i + (size_t)q * ldxs] = make_double2(c * v.x, c * v.y);
}

// Skinny product Y = A X: a CTA owns 128 rows and one segment of the columns of
// A; the segment's rows of X are staged in shared memory; partial sums meet in
// FP64 atomics.  Every A entry is read once and feeds NR complex FMAs.
constexpr int MV_ROWS = 128, MV_KT = 64;
template <int NR>
__global__ void __launch_bounds__(MV_ROWS) k_dense_matvec(const float2* __restrict__ Ah, const float2* __restrict__ Al,
                                                          size_t lda, int N,
                                                          const double2* __restrict__ X, int ldx, double2* __restrict__ Y,
                                                          int ldy, int seg) {
  __shared__ double2 xs[NR][MV_KT];
  const int row = blockIdx.x * MV_ROWS + threadIdx.x;
  const int k0 = blockIdx.y * seg, k1 = min(N, k0 + seg);
  double2 acc[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) acc[q] = make_double2(0, 0);
  for (int kb = k0; kb < k1; kb += MV_KT) {
    __syncthreads();
    for (int e = threadIdx.x; e < NR * MV_KT; e += MV_ROWS) {
      const int q = e / MV_KT, kk = e % MV_KT;
      xs[q][kk] = (kb + kk < k1) ? X[kb + kk + (size_t)q * ldx] : make_double2(0, 0);
    }
    __syncthreads();
    if (row < N) {
      const int cnt = min(MV_KT, k1 - kb);
      const float2* colh = Ah + row + (size_t)kb * lda;
      const float2* coll = Al + row + (size_t)kb * lda;
      for (int kk = 0; kk < cnt; ++kk) {
        const float2 h = __ldg(colh + (size_t)kk * lda), l = __ldg(coll + (size_t)kk * lda);
        const double2 a = make_double2(join_trunc(h.x, l.x), join_trunc(h.y, l.y));
#pragma unroll
        for (int q = 0; q < NR; ++q) cfma(acc[q], a, xs[q][kk]);
      }
    }
  }
  if (row >= N) return;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    atomicAdd(&Y[row + (size_t)q * ldy].x, acc[q].x);
    atomicAdd(&Y[row + (size_t)q * ldy].y, acc[q].y);
  }
}

// The same product with the hi parts only (one read of the hi plane, 8
// bytes per entry), in FP32 arithmetic over runs of MV32_KT columns whose
// sums are folded into FP64 accumulators (~1e-7 relative to |A| |X|
// typically, not growing with N): for the first refinement residual, which
// is ~1e-3 of the right-hand side, and for residual updates r - A dx.  The
// column loads are software-pipelined (the next MV32_G entries of the row
// are in flight while the current ones are multiplied), the next run's X
// values are fetched into registers during the current run, and the FP64
// accumulators live in shared memory (touched once per run).
constexpr int MV32_KT = 128, MV32_G = 8;
static_assert(MV32_KT == MV_ROWS, "one staged column of X per thread and right-hand side");
static_assert(MV32_KT % MV32_G == 0, "runs hold whole load groups");
template <int NR>
__global__ void __launch_bounds__(MV_ROWS) k_dense_matvec32(const float2* __restrict__ Ah, size_t lda, int N,
                                                            const double2* __restrict__ X, int ldx,
                                                            double2* __restrict__ Y, int ldy, int seg) {
  __shared__ float2 xs[MV32_KT][NR];
  __shared__ double2 accd[NR][MV_ROWS];   // this thread's FP64 sums: accd[q][threadIdx.x]
  const int row = blockIdx.x * MV_ROWS + threadIdx.x;
  const int k0 = blockIdx.y * seg, k1 = min(N, k0 + seg);
  float2 pre[NR];   // X[kb + threadIdx.x, q] of the next run, in FP32
#pragma unroll
  for (int q = 0; q < NR; ++q) accd[q][threadIdx.x] = make_double2(0.0, 0.0);
  auto fetch = [&](int kb) {
    const int kk = kb + threadIdx.x;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const double2 v = kk < k1 ? X[kk + (size_t)q * ldx] : make_double2(0, 0);
      pre[q] = make_float2((float)v.x, (float)v.y);
    }
  };
  if (k0 < k1) fetch(k0);
  for (int kb = k0; kb < k1; kb += MV32_KT) {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NR; ++q) xs[threadIdx.x][q] = pre[q];
    __syncthreads();
    if (kb + MV32_KT < k1) fetch(kb + MV32_KT);
    if (row < N) {
      // columns at or past cnt load as zero and meet zero X entries: they add 0
      const int cnt = min(MV32_KT, k1 - kb);
      const float2* col = Ah + row + (size_t)kb * lda;
      float2 acc[NR];
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[q] = make_float2(0.f, 0.f);
      float2 nxt[MV32_G];
#pragma unroll
      for (int g = 0; g < MV32_G; ++g) nxt[g] = g < cnt ? __ldg(col + (size_t)g * lda) : make_float2(0.f, 0.f);
      for (int kk = 0; kk < cnt; kk += MV32_G) {
        float2 cur[MV32_G];
#pragma unroll
        for (int g = 0; g < MV32_G; ++g) cur[g] = nxt[g];
#pragma unroll
        for (int g = 0; g < MV32_G; ++g) {
          const int kn = kk + MV32_G + g;
          nxt[g] = kn < cnt ? __ldg(col + (size_t)kn * lda) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int g = 0; g < MV32_G; ++g)
#pragma unroll
          for (int q = 0; q < NR; ++q) cfma(acc[q], cur[g], xs[kk + g][q]);
      }
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        double2 d = accd[q][threadIdx.x];
        d.x += (double)acc[q].x;
        d.y += (double)acc[q].y;
        accd[q][threadIdx.x] = d;
      }
    }
  }
  if (row >= N) return;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    atomicAdd(&Y[row + (size_t)q * ldy].x, accd[q][threadIdx.x].x);
    atomicAdd(&Y[row + (size_t)q * ldy].y, accd[q][threadIdx.x].y);
  }
}

// Float-float building blocks (Dekker / Knuth): exact FP32 product error via
// FMA, exact sum error via TwoSum.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// acc (hi, lo) += a * x for split a = (ah, al), x = (xh, xl): the hi products
// are split exactly (fmaf); their error and the cross terms are gathered in
// one FMA chain, which goes to lo with the TwoSum error (12 FP32 operations).
__device__ __forceinline__ void ff_mac(float& hi, float& lo, float ah, float al, float xh, float xl, float sgn) {
  const float p = ah * xh;
  float t = fmaf(ah, xh, -p);   // the exact error of ah xh
  t = fmaf(ah, xl, t);
  t = fmaf(al, xh, t);
  float s, e;
  two_sum(hi, sgn * p, s, e);
  hi = s;
  lo += e + sgn * t;
}

template <int NR>
__global__ void __launch_bounds__(MV_ROWS) k_dense_matvec_ff(const float2* __restrict__ Ah,
                                                             const float2* __restrict__ Al, size_t lda, int N,
                                                             const double2* __restrict__ X, int ldx,
                                                             double2* __restrict__ Y, int ldy, int seg) {
  __shared__ float4 xs[NR][MV_KT];   // {hi(re), hi(im), lo(re), lo(im)} of x
  const int row = blockIdx.x * MV_ROWS + threadIdx.x;
  const int k0 = blockIdx.y * seg, k1 = min(N, k0 + seg);
  float rh[NR], rl[NR], ih[NR], il[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) { rh[q] = rl[q] = ih[q] = il[q] = 0.f; }
  for (int kb = k0; kb < k1; kb += MV_KT) {
    __syncthreads();
    for (int e = threadIdx.x; e < NR * MV_KT; e += MV_ROWS) {
      const int q = e / MV_KT, kk = e % MV_KT;
      const double2 v = (kb + kk < k1) ? X[kb + kk + (size_t)q * ldx] : make_double2(0, 0);
      xs[q][kk] = split4(v.x, v.y);
    }
    __syncthreads();
    if (row < N) {
      const int cnt = min(MV_KT, k1 - kb);
      const float2* colh = Ah + row + (size_t)kb * lda;
      const float2* coll = Al + row + (size_t)kb * lda;
      for (int kk = 0; kk < cnt; ++kk) {
        const float2 h = __ldg(colh + (size_t)kk * lda), l = __ldg(coll + (size_t)kk * lda);
        const float4 a = make_float4(h.x, h.y, l.x, l.y);
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const float4 x = xs[q][kk];
          // re += a.re x.re - a.im x.im ;  im += a.re x.im + a.im x.re
          ff_mac(rh[q], rl[q], a.x, a.z, x.x, x.z, 1.f);
          ff_mac(rh[q], rl[q], a.y, a.w, x.y, x.w, -1.f);
          ff_mac(ih[q], il[q], a.x, a.z, x.y, x.w, 1.f);
          ff_mac(ih[q], il[q], a.y, a.w, x.x, x.z, 1.f);
        }
      }
    }
  }
  if (row >= N) return;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    atomicAdd(&Y[row + (size_t)q * ldy].x, (double)rh[q] + (double)rl[q]);
    atomicAdd(&Y[row + (size_t)q * ldy].y, (double)ih[q] + (double)il[q]);
  }
}

// The float-float product with its (hi, lo) sums restarted every FFC_FOLD
// columns and folded into FP64.  Within a group of m terms lo's own rounding
// is at most ~(m^2/2 + 7m) u^2 sum |a||x| (u = 2^-24): with m = 16 about 9e-13
// of sum_j |a_ij||x_j| per row, below the n 2^-53 worst case of a sequential
// FP64 sum over a ~20,000-term segment, so this product can end the
// refinement in place of the FP64 one.
constexpr int FFC_FOLD = 16;
template <int NR>
__global__ void __launch_bounds__(MV_ROWS) k_dense_matvec_ffc(const float2* __restrict__ Ah,
                                                              const float2* __restrict__ Al, size_t lda, int N,
                                                              const double2* __restrict__ X, int ldx,
                                                              double2* __restrict__ Y, int ldy, int seg) {
  __shared__ float4 xs[NR][MV_KT];   // {hi(re), hi(im), lo(re), lo(im)} of x
  const int row = blockIdx.x * MV_ROWS + threadIdx.x;
  const int k0 = blockIdx.y * seg, k1 = min(N, k0 + seg);
  double2 accd[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) accd[q] = make_double2(0.0, 0.0);
  for (int kb = k0; kb < k1; kb += MV_KT) {
    __syncthreads();
    for (int e = threadIdx.x; e < NR * MV_KT; e += MV_ROWS) {
      const int q = e / MV_KT, kk = e % MV_KT;
      const double2 v = (kb + kk < k1) ? X[kb + kk + (size_t)q * ldx] : make_double2(0, 0);
      xs[q][kk] = split4(v.x, v.y);
    }
    __syncthreads();
    if (row < N) {
      const int cnt = min(MV_KT, k1 - kb);
      const float2* colh = Ah + row + (size_t)kb * lda;
      const float2* coll = Al + row + (size_t)kb * lda;
      for (int kf = 0; kf < cnt; kf += FFC_FOLD) {
        const int kend = min(cnt, kf + FFC_FOLD);
        float rh[NR], rl[NR], ih[NR], il[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) { rh[q] = rl[q] = ih[q] = il[q] = 0.f; }
        for (int kk = kf; kk < kend; ++kk) {
          const float2 h = __ldg(colh + (size_t)kk * lda), l = __ldg(coll + (size_t)kk * lda);
          const float4 a = make_float4(h.x, h.y, l.x, l.y);
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            const float4 x = xs[q][kk];
            ff_mac(rh[q], rl[q], a.x, a.z, x.x, x.z, 1.f);
            ff_mac(rh[q], rl[q], a.y, a.w, x.y, x.w, -1.f);
            ff_mac(ih[q], il[q], a.x, a.z, x.y, x.w, 1.f);
            ff_mac(ih[q], il[q], a.y, a.w, x.x, x.z, 1.f);
          }
        }
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          accd[q].x += (double)rh[q] + (double)rl[q];
          accd[q].y += (double)ih[q] + (double)il[q];
        }
      }
    }
  }
  if (row >= N) return;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    atomicAdd(&Y[row + (size_t)q * ldy].x, accd[q].x);
    atomicAdd(&Y[row + (size_t)q * ldy].y, accd[q].y);
  }
}

// dst = split(src diag(1 / cs)): a self block into the column-scaled operator.
__global__ void k_split_copy(const double2* __restrict__ src, int lds, SplitOp dst, int m, int n,
                             const double* __restrict__ cs) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * n) return;
  const int i = e % m, j = e / m;
  const double2 v = src[i + (size_t)j * lds];
  if (cs) {
    const double c = 1.0 / cs[j];
    store_split(dst, i + (size_t)j * dst.ld, v.x * c, v.y * c);
  } else {
    store_split(dst, i + (size_t)j * dst.ld, v.x, v.y);
  }
}

__global__ void k_residual(const double2* __restrict__ B, const double2* __restrict__ Y, double2* __restrict__ R, int N,
                           double* norms2) {
  const int r = blockIdx.y;
  double sr = 0, sb = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double2 b = B[i + (size_t)r * N], y = Y[i + (size_t)r * N];
    const double2 v = make_double2(b.x - y.x, b.y - y.y);
    R[i + (size_t)r * N] = v;
    sr += v.x * v.x + v.y * v.y;
    sb += b.x * b.x + b.y * b.y;
  }
  sr = warp_sum(sr); sb = warp_sum(sb);
  if ((threadIdx.x & 31) == 0) { atomicAdd(&norms2[2 * r], sr); atomicAdd(&norms2[2 * r + 1], sb); }
}

__global__ void k_scale_to32(const double2* __restrict__ src, float2* __restrict__ dst, int N, const double* scale) {
  const int r = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double s = scale[r];
  const double2 v = src[i + (size_t)r * N];
  dst[i + (size_t)r * N] = make_float2((float)(v.x * s), (float)(v.y * s));
}

__global__ void k_axpy_from32(double2* __restrict__ x, const float2* __restrict__ d, int N, const double* scale) {
  const int r = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double s = scale[r];
  const float2 v = d[i + (size_t)r * N];
  double2& o = x[i + (size_t)r * N];
  o.x += s * (double)v.x;
  o.y += s * (double)v.y;
}

__global__ void k_axpy64(double2* __restrict__ X, const double2* __restrict__ D, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  X[i].x += D[i].x;
  X[i].y += D[i].y;
}

template <int NR>
void launch_apply(OpNodes nd, int total, double k0, const double2* X, int ldx, double2* Y, int ldy, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = (total + OP_T - 1) / OP_T;
  // enough CTAs for several per SM: split the sources into segments
  int segs = std::max(1, std::min(64, (sms * 8 + tiles - 1) / tiles));
  int seg_len = (total + segs - 1) / segs;
  seg_len = ((seg_len + OP_S - 1) / OP_S) * OP_S;
  segs = (total + seg_len - 1) / seg_len;
  dim3 g(tiles, segs);
  k_apply_offdiag<NR><<<g, OP_T, 0, st>>>(nd, total, k0, X, ldx, Y, ldy, seg_len);
  pm_launch_count_add(1);
}

}  // namespace

void apply_offdiag64(OpNodes nd, int total, double k0, const double2* X, int ldx, double2* Y, int ldy, int nrhs,
                     cudaStream_t st) {
  if (total <= 0 || nrhs <= 0) return;
  KPROF_BEGIN(st);
  for (int r0 = 0; r0 < nrhs;) {
    const int left = nrhs - r0;
    const double2* Xr = X + (size_t)r0 * ldx;
    double2* Yr = Y + (size_t)r0 * ldy;
    if (left >= 8) { launch_apply<8>(nd, total, k0, Xr, ldx, Yr, ldy, st); r0 += 8; }
    else if (left >= 4) { launch_apply<4>(nd, total, k0, Xr, ldx, Yr, ldy, st); r0 += 4; }
    else if (left >= 2) { launch_apply<2>(nd, total, k0, Xr, ldx, Yr, ldy, st); r0 += 2; }
    else { launch_apply<1>(nd, total, k0, Xr, ldx, Yr, ldy, st); r0 += 1; }
  }
  KPROF_END(st, "apply_offdiag64", 0.0);
}

void split_copy(const double2* src, int lds, SplitOp dst, int m, int n, const double* cs, cudaStream_t st) {
  if (m <= 0 || n <= 0) return;
  k_split_copy<<<(m * n + 255) / 256, 256, 0, st>>>(src, lds, dst, m, n, cs);
  pm_launch_count_add(1);
}

void dense_colscale(const double* w, const int* iu, const int* iq, int total_nodes, double k0, double* cs,
                    cudaStream_t st) {
  if (total_nodes <= 0) return;
  k_dense_colscale<<<(total_nodes + 255) / 256, 256, 0, st>>>(w, iu, iq, total_nodes, k0, cs);
  pm_launch_count_add(1);
}

void scale_rows(const double* cs, const double2* X, int ldx, double2* Xs, int ldxs, int N, int nrhs,
                cudaStream_t st) {
  if (N <= 0 || nrhs <= 0) return;
  k_scale_rows<<<dim3((N + 255) / 256, nrhs), 256, 0, st>>>(cs, X, ldx, Xs, ldxs, N);
  pm_launch_count_add(1);
}

void assemble_dense_offdiag64(OpNodes nd, int total, double k0, SplitOp A, cudaStream_t st) {
  if (total <= 0) return;
  dim3 g((total + 63) / 64, (total + 3) / 4);
  KPROF_BEGIN(st);
  k_dense_offdiag<<<g, 256, 0, st>>>(nd, total, k0, 1.0 / k0, A);
  pm_launch_count_add(1);
  KPROF_END(st, "dense_offdiag64", 0.0);
}

void assemble_dense_offdiag64_rows(OpNodes nd, int total, double k0, SplitOp A, int* counter, cudaStream_t st) {
  if (total <= 0) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaMemsetAsync(counter, 0, sizeof(int), st);
  // an SM changes its shared-memory carveout only when it is empty: the
  // persistent CTAs keep it at the maximum so that other kernels' shared
  // memory still fits beside them (the same value every time)
  cudaFuncSetAttribute(k_dense_offdiag_rows, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  KPROF_BEGIN(st);
  k_dense_offdiag_rows<<<sms, 128, 0, st>>>(nd, total, k0, 1.0 / k0, A, counter);
  pm_launch_count_add(1);
  KPROF_END(st, "dense_offdiag64", 0.0);
}

template <int NR>
void launch_matvec(SplitOp A, int N, const double2* X, int ldx, double2* Y, int ldy, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int rb = (N + MV_ROWS - 1) / MV_ROWS;
  int segs = std::max(1, (sms * 12 + rb - 1) / rb);
  int seg = (N + segs - 1) / segs;
  seg = ((seg + MV_KT - 1) / MV_KT) * MV_KT;
  segs = (N + seg - 1) / seg;
  dim3 g(rb, segs);
  k_dense_matvec<NR><<<g, MV_ROWS, 0, st>>>(A.hi, A.lo, A.ld, N, X, ldx, Y, ldy, seg);
  pm_launch_count_add(1);
}

void dense_matvec64(SplitOp A, int N, const double2* X, int ldx, double2* Y, int ldy, int nrhs,
                    cudaStream_t st) {
  if (N <= 0 || nrhs <= 0) return;
  for (int q = 0; q < nrhs; ++q) cudaMemsetAsync(Y + (size_t)q * ldy, 0, sizeof(double2) * N, st);
  KPROF_BEGIN(st);
  for (int r0 = 0; r0 < nrhs;) {
    const int left = nrhs - r0;
    const double2* Xr = X + (size_t)r0 * ldx;
    double2* Yr = Y + (size_t)r0 * ldy;
    if (left >= 8) { launch_matvec<8>(A, N, Xr, ldx, Yr, ldy, st); r0 += 8; }
    else if (left >= 4) { launch_matvec<4>(A, N, Xr, ldx, Yr, ldy, st); r0 += 4; }
    else if (left >= 2) { launch_matvec<2>(A, N, Xr, ldx, Yr, ldy, st); r0 += 2; }
    else { launch_matvec<1>(A, N, Xr, ldx, Yr, ldy, st); r0 += 1; }
  }
  KPROF_END(st, "dense_matvec64", 0.0);
}

template <int NR>
void launch_matvec_ff(SplitOp A, int N, const double2* X, int ldx, double2* Y, int ldy,
                      cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int rb = (N + MV_ROWS - 1) / MV_ROWS;
  int segs = std::max(1, (sms * 12 + rb - 1) / rb);
  int seg = (N + segs - 1) / segs;
  seg = ((seg + MV_KT - 1) / MV_KT) * MV_KT;
  segs = (N + seg - 1) / seg;
  dim3 g(rb, segs);
  k_dense_matvec_ff<NR><<<g, MV_ROWS, 0, st>>>(A.hi, A.lo, A.ld, N, X, ldx, Y, ldy, seg);
  pm_launch_count_add(1);
}

template <int NR>
void launch_matvec32(SplitOp A, int N, const double2* X, int ldx, double2* Y, int ldy,
                     cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int rb = (N + MV_ROWS - 1) / MV_ROWS;
  int segs = std::max(1, (sms * 12 + rb - 1) / rb);
  int seg = (N + segs - 1) / segs;
  seg = ((seg + MV32_KT - 1) / MV32_KT) * MV32_KT;
  segs = (N + seg - 1) / seg;
  k_dense_matvec32<NR><<<dim3(rb, segs), MV_ROWS, 0, st>>>(A.hi, A.ld, N, X, ldx, Y, ldy, seg);
  pm_launch_count_add(1);
}

void dense_matvec32(SplitOp A, int N, const double2* X, int ldx, double2* Y, int ldy, int nrhs,
                    cudaStream_t st) {
  if (N <= 0 || nrhs <= 0) return;
  for (int q = 0; q < nrhs; ++q) cudaMemsetAsync(Y + (size_t)q * ldy, 0, sizeof(double2) * N, st);
  KPROF_BEGIN(st);
  for (int r0 = 0; r0 < nrhs;) {
    const int left = nrhs - r0;
    const double2* Xr = X + (size_t)r0 * ldx;
    double2* Yr = Y + (size_t)r0 * ldy;
    if (left >= 8) { launch_matvec32<8>(A, N, Xr, ldx, Yr, ldy, st); r0 += 8; }
    else if (left >= 4) { launch_matvec32<4>(A, N, Xr, ldx, Yr, ldy, st); r0 += 4; }
    else if (left >= 2) { launch_matvec32<2>(A, N, Xr, ldx, Yr, ldy, st); r0 += 2; }
    else { launch_matvec32<1>(A, N, Xr, ldx, Yr, ldy, st); r0 += 1; }
  }
  KPROF_END(st, "dense_matvec32", 0.0);
}

void dense_matvec_ff(SplitOp A, int N, const double2* X, int ldx, double2* Y, int ldy, int nrhs,
                     cudaStream_t st) {
  if (N <= 0 || nrhs <= 0) return;
  for (int q = 0; q < nrhs; ++q) cudaMemsetAsync(Y + (size_t)q * ldy, 0, sizeof(double2) * N, st);
  KPROF_BEGIN(st);
  for (int r0 = 0; r0 < nrhs;) {
    const int left = nrhs - r0;
    const double2* Xr = X + (size_t)r0 * ldx;
    double2* Yr = Y + (size_t)r0 * ldy;
    if (left >= 8) { launch_matvec_ff<8>(A, N, Xr, ldx, Yr, ldy, st); r0 += 8; }
    else if (left >= 4) { launch_matvec_ff<4>(A, N, Xr, ldx, Yr, ldy, st); r0 += 4; }
    else if (left >= 2) { launch_matvec_ff<2>(A, N, Xr, ldx, Yr, ldy, st); r0 += 2; }
    else { launch_matvec_ff<1>(A, N, Xr, ldx, Yr, ldy, st); r0 += 1; }
  }
  KPROF_END(st, "dense_matvec_ff", 0.0);
}

template <int NR>
void launch_matvec_ffc(SplitOp A, int N, const double2* X, int ldx, double2* Y, int ldy,
                       cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int rb = (N + MV_ROWS - 1) / MV_ROWS;
  int segs = std::max(1, (sms * 12 + rb - 1) / rb);
  int seg = (N + segs - 1) / segs;
  seg = ((seg + MV_KT - 1) / MV_KT) * MV_KT;
  segs = (N + seg - 1) / seg;
  k_dense_matvec_ffc<NR><<<dim3(rb, segs), MV_ROWS, 0, st>>>(A.hi, A.lo, A.ld, N, X, ldx, Y, ldy, seg);
  pm_launch_count_add(1);
}

void dense_matvec_ffc(SplitOp A, int N, const double2* X, int ldx, double2* Y, int ldy, int nrhs,
                      cudaStream_t st) {
  if (N <= 0 || nrhs <= 0) return;
  for (int q = 0; q < nrhs; ++q) cudaMemsetAsync(Y + (size_t)q * ldy, 0, sizeof(double2) * N, st);
  KPROF_BEGIN(st);
  for (int r0 = 0; r0 < nrhs;) {
    const int left = nrhs - r0;
    const double2* Xr = X + (size_t)r0 * ldx;
    double2* Yr = Y + (size_t)r0 * ldy;
    if (left >= 8) { launch_matvec_ffc<8>(A, N, Xr, ldx, Yr, ldy, st); r0 += 8; }
    else if (left >= 4) { launch_matvec_ffc<4>(A, N, Xr, ldx, Yr, ldy, st); r0 += 4; }
    else if (left >= 2) { launch_matvec_ffc<2>(A, N, Xr, ldx, Yr, ldy, st); r0 += 2; }
    else { launch_matvec_ffc<1>(A, N, Xr, ldx, Yr, ldy, st); r0 += 1; }
  }
  KPROF_END(st, "dense_matvec_ffc", 0.0);
}

void residual64(const double2* B, const double2* Y, double2* R, int N, int nrhs, double* norms2, cudaStream_t st) {
  if (N <= 0 || nrhs <= 0) return;
  dim3 g(std::min(1024, (N + 255) / 256), nrhs);
  k_residual<<<g, 256, 0, st>>>(B, Y, R, N, norms2);
  pm_launch_count_add(1);
}

void scale_to32(const double2* src, float2* dst, int N, int nrhs, const double* scale, cudaStream_t st) {
  if (N <= 0 || nrhs <= 0) return;
  dim3 g((N + 255) / 256, nrhs);
  k_scale_to32<<<g, 256, 0, st>>>(src, dst, N, scale);
  pm_launch_count_add(1);
}

void axpy_from32(double2* x, const float2* d, int N, int nrhs, const double* scale, cudaStream_t st) {
  if (N <= 0 || nrhs <= 0) return;
  dim3 g((N + 255) / 256, nrhs);
  k_axpy_from32<<<g, 256, 0, st>>>(x, d, N, scale);
  pm_launch_count_add(1);
}

void axpy64(double2* X, const double2* D, int N, int nrhs, cudaStream_t st) {
  const size_t n = (size_t)N * nrhs;
  if (n == 0) return;
  k_axpy64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, D, n);
  pm_launch_count_add(1);
}
