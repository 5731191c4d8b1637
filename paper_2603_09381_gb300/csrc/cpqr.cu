// Column-pivoted Householder QR, one launch per elimination step.
//
// Each CTA owns up to 32 columns of one matrix.  At step s every CTA of the
// matrix reads the same squared trailing norms, picks the same pivot
// (largest norm; norms within a factor 1 - 1e-12 of the largest count as
// tied and the lowest column index wins), forms the Householder reflector of
// the pivot column (LAPACK zlarfg phase convention) and applies H^H to its
// own columns, recomputing their trailing norms from scratch for step s+1.
// The pivot column itself is left in place; R_ss goes to rdiag[s].  Because
// consecutive steps are consecutive launches no grid-wide barrier is needed.
// Work per entry and step: ~10 real FMAs on 48 bytes, so the FP64 pipe, not
// HBM, bounds it on GB300.
#include "cpqr.cuh"
#include "prof.cuh"
#include <algorithm>
#include <atomic>
#include <mutex>

namespace {

constexpr double TIE = 1e-12;

template <typename C>
__global__ void __launch_bounds__(256) k_init_norms(const CpqrProb<C>* __restrict__ P, const CpqrChunk* __restrict__ chunks) {
  typedef typename real_of<C>::type R;
  const CpqrChunk ch = chunks[blockIdx.x];
  const CpqrProb<C> p = P[ch.id];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = ch.c0 + warp; c < ch.c1; c += 8) {
    const C* col = p.Z + (size_t)c * p.ld;
    R acc = 0;
    for (int r = lane; r < p.W; r += 32) acc += abs2(col[r]);
    acc = warp_sum(acc);
    if (lane == 0) p.norm2[c] = (double)acc;
  }
}

// Sum of one value over the 256 threads of the CTA (every thread gets it).
template <typename R>
__device__ __forceinline__ R block_sum(R v, R* sh) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  R t = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) t += sh[w];
  return t;
}

// The chunk's columns one at a time, each held by the whole CTA in registers
// (RPT rows per thread): one read and one write of every trailing entry, with
// all of a thread's loads in flight together.  Requires W - s - 1 <= 256 RPT.
template <typename C, int RPT>
__device__ void cta_columns(const CpqrProb<C>& p, const CpqrChunk& ch, int s, int q, const C* xq, C ctau, C csc,
                            C sc, const double* cur, double* nxt) {
  typedef typename real_of<C>::type R;
  __shared__ R shx[8], shy[8], shn[8];
  const int tid = threadIdx.x;
  for (int c = ch.c0; c < ch.c1; ++c) {
    if (cur[c] < 0 || c == q) { if (tid == 0) nxt[c] = -1.0; continue; }
    C* col = p.Z + (size_t)c * p.ld;
    C v[RPT];
    C dot = czero<C>();
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = s + 1 + tid + 256 * i;
      v[i] = (r < p.W) ? col[r] : czero<C>();
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = s + 1 + tid + 256 * i;
      if (r < p.W) cfma_conj(dot, __ldg(&xq[r]), v[i]);
    }
    dot.x = block_sum(dot.x, shx);
    dot.y = block_sum(dot.y, shy);
    const C a_s = col[s];
    const C d = a_s + csc * dot;     // v^H a with v = [1; x/(alpha - beta)]
    const C f = ctau * d;            // H^H a = a - conj(tau) v (v^H a)
    const C fs = f * sc;
    R e = 0;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = s + 1 + tid + 256 * i;
      if (r < p.W) {
        cfms(v[i], fs, __ldg(&xq[r]));
        col[r] = v[i];
        e += abs2(v[i]);
      }
    }
    e = block_sum(e, shn);
    if (tid == 0) {
      col[s] = a_s - f;
      nxt[c] = (double)e;
    }
    __syncthreads();
  }
}

// One elimination step of the chunk's matrix on the chunk's columns (all 256
// threads of the CTA take the same path through the barriers).
template <typename C, bool TALL>
__device__ void cpqr_chunk_step(const CpqrProb<C>& p, const CpqrChunk& ch, int t) {
  typedef typename real_of<C>::type R;
  const int s = p.base + t;
  if (s >= p.target) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ double red[8];
  __shared__ int redi[8];
  __shared__ double s_mx;
  __shared__ int s_q;
  __shared__ int s_done;
  // Another CTA may set the rank during this launch: read it once so that the
  // whole CTA takes the same path through the barriers below.
  if (tid == 0) s_done = (p.mode == CPQR_FIND_RANK) && (*(volatile int*)p.rank >= 0);
  __syncthreads();
  if (s_done) return;
  const int n = p.n;
  const double* cur = p.norm2 + (s & 1) * n;
  double* nxt = p.norm2 + ((s + 1) & 1) * n;
  // pass 1: largest squared norm among unpivoted columns
  double mx = -1.0;
  for (int c = tid; c < n; c += 256) mx = fmax(mx, cur[c]);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    double m2 = red[0];
    for (int w = 1; w < 8; ++w) m2 = fmax(m2, red[w]);
    s_mx = m2;
  }
  __syncthreads();
  mx = s_mx;
  // pass 2: lowest index within the tie band
  const double band = (1.0 - TIE) * mx;
  int qi = n;
  for (int c = tid; c < n; c += 256) if (cur[c] >= 0 && cur[c] >= band) { qi = c; break; }
  for (int o = 16; o > 0; o >>= 1) qi = min(qi, __shfl_xor_sync(0xffffffffu, qi, o));
  if (lane == 0) redi[warp] = qi;
  __syncthreads();
  if (tid == 0) {
    int q2 = redi[0];
    for (int w = 1; w < 8; ++w) q2 = min(q2, redi[w]);
    s_q = q2;
  }
  __syncthreads();
  const int q = s_q;
  if (mx < 0 || q >= n) return;  // no unpivoted column left
  if (p.mode == CPQR_FIND_RANK) {
    double ref = (s == 0) ? sqrt(mx) : *p.ref;
    if (s == 0 && ch.first && tid == 0) *p.ref = ref;
    if (!(sqrt(mx) > p.tol * ref)) {
      if (ch.first && tid == 0) *p.rank = s;
      return;
    }
  }
  const C* xq = p.Z + (size_t)q * p.ld;
  const C alpha = xq[s];
  const R xnorm = (R)sqrt(cur[q]);
  const R beta = -copysign(xnorm, alpha.x);
  C tau = czero<C>(), sc = czero<C>();
  const bool reflect = xnorm > 0;
  if (reflect) {
    C bm = mk(beta, (R)0);
    tau = cdiv(bm - alpha, bm);
    sc = cdiv(mk((R)1, (R)0), alpha - bm);
  }
  const C ctau = conj(tau), csc = conj(sc);
  // complex64 tall enough to fill the CTA (short columns are barrier-bound) and fitting in registers
  if (TALL && sizeof(C) == 8 && reflect && p.W >= 2048 && p.W <= 256 * 32) {
    cta_columns<C, 32>(p, ch, s, q, xq, ctau, csc, sc, cur, nxt);
    if (tid == 0 && q >= ch.c0 && q < ch.c1) {
      p.rdiag[s] = mk(beta, (R)0);
      p.perm[s] = q;
    }
    return;
  }
  for (int c = ch.c0 + warp; c < ch.c1; c += 8) {
    if (cur[c] < 0 || c == q) { if (lane == 0) nxt[c] = -1.0; continue; }
    C* col = p.Z + (size_t)c * p.ld;
    if (!reflect) {
      R acc = 0;
      for (int r = s + 1 + lane; r < p.W; r += 32) acc += abs2(col[r]);
      acc = warp_sum(acc);
      if (lane == 0) nxt[c] = (double)acc;
      continue;
    }
    // four independent partial sums keep several loads in flight per lane
    C d0 = czero<C>(), d1 = czero<C>(), d2 = czero<C>(), d3 = czero<C>();
    int r = s + 1 + lane;
    for (; r + 96 < p.W; r += 128) {
      const C x0 = __ldg(&xq[r]), x1 = __ldg(&xq[r + 32]), x2 = __ldg(&xq[r + 64]), x3 = __ldg(&xq[r + 96]);
      const C a0 = col[r], a1 = col[r + 32], a2 = col[r + 64], a3 = col[r + 96];
      cfma_conj(d0, x0, a0); cfma_conj(d1, x1, a1); cfma_conj(d2, x2, a2); cfma_conj(d3, x3, a3);
    }
    for (; r < p.W; r += 32) cfma_conj(d0, __ldg(&xq[r]), col[r]);
    C dot = (d0 + d1) + (d2 + d3);
    dot.x = warp_sum(dot.x); dot.y = warp_sum(dot.y);
    const C a_s = col[s];
    __syncwarp();                   // every lane has read col[s] before lane 0 rewrites it
    dot = a_s + csc * dot;          // v^H a with v = [1; x/(alpha - beta)]
    const C f = ctau * dot;         // H^H a = a - conj(tau) v (v^H a)
    const C fs = f * sc;
    if (lane == 0) col[s] = a_s - f;
    R e0 = 0, e1 = 0, e2 = 0, e3 = 0;
    r = s + 1 + lane;
    for (; r + 96 < p.W; r += 128) {
      C v0 = col[r], v1 = col[r + 32], v2 = col[r + 64], v3 = col[r + 96];
      cfms(v0, fs, __ldg(&xq[r])); cfms(v1, fs, __ldg(&xq[r + 32]));
      cfms(v2, fs, __ldg(&xq[r + 64])); cfms(v3, fs, __ldg(&xq[r + 96]));
      col[r] = v0; col[r + 32] = v1; col[r + 64] = v2; col[r + 96] = v3;
      e0 += abs2(v0); e1 += abs2(v1); e2 += abs2(v2); e3 += abs2(v3);
    }
    for (; r < p.W; r += 32) {
      C v = col[r];
      cfms(v, fs, __ldg(&xq[r]));
      col[r] = v;
      e0 += abs2(v);
    }
    R acc = (e0 + e1) + (e2 + e3);
    acc = warp_sum(acc);
    if (lane == 0) nxt[c] = (double)acc;
  }
  if (tid == 0 && q >= ch.c0 && q < ch.c1) {
    p.rdiag[s] = mk(beta, (R)0);
    p.perm[s] = q;
  }
}

// Persistent grid (a multiple of the SM count): CTAs take chunks from a
// per-launch counter, largest matrices first, until none is left.  TALL
// compiles in the register-resident path for tall complex64 columns; without
// it the kernel needs far fewer registers (more resident CTAs), which is what
// the n x n triangles of the QR-first path want.
template <typename C, bool TALL>
__global__ void __launch_bounds__(256) k_cpqr_step(const CpqrProb<C>* __restrict__ P, const CpqrChunk* __restrict__ chunks,
                                                   int nchunk, int t, int* __restrict__ counter) {
  __shared__ int s_ci;
  for (;;) {
    if (threadIdx.x == 0) s_ci = atomicAdd(counter, 1);
    __syncthreads();
    const int ci = s_ci;
    if (ci >= nchunk) break;
    const CpqrChunk ch = chunks[ci];
    const CpqrProb<C> p = P[ch.id];
    cpqr_chunk_step<C, TALL>(p, ch, t);
    __syncthreads();
  }
}

// R11 (k x k, upper, diagonal from rdiag, zero below) and R12 (into T) in
// pivot order, both with leading dimension k.
template <typename C>
__global__ void k_interp_gather(const InterpProb<C>* __restrict__ P) {
  const InterpProb<C> p = P[blockIdx.y];
  const int k = p.k;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k <= 0 || e >= (size_t)k * p.n) return;
  const int i = (int)(e % k), j = (int)(e / k);
  const C v = p.Z[i + (size_t)p.perm[j] * p.ld];
  if (j < k) p.R11[i + (size_t)j * k] = i < j ? v : (i == j ? p.rdiag[i] : czero<C>());
  else p.T[i + (size_t)(j - k) * p.ldt] = v;
}

template <typename C>
__global__ void k_scatter(const ScatterProb<C>* __restrict__ P) {
  typedef typename real_of<C>::type R;
  const ScatterProb<C> p = P[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.k * p.ng) return;
  const int j = e % p.k, c = e / p.k;
  C v;
  if (c < p.k) {
    if (c != j) return;
    v = mk((R)1, (R)0);
  } else {
    v = p.T[j + (size_t)(c - p.k) * p.ldt];
  }
  const int row = p.pos[p.perm[c]];
  if (p.isL) p.out[row + (size_t)(p.off + j) * p.ld] = v;
  else p.out[(p.off + j) + (size_t)row * p.ld] = v;
}

__device__ __forceinline__ double2 cvt(double2 a, double2*) { return a; }
__device__ __forceinline__ float2 cvt(float2 a, float2*) { return a; }
__device__ __forceinline__ double2 cvt(float2 a, double2*) { return make_double2(a.x, a.y); }
__device__ __forceinline__ float2 cvt(double2 a, float2*) { return make_float2((float)a.x, (float)a.y); }

template <typename S, typename D>
__global__ void k_copy(const CopyProb<S, D>* __restrict__ P) {
  const CopyProb<S, D> p = P[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.m * p.n) return;
  const int i = e % p.m, j = e / p.m;
  p.dst[i + (size_t)j * p.ldd] = cvt(p.src[i + (size_t)j * p.lds], (D*)nullptr);
}

// Completes a permutation: after `done` pivot steps, the remaining columns in
// ascending order (one CTA per matrix).
__global__ void k_complete_perm(const PermFill* __restrict__ P) {
  extern __shared__ unsigned char used[];
  const PermFill p = P[blockIdx.x];
  for (int c = threadIdx.x; c < p.n; c += blockDim.x) used[c] = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < p.done; s += blockDim.x) used[p.perm[s]] = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    int o = p.done;
    for (int c = 0; c < p.n; ++c) if (!used[c]) p.perm[o++] = c;
  }
}

}  // namespace

void complete_perm(const PermFill* d_prob, int nprob, cudaStream_t st) {
  if (nprob <= 0) return;
  static std::once_flag attr;
  std::call_once(attr, [] { cudaFuncSetAttribute(k_complete_perm, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536); });
  k_complete_perm<<<nprob, 256, 65536, st>>>(d_prob);
  pm_launch_count_add(1);
}

template <typename C>
void cpqr_init_norms(const CpqrProb<C>* d_prob, const CpqrChunk* d_chunk, int nchunk, cudaStream_t st) {
  if (nchunk <= 0) return;
  k_init_norms<C><<<nchunk, 256, 0, st>>>(d_prob, d_chunk);
  pm_launch_count_add(1);
}
template <typename C, bool TALL>
int cpqr_grid() {   // SMs x resident CTAs, once per instance
  static std::atomic<int> grid_cache{0};
  int grid = grid_cache.load();
  if (grid == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cpqr_step<C, TALL>, 256, 0);
    grid = std::max(1, sms * std::max(per, 1));
    grid_cache.store(grid);
  }
  return grid;
}

template <typename C>
void cpqr_step(const CpqrProb<C>* d_prob, const CpqrChunk* d_chunk, int nchunk, int t, int* d_counter,
               cudaStream_t st, bool tall) {
  if (nchunk <= 0) return;
  KPROF_BEGIN(st);
  if (tall) k_cpqr_step<C, true><<<std::min(cpqr_grid<C, true>(), nchunk), 256, 0, st>>>(d_prob, d_chunk, nchunk, t, d_counter);
  else k_cpqr_step<C, false><<<std::min(cpqr_grid<C, false>(), nchunk), 256, 0, st>>>(d_prob, d_chunk, nchunk, t, d_counter);
  pm_launch_count_add(1);
  KPROF_END(st, kname<C>("cpqr_step", "cpqr_step32"), 0.0);   // work is added per level from the steps performed
}
template <typename C>
void interp_gather(const InterpProb<C>* d_prob, int nprob, size_t max_elems, cudaStream_t st) {
  if (nprob <= 0 || max_elems == 0) return;
  dim3 g((unsigned)((max_elems + 255) / 256), nprob);
  k_interp_gather<C><<<g, 256, 0, st>>>(d_prob);
  pm_launch_count_add(1);
}
template <typename C>
void scatter_interp(const ScatterProb<C>* d_prob, int nprob, int max_elems, cudaStream_t st) {
  if (nprob <= 0 || max_elems <= 0) return;
  dim3 g((max_elems + 255) / 256, nprob);
  k_scatter<C><<<g, 256, 0, st>>>(d_prob);
  pm_launch_count_add(1);
}
template <typename S, typename D>
void copy_batched(const CopyProb<S, D>* d_prob, int nprob, int max_elems, cudaStream_t st) {
  if (nprob <= 0 || max_elems <= 0) return;
  dim3 g((max_elems + 255) / 256, nprob);
  k_copy<S, D><<<g, 256, 0, st>>>(d_prob);
  pm_launch_count_add(1);
}

template void cpqr_init_norms<double2>(const CpqrProb<double2>*, const CpqrChunk*, int, cudaStream_t);
template void cpqr_step<double2>(const CpqrProb<double2>*, const CpqrChunk*, int, int, int*, cudaStream_t, bool);
template void interp_gather<double2>(const InterpProb<double2>*, int, size_t, cudaStream_t);
template void scatter_interp<double2>(const ScatterProb<double2>*, int, int, cudaStream_t);
template void copy_batched<double2, double2>(const CopyProb<double2, double2>*, int, int, cudaStream_t);
template void copy_batched<float2, float2>(const CopyProb<float2, float2>*, int, int, cudaStream_t);
template void copy_batched<float2, double2>(const CopyProb<float2, double2>*, int, int, cudaStream_t);
template void copy_batched<double2, float2>(const CopyProb<double2, float2>*, int, int, cudaStream_t);
template void cpqr_init_norms<float2>(const CpqrProb<float2>*, const CpqrChunk*, int, cudaStream_t);
template void cpqr_step<float2>(const CpqrProb<float2>*, const CpqrChunk*, int, int, int*, cudaStream_t, bool);
template void interp_gather<float2>(const InterpProb<float2>*, int, size_t, cudaStream_t);
template void scatter_interp<float2>(const ScatterProb<float2>*, int, int, cudaStream_t);
