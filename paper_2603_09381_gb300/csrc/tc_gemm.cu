// Batched complex64 GEMM on the tcgen05 tensor cores.
//
// A complex product is a real one of twice the size:
//   [Re D; Im D] = [[Re A, -Im A], [Im A, Re A]] [Re B; Im B],
// so a 64 x 32 complex output tile is one 128 x 32 real accumulator in tensor
// memory (TMEM), and every 16-wide complex k chunk is a 32-wide real k chunk.
// Each FP32 operand x is split into tf32 parts x = hi + lo (both exactly
// representable), and hi*hi + hi*lo + lo*hi are accumulated in FP32: the
// dropped lo*lo term is below FP32 rounding, so the product has FP32 accuracy
// (the "3xTF32" scheme).
//
// Per CTA (128 threads, one tile): the threads stage chunk c of op(A) and
// op(B), split, into shared memory in the K-major, non-swizzled canonical
// layout (8-row x 16-byte core matrices); one thread issues the 12 MMAs of
// the chunk (4 k-steps of 8 x 3 products) and commits them to the chunk
// buffer's mbarrier, so staging chunk c+1 into the other buffer overlaps
// them.  The epilogue reads the accumulator with tcgen05.ld (thread i of the
// CTA owns TMEM lane i = real row i) and writes alpha D + beta C.  Every
// mbarrier wait is bounded; a wait that runs out sets the caller's error flag.
#include "tc_gemm.cuh"
#include "tc_common.cuh"
#include "prof.cuh"
#include <cstdint>

namespace {

constexpr int TC_T = 128;                 // threads: warp w reads TMEM lanes [32w, 32w + 32)
constexpr int KC = 16;                    // complex k per chunk
constexpr int KR = 2 * KC;                // real k per chunk
constexpr int A_ROWS = 2 * TC_TM;         // 128
constexpr int B_ROWS = TC_TN;             // 32
constexpr uint32_t A_BYTES = A_ROWS * KR * 4;
constexpr uint32_t B_BYTES = B_ROWS * KR * 4;
constexpr uint32_t BUF = 2 * A_BYTES + 2 * B_BYTES;   // hi and lo of both operands
constexpr uint32_t TMEM_COLS = 32;
constexpr int WAIT_LIMIT = 1 << 20;       // x ~1 us suspend hint: about a second
constexpr int SMEM_BYTES = 2 * BUF + 64;
constexpr uint32_t IDESC = tcx::idesc_tf32(A_ROWS, TC_TN);
constexpr uint32_t LBO = tcx::LBO;

using tcx::smem_u32;
using tcx::put_split;
__device__ __forceinline__ uint32_t core_off(int row, int k) { return tcx::core_off<KR>(row, k); }
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) { return tcx::sdesc<KR>(saddr); }
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit = WAIT_LIMIT) {
  return tcx::mbar_wait(bar, parity, limit);
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t accumulate) {
  tcx::mma_tf32<IDESC>(tmem, ad, bd, accumulate);
}

__global__ void __launch_bounds__(TC_T) k_tc_gemm(const TcGemmProb* __restrict__ P, const int* __restrict__ tile_off,
                                                  int nprob, int tile_base, int* err, int no_arrive) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int t = tile_base + (int)blockIdx.x;
  int lo_p = 0, hi_p = nprob;
  while (hi_p - lo_p > 1) {
    const int mid = (lo_p + hi_p) >> 1;
    if (tile_off[mid] <= t) lo_p = mid; else hi_p = mid;
  }
  const TcGemmProb g = P[lo_p];
  const int local = t - tile_off[lo_p];
  const int tiles_m = (g.m + TC_TM - 1) / TC_TM;
  const int m0 = (local % tiles_m) * TC_TM, n0 = (local / tiles_m) * TC_TN;
  const int tid = threadIdx.x, warp = tid >> 5;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 2 * BUF);
  uint32_t* s_taddr = reinterpret_cast<uint32_t*>(sm + 2 * BUF + 24);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[2])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_taddr)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *s_taddr;

  bool ok = true;
  // timeout-path test: a barrier that nothing arrives at, waited on before any work is issued
  if (no_arrive) ok = mbar_wait(&mbar[2], 0, 1 << 10);
  const int nchunks = __syncthreads_and(ok ? 1 : 0) ? (g.k + KC - 1) / KC : 0;
  uint32_t phase0 = 0, phase1 = 0;
  for (int c = 0; c < nchunks; ++c) {
    const int b = c & 1;
    unsigned char* Ahi = sm + b * BUF;
    unsigned char* Alo = Ahi + A_BYTES;
    unsigned char* Bhi = Alo + A_BYTES;
    unsigned char* Blo = Bhi + B_BYTES;
    if (c >= 2) {   // the MMAs of chunk c - 2 read this buffer
      if (b == 0) { ok = mbar_wait(&mbar[0], phase0) && ok; phase0 ^= 1; }
      else { ok = mbar_wait(&mbar[1], phase1) && ok; phase1 ^= 1; }
    }
    const int k0 = c * KC;
    // op(A) chunk: 64 x 16 complex
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int mm, kk;
      float2 a = make_float2(0.f, 0.f);
      if (!g.conj_a) {
        mm = tid & 63; kk = (tid >> 6) + 2 * i;
        if (m0 + mm < g.m && k0 + kk < g.k) a = g.A[(m0 + mm) + (size_t)(k0 + kk) * g.lda];
      } else {
        kk = tid & 15; mm = (tid >> 4) + 8 * i;
        if (m0 + mm < g.m && k0 + kk < g.k) {
          a = g.A[(k0 + kk) + (size_t)(m0 + mm) * g.lda];
          a.y = -a.y;
        }
      }
      put_split(Ahi, Alo, core_off(mm, kk), a.x);
      put_split(Ahi, Alo, core_off(mm, KC + kk), -a.y);
      put_split(Ahi, Alo, core_off(TC_TM + mm, kk), a.y);
      put_split(Ahi, Alo, core_off(TC_TM + mm, KC + kk), a.x);
    }
    // op(B) chunk: 16 x 32 complex, stored transposed (row = output column)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int kk, nn;
      float2 v = make_float2(0.f, 0.f);
      if (!g.conj_b) {
        kk = tid & 15; nn = (tid >> 4) + 8 * i;
        if (n0 + nn < g.n && k0 + kk < g.k) v = g.B[(k0 + kk) + (size_t)(n0 + nn) * g.ldb];
      } else {
        nn = tid & 31; kk = (tid >> 5) + 4 * i;
        if (n0 + nn < g.n && k0 + kk < g.k) {
          v = g.B[(n0 + nn) + (size_t)(k0 + kk) * g.ldb];
          v.y = -v.y;
        }
      }
      put_split(Bhi, Blo, core_off(nn, kk), v.x);
      put_split(Bhi, Blo, core_off(nn, KC + kk), v.y);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
      for (int s = 0; s < KR / 8; ++s) {
        const uint32_t o = s * 2 * LBO;   // 8 tf32 along k = two core matrices
        mma_tf32(tmem, sdesc(ah + o), sdesc(bh + o), (c > 0 || s > 0) ? 1u : 0u);
        mma_tf32(tmem, sdesc(ah + o), sdesc(bl + o), 1u);
        mma_tf32(tmem, sdesc(al + o), sdesc(bh + o), 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[b]))
                   : "memory");
    }
  }
  // the last commit tracks every MMA issued before it
  float d[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) d[j] = 0.f;
  if (nchunks > 0) {
    const int b = (nchunks - 1) & 1;
    ok = mbar_wait(&mbar[b], b == 0 ? phase0 : phase1) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // tcgen05.ld is warp-collective: the whole warp takes the same branch
    if (__all_sync(0xffffffffu, ok ? 1 : 0)) {
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16);
      tcx::tmem_ld32(ta, d);
    }
  }
  // ok is per thread: make the CTA agree before branching on it
  const int all_ok = __syncthreads_and(ok ? 1 : 0);
  float* s_d = reinterpret_cast<float*>(sm);   // buffer 0 is free: every MMA has completed
  if (all_ok) {
#pragma unroll
    for (int j = 0; j < 32; ++j) s_d[tid * 33 + j] = d[j];
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  if (!all_ok) {
    if (tid == 0) atomicExch(err, 1);
    return;
  }
#pragma unroll 4
  for (int i = 0; i < 16; ++i) {
    const int mm = tid & 63, nn = (tid >> 6) + 2 * i;
    if (m0 + mm < g.m && n0 + nn < g.n) {
      const float re = s_d[mm * 33 + nn], im = s_d[(TC_TM + mm) * 33 + nn];
      float2* cp = g.C + (m0 + mm) + (size_t)(n0 + nn) * g.ldc;
      float2 v = make_float2(g.alpha.x * re - g.alpha.y * im, g.alpha.x * im + g.alpha.y * re);
      if (g.beta.x != 0.f || g.beta.y != 0.f) {
        const float2 c0 = *cp;
        v.x += g.beta.x * c0.x - g.beta.y * c0.y;
        v.y += g.beta.x * c0.y + g.beta.y * c0.x;
      }
      *cp = v;
    }
  }
}

}  // namespace

void tc_gemm_batched(const TcGemmProb* d_prob, const int* d_tile_off, int nprob, int total_tiles, int* d_err,
                     cudaStream_t st, int tile_base, bool no_arrive) {
  if (nprob <= 0 || total_tiles <= 0) return;
  // the same value every time: idempotent across threads and devices
  cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  KPROF_BEGIN(st);
  k_tc_gemm<<<total_tiles, TC_T, SMEM_BYTES, st>>>(d_prob, d_tile_off, nprob, tile_base, d_err, no_arrive ? 1 : 0);
  pm_launch_count_add(1);
  KPROF_END(st, "tc_gemm32", 0.0);
}
