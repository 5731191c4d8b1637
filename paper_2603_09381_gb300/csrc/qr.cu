// Blocked, unpivoted Householder QR of the tall ID inputs (W x n, W > n),
// ahead of their column-pivoted QR (paper Sec. 3 computes the ID by CPQR).
// Q^H preserves the norm of every trailing column block, so the pivoted
// factorization of the n x n triangle R picks the pivots of Z and returns its
// R (exact arithmetic); the pivoted steps then stream n instead of W rows.
//
// Per panel of QR_NB columns: a cluster of 1-8 CTAs per matrix factors the
// panel (LAPACK zlarfg phase convention, H = I - tau v v^H, Q^H applied) with
// one pass over the panel per reflector (the pass that applies reflector j
// also sums the norm and the dot products that define reflector j+1); the
// cluster's CTAs split the rows and add their partial sums through
// distributed shared memory, every CTA forming the same reflector from the
// same sums.  It then forms the compact-WY factor T (Q = I - V T V^H).
// Q^H = I - V T^H V^H is applied to every 32-column tile of the trailing
// block in three launches: partial products Y_b = V_b^H C_b per (tile,
// QR_RB-row block), their sum in block order times T^H, and C_b -= V_b Y per
// (tile, block), so that the rows of a tall matrix spread over many CTAs.
#include "cpqr.cuh"
#include "prof.cuh"
#include "tc_common.cuh"
#include <cooperative_groups.h>
#include <type_traits>

namespace cg = cooperative_groups;

namespace {

constexpr int PT = 512;      // panel CTA: two threads per row, 16 panel columns each
constexpr int PR = PT / 2;   // rows per sweep of the panel CTA
constexpr int UT = 256;      // update CTA
constexpr int RC = 32;       // rows per staged chunk
constexpr int HB = QR_NB / 2;

// V entry (row r, panel column j) of a panel starting at j0: unit diagonal,
// zero above, the stored reflector below.
template <typename C>
__device__ __forceinline__ C v_entry(const QrProb<C>& p, int j0, int jb, int r, int j) {
  typedef typename real_of<C>::type R;
  if (j >= jb || r >= p.W) return czero<C>();
  const int d = j0 + j;
  if (r < d) return czero<C>();
  if (r == d) return mk((R)1, (R)0);
  return p.Z[r + (size_t)d * p.ld];
}

// One pass over the panel rows: applies reflector `ja` (if ja >= 0; its
// factors f_k in s_f, its column scaled by sc into v) and accumulates the
// inputs of step jn = ja + 1: N = sum_{r >= c'} |a_jn[r]|^2 and
// S_k = sum_{r > c'} conj(a_jn[r]) a_k[r] for k > jn (c' = j0 + jn), with row
// c' itself stored to s_row.  Lanes 0-15 of a warp hold panel columns 0-15 of
// 16 rows, lanes 16-31 columns 16-31 of the same rows; every entry a thread
// needs is loaded before the pair stores anything.
template <typename C>
__device__ __forceinline__ void panel_pass(const QrProb<C>& p, int j0, int jb, int ja, const C* s_f, C sc,
                                           C* s_row, typename real_of<C>::type& N, C* S, int rank, int csize) {
  typedef typename real_of<C>::type R;
  const int jn = ja + 1;
  const int ca = j0 + ja, cn = j0 + jn;
  C* Zp = p.Z + (size_t)j0 * p.ld;
  const size_t ld = p.ld;
  const int lane = threadIdx.x & 31, half = lane >> 4;
  const int kb = half * HB;
  const int kmin = ja >= 0 ? ja : jn;
  const C fjn = (ja >= 0 && jn < jb) ? s_f[jn] : czero<C>();
  // warp-uniform sweep (the __syncwarp below needs every lane), rows guarded
  for (int r0 = (ja >= 0 ? ca : cn) + (threadIdx.x >> 5) * 16 + rank * PR; r0 < p.W; r0 += PR * csize) {
    const int r = r0 + (lane & 15);
    const bool act = r < p.W;
    C v[HB];
#pragma unroll
    for (int k = 0; k < HB; ++k)
      if (act && kb + k >= kmin && kb + k < jb) v[k] = Zp[r + (size_t)(kb + k) * ld];
    const C x = (act && ja >= 0) ? Zp[r + (size_t)ja * ld] : czero<C>();
    const C yold = (act && jn < jb) ? Zp[r + (size_t)jn * ld] : czero<C>();
    __syncwarp();   // both threads of the pair have read the row before either writes it
    if (!act) continue;
    C vr = czero<C>();
    if (ja >= 0) {
      vr = (r == ca) ? mk((R)1, (R)0) : x * sc;
      if (r > ca && half == (ja >= HB)) Zp[r + (size_t)ja * ld] = vr;
#pragma unroll
      for (int k = 0; k < HB; ++k)
        if (kb + k > ja && kb + k < jb) {
          cfms(v[k], s_f[kb + k], vr);
          Zp[r + (size_t)(kb + k) * ld] = v[k];
        }
    }
    if (jn < jb && r >= cn) {
      C y = yold;
      if (ja >= 0) cfms(y, fjn, vr);
      if (half == 0) N += abs2(y);
      if (r == cn) {
#pragma unroll
        for (int k = 0; k < HB; ++k) if (kb + k >= jn && kb + k < jb) s_row[kb + k] = v[k];
      } else {
#pragma unroll
        for (int k = 0; k < HB; ++k) if (kb + k > jn && kb + k < jb) cfma_conj(S[k], y, v[k]);
      }
    }
  }
}

template <typename C>
// At most 112 registers: 512 x 112 leaves room on the SM for one CTA of the
// operator assembly that may run beside the factorization.
__global__ void __maxnreg__(112) k_qr_panel(const QrProb<C>* __restrict__ P, int j0) {
  typedef typename real_of<C>::type R;
  cg::cluster_group cluster = cg::this_cluster();
  const int csize = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const QrProb<C> p = P[blockIdx.x / csize];
  if (j0 >= p.n) return;   // the whole cluster (same matrix) leaves
  const int jb = min(QR_NB, p.n - j0);
  const int W = p.W;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, half = lane >> 4;
  constexpr int NV = 4 * QR_NB + 1;   // S (re, im), N, row c' (re, im)
  __shared__ R s_red[PT / 32][2 * QR_NB + 1];
  __shared__ R s_part[2][NV];         // this CTA's partial sums, by pass parity
  __shared__ R s_tot[NV];
  __shared__ C s_f[QR_NB];
  __shared__ C s_row[QR_NB];          // row c' entries held by this CTA (zero elsewhere)
  __shared__ C s_tau[QR_NB];
  __shared__ C s_sc;
  __shared__ C s_v[RC][QR_NB + 1];
  __shared__ C s_g[QR_NB][QR_NB + 1];
  __shared__ C s_t[QR_NB][QR_NB + 1];
  if (tid < QR_NB) s_row[tid] = czero<C>();
  __syncthreads();
  C sc = czero<C>();
  int par = 0;
  for (int ja = -1; ja < jb; ++ja, par ^= 1) {
    R N = 0;
    C S[HB];
#pragma unroll
    for (int k = 0; k < HB; ++k) S[k] = czero<C>();
    panel_pass(p, j0, jb, ja, s_f, sc, s_row, N, S, rank, csize);
    const int jn = ja + 1;
    if (jn >= jb) break;
    // CTA sums: N over all lanes, S_k over the 16 lanes of each half
    N = warp_sum(N);
#pragma unroll
    for (int k = 0; k < HB; ++k)
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        S[k].x += __shfl_xor_sync(0xffffffffu, S[k].x, o);
        S[k].y += __shfl_xor_sync(0xffffffffu, S[k].y, o);
      }
    if ((lane & 15) == 0) {
#pragma unroll
      for (int k = 0; k < HB; ++k) {
        s_red[warp][2 * (half * HB + k)] = S[k].x;
        s_red[warp][2 * (half * HB + k) + 1] = S[k].y;
      }
      if (half == 0) s_red[warp][2 * QR_NB] = N;
    }
    __syncthreads();
    if (tid < 2 * QR_NB + 1) {
      R t = 0;
#pragma unroll
      for (int w = 0; w < PT / 32; ++w) t += s_red[w][tid];
      s_part[par][tid] = t;
    } else if (tid < NV) {
      const int k = (tid - 2 * QR_NB - 1) >> 1;
      s_part[par][tid] = ((tid - 2 * QR_NB - 1) & 1) ? s_row[k].y : s_row[k].x;
    }
    cluster.sync();   // every CTA's partials of this pass are written
    if (tid < NV) {
      R t = 0;
      for (int q = 0; q < csize; ++q) t += cluster.map_shared_rank(&s_part[par][0], q)[tid];   // rank order
      s_tot[tid] = t;
    }
    if (tid < QR_NB) s_row[tid] = czero<C>();
    __syncthreads();
    if (tid == 0) {
      // reflector of column jn (LAPACK zlarfg phase), factors of the next pass
      const int c = j0 + jn;
      const C alpha = mk(s_tot[2 * QR_NB + 1 + 2 * jn], s_tot[2 * QR_NB + 2 + 2 * jn]);
      const R xnorm = sqrt(s_tot[2 * QR_NB]);
      C tau = czero<C>(), scn = czero<C>();
      R beta = 0;
      if (xnorm > 0) {
        beta = -copysign(xnorm, alpha.x);
        const C bm = mk(beta, (R)0);
        tau = cdiv(bm - alpha, bm);
        scn = cdiv(mk((R)1, (R)0), alpha - bm);
      }
      if (rank == 0) p.Z[c + (size_t)c * p.ld] = mk(beta, (R)0);
      s_tau[jn] = tau;
      s_sc = scn;
      const C ctau = conj(tau), cscn = conj(scn);
      for (int k = jn + 1; k < jb; ++k) {
        const C rowk = mk(s_tot[2 * QR_NB + 1 + 2 * k], s_tot[2 * QR_NB + 2 + 2 * k]);
        s_f[k] = ctau * (rowk + cscn * mk(s_tot[2 * k], s_tot[2 * k + 1]));
      }
    }
    __syncthreads();
    sc = s_sc;
  }
  // the last pass stored its reflector in rows that other CTAs of the
  // cluster read below (rows are dealt out differently there)
  cluster.sync();
  // G = V^H V over chunks of this CTA's rows staged in shared memory (V also
  // written out), then summed over the cluster
  {
    const int gi = tid & 31, gj = tid >> 5;   // G[gi][gj] and G[gi][gj + 16]
    C g0 = czero<C>(), g1 = czero<C>();
    for (int r0 = j0 + rank * RC; r0 < W; r0 += RC * csize) {
      for (int e = tid; e < RC * QR_NB; e += PT) {
        const int i = e % RC, j = e / RC;
        const C v = v_entry(p, j0, jb, r0 + i, j);
        s_v[i][j] = v;
        if (p.V && r0 + i < W) p.V[(r0 + i - j0) + (size_t)j * p.W] = v;
      }
      __syncthreads();
#pragma unroll 8
      for (int i = 0; i < RC; ++i) {
        const C a = s_v[i][gi];
        cfma_conj(g0, a, s_v[i][gj]);
        cfma_conj(g1, a, s_v[i][gj + 16]);
      }
      __syncthreads();
    }
    s_t[gi][gj] = g0;   // s_t holds this CTA's partial G until T is built
    s_t[gi][gj + 16] = g1;
    cluster.sync();
    C a0 = czero<C>(), a1 = czero<C>();
    for (int q = 0; q < csize; ++q) {
      const C* rt = &cluster.map_shared_rank(&s_t[0][0], q)[0];
      a0 = a0 + rt[gi * (QR_NB + 1) + gj];
      a1 = a1 + rt[gi * (QR_NB + 1) + gj + 16];
    }
    s_g[gi][gj] = a0;
    s_g[gi][gj + 16] = a1;
    cluster.sync();   // no CTA reuses s_t (or leaves) while another still reads it
  }
  // T: T_jj = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] G[0:j, j]
  for (int e = tid; e < QR_NB * QR_NB; e += PT) {
    const int i = e % QR_NB, j = e / QR_NB;
    s_t[i][j] = (i == j && i < jb) ? s_tau[i] : czero<C>();
  }
  __syncthreads();
  for (int j = 1; j < jb; ++j) {
    if (tid < j) {
      C acc = czero<C>();
      for (int l = tid; l < j; ++l) cfma(acc, s_t[tid][l], s_g[l][j]);
      s_t[tid][j] = -(s_tau[j] * acc);
    }
    __syncthreads();
  }
  if (rank == 0)
    for (int e = tid; e < QR_NB * QR_NB; e += PT) p.T[e] = s_t[e % QR_NB][e / QR_NB];
}

// Trailing update Q^H C = C - V (T^H (V^H C)) for every 32-column tile of
// the trailing block, in three launches so that the rows of a tall matrix
// spread over many CTAs: partial products Y_b = V_b^H C_b of each block of
// QR_RB rows; their sum (fixed order) times T^H; C_b -= V_b Y.
template <typename C>
__global__ void __launch_bounds__(UT) k_qr_ypart(const QrProb<C>* __restrict__ P, int j0) {
  const QrProb<C> p = P[blockIdx.z];
  if (j0 >= p.n) return;
  const int jb = min(QR_NB, p.n - j0);
  const int tile = blockIdx.x, rb = blockIdx.y;
  const int c0 = j0 + jb + tile * 32;
  const int rbeg = j0 + rb * QR_RB;
  if (c0 >= p.n || rbeg >= p.W) return;
  const int nc = min(32, p.n - c0), rend = min(p.W, rbeg + QR_RB);
  const int tid = threadIdx.x;
  __shared__ C s_v[RC][QR_NB + 1];
  __shared__ C s_c[RC][33];
  const int tx = tid & 15, ty = tid >> 4;
  C y00 = czero<C>(), y01 = czero<C>(), y10 = czero<C>(), y11 = czero<C>();
  for (int r0 = rbeg; r0 < rend; r0 += RC) {
    for (int e = tid; e < RC * 32; e += UT) {
      const int i = e % RC, j = e / RC, r = r0 + i;
      s_v[i][j] = r < rend ? v_entry(p, j0, jb, r, j) : czero<C>();
      s_c[i][j] = (j < nc && r < rend) ? p.Z[r + (size_t)(c0 + j) * p.ld] : czero<C>();
    }
    __syncthreads();
#pragma unroll 8
    for (int i = 0; i < RC; ++i) {
      const C a0 = s_v[i][tx], a1 = s_v[i][tx + 16], b0 = s_c[i][ty], b1 = s_c[i][ty + 16];
      cfma_conj(y00, a0, b0); cfma_conj(y01, a0, b1);
      cfma_conj(y10, a1, b0); cfma_conj(y11, a1, b1);
    }
    __syncthreads();
  }
  C* yp = p.Yp + ((size_t)tile * p.mrb + rb) * (QR_NB * 32);
  yp[tx + QR_NB * ty] = y00;
  yp[tx + QR_NB * (ty + 16)] = y01;
  yp[tx + 16 + QR_NB * ty] = y10;
  yp[tx + 16 + QR_NB * (ty + 16)] = y11;
}

// Y = sum of the row blocks' partials (in block order), then T^H Y into the
// tile's first partial slot.
template <typename C>
__global__ void __launch_bounds__(UT) k_qr_yreduce(const QrProb<C>* __restrict__ P, int j0) {
  const QrProb<C> p = P[blockIdx.y];
  if (j0 >= p.n) return;
  const int jb = min(QR_NB, p.n - j0);
  const int tile = blockIdx.x;
  if (j0 + jb + tile * 32 >= p.n) return;
  const int nrb = (p.W - j0 + QR_RB - 1) / QR_RB;
  const int tid = threadIdx.x;
  __shared__ C s_y[QR_NB][33];
  __shared__ C s_t[QR_NB][QR_NB + 1];
  C* yp = p.Yp + (size_t)tile * p.mrb * (QR_NB * 32);
  for (int e = tid; e < QR_NB * 32; e += UT) {
    C acc = czero<C>();
    for (int b = 0; b < nrb; ++b) acc = acc + yp[(size_t)b * (QR_NB * 32) + e];
    s_y[e % QR_NB][e / QR_NB] = acc;
  }
  for (int e = tid; e < QR_NB * QR_NB; e += UT) s_t[e % QR_NB][e / QR_NB] = p.T[e];
  __syncthreads();
  for (int e = tid; e < QR_NB * 32; e += UT) {
    const int i = e % QR_NB, cc = e / QR_NB;
    C acc = czero<C>();
    for (int l = 0; l <= i; ++l) cfma_conj(acc, s_t[l][i], s_y[l][cc]);
    yp[e] = acc;
  }
}

template <typename C>
__global__ void __launch_bounds__(UT) k_qr_apply(const QrProb<C>* __restrict__ P, int j0) {
  const QrProb<C> p = P[blockIdx.z];
  if (j0 >= p.n) return;
  const int jb = min(QR_NB, p.n - j0);
  const int tile = blockIdx.x, rb = blockIdx.y;
  const int c0 = j0 + jb + tile * 32;
  const int rbeg = j0 + rb * QR_RB;
  if (c0 >= p.n || rbeg >= p.W) return;
  const int nc = min(32, p.n - c0), rend = min(p.W, rbeg + QR_RB);
  const int tid = threadIdx.x;
  __shared__ C s_v[RC][QR_NB + 1];
  __shared__ C s_y[QR_NB][33];
  const C* yp = p.Yp + (size_t)tile * p.mrb * (QR_NB * 32);
  for (int e = tid; e < QR_NB * 32; e += UT) s_y[e % QR_NB][e / QR_NB] = yp[e];
  const int ri = tid & 31, g = tid >> 5;
  for (int r0 = rbeg; r0 < rend; r0 += RC) {
    __syncthreads();
    for (int e = tid; e < RC * QR_NB; e += UT) {
      const int i = e % RC, j = e / RC;
      s_v[i][j] = v_entry(p, j0, jb, r0 + i, j);
    }
    __syncthreads();
    C acc[4] = {czero<C>(), czero<C>(), czero<C>(), czero<C>()};
    for (int j = 0; j < jb; ++j) {
      const C v = s_v[ri][j];
#pragma unroll
      for (int q = 0; q < 4; ++q) cfma(acc[q], v, s_y[j][4 * g + q]);
    }
    const int r = r0 + ri;
    if (r < rend) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (4 * g + q < nc) {
          C* pz = p.Z + r + (size_t)(c0 + 4 * g + q) * p.ld;
          *pz = *pz - acc[q];
        }
    }
  }
}

// C_b -= V_b Y on the fifth-generation tensor cores (complex64, the default
// path): one CTA per 64-row block of a matrix walks all 32-column tiles of
// its trailing block.  The complex product is a real one of twice the size,
// [Re D; Im D] = [[Re V, -Im V], [Im V, Re V]] [Re Y; Im Y], i.e. an
// M = 128, N = 32, K = 64 real MMA; every FP32 operand is split into tf32
// parts x = hi + lo and hi*hi + hi*lo + lo*hi are accumulated in FP32 (the
// 3xTF32 scheme, FP32 accuracy), and each tile's accumulation is only 64
// real terms long.  V_b is split into shared memory once; per tile the CTA
// stages Y (from the row-block reduction) into one of two buffers, one
// thread issues the 24 MMAs into one of two TMEM accumulators and commits
// them to that buffer's mbarrier, and the epilogue of the previous tile
// (tcgen05.ld by all eight warps, each with a quarter of the rows and half
// of the columns, then each thread's component of C -= D, with C loaded one
// tile ahead) overlaps them.  Every wait is bounded; a wait that runs out
// sets *err and the CTA stops writing.
namespace tcq {
constexpr int T = 256;                         // threads: warp w reads TMEM lanes [32 (w % 4), + 32), columns 16 (w / 4) ..
constexpr int ROWS = 64;                       // complex rows per CTA
constexpr int KR = 2 * QR_NB;                  // real k: real and imaginary parts of the reflectors
constexpr uint32_t A_BYTES = 2 * ROWS * KR * 4;    // one of hi / lo: 128 x 64 tf32
constexpr uint32_t B_BYTES = 32 * KR * 4;          // one of hi / lo: 32 x 64 tf32
constexpr uint32_t OFF_B = 2 * A_BYTES;            // two buffers of (hi, lo)
constexpr uint32_t OFF_BAR = OFF_B + 4 * B_BYTES;
constexpr int SMEM = OFF_BAR + 64;
constexpr uint32_t IDESC = tcx::idesc_tf32(2 * ROWS, 32);
constexpr uint32_t TMEM_COLS = 64;             // two 32-column accumulators
constexpr int WAIT = 1 << 20;                  // x ~1 us suspend hint: about a second
}  // namespace tcq

// no_arrive (tests of the timeout path): every CTA first waits, with a bound
// of about a millisecond, on a barrier that nothing arrives at, then issues
// nothing, frees its tensor memory and sets *err.
// At most 112 registers: two CTAs per SM beside one CTA of the operator assembly.
__global__ void __maxnreg__(112) k_qr_apply_tc(const QrProb<float2>* __restrict__ P, int j0, int* err,
                                                        int no_arrive) {
  using namespace tcq;
  extern __shared__ __align__(1024) unsigned char sm[];
  const QrProb<float2> p = P[blockIdx.y];
  if (j0 >= p.n) return;
  const int jb = min(QR_NB, p.n - j0);
  const int cfirst = j0 + jb;
  const int ntiles = (p.n - cfirst + 31) / 32;
  const int rbeg = j0 + (int)blockIdx.x * ROWS;
  if (ntiles <= 0 || rbeg >= p.W) return;
  const int rend = min(p.W, rbeg + ROWS);
  const int tid = threadIdx.x, warp = tid >> 5;
  unsigned char* Ahi = sm;
  unsigned char* Alo = sm + A_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + OFF_BAR);
  uint32_t* s_taddr = reinterpret_cast<uint32_t*>(sm + OFF_BAR + 24);
  if (tid == 0) {
    tcx::mbar_init(&mbar[0]);
    tcx::mbar_init(&mbar[1]);
    tcx::mbar_init(&mbar[2]);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tcx::smem_u32(s_taddr)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // A: the block's reflector rows (unit diagonal, zeros above it and past W)
#pragma unroll 4
  for (int i = 0; i < 8; ++i) {
    const int mm = tid & 63, kk = (tid >> 6) + 4 * i;
    const float2 v = v_entry(p, j0, jb, rbeg + mm, kk);
    tcx::put_split(Ahi, Alo, tcx::core_off<KR>(mm, kk), v.x);
    tcx::put_split(Ahi, Alo, tcx::core_off<KR>(mm, QR_NB + kk), -v.y);
    tcx::put_split(Ahi, Alo, tcx::core_off<KR>(ROWS + mm, kk), v.y);
    tcx::put_split(Ahi, Alo, tcx::core_off<KR>(ROWS + mm, QR_NB + kk), v.x);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *s_taddr;
  bool ok = true;
  if (no_arrive) ok = tcx::mbar_wait(&mbar[2], 0, 1 << 10);
  const int nt = __syncthreads_and(ok ? 1 : 0) ? ntiles : -1;
  // Epilogue work split: warp w reads TMEM lanes 32 (w % 4) .. + 32, i.e.
  // D's real row lane = 32 (w % 4) + (tid & 31): the real (lane < 64) or
  // imaginary (lane >= 64) part of complex row rbeg + (lane & 63), columns
  // 16 (w / 4) .. + 16 of the tile; each thread updates that component of C
  // itself (no exchange).  C of tile t is loaded at iteration t and updated
  // at iteration t + 1, and Y of tile t + 1 is loaded at iteration t, so
  // their latency overlaps the MMAs and the previous epilogue.
  const int lane_row = 32 * (warp & 3) + (tid & 31), hcol = 16 * (warp >> 2);
  const int r = lane_row & 63, comp = lane_row >> 6;
  const int row = rbeg + r;
  const bool row_ok = row < rend;
  float cnext[16], ccur[16];
  float2 ynext[4];
  auto load_y = [&](int t) {
    const float2* yp = p.Yp + (size_t)t * p.mrb * (QR_NB * 32);
#pragma unroll
    for (int i = 0; i < 4; ++i) ynext[i] = yp[(tid & 31) + QR_NB * ((tid >> 5) + 8 * i)];
  };
  if (nt > 0) load_y(0);
  for (int t = 0; t <= nt; ++t) {
    if (t < nt) {
      const int b = t & 1;
      unsigned char* Bhi = sm + OFF_B + b * 2 * B_BYTES;
      unsigned char* Blo = Bhi + B_BYTES;
      // Y of tile t (rows: reflectors, columns: the tile's columns), stored transposed;
      // buffer b was last read by the MMAs of tile t - 2, waited for at iteration t - 1
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int kk = tid & 31, nn = (tid >> 5) + 8 * i;
        tcx::put_split(Bhi, Blo, tcx::core_off<KR>(nn, kk), ynext[i].x);
        tcx::put_split(Bhi, Blo, tcx::core_off<KR>(nn, QR_NB + kk), ynext[i].y);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t acc = tmem + (uint32_t)(b * 32);
        const uint32_t ah = tcx::smem_u32(Ahi), al = tcx::smem_u32(Alo);
        const uint32_t bh = tcx::smem_u32(Bhi), bl = tcx::smem_u32(Blo);
#pragma unroll
        for (int s = 0; s < KR / 8; ++s) {
          const uint32_t o = s * 2 * tcx::LBO;   // 8 tf32 along k = two core matrices
          tcx::mma_tf32<IDESC>(acc, tcx::sdesc<KR>(ah + o), tcx::sdesc<KR>(bh + o), s > 0 ? 1u : 0u);
          tcx::mma_tf32<IDESC>(acc, tcx::sdesc<KR>(ah + o), tcx::sdesc<KR>(bl + o), 1u);
          tcx::mma_tf32<IDESC>(acc, tcx::sdesc<KR>(al + o), tcx::sdesc<KR>(bh + o), 1u);
        }
        tcx::mma_commit(&mbar[b]);
      }
      if (t + 1 < nt) load_y(t + 1);
      // this thread's component of C, tile t, its 16 columns
      const int c0 = cfirst + t * 32 + hcol, nc = min(16, p.n - c0);
      const float* cz = reinterpret_cast<const float*>(p.Z + row + (size_t)c0 * p.ld) + comp;
#pragma unroll
      for (int j = 0; j < 16; ++j) cnext[j] = (row_ok && j < nc) ? cz[(size_t)j * 2 * p.ld] : 0.f;
    }
    if (t >= 1) {   // epilogue of tile u = t - 1
      const int u = t - 1, b = u & 1;
      ok = ok && tcx::mbar_wait(&mbar[b], (uint32_t)((u >> 1) & 1), WAIT);   // after a failure: no more waits
      asm volatile("tcgen05.fence::after_thread_sync;");
      float d[16];
      const bool wok = __all_sync(0xffffffffu, ok ? 1 : 0);
      if (wok) {
        tcx::tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(b * 32 + hcol), d);
        const int c0 = cfirst + u * 32 + hcol, nc = min(16, p.n - c0);
        float* cz = reinterpret_cast<float*>(p.Z + row + (size_t)c0 * p.ld) + comp;
        if (row_ok) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (j < nc) cz[(size_t)j * 2 * p.ld] = ccur[j] - d[j];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) ccur[j] = cnext[j];
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  const int all_ok = __syncthreads_and(ok ? 1 : 0);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  if (!all_ok && tid == 0) atomicExch(err, 1);
}

// Zeros below the diagonal of the top n x n block (the reflectors' storage).
template <typename C>
__global__ void k_qr_zero_lower(const QrProb<C>* __restrict__ P) {
  const QrProb<C> p = P[blockIdx.y];
  const int j = blockIdx.x;
  if (j >= p.n) return;
  C* col = p.Z + (size_t)j * p.ld;
  for (int r = j + 1 + threadIdx.x; r < p.n; r += blockDim.x) col[r] = czero<C>();
}

}  // namespace

template <typename C>
void qr_panel(const QrProb<C>* d_prob, int nprob, int j0, cudaStream_t st) {
  if (nprob <= 0) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // cluster of up to 8 CTAs per matrix, enough to fill the SMs (one CTA per SM)
  int cs = 1;
  while (cs < 8 && (long)nprob * cs * 2 <= sms) cs *= 2;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nprob * cs);
  cfg.blockDim = dim3(PT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  KPROF_BEGIN(st);
  cudaLaunchKernelEx(&cfg, k_qr_panel<C>, d_prob, j0);
  pm_launch_count_add(1);
  KPROF_END(st, kname<C>("qr_panel", "qr_panel32"), 0.0);
}
template <typename C>
void qr_update(const QrProb<C>* d_prob, int nprob, int j0, int max_tiles, int max_rb, cudaStream_t st,
               int* tc_err, int max_w, bool no_arrive) {
  if (nprob <= 0 || max_tiles <= 0 || max_rb <= 0) return;
  KPROF_BEGIN(st);
  k_qr_ypart<C><<<dim3(max_tiles, max_rb, nprob), UT, 0, st>>>(d_prob, j0);
  k_qr_yreduce<C><<<dim3(max_tiles, nprob), UT, 0, st>>>(d_prob, j0);
  bool on_tc = false;
  if constexpr (std::is_same<C, float2>::value) {
    if (tc_err) {
      // the same value every time: idempotent across threads and devices
      cudaFuncSetAttribute(k_qr_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tcq::SMEM);
      const int rblocks = (max_w - j0 + tcq::ROWS - 1) / tcq::ROWS;
      if (rblocks > 0) k_qr_apply_tc<<<dim3(rblocks, nprob), tcq::T, tcq::SMEM, st>>>(d_prob, j0, tc_err,
                                                                                       no_arrive ? 1 : 0);
      on_tc = true;
    }
  }
  if (!on_tc) k_qr_apply<C><<<dim3(max_tiles, max_rb, nprob), UT, 0, st>>>(d_prob, j0);
  pm_launch_count_add(3);
  KPROF_END(st, on_tc ? "qr_update_tc32" : kname<C>("qr_update", "qr_update32"), 0.0);
}
template <typename C>
void qr_zero_lower(const QrProb<C>* d_prob, int nprob, int max_n, cudaStream_t st) {
  if (nprob <= 0 || max_n <= 0) return;
  k_qr_zero_lower<C><<<dim3(max_n, nprob), 256, 0, st>>>(d_prob);
  pm_launch_count_add(1);
}

template void qr_panel<float2>(const QrProb<float2>*, int, int, cudaStream_t);
template void qr_update<float2>(const QrProb<float2>*, int, int, int, int, cudaStream_t, int*, int, bool);
template void qr_zero_lower<float2>(const QrProb<float2>*, int, int, cudaStream_t);
