// Host runtime of the PMCHWT (Omit) proxy fast direct solver: C ABI entry
// points, quadtree planner, level scheduler and device memory arenas.
// Every numerical step runs in the CUDA kernels of assemble.cu, cpqr.cu and
// dense_la.cu; this file only plans index lists and launches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <tuple>
#include <mutex>
#include <thread>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/pmchwt.h"
#include "assemble.cuh"
#include "cpqr.cuh"
#include "tc_gemm.cuh"
#include "dense_la.cuh"
#include "field.cuh"
#include "mlp.cuh"
#include "operator.cuh"
#include "prof.cuh"

typedef double2 Cd;

thread_local KProf* g_kprof = nullptr;
static std::atomic<unsigned long long> g_launches{0};
void pm_launch_count_add(long n) { g_launches += (unsigned long long)n; }

namespace {

thread_local std::string g_err;

struct PmError {
  pm_status st;
  std::string msg;
};

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    pm_status s = (e == cudaErrorMemoryAllocation) ? PM_ERR_OOM : PM_ERR_CUDA;
    cudaGetLastError();
    throw PmError{s, std::string(what) + ": " + cudaGetErrorString(e)};
  }
}
#define CK(x) ck((x), #x)

void fail(pm_status s, const std::string& m) { throw PmError{s, m}; }

// Process-wide cache of freed device blocks.  Returning a large block with
// cudaFree unmaps it (25 ms for the 69 GB operator of a 65,536-unknown
// problem, 6 ms for 16 GB on GB300) and synchronises the device, and the next
// factorization of the same problem asks for the same sizes again.  A freed
// block is kept with an event recorded on the stream that last used it (only
// while the caller knows that stream to be alive), as idle when the caller has
// synchronised, or else after a device synchronisation (as cudaFree would
// do), and handed out again, best fit within 1.5x of the request, once that
// event has completed.  At most 45% of the device's memory stays cached; a cudaMalloc
// that fails releases this device's cached blocks and retries;
// pm_release_cached_memory releases them all.
struct PoolBlk {
  void* p;
  size_t size;
  int dev;
  cudaEvent_t ev;   // null: idle when cached
};
std::mutex g_pool_mu;
std::multimap<size_t, PoolBlk> g_pool;   // by size
size_t g_pool_bytes[64] = {};            // cached bytes per device

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d < 0 || d >= 64 ? 0 : d;
}

size_t pool_cached_bytes(int dev) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  return g_pool_bytes[dev];
}

// Frees every cached block of device dev (all devices: dev < 0); returns the bytes freed.
size_t pool_trim(int dev) {
  std::vector<PoolBlk> out;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto it = g_pool.begin(); it != g_pool.end();) {
      if (dev < 0 || it->second.dev == dev) {
        out.push_back(it->second);
        g_pool_bytes[it->second.dev] -= it->second.size;
        it = g_pool.erase(it);
      } else {
        ++it;
      }
    }
  }
  size_t n = 0;
  const int cur = current_device();
  for (auto& b : out) {
    if (b.dev != cur) cudaSetDevice(b.dev);
    if (b.ev) { cudaEventSynchronize(b.ev); cudaEventDestroy(b.ev); }
    cudaFree(b.p);
    if (b.dev != cur) cudaSetDevice(cur);
    n += b.size;
  }
  return n;
}

void* pool_malloc(size_t bytes) {
  const int dev = current_device();
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto it = g_pool.lower_bound(bytes); it != g_pool.end() && it->first <= bytes + bytes / 2; ++it) {
      const PoolBlk& b = it->second;
      if (b.dev != dev) continue;
      if (b.ev && cudaEventQuery(b.ev) != cudaSuccess) { cudaGetLastError(); continue; }
      void* p = b.p;
      if (b.ev) cudaEventDestroy(b.ev);
      g_pool_bytes[dev] -= it->first;
      g_pool.erase(it);
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) == cudaSuccess) return p;
  cudaGetLastError();
  if (pool_trim(dev) == 0) return nullptr;
  if (cudaMalloc(&p, bytes) == cudaSuccess) return p;
  cudaGetLastError();
  return nullptr;
}

// How the caller knows that the work using a block has finished.
enum class Done { Unknown, Idle, Stream };
// Done::Stream: st is a live stream whose work last used the block (an event
// is recorded on it); Done::Idle: the caller has synchronised; Done::Unknown:
// the device is synchronised here.
void pool_free(void* p, size_t bytes, Done how, cudaStream_t st = nullptr) {
  if (!p) return;
  const int dev = current_device();
  cudaEvent_t ev = nullptr;
  if (how == Done::Stream && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
    if (cudaEventRecord(ev, st) != cudaSuccess) { cudaEventDestroy(ev); ev = nullptr; cudaDeviceSynchronize(); }
  } else if (how != Done::Idle) {
    cudaDeviceSynchronize();
  }
  cudaGetLastError();
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  std::vector<PoolBlk> evict;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    g_pool.emplace(bytes, PoolBlk{p, bytes, dev, ev});
    g_pool_bytes[dev] += bytes;
    // over the cap: the largest other blocks of this device go first
    for (auto it = g_pool.end(); g_pool_bytes[dev] > tot / 100 * 45 && it != g_pool.begin();) {
      --it;
      if (it->second.dev != dev || it->second.p == p) continue;
      evict.push_back(it->second);
      g_pool_bytes[dev] -= it->first;
      it = g_pool.erase(it);
    }
  }
  for (auto& b : evict) {
    if (b.ev) { cudaEventSynchronize(b.ev); cudaEventDestroy(b.ev); }
    cudaFree(b.p);
  }
}

// Bump allocator over large device blocks (from the pool above); reset()
// keeps the blocks for reuse.  release() tells the pool how the blocks' work
// ends (the destructor: not known, so the device is synchronised).
struct Arena {
  struct Blk { char* p; size_t size; };
  std::vector<Blk> blks;
  size_t cur = 0, off = 0;
  size_t min_block = (size_t)64 << 20;
  void* alloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    while (cur < blks.size() && off + bytes > blks[cur].size) { ++cur; off = 0; }
    if (cur == blks.size()) {
      size_t sz = std::max(bytes, min_block);
      void* p = pool_malloc(sz);
      if (!p) fail(PM_ERR_OOM, "device memory: " + std::to_string(sz) + " bytes");
      blks.push_back({(char*)p, sz});
      off = 0;
    }
    void* r = blks[cur].p + off;
    off += bytes;
    return r;
  }
  template <class T> T* get(size_t n) { return (T*)alloc(n * sizeof(T)); }
  void reset() { cur = 0; off = 0; }
  void release(Done how = Done::Unknown, cudaStream_t st = nullptr) {
    for (auto& b : blks) {
      pool_free(b.p, b.size, how, st);
      if (how == Done::Unknown) how = Done::Idle;   // one device synchronisation covers the rest
    }
    blks.clear();
    cur = off = 0;
  }
  ~Arena() { release(); }
};

// While a solve plan is being captured into a CUDA graph, descriptor uploads
// must not become graph nodes (they read pageable host memory that is gone
// when the graph replays): they go, synchronously, through this side stream
// into plan-owned device memory that the graph's kernels then read.
thread_local cudaStream_t g_capture_side = nullptr;

template <class T>
T* upload(Arena& a, const std::vector<T>& v, cudaStream_t st) {
  T* d = a.get<T>(std::max<size_t>(v.size(), 1));
  if (v.empty()) return d;
  if (g_capture_side) {
    CK(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, g_capture_side));
    CK(cudaStreamSynchronize(g_capture_side));
  } else {
    CK(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  }
  return d;
}

template <class C>
__global__ void k_identity(C* A, int m, int ld) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  int i = e % m, j = e / m;
  A[i + (size_t)j * ld] = mk((typename real_of<C>::type)(i == j ? 1 : 0), (typename real_of<C>::type)0);
}

uint64_t morton(uint32_t x, uint32_t y) {
  uint64_t c = 0;
  for (int b = 0; b < 32; ++b) {
    c |= (uint64_t)((x >> b) & 1) << (2 * b);
    c |= (uint64_t)((y >> b) & 1) << (2 * b + 1);
  }
  return c;
}

struct Box {
  int bx, by;
  std::vector<int> leaves;    // inclusion ids
  std::vector<int> children;  // indices into the level below
  double cx = 0, cy = 0, r_cell = 0, R_p = 0;
  int p = 0;
  int p_rule = 0;        // the closed-form proxy count (or the fixed one)
  bool locked = false;   // proxy count fixed to p_rule after a failed held-out check
  std::vector<int> near;
};

}  // namespace

struct pm_geometry {
  int device = 0;       // the CUDA device the geometry (and its factors) live on
  int m = 0;
  double k0 = 0, spacing = 1;
  int gnx = 0, gny = 0;
  std::vector<pm_inclusion> inc;
  std::vector<int> node_off, row_off;
  int total_nodes = 0, N = 0, maxn = 0;
  std::vector<double> hx, hy, hnx, hny, hw;
  std::vector<InclDev> hinc;
  Arena arena;
  InclDev* d_inc = nullptr;
  NodesDev nodes{};
  // quadtree (paper Sec. 3; grid cells padded to 2^L x 2^L, Morton order)
  int L = 0;
  double ox = 0, oy = 0;
  bool general = false;   // spacing 0: an arbitrary arrangement, cells of the centres' bounding square
  std::vector<std::vector<Box>> levels;  // levels[l], l = 0..L

  // global index -> packed point code (node * 2 + group)
  int code_of(int g) const {
    int j = int(std::upper_bound(row_off.begin(), row_off.end(), g) - row_off.begin()) - 1;
    int loc = g - row_off[j];
    int n = inc[j].n_nodes;
    return (node_off[j] + loc % n) * 2 + (loc >= n ? 1 : 0);
  }
};

namespace {

template <class C>
struct BoxF {
  std::vector<int> rows, rgrp, cols, cgrp;
  int mb = 0, kb = 0, kg[2] = {0, 0};
  C *D = nullptr, *X = nullptr, *Rm = nullptr, *At = nullptr;
  int* ipiv = nullptr;
  std::vector<int> srows, scols;
  std::vector<int> srgrp, scgrp;
  std::vector<int> child_off;  // offsets of the children's blocks in rows/cols
};

typedef float2 Cf;

template <class C> inline C cone();
template <> inline double2 cone<double2>() { return make_double2(1, 0); }
template <> inline float2 cone<float2>() { return make_float2(1, 0); }
template <class C> inline C cmone();
template <> inline double2 cmone<double2>() { return make_double2(-1, 0); }
template <> inline float2 cmone<float2>() { return make_float2(-1, 0); }
template <class C> inline C czero_h();
template <> inline double2 czero_h<double2>() { return make_double2(0, 0); }
template <> inline float2 czero_h<float2>() { return make_float2(0, 0); }

}  // namespace

struct pm_factor {
  const pm_geometry* g = nullptr;
  pm_factor_opts opts{};
  cudaStream_t st = nullptr;
  int L = 0;
  int precision = PM_FP64;
  std::vector<std::vector<BoxF<double2>>> lev64;   // FP64 mode
  std::vector<std::vector<BoxF<float2>>> lev32;    // mixed mode (FP32 factorization)
  BoxF<double2> root;                              // top-level system, assembled in FP64
  float2* root32 = nullptr;                        // mixed mode: its complex64 LU factors
  int* ipiv32 = nullptr;
  SplitOp root_op{};                               // and the FP64 system (hi / lo planes) for one correction
  Arena arena, scratch;
  pm_stats stats{};
  std::vector<std::vector<Box>> tree;  // the geometry's quadtree with this factorization's proxies
  KProf prof;
  bool profiling = false;
  // learned rank predictor: features and adaptive ranks of every (box, group)
  std::vector<float> rank_X, rank_T;
  // per (box, group) sample: held-out proxy check ratio (-1: not run), box redone with the rule
  std::vector<float> proxy_ratio;
  std::vector<int> proxy_redone;
  // mixed mode: FP64 self blocks (operator for the refinement residual)
  std::vector<double2*> self64;
  int* d_iu = nullptr;
  int* d_iq = nullptr;
  float2* dense64 = nullptr;    // the whole FP64 operator, N x N, split: hi plane then lo plane, when it fits
  SplitOp dense_op{};           // its two planes
  bool op_started = false;      // index maps, column scales and the operator's assembly are enqueued
  bool op_pending = false;      // start the assembly beside the factorization once the leaves are assembled
  cudaStream_t op_st = nullptr; // the operator's assembly beside the factorization (low priority)
  cudaEvent_t op_done = nullptr;
  double* d_colscale = nullptr; // its column scales: A = dense64 diag(d_colscale)
  size_t dense_bytes = 0;
  // CUDA graphs of the compressed inverse (FP64) or the mixed preconditioner,
  // one per right-hand-side count; solves of one factor are serialised by plan_mu
  std::mutex plan_mu;
  std::map<std::pair<int, int>, std::unique_ptr<struct SolvePlan>> plans;   // (kind, nrhs)
  int graph_launches = 0, graph_captures = 0;
  // set by a bounded wait of the chained top-level solve that ran out (checked after every solve)
  int* d_wait_err = nullptr;
  ~pm_factor();
};

// A captured solve: plan-owned input / output / scale buffers, the arena of
// the captured launches (descriptors and workspace, never reused by anything
// else), and the instantiated graph.
struct SolvePlan {
  int uses = 0;
  Arena io, ws;
  double2* in = nullptr;
  double2* out = nullptr;
  double* scal = nullptr;
  cudaStream_t cap = nullptr, side = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~SolvePlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
    if (side) cudaStreamDestroy(side);
  }
};

namespace {
// Dense operators held by live factorizations, process-wide: concurrent
// factorizations (batches) must not each take a share of the same free memory.
std::mutex g_dense_mu;
size_t g_dense_held = 0;
}  // namespace

pm_factor::~pm_factor() {
  if (op_st) {
    cudaStreamSynchronize(op_st);
    cudaStreamDestroy(op_st);
  }
  if (op_done) cudaEventDestroy(op_done);
  if (dense64) {
    pool_free(dense64, dense_bytes, Done::Unknown);   // the caller's stream may be gone
    std::lock_guard<std::mutex> lk(g_dense_mu);
    g_dense_held -= dense_bytes;
  }
}

template <class C> std::vector<std::vector<BoxF<C>>>& levels_of(pm_factor* F);
namespace {
void start_mixed_operator(pm_factor* F, bool beside);
}
template <> std::vector<std::vector<BoxF<double2>>>& levels_of<double2>(pm_factor* F) { return F->lev64; }
template <> std::vector<std::vector<BoxF<float2>>>& levels_of<float2>(pm_factor* F) { return F->lev32; }

namespace {

void build_tree(pm_geometry* g, const pm_factor_opts* o) {
  // grid indices
  double ox = 1e300, oy = 1e300, mx = -1e300, my = -1e300;
  for (auto& c : g->inc) {
    ox = std::min(ox, c.cx); oy = std::min(oy, c.cy);
    mx = std::max(mx, c.cx); my = std::max(my, c.cy);
  }
  g->ox = ox; g->oy = oy;
  std::vector<int> ix(g->m), iy(g->m);
  int L = 0;
  if (g->general) {
    // the centres' bounding square (side = the larger extent, widened by
    // 1 + 2^-30) in 2^L x 2^L cells, L the smallest depth up to 20 that puts
    // every centre in a cell of its own
    const double ext = std::max(mx - ox, my - oy);
    g->spacing = 1.0;
    if (g->m > 1 && ext > 0) {
      const double side = ext * (1.0 + std::ldexp(1.0, -30));
      bool ok = false;
      for (L = 1; L <= 20 && !ok; ++L) {
        const double cell = side / (double)(1 << L);
        std::map<std::pair<int, int>, int> seen;
        ok = true;
        for (int j = 0; j < g->m && ok; ++j) {
          ix[j] = (int)std::floor((g->inc[j].cx - ox) / cell);
          iy[j] = (int)std::floor((g->inc[j].cy - oy) / cell);
          ok = seen.emplace(std::make_pair(ix[j], iy[j]), j).second;
        }
        if (ok) { g->spacing = cell; break; }
      }
      if (!ok) fail(PM_ERR_GEOMETRY, "inclusion centres too close to separate");
    } else {
      for (int j = 0; j < g->m; ++j) ix[j] = iy[j] = 0;
    }
  } else {
    const double s = g->spacing;
    int side = 1;
    std::map<std::pair<int, int>, int> seen;
    for (int j = 0; j < g->m; ++j) {
      ix[j] = (int)std::lround((g->inc[j].cx - ox) / s);
      iy[j] = (int)std::lround((g->inc[j].cy - oy) / s);
      if (ix[j] < 0 || iy[j] < 0 || ix[j] > (1 << 20) || iy[j] > (1 << 20)) fail(PM_ERR_GEOMETRY, "grid index out of range");
      if (!seen.emplace(std::make_pair(ix[j], iy[j]), j).second) fail(PM_ERR_GEOMETRY, "two inclusions share a grid cell");
      side = std::max(side, std::max(ix[j], iy[j]) + 1);
    }
    while ((1 << L) < side) ++L;
  }
  g->L = L;
  g->levels.assign(L + 1, {});
  std::vector<int> order(g->m);
  for (int j = 0; j < g->m; ++j) order[j] = j;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return morton(ix[a], iy[a]) < morton(ix[b], iy[b]); });
  for (int j : order) {
    Box b; b.bx = ix[j]; b.by = iy[j]; b.leaves = {j};
    g->levels[L].push_back(b);
  }
  for (int l = L - 1; l >= 0; --l) {
    auto& ch = g->levels[l + 1];
    std::vector<Box> par;
    for (int c = 0; c < (int)ch.size(); ++c) {
      int px = ch[c].bx >> 1, py = ch[c].by >> 1;
      if (par.empty() || par.back().bx != px || par.back().by != py) {
        Box b; b.bx = px; b.by = py;
        par.push_back(b);
      }
      par.back().children.push_back(c);
      for (int j : ch[c].leaves) par.back().leaves.push_back(j);
    }
    g->levels[l] = par;  // children of a Morton-ordered level are contiguous and ordered
  }
  (void)o;
}

// Proxy count for a fraction s of the rule's count: max(16, 8 ceil(s p / 8)).
int proxy_count(double s, int p_rule) { return std::max(16, 8 * (int)std::ceil(s * p_rule / 8.0)); }

// Proxy circles and near lists (depend on the tolerance and the proxy options).
void plan_proxies(const pm_geometry* g, std::vector<std::vector<Box>>& levels, const pm_factor_opts* o) {
  const double f = o->proxy_factor > 0 ? o->proxy_factor : 1.5;
  const int ctol = (int)std::ceil(std::log(1.0 / o->tol) / std::log(f));
  // PMCHWT (All) and Burton-Miller proxies carry the interior kernel too: the
  // closed-form count resolves the largest wavenumber
  double krule = g->k0;
  if (o->formulation != PM_FORM_OMIT)
    for (const auto& c : g->inc) krule = std::max(krule, c.k_in.re);
  const double s = g->spacing;
  for (int l = 0; l <= g->L; ++l) {
    const double scale = std::ldexp(1.0, g->L - l);
    auto& boxes = levels[l];
    for (auto& b : boxes) {
      if (!g->general) {
        b.cx = g->ox + s * (b.bx * scale + (scale - 1) / 2.0);
        b.cy = g->oy + s * (b.by * scale + (scale - 1) / 2.0);
      } else if (l == g->L) {   // a leaf's proxy circle around its inclusion
        b.cx = g->inc[b.leaves[0]].cx;
        b.cy = g->inc[b.leaves[0]].cy;
      } else {                  // a parent's around its cell
        b.cx = g->ox + s * (b.bx * scale + scale / 2.0);
        b.cy = g->oy + s * (b.by * scale + scale / 2.0);
      }
      double r = 0;
      for (int j : b.leaves)
        for (int q = g->node_off[j]; q < g->node_off[j + 1]; ++q)
          r = std::max(r, std::hypot(g->hx[q] - b.cx, g->hy[q] - b.cy));
      b.r_cell = r;
      b.R_p = f * r;
      int p = o->proxy_points;
      if (p <= 0) {
        p = std::max(32, 8 * (int)std::ceil((2 * krule * b.R_p + ctol) / 8.0));
        b.p_rule = p;
        if (o->proxy_scale > 0 && o->proxy_scale != 1.0) p = proxy_count(o->proxy_scale, p);
      } else {
        b.p_rule = p;
      }
      b.p = p;
    }
    for (int i = 0; i < (int)boxes.size(); ++i) {
      auto& b = boxes[i];
      b.near.clear();
      for (int j = 0; j < (int)boxes.size(); ++j) {
        if (j == i) continue;
        const auto& o2 = boxes[j];
        int dk = std::abs(o2.bx - b.bx) + std::abs(o2.by - b.by);
        if (dk == 1) { b.near.push_back(j); continue; }
        if (std::hypot(o2.cx - b.cx, o2.cy - b.cy) - o2.r_cell >= b.R_p) continue;
        bool inside = false;
        for (int jj : o2.leaves) {
          for (int q = g->node_off[jj]; q < g->node_off[jj + 1] && !inside; ++q)
            if (std::hypot(g->hx[q] - b.cx, g->hy[q] - b.cy) < b.R_p) inside = true;
          if (inside) break;
        }
        if (inside) b.near.push_back(j);
      }
    }
  }
}

void upload_inclusions(pm_geometry* g) {
  g->hinc.resize(g->m);
  for (int j = 0; j < g->m; ++j) {
    const pm_inclusion& c = g->inc[j];
    InclDev d{};
    d.shape = c.shape; d.n = c.n_nodes; d.node_off = g->node_off[j]; d.row_off = g->row_off[j];
    d.cx = c.cx; d.cy = c.cy; d.rot = c.rot;
    for (int i = 0; i < 16; ++i) d.prm[i] = c.prm[i];
    d.k_in_re = c.k_in.re; d.k_in_im = c.k_in.im;
    // eps- = (k- / k+)^2 (eps+ = 1), complex for a lossy interior
    const double a = c.k_in.re / g->k0, b = c.k_in.im / g->k0;
    d.eps_in_re = a * a - b * b; d.eps_in_im = 2 * a * b;
    g->hinc[j] = d;
  }
}

// Self blocks A_jj of the listed inclusions into A[i] (leading dims lda[i]).
// bm: the Burton-Miller self blocks (the Maue product goes to the (exterior, u) block).
template <class C>
void assemble_self(const pm_geometry* g, const std::vector<int>& incl, const std::vector<C*>& A,
                   const std::vector<int>& lda, Arena& scr, cudaStream_t st, int bm = 0) {
  const int m = (int)incl.size();
  if (m == 0) return;
  std::vector<InclDev> sub(m);
  int maxn = 0;
  std::map<int, C*> dts;
  std::vector<C*> Cm(m), DtS(m), E(m);
  for (int i = 0; i < m; ++i) {
    sub[i] = g->hinc[incl[i]];
    int n = sub[i].n;
    maxn = std::max(maxn, n);
    Cm[i] = scr.get<C>((size_t)n * n);
    DtS[i] = scr.get<C>((size_t)n * n);
    E[i] = scr.get<C>((size_t)n * n);
    if (!dts.count(n)) {
      C* d = scr.get<C>((size_t)n * n);
      diff_matrices<C>(n, d, st);
      dts[n] = d;
    }
  }
  InclDev* d_sub = upload(scr, sub, st);
  C** dA = upload(scr, A, st);
  int* dlda = upload(scr, lda, st);
  C** dC = upload(scr, Cm, st);
  C** dD = upload(scr, DtS, st);
  self_pointwise<C>(d_sub, m, maxn, g->nodes, g->k0, dA, dlda, dC, st, bm);
  if (g_kprof) {
    double e = 0;
    for (auto& c : sub) e += (double)c.n * c.n;
    g_kprof->add_flops("self_pointwise", e);   // work unit: node pairs (two wavenumbers each)
  }
  scaled_diff<C>(d_sub, m, maxn, g->nodes, dD, st);
  CK(cudaGetLastError());
  // Maue: N-block += diag(1/|x'|) Dt (S0+/e+ + S0-/e-) Dt
  std::vector<GemmDesc<C>> d1(m), d2(m);
  std::vector<int> off1(m + 1, 0), off2(m + 1, 0);
  for (int i = 0; i < m; ++i) {
    int n = sub[i].n;
    d1[i] = GemmDesc<C>{n, n, n, Cm[i], n, dts[n], n, E[i], n, cone<C>(), czero_h<C>(), 1};
    C* tgt = bm ? A[i] : A[i] + n + (size_t)n * lda[i];
    d2[i] = GemmDesc<C>{n, n, n, DtS[i], n, E[i], n, tgt, lda[i], cone<C>(), cone<C>(), 0};
    off1[i + 1] = off1[i] + gemm_tiles(n, n);
    off2[i + 1] = off2[i] + gemm_tiles(n, n);
  }
  auto* dd1 = upload(scr, d1, st); auto* do1 = upload(scr, off1, st);
  la_gemm_batched<C>(dd1, do1, m, off1[m], st);
  auto* dd2 = upload(scr, d2, st); auto* do2 = upload(scr, off2, st);
  la_gemm_batched<C>(dd2, do2, m, off2[m], st);
  CK(cudaGetLastError());
}

template <class C>
struct GatherBatch {
  int mode = GATHER_OMIT;          // entry formula of the products added from now on
  double k_in = 0, eps_in = 1;     // interior wavenumber and eps- (real) of the non-Omit formulas
  std::vector<GatherProb<C>> probs;
  std::vector<int> tile_off{0};
  std::vector<int> codes;                 // all target / source lists
  std::vector<std::pair<size_t, size_t>> lists;  // (tgt offset, src offset) per prob
  // code_off: added to every packed code (the problem's first point in a joint
  // point table, times 2); k: the problem's exterior wavenumber (0: run()'s k0)
  void add(C* out, int ld, int M, int N, const std::vector<int>& tgt, const std::vector<int>& src, int trans,
           int code_off = 0, double k = 0.0) {
    if (M <= 0 || N <= 0) return;
    size_t to = codes.size();
    for (int c : tgt) codes.push_back(c + code_off);
    size_t so = codes.size();
    for (int c : src) codes.push_back(c + code_off);
    probs.push_back(GatherProb<C>{out, ld, M, N, nullptr, nullptr, trans, k, mode, k_in, eps_in});
    lists.push_back({to, so});
    tile_off.push_back(tile_off.back() + gather_tiles(M, N));
  }
  void run(Arena& scr, PointsDev pts, double k0, cudaStream_t st) {
    if (probs.empty()) return;
    int* dcodes = upload(scr, codes, st);
    for (size_t i = 0; i < probs.size(); ++i) {
      probs[i].tgt = dcodes + lists[i].first;
      probs[i].src = dcodes + lists[i].second;
    }
    auto* dp = upload(scr, probs, st);
    int* dt = upload(scr, tile_off, st);
    gather_assemble<C>(dp, dt, (int)probs.size(), tile_off.back(), pts, k0, st);
    if (g_kprof) {
      double e = 0;
      for (auto& x : probs) e += (double)x.M * x.N;
      g_kprof->add_flops(kname<C>("gather_entries", "gather_entries32"), e);   // work unit: matrix entries
    }
    CK(cudaGetLastError());
  }
};

// Autotuner of the batched GEMM's output tile (no counterpart in the paper).
// Batches are classed by (device, precision, ceil log2 of the largest m, of
// the largest n, of the mean k, of the problem count).  The first
// write-only batch of a class (every C overwritten, no C aliasing an
// operand, so running it again gives the same result) times every tile shape
// once after a warm-up launch with CUDA events and keeps the fastest; later
// batches of the class use it.  All shapes sum over k in the same order, so
// the choice changes speed only, never a result.  A class not tuned yet runs
// the 32 x 32 shape.
struct TuneKey {
  int dev, bytes, lm, ln, lk, lc;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, bytes, lm, ln, lk, lc) < std::tie(o.dev, o.bytes, o.lm, o.ln, o.lk, o.lc);
  }
};
struct TuneEntry {
  int shape = 0;
  float ms[GEMM_NSHAPES] = {};
  long long uses = 0;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneEntry> g_tune;
thread_local bool g_tune_off = false;    // PM_FLAG_NO_AUTOTUNE of the running call

int ceil_log2(double x) { return x <= 1 ? 0 : (int)std::ceil(std::log2(x)); }

struct TuneScope {   // the running call's PM_FLAG_NO_AUTOTUNE, restored on exit
  bool prev;
  explicit TuneScope(bool off) : prev(g_tune_off) { g_tune_off = off; }
  ~TuneScope() { g_tune_off = prev; }
};

template <class C>
struct GemmBatch {
  std::vector<GemmDesc<C>> d;
  std::vector<int> off{0};
  void add(int m, int n, int k, const C* A, int lda, const C* B, int ldb, C* Cp, int ldc, C alpha, C beta,
           int beta_zero) {
    if (m <= 0 || n <= 0) return;
    if (k <= 0) {
      if (beta_zero) k = 0; else return;
    }
    d.push_back(GemmDesc<C>{m, n, k, A, lda, B, ldb, Cp, ldc, alpha, beta, beta_zero});
    off.push_back(off.back() + gemm_tiles(m, n));
  }
  std::vector<int> offsets(int shape) const {
    std::vector<int> o{0};
    for (auto& x : d) o.push_back(o.back() + gemm_tiles_shape(shape, x.m, x.n));
    return o;
  }
  void run(Arena& scr, cudaStream_t st) {
    if (d.empty()) return;
    auto* dd = upload(scr, d, st);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    int mm = 0, mn = 0;
    double ks = 0;
    bool write_only = true;
    for (auto& x : d) {
      mm = std::max(mm, x.m); mn = std::max(mn, x.n); ks += x.k;
      write_only = write_only && x.beta_zero && (const void*)x.Cm != (const void*)x.A && (const void*)x.Cm != (const void*)x.B;
    }
    const TuneKey key{dev, (int)sizeof(C), ceil_log2(mm), ceil_log2(mn), ceil_log2(ks / d.size()), ceil_log2((double)d.size())};
    int shape = 0;
    bool tune = false;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) { shape = it->second.shape; it->second.uses++; }
      else tune = write_only && !g_tune_off && !g_kprof && !g_capture_side;
    }
    if (tune) {
      TuneEntry e;
      cudaEvent_t a, b;
      CK(cudaEventCreate(&a)); CK(cudaEventCreate(&b));
      for (int sh = 0; sh < GEMM_NSHAPES; ++sh) {
        const std::vector<int> o = offsets(sh);
        int* dof = upload(scr, o, st);
        la_gemm_batched_shape<C>(sh, dd, dof, (int)d.size(), o.back(), st);   // warm-up
        CK(cudaEventRecord(a, st));
        la_gemm_batched_shape<C>(sh, dd, dof, (int)d.size(), o.back(), st);
        CK(cudaEventRecord(b, st));
        CK(cudaEventSynchronize(b));
        CK(cudaEventElapsedTime(&e.ms[sh], a, b));
        if (e.ms[sh] < e.ms[e.shape]) e.shape = sh;
      }
      cudaEventDestroy(a); cudaEventDestroy(b);
      e.uses = 1;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune.emplace(key, e);   // the result is in C: every shape wrote the same values
    } else {
      const std::vector<int> o = shape == 0 ? off : offsets(shape);
      int* dof = upload(scr, o, st);
      la_gemm_batched_shape<C>(shape, dd, dof, (int)d.size(), o.back(), st);
    }
    if (g_kprof) {
      double f = 0;
      for (auto& x : d) f += 8.0 * x.m * x.n * x.k;
      g_kprof->add_flops(kname<C>("gemm_batched", "gemm_batched32"), f);
    }
    CK(cudaGetLastError());
  }
};

template <class S, class D = S>
struct CopyBatch {
  std::vector<CopyProb<S, D>> p;
  int maxe = 0;
  void add(const S* src, int lds, D* dst, int ldd, int m, int n) {
    if (m <= 0 || n <= 0) return;
    p.push_back(CopyProb<S, D>{src, lds, dst, ldd, m, n});
    maxe = std::max(maxe, m * n);
  }
  void run(Arena& scr, cudaStream_t st) {
    if (p.empty()) return;
    auto* dp = upload(scr, p, st);
    copy_batched<S, D>(dp, (int)p.size(), maxe, st);
    CK(cudaGetLastError());
  }
};

template <class C>
void lu_batch(std::vector<LuProb<C>>& probs, Arena& scr, cudaStream_t st, const char* what) {
  if (probs.empty()) return;
  int n = (int)probs.size();
  int* info = scr.get<int>(n);
  CK(cudaMemsetAsync(info, 0, n * sizeof(int), st));
  int maxm = 0;
  for (int i = 0; i < n; ++i) { probs[i].info = info + i; maxm = std::max(maxm, probs[i].m); }
  auto* dp = upload(scr, probs, st);
  std::vector<int> hm(n);
  for (int i = 0; i < n; ++i) hm[i] = probs[i].m;
  la_getrf_batched<C>(dp, n, maxm, hm.data(), st);
  CK(cudaGetLastError());
  std::vector<int> h(n);
  CK(cudaMemcpyAsync(h.data(), info, n * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int i = 0; i < n; ++i)
    if (h[i] != 0) fail(PM_ERR_SINGULAR, std::string(what) + ": exactly singular pivot in LU");
}

// wait_err (optional): lets batches with at most 8 right-hand sides take the
// chained triangular solves (one launch per triangle for all matrices),
// whose bounded waits report there.
template <class C>
void solve_batch(std::vector<SolveProb<C>>& probs, Arena& scr, cudaStream_t st, int* wait_err = nullptr,
                 bool debug_no_flag = false) {
  if (probs.empty()) return;
  int maxm = 0, maxr = 0;
  std::vector<int> hm, hr;
  for (auto& p : probs) {
    maxm = std::max(maxm, p.m); maxr = std::max(maxr, p.nrhs);
    hm.push_back(p.m); hr.push_back(p.nrhs);
  }
  auto* dp = upload(scr, probs, st);
  if (wait_err && maxr <= 8) {
    std::vector<int4> items;
    ChainArgs ch;
    // FP64: two columns per CTA (the links of the chain are bound by one SM's
    // FP64 rate); complex64: all columns in one CTA
    ch.rhs_per_cta = sizeof(C) == sizeof(double2) ? 2 : 8;
    ch.total_blocks = la_chain_items(hm.data(), (int)probs.size(), (maxr + ch.rhs_per_cta - 1) / ch.rhs_per_cta, items);
    ch.items = items.empty() ? nullptr : upload(scr, items, st);
    ch.sync = scr.get<int>(la_chain_sync_ints(ch.total_blocks));
    ch.err = wait_err;
    ch.no_flag = debug_no_flag ? 1 : 0;
    la_getrs_batched<C>(dp, (int)probs.size(), maxm, maxr, hm.data(), hr.data(), st, &ch);
  } else {
    la_getrs_batched<C>(dp, (int)probs.size(), maxm, maxr, hm.data(), hr.data(), st);
  }
  CK(cudaGetLastError());
}

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) { cudaEventCreate(&a); cudaEventCreate(&b); cudaEventRecord(a, st); }
  double stop() {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a); cudaEventDestroy(b);
    return ms;
  }
};

// Active sets and D_b of a parent (or the root) from its children's compressed blocks.
// Cc: the children's arithmetic, Cp: the parent's.
// Active sets of a parent (or the root): its children's skeletons, in order.
template <class Cc, class Cp>
void active_sets(const std::vector<BoxF<Cc>>& kids, const Box& box, BoxF<Cp>& bf) {
  bf.rows.clear(); bf.rgrp.clear(); bf.cols.clear(); bf.cgrp.clear(); bf.child_off.clear();
  for (int c : box.children) {
    bf.child_off.push_back((int)bf.rows.size());
    const BoxF<Cc>& k = kids[c];
    bf.rows.insert(bf.rows.end(), k.srows.begin(), k.srows.end());
    bf.rgrp.insert(bf.rgrp.end(), k.srgrp.begin(), k.srgrp.end());
    bf.cols.insert(bf.cols.end(), k.scols.begin(), k.scols.end());
    bf.cgrp.insert(bf.cgrp.end(), k.scgrp.begin(), k.scgrp.end());
  }
  bf.mb = (int)bf.rows.size();
}

template <class Cc, class Cp>
void merge_children(pm_factor* F, const std::vector<BoxF<Cc>>& kids, const Box& box, BoxF<Cp>& bf,
                    GatherBatch<Cp>& gb, CopyBatch<Cc, Cp>& cb, int code_off = 0) {
  active_sets<Cc, Cp>(kids, box, bf);
  bf.D = F->arena.get<Cp>((size_t)std::max(bf.mb, 1) * std::max(bf.mb, 1));
  const pm_geometry* g = F->g;
  for (size_t a = 0; a < box.children.size(); ++a) {
    const BoxF<Cc>& ka = kids[box.children[a]];
    std::vector<int> tcodes(ka.srows.size());
    for (size_t i = 0; i < ka.srows.size(); ++i) tcodes[i] = g->code_of(ka.srows[i]);
    for (size_t b = 0; b < box.children.size(); ++b) {
      const BoxF<Cc>& kb = kids[box.children[b]];
      Cp* dst = bf.D + bf.child_off[a] + (size_t)bf.child_off[b] * bf.mb;
      if (a == b) {
        cb.add(ka.At, ka.kb, dst, bf.mb, ka.kb, ka.kb);
      } else {
        std::vector<int> scodes(kb.scols.size());
        for (size_t i = 0; i < kb.scols.size(); ++i) scodes[i] = g->code_of(kb.scols[i]);
        gb.add(dst, bf.mb, ka.kb, kb.kb, tcodes, scodes, 0, code_off, g->k0);
      }
    }
  }
}

PointsDev make_points(const pm_geometry* g, const std::vector<Box>& boxes, Arena& scr, cudaStream_t st,
                      std::vector<int>& proxy_off) {
  int total_proxy = 0;
  proxy_off.assign(boxes.size(), 0);
  std::vector<ProxyBoxDev> pb(boxes.size());
  for (size_t b = 0; b < boxes.size(); ++b) {
    proxy_off[b] = total_proxy;
    pb[b] = ProxyBoxDev{boxes[b].cx, boxes[b].cy, boxes[b].R_p, boxes[b].p, total_proxy, 0.0};
    total_proxy += boxes[b].p;
  }
  const size_t np = (size_t)g->total_nodes + total_proxy;
  PointsDev P;
  P.x = scr.get<double>(np); P.y = scr.get<double>(np); P.nx = scr.get<double>(np);
  P.ny = scr.get<double>(np); P.w = scr.get<double>(np);
  geom_points_from_nodes(g->nodes, P, g->total_nodes, st);
  auto* dpb = upload(scr, pb, st);
  geom_proxy_points(dpb, (int)boxes.size(), P, total_proxy, g->total_nodes, st);
  CK(cudaGetLastError());
  return P;
}

// One level of one problem's factorization; several jobs (independent
// problems, possibly at different depths of their trees) are processed in
// shared launches.
// boxes [b0, b1) of the level (b1 < 0: to the last); the call with b0 = 0 also
// sets up the active sets of all of the level's boxes (the near lists of later
// chunks read them)
struct LevelJob {
  pm_factor* F;
  int lev;
  int b0 = 0, b1 = -1;
};

// Points of several problems in one table: every problem's nodes first
// (problem j's from nbase[j]), then, per problem from pbase[j], the proxy
// points of its boxes at its job's level (box b's first at pbase[j] +
// poff[j][b]) and, with hoff, each box's held-out ring (its proxy count,
// turned half a spacing; first at pbase[j] + hoff[j][b]).  Node positions do
// not depend on the proxy counts.
PointsDev make_points_joint(const std::vector<LevelJob>& jobs, bool proxies, Arena& scr, cudaStream_t st,
                            std::vector<int>& nbase, std::vector<int>& pbase, std::vector<std::vector<int>>& poff,
                            std::vector<std::vector<int>>* hoff = nullptr) {
  const int nj = (int)jobs.size();
  nbase.assign(nj, 0);
  pbase.assign(nj, 0);
  poff.assign(nj, {});
  if (hoff) hoff->assign(nj, {});
  std::vector<std::vector<ProxyBoxDev>> pb(nj);
  std::vector<int> nprox(nj, 0);
  size_t np = 0;
  for (int j = 0; j < nj; ++j) {
    nbase[j] = (int)np;
    np += (size_t)jobs[j].F->g->total_nodes;
  }
  for (int j = 0; j < nj; ++j) {
    pbase[j] = (int)np;
    if (proxies) {
      const auto& boxes = jobs[j].F->tree[jobs[j].lev];
      poff[j].assign(boxes.size(), 0);
      for (size_t b = 0; b < boxes.size(); ++b) {
        poff[j][b] = nprox[j];
        pb[j].push_back(ProxyBoxDev{boxes[b].cx, boxes[b].cy, boxes[b].R_p, boxes[b].p, nprox[j], 0.0});
        nprox[j] += boxes[b].p;
      }
      if (hoff) {
        (*hoff)[j].assign(boxes.size(), 0);
        for (size_t b = 0; b < boxes.size(); ++b) {
          (*hoff)[j][b] = nprox[j];
          pb[j].push_back(ProxyBoxDev{boxes[b].cx, boxes[b].cy, boxes[b].R_p, boxes[b].p, nprox[j], 0.5});
          nprox[j] += boxes[b].p;
        }
      }
    }
    np += nprox[j];
  }
  if (np > (size_t)(1 << 30)) fail(PM_ERR_UNSUPPORTED, "more than 2^30 points in one launch");
  PointsDev P;
  P.x = scr.get<double>(np); P.y = scr.get<double>(np); P.nx = scr.get<double>(np);
  P.ny = scr.get<double>(np); P.w = scr.get<double>(np);
  for (int j = 0; j < nj; ++j) {
    const pm_geometry* g = jobs[j].F->g;
    const size_t o = nbase[j];
    geom_points_from_nodes(g->nodes, PointsDev{P.x + o, P.y + o, P.nx + o, P.ny + o, P.w + o}, g->total_nodes, st);
    if (nprox[j] > 0) {
      const size_t q = pbase[j];
      auto* dpb = upload(scr, pb[j], st);
      geom_proxy_points(dpb, (int)pb[j].size(), PointsDev{P.x + q, P.y + q, P.nx + q, P.ny + q, P.w + q}, nprox[j], 0,
                        st);
    }
  }
  CK(cudaGetLastError());
  return P;
}

// Entry formula of the off-diagonal blocks of a factorization's formulation,
// and its interior medium (one real k- for all inclusions off PMCHWT (Omit)).
int gather_mode_of(const pm_factor_opts& O) {
  switch (O.formulation) {
    case PM_FORM_ALL: return GATHER_ALL;
    case PM_FORM_BM: return GATHER_BM;
    case PM_FORM_BM_SIMPLIFIED: return GATHER_BM_SIMPLIFIED;
    default: return GATHER_OMIT;
  }
}
template <class C>
void set_form(GatherBatch<C>& gb, const pm_factor* F) {
  gb.mode = gather_mode_of(F->opts);
  gb.k_in = F->g->inc[0].k_in.re;
  gb.eps_in = (gb.k_in / F->g->k0) * (gb.k_in / F->g->k0);
}

// Squared Frobenius norms of many column-major blocks: out[i] += sum |A_i|^2.
struct SqNormProb { const void* A; int ld; int m; int n; double* out; };
template <class C>
__global__ void __launch_bounds__(256) k_sqnorm(const SqNormProb* __restrict__ P) {
  const SqNormProb p = P[blockIdx.y];
  const C* A = (const C*)p.A;
  double acc = 0;
  for (int j = blockIdx.x; j < p.n; j += gridDim.x)
    for (int i = threadIdx.x; i < p.m; i += 256) acc += (double)abs2(A[i + (size_t)j * p.ld]);
  acc = warp_sum(acc);
  __shared__ double sh[8];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    atomicAdd(p.out, t);
  }
}

template <class C>
void sqnorm_batch(const std::vector<SqNormProb>& probs, Arena& scr, cudaStream_t st) {
  if (probs.empty()) return;
  auto* d = upload(scr, probs, st);
  k_sqnorm<C><<<dim3(64, (unsigned)probs.size()), 256, 0, st>>>(d);
  pm_launch_count_add(1);
  CK(cudaGetLastError());
}

// Held-out proxy check bound: an ID passes while ||H_J - H_S T|| <= PROXY_CHECK_BOUND tol ||H||.
constexpr double PROXY_CHECK_BOUND = 200.0;

// failed (optional): receives (job, box) of every box whose predicted proxy
// count failed the held-out check; the call then returns before the Schur
// steps, and the caller redoes the level with those boxes at the rule's count.
template <class C>
void process_levels(const std::vector<LevelJob>& jobs, Arena& scr, cudaStream_t st, double tol,
                    std::vector<std::pair<int, int>>* failed = nullptr) {
  scr.reset();
  const int nj = (int)jobs.size();
  const pm_factor_opts& O = jobs[0].F->opts;   // the jobs of one call share their options
  // boxes of all jobs (each job's range [b0, b1)), flattened: global box
  // gb = jb_off[j] + (b - b0[j])
  std::vector<int> jb_off(nj + 1, 0), jb0(nj), jb1(nj);
  for (int j = 0; j < nj; ++j) {
    const int nbj = (int)jobs[j].F->tree[jobs[j].lev].size();
    jb0[j] = jobs[j].b0;
    jb1[j] = jobs[j].b1 < 0 ? nbj : std::min(jobs[j].b1, nbj);
    if (jb0[j] == 0) levels_of<C>(jobs[j].F)[jobs[j].lev].assign(nbj, BoxF<C>());
    jb_off[j + 1] = jb_off[j] + (jb1[j] - jb0[j]);
  }
  const int nb = jb_off[nj];
  std::vector<int> job_of(nb);
  for (int j = 0; j < nj; ++j)
    for (int b = jb_off[j]; b < jb_off[j + 1]; ++b) job_of[b] = j;
  auto lbox = [&](int x) { return x - jb_off[job_of[x]] + jb0[job_of[x]]; };   // box index within its level
  auto BFx = [&](int x) -> BoxF<C>& {
    const LevelJob& J = jobs[job_of[x]];
    return levels_of<C>(J.F)[J.lev][lbox(x)];
  };
  auto BOX = [&](int x) -> const Box& {
    const LevelJob& J = jobs[job_of[x]];
    return J.F->tree[J.lev][lbox(x)];
  };
  auto GEO = [&](int x) -> const pm_geometry* { return jobs[job_of[x]].F->g; };
  Timer t_asm(st);
  // node positions in the level's point table (the proxy points follow all nodes)
  std::vector<int> nbase(nj, 0);
  for (int j = 1; j < nj; ++j) nbase[j] = nbase[j - 1] + jobs[j - 1].F->g->total_nodes;
  // 1. active sets and diagonal blocks (the merges' gathers run once the points exist)
  GatherBatch<C> gm; CopyBatch<C, C> cm;
  {
    for (int j = 0; j < nj; ++j) {
      pm_factor* F = jobs[j].F;
      const int lev = jobs[j].lev;
      const pm_geometry* g = F->g;
      auto& LV = levels_of<C>(F);
      auto& BF = LV[lev];
      const auto& boxes = F->tree[lev];
      const int nbj = (int)boxes.size();
      if (lev == F->L) {
        if (jb0[j] == 0)
          for (int b = 0; b < nbj; ++b) {   // active sets of every box of the level
            int i0 = boxes[b].leaves[0];
            int n = g->inc[i0].n_nodes;
            BoxF<C>& bf = BF[b];
            bf.mb = 2 * n;
            for (int i = 0; i < 2 * n; ++i) {
              bf.rows.push_back(g->row_off[i0] + i);
              bf.rgrp.push_back(i >= n);
            }
            bf.cols = bf.rows; bf.cgrp = bf.rgrp;
          }
        std::vector<int> incl, lda;
        std::vector<C*> A;
        for (int b = jb0[j]; b < jb1[j]; ++b) {
          BoxF<C>& bf = BF[b];
          bf.D = F->arena.get<C>((size_t)bf.mb * bf.mb);
          incl.push_back(boxes[b].leaves[0]); A.push_back(bf.D); lda.push_back(bf.mb);
        }
        if constexpr (std::is_same<C, float2>::value) {
          // mixed mode: the FP64 self blocks (kept for the refinement's operator)
          // rounded to complex64, instead of a second assembly in complex64
          if (F->self64.size() != (size_t)g->m) F->self64.assign(g->m, nullptr);
          std::vector<double2*> A64;
          for (size_t i = 0; i < incl.size(); ++i) {
            double2*& d = F->self64[incl[i]];
            if (!d) d = F->arena.get<double2>((size_t)lda[i] * lda[i]);
            A64.push_back(d);
          }
          assemble_self<double2>(g, incl, A64, lda, scr, st, F->opts.formulation >= PM_FORM_BM);
          const int maxn = *std::max_element(lda.begin(), lda.end());
          round_blocks(upload(scr, A64, st), upload(scr, A, st), upload(scr, lda, st), (int)incl.size(), maxn, st);
          CK(cudaGetLastError());
        } else {
          assemble_self<C>(g, incl, A, lda, scr, st, F->opts.formulation >= PM_FORM_BM);
        }
      } else {
        if (jb0[j] == 0)
          for (int b = 0; b < nbj; ++b) active_sets<C, C>(LV[lev + 1], boxes[b], BF[b]);
        set_form(gm, F);
        for (int b = jb0[j]; b < jb1[j]; ++b)
          merge_children<C, C>(F, LV[lev + 1], boxes[b], BF[b], gm, cm, 2 * nbase[j]);
      }
    }
  }
  const int nid = 4 * nb;
  // 1b. candidate counts, input rows at the rule's proxy count and the learned
  // predictor's features of every (box, group); the predictor may then lower
  // the boxes' proxy counts before the proxy points are made
  std::vector<int> nn(nid), Wr(nid);
  for (int b = 0; b < nb; ++b) {
    const int jj = job_of[b];
    const Box& box = BOX(b);
    const BoxF<C>& bf = BFx(b);
    const auto& BFj = levels_of<C>(jobs[jj].F)[jobs[jj].lev];
    int ncol = 0, nrow = 0;
    for (int o : box.near) { ncol += (int)BFj[o].cols.size(); nrow += (int)BFj[o].rows.size(); }
    for (int grp = 0; grp < 2; ++grp) {
      nn[4 * b + grp] = (int)std::count(bf.rgrp.begin(), bf.rgrp.end(), grp);
      nn[4 * b + 2 + grp] = (int)std::count(bf.cgrp.begin(), bf.cgrp.end(), grp);
      Wr[4 * b + grp] = ncol + 2 * box.p_rule;
      Wr[4 * b + 2 + grp] = nrow + 2 * box.p_rule;
    }
  }
  std::vector<float> feat(2 * (size_t)nb * MLP_IN);
  for (int b = 0; b < nb; ++b) {
    const pm_geometry* g = GEO(b);
    const Box& box = BOX(b);
    double kin = 0;
    for (int j : box.leaves) kin += g->inc[j].k_in.re;
    kin /= std::max<size_t>(box.leaves.size(), 1);
    for (int grp = 0; grp < 2; ++grp) {
      float* f = &feat[(2 * (size_t)b + grp) * MLP_IN];
      f[0] = (float)std::log((double)std::max(nn[4 * b + grp], 1));
      f[1] = (float)std::log((double)std::max(Wr[4 * b + grp], 1));
      f[2] = (float)std::log((double)std::max(Wr[4 * b + 2 + grp], 1));
      f[3] = (float)(g->k0 * box.r_cell);
      f[4] = (float)std::log10(tol);
      f[5] = (float)std::log2((double)box.leaves.size());
      f[6] = (float)grp;
      f[7] = (float)(kin / g->k0);
    }
  }
  std::vector<int> khat;   // predicted rank bound per ID (empty: no predictor)
  bool lowered = false;    // some box runs below the rule's proxy count
  for (int b = 0; b < nb; ++b) lowered = lowered || BOX(b).p < BOX(b).p_rule;
  if (O.rank_model && O.formulation == PM_FORM_OMIT) {   // trained on PMCHWT (Omit) factorizations
    const float* mdl = O.rank_model;   // theta | mean (8) | std (8), device
    std::vector<float> musd(2 * MLP_IN);
    CK(cudaMemcpyAsync(musd.data(), mdl + MLP_NPARAM, sizeof(float) * 2 * MLP_IN, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<float> xn(feat.size());
    for (size_t i = 0; i < feat.size(); ++i) {
      const int c = (int)(i % MLP_IN);
      xn[i] = (feat[i] - musd[c]) / (musd[MLP_IN + c] > 0 ? musd[MLP_IN + c] : 1.f);
    }
    float* dx = upload(scr, xn, st);
    float* dy = scr.get<float>(2 * (size_t)nb * MLP_OUT);
    mlp_forward<float>(mdl, 2 * nb, dx, dy, st);
    std::vector<float> yp(2 * (size_t)nb * MLP_OUT);
    CK(cudaMemcpyAsync(yp.data(), dy, sizeof(float) * yp.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    khat.assign(nid, 0);
    for (int b = 0; b < nb; ++b) {
      double pfrac = 0;
      for (int grp = 0; grp < 2; ++grp) {
        const float* y = &yp[(2 * (size_t)b + grp) * MLP_OUT];
        const int n = nn[4 * b + grp];
        const double frac = std::min(1.0, std::max(0.0, (double)y[0]));
        const int k = std::min(n, (int)std::ceil(frac * n + 2 + 0.02 * n));
        khat[4 * b + grp] = khat[4 * b + 2 + grp] = k;
        pfrac = std::max(pfrac, (double)y[1]);
      }
      // learned proxy count, unless the count is fixed or the box failed the check before
      Box& box = jobs[job_of[b]].F->tree[jobs[job_of[b]].lev][lbox(b)];
      if (O.proxy_points == 0 && !box.locked) {
        box.p = std::min(box.p_rule, proxy_count(std::min(1.0, std::max(0.25, pfrac + 0.1)), box.p_rule));
        lowered = lowered || box.p < box.p_rule;
      }
    }
    if (O.debug_flags & PM_DEBUG_UNDERPREDICT) std::fill(khat.begin(), khat.end(), 1);   // injected
  }
  // the held-out proxy check: asked for, or what decides lowered counts in FP64
  const bool check_on = O.formulation == PM_FORM_OMIT &&
                        ((O.flags & PM_FLAG_PROXY_CHECK) ||
                         (lowered && O.rank_model && O.precision == PM_FP64 && O.proxy_points == 0));
  // one point table for the level: every job's nodes, then its boxes' proxy points (and held-out rings)
  std::vector<int> pbase;
  std::vector<std::vector<int>> poff, hoff;
  PointsDev P = make_points_joint(jobs, true, scr, st, nbase, pbase, poff, check_on ? &hoff : nullptr);
  gm.run(scr, P, 0.0, st);
  cm.run(scr, st);
  // 2. ID inputs: per box 4 IDs (row u-eq, row q-eq, col q, col u)
  std::vector<int> W(nid);
  std::vector<C*> Z(nid);
  std::vector<std::vector<int>> pos(nid);
  GatherBatch<C> gb;
  for (int b = 0; b < nb; ++b) {
    const int jj = job_of[b], lb = lbox(b);
    const pm_geometry* g = GEO(b);
    const Box& box = BOX(b);
    const BoxF<C>& bf = BFx(b);
    const auto& BFj = levels_of<C>(jobs[jj].F)[jobs[jj].lev];
    const int co = 2 * nbase[jj];
    std::vector<int> ncols, nrows;
    for (int o : box.near) {
      for (int c : BFj[o].cols) ncols.push_back(g->code_of(c) + co);
      for (int r : BFj[o].rows) nrows.push_back(g->code_of(r) + co);
    }
    const int pb0 = pbase[jj] + poff[jj][lb];   // absolute point index of the box's first proxy
    std::vector<int> pcols, prows;
    for (int grp = 0; grp < 2; ++grp)
      for (int s = 0; s < box.p; ++s) { pcols.push_back((pb0 + s) * 2 + grp); prows.push_back((pb0 + s) * 2 + grp); }
    // rows of the ID inputs: near entries of the formulation, then the proxy
    // densities (PMCHWT (All): an exterior and an interior family)
    const pm_factor* Fj = jobs[jj].F;
    const int form = Fj->opts.formulation;
    const int nfam = form == PM_FORM_ALL ? 2 : 1;
    auto add_proxies = [&](C* Zp, int ld, int n_cand, const std::vector<int>& cand, const std::vector<int>& prox,
                           int trans) {
      for (int fam = 0; fam < nfam; ++fam) {
        set_form(gb, Fj);
        if (form == PM_FORM_ALL) gb.mode = fam == 0 ? GATHER_OMIT : GATHER_INTERIOR;
        C* out = Zp + (size_t)fam * prox.size();
        if (trans) gb.add(out, ld, (int)prox.size(), n_cand, cand, prox, 1, 0, g->k0);
        else gb.add(out, ld, (int)prox.size(), n_cand, prox, cand, 0, 0, g->k0);
      }
    };
    for (int grp = 0; grp < 2; ++grp) {
      // row ID of group grp: Z[w, c] = A(row c, source w), sources = near columns + proxy
      int id = 4 * b + grp;
      std::vector<int> tgt;
      for (int i = 0; i < bf.mb; ++i) if (bf.rgrp[i] == grp) { pos[id].push_back(i); tgt.push_back(g->code_of(bf.rows[i]) + co); }
      W[id] = (int)(ncols.size() + nfam * pcols.size());
      Z[id] = scr.get<C>((size_t)W[id] * std::max(nn[id], 1));
      set_form(gb, Fj);
      gb.add(Z[id], W[id], (int)ncols.size(), nn[id], tgt, ncols, 1, 0, g->k0);
      add_proxies(Z[id] + ncols.size(), W[id], nn[id], tgt, pcols, 1);
      // column ID of group grp: Z[w, c] = A(target w, column c), targets = near rows + proxy
      id = 4 * b + 2 + grp;
      std::vector<int> srcc;
      for (int i = 0; i < bf.mb; ++i) if (bf.cgrp[i] == grp) { pos[id].push_back(i); srcc.push_back(g->code_of(bf.cols[i]) + co); }
      W[id] = (int)(nrows.size() + nfam * prows.size());
      Z[id] = scr.get<C>((size_t)W[id] * std::max(nn[id], 1));
      set_form(gb, Fj);
      gb.add(Z[id], W[id], (int)nrows.size(), nn[id], nrows, srcc, 0, 0, g->k0);
      add_proxies(Z[id] + nrows.size(), W[id], nn[id], srcc, prows, 0);
    }
  }
  gb.run(scr, P, 0.0, st);
  for (int i = 0; i < nid; ++i) jobs[job_of[i / 4]].F->stats.id_rows += W[i];
  const double ms_asm = t_asm.stop();
  for (const auto& J : jobs) J.F->stats.ms_assemble += ms_asm;
  // the operator's FP64 assembly starts beside the factorization once the
  // leaf level's FP64 work (self blocks, Maue products) is done
  for (const auto& J : jobs)
    if (J.F->op_pending) {
      J.F->op_pending = false;
      start_mixed_operator(J.F, true);
    }
  Timer t_id(st);
  // 3a. complex64: tall inputs reduced to their triangular factor first, so
  // that the pivoted steps stream n instead of W rows
  std::vector<int> We(W);   // rows the pivoted QR runs on (leading dimension stays W)
  if constexpr (std::is_same<C, float2>::value) {
    if (!(O.flags & PM_FLAG_NO_QR_FIRST)) {
      std::vector<QrProb<C>> qp;
      int maxn = 0;
      double fl = 0;
      for (int i = 0; i < nid; ++i)
        if (nn[i] > 0 && W[i] >= 2 * nn[i]) {
          qp.push_back(QrProb<C>{Z[i], W[i], W[i], nn[i], nullptr, nullptr, nullptr, 0});
          We[i] = nn[i];
          maxn = std::max(maxn, nn[i]);
          for (int j0 = 0; j0 < nn[i]; j0 += QR_NB) {
            const double jb = std::min(QR_NB, nn[i] - j0);
            fl += 16.0 * (double)(W[i] - j0) * jb * (nn[i] - j0 - jb);   // two passes, 8 flops per complex MAC
          }
        }
      if (!qp.empty()) {
        const int nq = (int)qp.size();
        C* tws = scr.get<C>((size_t)nq * QR_NB * QR_NB);
        for (int q = 0; q < nq; ++q) qp[q].T = tws + (size_t)q * QR_NB * QR_NB;
        if (!(O.flags & PM_FLAG_TENSOR_CORES)) {
          int maxW = 0;
          for (int q = 0; q < nq; ++q) {
            qp[q].mrb = (qp[q].W + QR_RB - 1) / QR_RB;
            qp[q].Yp = scr.get<C>((size_t)((qp[q].n + 31) / 32) * qp[q].mrb * QR_NB * 32);
            maxW = std::max(maxW, qp[q].W);
          }
          auto* dqp = upload(scr, qp, st);
          // C -= V Y on the tensor cores unless PM_FLAG_QR_CUDA_CORES
          int* terr = nullptr;
          if (!(O.flags & PM_FLAG_QR_CUDA_CORES)) {
            terr = scr.get<int>(1);
            CK(cudaMemsetAsync(terr, 0, sizeof(int), st));
          }
          for (int j0 = 0; j0 < maxn; j0 += QR_NB) {
            qr_panel<C>(dqp, nq, j0, st);
            const int tiles = (maxn - j0 - QR_NB + 31) / 32;
            const int rbs = (maxW - j0 + QR_RB - 1) / QR_RB;
            if (tiles > 0)
              qr_update<C>(dqp, nq, j0, tiles, rbs, st, terr, maxW, (O.debug_flags & PM_DEBUG_TC_NO_ARRIVE) != 0);
          }
          qr_zero_lower<C>(dqp, nq, maxn, st);
          if (terr) {
            int herr = 0;
            CK(cudaMemcpyAsync(&herr, terr, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (herr) fail(PM_ERR_TIMEOUT, "a wait on the tensor cores ran out (QR update)");
          }
          if (g_kprof) g_kprof->add_flops(terr ? "qr_update_tc32" : "qr_update32", fl);
        } else {
          // Trailing update of every panel on the tensor cores: with V the
          // panel's reflectors (unit diagonal) and C its trailing block,
          // Y^H = C^H V, Y^H <- Y^H T, C -= V Y.  All panels' problem lists
          // are built and uploaded at once.
          std::vector<C*> yh(nq), y2h(nq);
          for (int q = 0; q < nq; ++q) {
            qp[q].V = scr.get<C>((size_t)qp[q].W * QR_NB);
            yh[q] = scr.get<C>((size_t)qp[q].n * QR_NB);
            y2h[q] = scr.get<C>((size_t)qp[q].n * QR_NB);
          }
          std::vector<TcGemmProb> gl[3];
          std::vector<int> toff[3];
          std::vector<int> pstart, pcount;   // per panel: first problem and problem count of each list
          const float2 one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f), mone = make_float2(-1.f, 0.f);
          for (int j0 = 0; j0 < maxn; j0 += QR_NB) {
            pstart.push_back((int)gl[0].size());
            int cnt = 0;
            for (int q = 0; q < nq; ++q) {
              const int n = qp[q].n, Wq = qp[q].W, ld = qp[q].ld;
              if (j0 >= n) continue;
              const int jb = std::min(QR_NB, n - j0), nt = n - j0 - jb;
              if (nt <= 0) continue;
              float2* Cb = (float2*)(qp[q].Z + j0 + (size_t)(j0 + jb) * ld);
              float2* V = (float2*)qp[q].V;
              gl[0].push_back(TcGemmProb{Cb, ld, 1, V, Wq, 0, (float2*)yh[q], n, nt, jb, Wq - j0, one, zero});
              gl[1].push_back(TcGemmProb{(float2*)yh[q], n, 0, (float2*)qp[q].T, QR_NB, 0, (float2*)y2h[q], n, nt, jb,
                                         jb, one, zero});
              gl[2].push_back(TcGemmProb{V, Wq, 0, (float2*)y2h[q], n, 1, Cb, ld, Wq - j0, nt, jb, mone, one});
              ++cnt;
            }
            pcount.push_back(cnt);
          }
          for (int l = 0; l < 3; ++l) {
            toff[l].assign(gl[l].size() + 1, 0);
            for (size_t i = 0; i < gl[l].size(); ++i) toff[l][i + 1] = toff[l][i] + tc_tiles(gl[l][i].m, gl[l][i].n);
          }
          TcGemmProb* dg[3];
          int* dt[3];
          for (int l = 0; l < 3; ++l) { dg[l] = upload(scr, gl[l], st); dt[l] = upload(scr, toff[l], st); }
          int* terr = scr.get<int>(1);
          CK(cudaMemsetAsync(terr, 0, sizeof(int), st));
          auto* dqp = upload(scr, qp, st);
          int pi = 0;
          for (int j0 = 0; j0 < maxn; j0 += QR_NB, ++pi) {
            qr_panel<C>(dqp, nq, j0, st);
            const int s0 = pstart[pi], c = pcount[pi];
            if (c == 0) continue;
            for (int l = 0; l < 3; ++l) {
              const int t0 = toff[l][s0], t1 = toff[l][s0 + c];
              tc_gemm_batched(dg[l] + s0, dt[l] + s0, c, t1 - t0, terr, st, t0,
                              (O.debug_flags & PM_DEBUG_TC_NO_ARRIVE) != 0);
            }
          }
          qr_zero_lower<C>(dqp, nq, maxn, st);
          CK(cudaGetLastError());
          int herr = 0;
          CK(cudaMemcpyAsync(&herr, terr, sizeof(int), cudaMemcpyDeviceToHost, st));
          CK(cudaStreamSynchronize(st));
          if (herr) fail(PM_ERR_TIMEOUT, "a wait on the tensor cores ran out (QR update)");
          if (g_kprof) g_kprof->add_flops("tc_gemm32", fl);
        }
        CK(cudaGetLastError());
      }
    }
  }
  // 3. CPQR with rank detection
  int total_n = 0;
  std::vector<int> noff(nid + 1, 0);
  for (int i = 0; i < nid; ++i) noff[i + 1] = noff[i] + nn[i];
  total_n = noff[nid];
  double* norm2 = scr.get<double>(2 * (size_t)std::max(total_n, 1));
  int* perm = scr.get<int>(std::max(total_n, 1));
  C* rdiag = scr.get<C>(std::max(total_n, 1));
  int* rank = scr.get<int>(nid);
  double* ref = scr.get<double>(nid);
  CK(cudaMemsetAsync(rank, 0xff, nid * sizeof(int), st));
  CK(cudaMemsetAsync(perm, 0, std::max(total_n, 1) * sizeof(int), st));
  std::vector<CpqrProb<C>> cp(nid);
  std::vector<CpqrChunk> chunks;
  int maxT = 0;
  for (int i = 0; i < nid; ++i) {
    int tgt = std::min(We[i], nn[i]);
    cp[i] = CpqrProb<C>{Z[i], W[i], We[i], nn[i], tol, CPQR_FIND_RANK, 0, tgt,
                        norm2 + 2 * (size_t)noff[i], perm + noff[i], rdiag + noff[i], rank + i, ref + i};
    maxT = std::max(maxT, tgt);
    for (int c0 = 0; c0 < nn[i]; c0 += CPQR_CB) chunks.push_back(CpqrChunk{i, c0, std::min(c0 + CPQR_CB, nn[i]), c0 == 0});
  }
  // tallest matrices first: their chunks carry the most work per step
  std::stable_sort(chunks.begin(), chunks.end(), [&](const CpqrChunk& a, const CpqrChunk& b) { return We[a.id] > We[b.id]; });
  bool tall = false;   // any complex64 input pivoted on >= 2048 rows
  for (int i = 0; i < nid; ++i) tall = tall || We[i] >= 2048;
  int* ctr = scr.get<int>(2 * (size_t)maxT + 2);
  CK(cudaMemsetAsync(ctr, 0, (2 * (size_t)maxT + 2) * sizeof(int), st));
  auto* dcp = upload(scr, cp, st);
  auto* dch = upload(scr, chunks, st);
  const int nch = (int)chunks.size();
  cpqr_init_norms<C>(dcp, dch, nch, st);
  std::vector<int> hr(nid);
  // With predicted ranks, run the predicted number of steps (+1, where the stop
  // test of the last rank happens) before the first check; otherwise check
  // every 16 steps.  Launches and results are the same either way.
  int first_check = 15;
  if (!khat.empty()) {
    // first check once half of the IDs should have found their rank; the rest
    // (over- or under-predicted bounds) finish under the regular 16-step checks
    std::vector<int> due;
    for (int i = 0; i < nid; ++i)
      if (cp[i].target > 0) due.push_back(std::min(cp[i].target, khat[i] + 1) - 1);
    if (!due.empty()) {
      std::sort(due.begin(), due.end());
      first_check = std::max(0, due[(due.size() - 1) / 2]);
    }
  }
  for (int t = 0; t < maxT; ++t) {
    cpqr_step<C>(dcp, dch, nch, t, ctr + t, st, tall);
    for (const auto& J : jobs) J.F->stats.cpqr_launches++;
    const bool check = khat.empty() ? ((t % 16 == 15) || t == maxT - 1)
                                    : (t == first_check || (t > first_check && ((t - first_check) % 16 == 0)) ||
                                       t == maxT - 1);
    if (check) {
      CK(cudaMemcpyAsync(hr.data(), rank, nid * sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (const auto& J : jobs) J.F->stats.rank_checks++;
      int pending = 0;
      for (int i = 0; i < nid; ++i) if (hr[i] < 0 && t + 1 < cp[i].target) ++pending;
      if (pending == 0) break;
    }
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(hr.data(), rank, nid * sizeof(int), cudaMemcpyDeviceToHost, st));
  // an exactly zero ID input (no far field at all: the interior rows of the
  // simplified Burton-Miller system) gets a zero interpolation, not an
  // identity on arbitrary pivots
  std::vector<double> href(nid);
  CK(cudaMemcpyAsync(href.data(), ref, nid * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<char> zero_in(nid);
  for (int i = 0; i < nid; ++i) zero_in[i] = nn[i] > 0 && !(href[i] > 0);
  std::vector<int> r(nid);
  for (int i = 0; i < nid; ++i) r[i] = hr[i] >= 0 ? hr[i] : cp[i].target;
  if (!khat.empty())
    for (int i = 0; i < nid; ++i) jobs[job_of[i / 4]].F->stats.predictor_fallbacks += r[i] > khat[i];   // above the bound
  // 4. pair ranks k_g = max(row rank, column rank); extend the shorter factorization
  std::vector<int> kk(nid);
  int maxExt = 0;
  for (int b = 0; b < nb; ++b)
    for (int grp = 0; grp < 2; ++grp) {
      int ir = 4 * b + grp, ic = 4 * b + 2 + grp;
      int k = std::min(std::max(r[ir], r[ic]), std::min(cp[ir].target, cp[ic].target));
      kk[ir] = kk[ic] = k;
      BFx(b).kg[grp] = k;
    }
  for (int i = 0; i < nid; ++i) {
    cp[i].mode = CPQR_EXTEND;
    cp[i].base = r[i];
    cp[i].target = std::max(kk[i], r[i]);
    maxExt = std::max(maxExt, cp[i].target - cp[i].base);
  }
  if (maxExt > 0) {
    dcp = upload(scr, cp, st);
    for (int t = 0; t < maxExt; ++t) cpqr_step<C>(dcp, dch, nch, t, ctr + maxT + t, st, tall);
    for (const auto& J : jobs) J.F->stats.cpqr_launches += maxExt;
    CK(cudaGetLastError());
  }
  // training data for the predictor: features -> (max(row rank, column rank) / n,
  // proxy count used / the rule's); the held-out check's ratio is filled in below
  std::vector<size_t> rec0(nj);
  for (int j = 0; j < nj; ++j) rec0[j] = jobs[j].F->proxy_ratio.size();
  for (int b = 0; b < nb; ++b)
    for (int grp = 0; grp < 2; ++grp) {
      const float* f = &feat[(2 * (size_t)b + grp) * MLP_IN];
      pm_factor* Fb = jobs[job_of[b]].F;
      Fb->rank_X.insert(Fb->rank_X.end(), f, f + MLP_IN);
      const double n = std::max(nn[4 * b + grp], 1);
      Fb->rank_T.push_back((float)(std::max(r[4 * b + grp], r[4 * b + 2 + grp]) / n));
      Fb->rank_T.push_back((float)BOX(b).p / (float)std::max(BOX(b).p_rule, 1));
      Fb->proxy_ratio.push_back(-1.f);
      Fb->proxy_redone.push_back(BOX(b).locked ? 1 : 0);
    }
  {
    // the unchosen columns follow the pivots, ascending (defines the column order of T)
    std::vector<PermFill> pf;
    for (int i = 0; i < nid; ++i) {
      if (nn[i] > 65536) fail(PM_ERR_UNSUPPORTED, "ID with more than 65536 candidate indices");
      pf.push_back(PermFill{perm + noff[i], nn[i], std::max(r[i], kk[i])});
    }
    auto* dpf = upload(scr, pf, st);
    complete_perm(dpf, nid, st);
    CK(cudaGetLastError());
  }
  if (g_kprof) {
    double f = 0, fi = 0;
    for (int i = 0; i < nid; ++i) {
      int S = std::max(r[i], kk[i]);
      for (int s2 = 0; s2 < S; ++s2) f += 20.0 * (double)(We[i] - s2 - 1) * (nn[i] - s2 - 1);
      fi += 4.0 * (double)kk[i] * kk[i] * (nn[i] - kk[i]);
    }
    // FP64: 20 flops per trailing entry and step; FP32 (memory-bound): the
    // algorithmic bytes, one read and one write of every trailing entry
    if (std::is_same<C, double2>::value) g_kprof->add_flops("cpqr_step", f);
    else g_kprof->add_flops("cpqr_step32", f / 20.0 * 2.0 * sizeof(C));
    g_kprof->add_flops(kname<C>("interp_solve", "interp_solve32"), fi);
  }
  std::vector<int> hperm(std::max(total_n, 1));
  CK(cudaMemcpyAsync(hperm.data(), perm, std::max(total_n, 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  // 5. interpolation matrices T = R11^{-1} R12: R11 and R12 gathered in pivot
  // order, then one blocked upper-triangular solve for all IDs
  std::vector<InterpProb<C>> ip;
  std::vector<SolveProb<C>> ts;
  std::vector<C*> T(nid, nullptr);
  int maxcols = 0, maxk = 0;
  size_t maxel = 0;
  for (int i = 0; i < nid; ++i) {
    int k = kk[i], n = nn[i];
    if (k <= 0 || n - k <= 0 || zero_in[i]) continue;
    T[i] = scr.get<C>((size_t)k * (n - k));
    C* r11 = scr.get<C>((size_t)k * k);
    ip.push_back(InterpProb<C>{Z[i], W[i], n, k, perm + noff[i], rdiag + noff[i], T[i], k, r11});
    ts.push_back(SolveProb<C>{r11, k, k, nullptr, T[i], k, n - k});
    maxcols = std::max(maxcols, n - k);
    maxk = std::max(maxk, k);
    maxel = std::max(maxel, (size_t)k * n);
  }
  if (!ip.empty()) {
    auto* dip = upload(scr, ip, st);
    interp_gather<C>(dip, (int)ip.size(), maxel, st);
    auto* dts = upload(scr, ts, st);
    la_trsm_upper_batched<C>(dts, (int)ts.size(), maxk, maxcols, kname<C>("interp_solve", "interp_solve32"), 0.0, st);
    CK(cudaGetLastError());
  }
  // 5b. held-out proxy check: each ID's candidates against its box's held-out
  // ring, gathered in pivot order so that H = [H_S | H_J]; then H_J -= H_S T
  // and ratio = ||H_J|| / (tol ||H||) (no counterpart in the paper)
  if (check_on) {
    GatherBatch<C> gh;
    GemmBatch<C> ge;
    std::vector<SqNormProb> nref, nerr;
    double* sums = scr.get<double>(2 * (size_t)nid);
    CK(cudaMemsetAsync(sums, 0, 2 * (size_t)nid * sizeof(double), st));
    std::vector<C*> H(nid, nullptr);
    std::vector<int> Wh(nid, 0);
    for (int b = 0; b < nb; ++b) {
      const int jj = job_of[b], lb = lbox(b);
      const pm_geometry* g = GEO(b);
      const Box& box = BOX(b);
      const BoxF<C>& bf = BFx(b);
      const int co = 2 * nbase[jj];
      const int h0 = pbase[jj] + hoff[jj][lb];
      std::vector<int> ring;
      for (int grp = 0; grp < 2; ++grp)
        for (int s2 = 0; s2 < box.p; ++s2) ring.push_back((h0 + s2) * 2 + grp);
      for (int q = 0; q < 4; ++q) {
        const int id = 4 * b + q;
        const int n = nn[id], k = kk[id];
        if (n <= 0) continue;
        const bool row_id = q < 2;
        std::vector<int> cand(n);
        for (int j2 = 0; j2 < n; ++j2) {
          const int pos_i = pos[id][hperm[noff[id] + j2]];
          cand[j2] = g->code_of(row_id ? bf.rows[pos_i] : bf.cols[pos_i]) + co;
        }
        Wh[id] = (int)ring.size();
        H[id] = scr.get<C>((size_t)Wh[id] * n);
        if (row_id) gh.add(H[id], Wh[id], Wh[id], n, cand, ring, 1, 0, g->k0);
        else gh.add(H[id], Wh[id], Wh[id], n, ring, cand, 0, 0, g->k0);
        nref.push_back(SqNormProb{H[id], Wh[id], Wh[id], n, sums + 2 * id});
        if (k > 0 && n - k > 0)
          ge.add(Wh[id], n - k, k, H[id], Wh[id], T[id], k, H[id] + (size_t)k * Wh[id], Wh[id], cmone<C>(), cone<C>(), 0);
        if (n - k > 0) nerr.push_back(SqNormProb{H[id] + (size_t)k * Wh[id], Wh[id], Wh[id], n - k, sums + 2 * id + 1});
      }
    }
    gh.run(scr, P, 0.0, st);
    sqnorm_batch<C>(nref, scr, st);
    ge.run(scr, st);
    sqnorm_batch<C>(nerr, scr, st);
    std::vector<double> hs(2 * (size_t)nid);
    CK(cudaMemcpyAsync(hs.data(), sums, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int b = 0; b < nb; ++b) {
      double ratio = 0;
      for (int q = 0; q < 4; ++q) {
        const int id = 4 * b + q;
        if (nn[id] <= 0) continue;
        const double ref = hs[2 * id], err = hs[2 * id + 1];
        ratio = std::max(ratio, ref > 0 ? std::sqrt(err / ref) / tol : 0.0);
      }
      const int jj = job_of[b];
      pm_factor* Fb = jobs[jj].F;
      Fb->stats.proxy_checked++;
      for (int grp = 0; grp < 2; ++grp) Fb->proxy_ratio[rec0[jj] + 2 * (b - jb_off[jj]) + grp] = (float)ratio;
      const Box& box = BOX(b);
      if (failed && ratio > PROXY_CHECK_BOUND && box.p < box.p_rule) failed->push_back({jj, lbox(b)});
    }
    if (failed && !failed->empty()) return;   // the caller redoes the level
  }
  const double ms_id = t_id.stop();
  for (const auto& J : jobs) J.F->stats.ms_id += ms_id;
  Timer t_sc(st);
  // 6. skeleton lists, L (into X) and R
  std::vector<ScatterProb<C>> sp;
  std::vector<int> posall;
  std::vector<size_t> posref;
  int maxe = 0;
  for (int b = 0; b < nb; ++b) {
    BoxF<C>& bf = BFx(b);
    Arena& ar = jobs[job_of[b]].F->arena;
    bf.kb = bf.kg[0] + bf.kg[1];
    bf.X = ar.get<C>((size_t)std::max(bf.mb, 1) * std::max(bf.kb, 1));
    bf.Rm = ar.get<C>((size_t)std::max(bf.kb, 1) * std::max(bf.mb, 1));
    bf.At = ar.get<C>((size_t)std::max(bf.kb, 1) * std::max(bf.kb, 1));
    bf.ipiv = ar.get<int>(std::max(bf.mb, 1));
    CK(cudaMemsetAsync(bf.X, 0, sizeof(C) * (size_t)bf.mb * bf.kb, st));
    CK(cudaMemsetAsync(bf.Rm, 0, sizeof(C) * (size_t)bf.mb * bf.kb, st));
    int off = 0;
    for (int grp = 0; grp < 2; ++grp) {
      int k = bf.kg[grp];
      int ir = 4 * b + grp, ic = 4 * b + 2 + grp;
      for (int j = 0; j < k; ++j) {
        int pr = pos[ir][hperm[noff[ir] + j]];
        bf.srows.push_back(bf.rows[pr]); bf.srgrp.push_back(grp);
        int pc = pos[ic][hperm[noff[ic] + j]];
        bf.scols.push_back(bf.cols[pc]); bf.scgrp.push_back(grp);
      }
      for (int side = 0; side < 2; ++side) {
        int id = side == 0 ? ir : ic;
        if (zero_in[id]) continue;   // zero interpolation: the block of X (L) or R stays zero
        size_t po = posall.size();
        posall.insert(posall.end(), pos[id].begin(), pos[id].end());
        ScatterProb<C> sc{side == 0 ? bf.X : bf.Rm, side == 0 ? bf.mb : bf.kb, off, side == 0,
                          nullptr, perm + noff[id], k, nn[id], T[id], k};
        sp.push_back(sc);
        posref.push_back(po);
        maxe = std::max(maxe, k * nn[id]);
      }
      off += k;
    }
  }
  if (!sp.empty()) {
    int* dpos = upload(scr, posall, st);
    for (size_t i = 0; i < sp.size(); ++i) sp[i].pos = dpos + posref[i];
    auto* dsp = upload(scr, sp, st);
    scatter_interp<C>(dsp, (int)sp.size(), maxe, st);
    CK(cudaGetLastError());
  }
  // 7. LU of D_b, X = D_b^{-1} L_b, Y = R_b X, A~_b = Y^{-1}
  // injected (tests): the first leaf box's self block zeroed
  const bool first_is_leaf = nb > 0 && jobs[0].lev == jobs[0].F->L;
  if ((O.debug_flags & PM_DEBUG_SINGULAR_BLOCK) && first_is_leaf)
    CK(cudaMemsetAsync(BFx(0).D, 0, sizeof(C) * (size_t)BFx(0).mb * BFx(0).mb, st));
  std::vector<LuProb<C>> lu;
  for (int b = 0; b < nb; ++b) lu.push_back(LuProb<C>{BFx(b).D, BFx(b).mb, BFx(b).mb, BFx(b).ipiv, nullptr});
  lu_batch<C>(lu, scr, st, "diagonal block");
  std::vector<SolveProb<C>> sv;
  for (int b = 0; b < nb; ++b)
    sv.push_back(SolveProb<C>{BFx(b).D, BFx(b).mb, BFx(b).mb, BFx(b).ipiv, BFx(b).X, BFx(b).mb, BFx(b).kb});
  solve_batch<C>(sv, scr, st);
  GemmBatch<C> gy;
  std::vector<C*> Y(nb);
  std::vector<int*> ypiv(nb);
  std::vector<CopyProb<C, C>> idp;
  for (int b = 0; b < nb; ++b) {
    BoxF<C>& bf = BFx(b);
    Y[b] = scr.get<C>((size_t)std::max(bf.kb, 1) * std::max(bf.kb, 1));
    ypiv[b] = scr.get<int>(std::max(bf.kb, 1));
    gy.add(bf.kb, bf.kb, bf.mb, bf.Rm, bf.kb, bf.X, bf.mb, Y[b], bf.kb, cone<C>(), czero_h<C>(), 1);
    if (bf.kb > 0) {
      k_identity<C><<<(bf.kb * bf.kb + 255) / 256, 256, 0, st>>>(bf.At, bf.kb, bf.kb);
      pm_launch_count_add(1);
    }
  }
  gy.run(scr, st);
  if ((O.debug_flags & PM_DEBUG_SINGULAR_COMPRESSED) && first_is_leaf && BFx(0).kb > 0)
    CK(cudaMemsetAsync(Y[0], 0, sizeof(C) * (size_t)BFx(0).kb * BFx(0).kb, st));   // injected: singular R A^-1 L
  std::vector<LuProb<C>> luy;
  std::vector<SolveProb<C>> svy;
  for (int b = 0; b < nb; ++b) {
    const BoxF<C>& bf = BFx(b);
    if (bf.kb <= 0) continue;
    luy.push_back(LuProb<C>{Y[b], bf.kb, bf.kb, ypiv[b], nullptr});
    svy.push_back(SolveProb<C>{Y[b], bf.kb, bf.kb, ypiv[b], bf.At, bf.kb, bf.kb});
  }
  lu_batch<C>(luy, scr, st, "R A^-1 L (compressed block)");
  solve_batch<C>(svy, scr, st);
  const double ms_sc = t_sc.stop();
  for (const auto& J : jobs) {
    J.F->stats.ms_schur += ms_sc;
    int sk = 0;
    for (auto& bf : levels_of<C>(J.F)[J.lev]) sk += bf.kb;
    if (J.lev < 16) J.F->stats.skeleton[J.lev] = sk;
  }
}

template <class C>
void process_level(pm_factor* F, int lev, double tol) {
  process_levels<C>({LevelJob{F, lev}}, F->scratch, F->st, tol);
}

// Top-level systems in FP64 from the level-1 boxes (arithmetic Cc), or the
// single inclusion's self block, of one or more factorizations: one gather,
// one copy and one batched LU for all of them.
template <class Cc>
void factor_tops(const std::vector<pm_factor*>& Fs, Arena& scr, cudaStream_t st) {
  scr.reset();
  Timer t(st);
  std::vector<LevelJob> jobs;
  for (pm_factor* F : Fs) jobs.push_back(LevelJob{F, 0});
  std::vector<int> base, pbase;
  std::vector<std::vector<int>> poff;
  PointsDev P = make_points_joint(jobs, false, scr, st, base, pbase, poff);
  GatherBatch<double2> gb;
  CopyBatch<Cc, double2> cb;
  std::vector<LuProb<double2>> lu;
  std::vector<LuProb<float2>> lu32;
  std::vector<const double2*> r64;
  std::vector<float2*> r32;
  std::vector<int> rn;
  for (size_t i = 0; i < Fs.size(); ++i) {
    pm_factor* F = Fs[i];
    const pm_geometry* g = F->g;
    BoxF<double2>& rt = F->root;
    if (F->L == 0) {
      int j = F->tree[0][0].leaves[0];
      int n = g->inc[j].n_nodes;
      rt.mb = 2 * n;
      for (int r = 0; r < 2 * n; ++r) { rt.rows.push_back(g->row_off[j] + r); rt.rgrp.push_back(r >= n); }
      rt.cols = rt.rows; rt.cgrp = rt.rgrp;
      rt.D = F->arena.get<double2>((size_t)rt.mb * rt.mb);
      assemble_self<double2>(g, {j}, {rt.D}, {rt.mb}, scr, st, F->opts.formulation >= PM_FORM_BM);
    } else {
      set_form(gb, F);
      merge_children<Cc, double2>(F, levels_of<Cc>(F)[1], F->tree[0][0], rt, gb, cb, 2 * base[i]);
    }
    if (F->precision == PM_MIXED && !(F->opts.flags & PM_FLAG_TOP_FP64)) {
      // mixed mode: a preconditioner whose levels carry ID errors of ~5e-6;
      // the top system is factored in complex64 from its FP64 assembly
      F->root32 = F->arena.get<float2>((size_t)std::max(rt.mb, 1) * rt.mb);
      F->ipiv32 = F->arena.get<int>(std::max(rt.mb, 1));
      lu32.push_back(LuProb<float2>{F->root32, rt.mb, rt.mb, F->ipiv32, nullptr});
      r64.push_back(rt.D); r32.push_back(F->root32); rn.push_back(rt.mb);
      continue;
    }
    rt.ipiv = F->arena.get<int>(std::max(rt.mb, 1));
    lu.push_back(LuProb<double2>{rt.D, rt.mb, rt.mb, rt.ipiv, nullptr});
  }
  gb.run(scr, P, 0.0, st);
  cb.run(scr, st);
  if (!r64.empty()) {
    const int maxn = *std::max_element(rn.begin(), rn.end());
    round_blocks(upload(scr, r64, st), upload(scr, r32, st), upload(scr, rn, st), (int)rn.size(), maxn, st);
    for (pm_factor* F : Fs)
      if (F->root32) {
        const int mb = F->root.mb;
        float2* planes = F->arena.get<float2>(2 * (size_t)std::max(mb, 1) * mb);
        F->root_op = SplitOp{planes, planes + (size_t)mb * mb, (size_t)std::max(mb, 1)};
        split_copy(F->root.D, mb, F->root_op, mb, mb, nullptr, st);
      }
    CK(cudaGetLastError());
    lu_batch<float2>(lu32, scr, st, "top-level system");
  }
  lu_batch<double2>(lu, scr, st, "top-level system");
  const double ms = t.stop();
  for (pm_factor* F : Fs) {
    F->stats.K = F->root.mb;
    F->stats.ms_top += ms;
  }
}

template <class Cc>
void factor_top(pm_factor* F) {
  factor_tops<Cc>({F}, F->scratch, F->st);
}

// ---------------------------------------------------------------------------------
// Solve (paper Sec. 3): upward RHS compression, top solve, downward recovery.
// C is the arithmetic of the compressed levels; the top system is FP64.
template <class C>
struct SolveWork {
  std::vector<std::vector<C*>> fin, ft;   // per level and box: f_b (-> g_b -> x_b), f~_b
  double2* froot = nullptr;
};

template <class C>
void solve_up(pm_factor* F, const C* rhs, int nrhs, SolveWork<C>& w, Arena& ws, cudaStream_t st) {
  const pm_geometry* g = F->g;
  const int N = g->N;
  const int L = F->L;
  auto& LV = levels_of<C>(F);
  w.fin.assign(L + 1, {}); w.ft.assign(L + 1, {});
  for (int l = 1; l <= L; ++l) {
    auto& BF = LV[l];
    w.fin[l].resize(BF.size()); w.ft[l].resize(BF.size());
    for (size_t b = 0; b < BF.size(); ++b) {
      w.fin[l][b] = ws.get<C>((size_t)std::max(BF[b].mb, 1) * nrhs);
      w.ft[l][b] = ws.get<C>((size_t)std::max(BF[b].kb, 1) * nrhs);
    }
  }
  BoxF<double2>& rt = F->root;
  w.froot = ws.get<double2>((size_t)std::max(rt.mb, 1) * nrhs);
  {
    CopyBatch<C, C> cb;
    auto& BF = LV[L];
    for (size_t b = 0; b < BF.size(); ++b) cb.add(rhs + BF[b].rows[0], N, w.fin[L][b], BF[b].mb, BF[b].mb, nrhs);
    cb.run(ws, st);
  }
  for (int l = L; l >= 1; --l) {
    auto& BF = LV[l];
    std::vector<SolveProb<C>> sv;
    for (size_t b = 0; b < BF.size(); ++b)
      sv.push_back(SolveProb<C>{BF[b].D, BF[b].mb, BF[b].mb, BF[b].ipiv, w.fin[l][b], BF[b].mb, nrhs});
    solve_batch<C>(sv, ws, st, F->d_wait_err, (F->opts.debug_flags & PM_DEBUG_SOLVE_NO_FLAG) != 0);  // g_b = D_b^{-1} f_b
    std::vector<C*> t(BF.size());
    GemmBatch<C> g1, g2;
    for (size_t b = 0; b < BF.size(); ++b) {
      t[b] = ws.get<C>((size_t)std::max(BF[b].kb, 1) * nrhs);
      g1.add(BF[b].kb, nrhs, BF[b].mb, BF[b].Rm, BF[b].kb, w.fin[l][b], BF[b].mb, t[b], BF[b].kb, cone<C>(),
             czero_h<C>(), 1);
      g2.add(BF[b].kb, nrhs, BF[b].kb, BF[b].At, BF[b].kb, t[b], BF[b].kb, w.ft[l][b], BF[b].kb, cone<C>(),
             czero_h<C>(), 1);
    }
    g1.run(ws, st);
    g2.run(ws, st);
    // f~ of every child into its parent's right-hand side
    const auto& parents = F->tree[l - 1];
    if (l - 1 == 0) {
      CopyBatch<C, double2> cb;
      for (size_t a = 0; a < parents[0].children.size(); ++a) {
        int c = parents[0].children[a];
        cb.add(w.ft[l][c], BF[c].kb, w.froot + rt.child_off[a], rt.mb, BF[c].kb, nrhs);
      }
      cb.run(ws, st);
    } else {
      CopyBatch<C, C> cb;
      for (size_t pidx = 0; pidx < parents.size(); ++pidx) {
        const BoxF<C>& pb = LV[l - 1][pidx];
        for (size_t a = 0; a < parents[pidx].children.size(); ++a) {
          int c = parents[pidx].children[a];
          cb.add(w.ft[l][c], BF[c].kb, w.fin[l - 1][pidx] + pb.child_off[a], pb.mb, BF[c].kb, nrhs);
        }
      }
      cb.run(ws, st);
    }
  }
}

template <class C>
void solve_down(pm_factor* F, int nrhs, SolveWork<C>& w, C* phi, Arena& ws, cudaStream_t st) {
  const pm_geometry* g = F->g;
  const int N = g->N;
  const int L = F->L;
  auto& LV = levels_of<C>(F);
  BoxF<double2>& rt = F->root;
  C* xroot = nullptr;
  if (std::is_same<C, double2>::value) {
    xroot = (C*)w.froot;
  } else {
    xroot = ws.get<C>((size_t)std::max(rt.mb, 1) * nrhs);
    CopyBatch<double2, C> cb;
    cb.add(w.froot, rt.mb, xroot, rt.mb, rt.mb, nrhs);
    cb.run(ws, st);
  }
  for (int l = 1; l <= L; ++l) {
    auto& BF = LV[l];
    const auto& parents = F->tree[l - 1];
    GemmBatch<C> g1, g2;
    for (size_t pidx = 0; pidx < parents.size(); ++pidx) {
      const int pmb = (l - 1 == 0) ? rt.mb : LV[l - 1][pidx].mb;
      const std::vector<int>& coff = (l - 1 == 0) ? rt.child_off : LV[l - 1][pidx].child_off;
      const C* px = (l - 1 == 0) ? xroot : w.fin[l - 1][pidx];
      for (size_t a = 0; a < parents[pidx].children.size(); ++a) {
        int c = parents[pidx].children[a];
        const C* y = px + coff[a];
        // f~ - A~ y, then x = g - X (f~ - A~ y)
        g1.add(BF[c].kb, nrhs, BF[c].kb, BF[c].At, BF[c].kb, y, pmb, w.ft[l][c], BF[c].kb, cmone<C>(), cone<C>(), 0);
        g2.add(BF[c].mb, nrhs, BF[c].kb, BF[c].X, BF[c].mb, w.ft[l][c], BF[c].kb, w.fin[l][c], BF[c].mb, cmone<C>(),
               cone<C>(), 0);
      }
    }
    g1.run(ws, st);
    g2.run(ws, st);
  }
  CopyBatch<C, C> cb;
  auto& BF = LV[L];
  for (size_t b = 0; b < BF.size(); ++b) cb.add(w.fin[L][b], BF[b].mb, phi + BF[b].cols[0], N, BF[b].mb, nrhs);
  cb.run(ws, st);
}

void root_solve(pm_factor* F, double2* x, int ldx, int nrhs, Arena& ws, cudaStream_t st) {
  BoxF<double2>& rt = F->root;
  const bool no_flag = (F->opts.debug_flags & PM_DEBUG_SOLVE_NO_FLAG) != 0;
  if (F->root32) {
    // complex64 top LU with one correction from the FP64 residual:
    // x0 = S(b), x = x0 + S(b - A x0), S = the complex64 LU solve (the
    // correction takes the top solve's error from ~kappa u32 to ~(kappa u32)^2)
    const int mb = rt.mb;
    const size_t len = (size_t)std::max(mb, 1) * nrhs;
    float2* x32 = ws.get<float2>(len);
    double2* b = ws.get<double2>(len);
    double2* y = ws.get<double2>(len);
    double* norms = ws.get<double>(2 * (size_t)nrhs);
    auto solve32 = [&](const double2* src, int lds, double2* dst, int ldd) {
      CopyBatch<double2, float2> down;
      down.add(src, lds, x32, mb, mb, nrhs);
      down.run(ws, st);
      std::vector<SolveProb<float2>> sv{SolveProb<float2>{F->root32, mb, mb, F->ipiv32, x32, mb, nrhs}};
      solve_batch<float2>(sv, ws, st, F->d_wait_err, no_flag);
      CopyBatch<float2, double2> up;
      up.add(x32, mb, dst, ldd, mb, nrhs);
      up.run(ws, st);
    };
    CopyBatch<double2, double2> keep;                         // b: the right-hand sides, leading dimension mb
    keep.add(x, ldx, b, mb, mb, nrhs);
    keep.run(ws, st);
    double2* x0 = ws.get<double2>(len);
    solve32(b, mb, x0, mb);                                  // x0 = S(b)
    dense_matvec64(F->root_op, mb, x0, mb, y, mb, nrhs, st);  // y = A x0
    CK(cudaMemsetAsync(norms, 0, 2 * nrhs * sizeof(double), st));
    residual64(b, y, b, mb, nrhs, norms, st);                // b = b - A x0
    solve32(b, mb, y, mb);                                   // y = S(b - A x0)
    axpy64(x0, y, mb, nrhs, st);                             // x0 += y
    CopyBatch<double2, double2> back;
    back.add(x0, mb, x, ldx, mb, nrhs);
    back.run(ws, st);
    CK(cudaGetLastError());
    return;
  }
  std::vector<SolveProb<double2>> sv{SolveProb<double2>{rt.D, rt.mb, rt.mb, rt.ipiv, x, ldx, nrhs}};
  solve_batch<double2>(sv, ws, st, F->d_wait_err, no_flag);
}

// phi = M^{-1} rhs with the compressed factorization (FP64 levels).
void apply_inverse64(pm_factor* F, const double2* rhs, int nrhs, double2* phi, Arena& ws, cudaStream_t st) {
  const int N = F->g->N;
  if (F->L == 0) {
    CopyBatch<double2, double2> cb;
    cb.add(rhs, N, phi, N, N, nrhs);
    cb.run(ws, st);
    root_solve(F, phi, N, nrhs, ws, st);
    return;
  }
  SolveWork<double2> w;
  solve_up<double2>(F, rhs, nrhs, w, ws, st);
  root_solve(F, w.froot, F->root.mb, nrhs, ws, st);
  solve_down<double2>(F, nrhs, w, phi, ws, st);
}

// phi = M^{-1} rhs with the mixed factorization (FP32 levels, FP64 top).
// rhs is FP64; each column is scaled to unit norm for the FP32 part.
void apply_inverse_mixed(pm_factor* F, const double2* rhs, int nrhs, double2* phi, const double* d_scale,
                         const double* d_unscale, Arena& ws, cudaStream_t st) {
  const int N = F->g->N;
  CK(cudaMemsetAsync(phi, 0, sizeof(double2) * (size_t)N * nrhs, st));
  if (F->L == 0) {
    CopyBatch<double2, double2> cb;
    cb.add(rhs, N, phi, N, N, nrhs);
    cb.run(ws, st);
    root_solve(F, phi, N, nrhs, ws, st);
    return;
  }
  Cf* r32 = ws.get<Cf>((size_t)N * nrhs);
  Cf* p32 = ws.get<Cf>((size_t)N * nrhs);
  scale_to32(rhs, r32, N, nrhs, d_scale, st);
  SolveWork<Cf> w;
  solve_up<Cf>(F, r32, nrhs, w, ws, st);
  root_solve(F, w.froot, F->root.mb, nrhs, ws, st);
  solve_down<Cf>(F, nrhs, w, p32, ws, st);
  axpy_from32(phi, p32, N, nrhs, d_unscale, st);
  CK(cudaGetLastError());
}

// phi = M^{-1} rhs through the factor's plan for (kind, nrhs): kind 0 the
// compressed inverse of an FP64 factorization, kind 1 the mixed
// preconditioner with per-column scales h_scale (2 nrhs host values: scale,
// unscale).  The first use runs the launches eagerly in the plan's arena
// (sizing it); the second captures the same launches into a CUDA graph on
// the plan's stream, with descriptor uploads done synchronously on a side
// stream into the arena, and instantiates it; later uses replay the graph on
// `st`.  The caller holds F->plan_mu; the body synchronises nothing.
void run_planned(pm_factor* F, int kind, const double2* rhs, int nrhs, double2* phi, const double* h_scale,
                 cudaStream_t st) {
  const int N = F->g->N;
  auto& up = F->plans[std::make_pair(kind, nrhs)];
  if (!up) up.reset(new SolvePlan());
  SolvePlan& P = *up;
  P.uses++;
  const size_t bytes = sizeof(double2) * (size_t)N * nrhs;
  if (!P.in) {
    P.io.min_block = 1 << 20;
    P.in = P.io.get<double2>((size_t)N * nrhs);
    P.out = P.io.get<double2>((size_t)N * nrhs);
    P.scal = P.io.get<double>(2 * (size_t)nrhs);
  }
  CK(cudaMemcpyAsync(P.in, rhs, bytes, cudaMemcpyDeviceToDevice, st));
  if (kind == 1) CK(cudaMemcpyAsync(P.scal, h_scale, 2 * nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
  auto body = [&](cudaStream_t s2) {
    if (kind == 0) apply_inverse64(F, P.in, nrhs, P.out, P.ws, s2);
    else apply_inverse_mixed(F, P.in, nrhs, P.out, P.scal, P.scal + nrhs, P.ws, s2);
  };
  const bool graphs = !F->profiling && !(F->opts.flags & PM_FLAG_NO_GRAPHS);
  if (!P.exec && graphs && P.uses >= 2) {
    if (!P.cap) CK(cudaStreamCreateWithFlags(&P.cap, cudaStreamNonBlocking));
    if (!P.side) CK(cudaStreamCreateWithFlags(&P.side, cudaStreamNonBlocking));
    CK(cudaStreamSynchronize(st));   // the eager run that used the arena has finished
    P.ws.reset();                    // the same launches again: the arena allocates nothing new
    CK(cudaStreamBeginCapture(P.cap, cudaStreamCaptureModeRelaxed));
    g_capture_side = P.side;
    cudaGraph_t graph = nullptr;
    try {
      body(P.cap);
    } catch (...) {
      g_capture_side = nullptr;
      cudaStreamEndCapture(P.cap, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      throw;
    }
    g_capture_side = nullptr;
    CK(cudaStreamEndCapture(P.cap, &graph));
    const cudaError_t e = cudaGraphInstantiate(&P.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) P.exec = nullptr;
    CK(e);
    F->graph_captures++;
  }
  if (P.exec) {
    CK(cudaGraphLaunch(P.exec, st));
    F->graph_launches++;
  } else {
    P.ws.reset();
    body(st);
  }
  CK(cudaMemcpyAsync(phi, P.out, bytes, cudaMemcpyDeviceToDevice, st));
}

double hankel_flops_per_pair(const pm_geometry* g);

// Y = A X with the FP64 operator (self blocks + on-the-fly off-diagonal kernels).
void apply_operator64(pm_factor* F, const double2* X, int nrhs, double2* Y, Arena& ws, cudaStream_t st) {
  const pm_geometry* g = F->g;
  const int N = g->N;
  if (F->dense64) {
    double2* Xs = ws.get<double2>((size_t)N * nrhs);
    scale_rows(F->d_colscale, X, N, Xs, N, N, nrhs, st);
    dense_matvec64(F->dense_op, N, Xs, N, Y, N, nrhs, st);
    if (g_kprof) g_kprof->add_flops("dense_matvec64", 8.0 * (double)N * N * nrhs);
    CK(cudaGetLastError());
    return;
  }
  GemmBatch<double2> gb;
  for (int j = 0; j < g->m; ++j) {
    const int r0 = g->row_off[j], m2 = 2 * g->inc[j].n_nodes;
    gb.add(m2, nrhs, m2, F->self64[j], m2, X + r0, N, Y + r0, N, cone<double2>(), czero_h<double2>(), 1);
  }
  gb.run(ws, st);
  OpNodes nd{g->nodes.x, g->nodes.y, g->nodes.nx, g->nodes.ny, g->nodes.w, g->nodes.incl, F->d_iu, F->d_iq};
  apply_offdiag64(nd, g->total_nodes, g->k0, X, N, Y, N, nrhs, st);
  if (g_kprof) {
    // algorithmic FP64 flops per ordered node pair: 47 for the geometry and
    // the four weighted entries, the Hankel pair, 32 per right-hand side (4
    // complex multiply-adds); special functions not counted
    double pairs = (double)g->total_nodes * g->total_nodes;
    for (int j = 0; j < g->m; ++j) pairs -= (double)g->inc[j].n_nodes * g->inc[j].n_nodes;
    g_kprof->add_flops("apply_offdiag64", pairs * (47.0 + hankel_flops_per_pair(g) + 32.0 * nrhs));
  }
  CK(cudaGetLastError());
}

// Iterative refinement (mixed mode): x <- x + M^{-1} (b - A x) until the
// relative residual of every column is below refine_tol.  With the dense
// operator the first residual is an FP32 product, the later intermediate ones
// float-float (~1e-13 relative) on the FP32 pipes, or, once the residual is
// small, the update r <- r - A dx with an FP32 product; only FP64 residuals
// decide convergence.
void solve_refined(pm_factor* F, const double2* B, int nrhs, double2* X, Arena& ws, cudaStream_t st,
                   pm_solve_info* info) {
  const pm_geometry* g = F->g;
  const int N = g->N;
  double2* Y = ws.get<double2>((size_t)N * nrhs);
  double2* R = ws.get<double2>((size_t)N * nrhs);
  double2* dX = ws.get<double2>((size_t)N * nrhs);
  double* norms = ws.get<double>(2 * (size_t)nrhs);
  double* scal = ws.get<double>(2 * (size_t)nrhs);
  std::vector<double> hn(2 * nrhs), hs(2 * nrhs);
  auto finish = [&]() {   // R = B - Y, column norms -> worst relative residual
    CK(cudaMemsetAsync(norms, 0, 2 * nrhs * sizeof(double), st));
    residual64(B, Y, R, N, nrhs, norms, st);
    CK(cudaMemcpyAsync(hn.data(), norms, 2 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double worst = 0;
    for (int r = 0; r < nrhs; ++r) worst = std::max(worst, std::sqrt(hn[2 * r]) / std::max(std::sqrt(hn[2 * r + 1]), 1e-300));
    return worst;
  };
  // The residual that can end the refinement: the float-float product folded
  // into FP64 every 16 columns (a smaller worst-case error bound than a
  // sequential FP64 sum, on the FP32 pipes), or with PM_FLAG_FP64_CONFIRM the
  // FP64 product.
  const bool ff_confirm = F->dense64 && !(F->opts.flags & PM_FLAG_FP64_CONFIRM);
  // the stored operator is column-scaled: its products take diag(cs) x
  double2* Xs = F->dense64 ? ws.get<double2>((size_t)N * nrhs) : nullptr;
  auto scaled = [&](const double2* x) -> const double2* {
    scale_rows(F->d_colscale, x, N, Xs, N, N, nrhs, st);
    return Xs;
  };
  auto residual = [&](const double2* x) {
    if (ff_confirm) {
      dense_matvec_ffc(F->dense_op, N, scaled(x), N, Y, N, nrhs, st);
      CK(cudaGetLastError());
    } else {
      apply_operator64(F, x, nrhs, Y, ws, st);
    }
    return finish();
  };
  auto residual_low = [&](const double2* x) {
    dense_matvec_ff(F->dense_op, N, scaled(x), N, Y, N, nrhs, st);
    CK(cudaGetLastError());
    return finish();
  };
  auto residual_f32 = [&](const double2* x) {
    dense_matvec32(F->dense_op, N, scaled(x), N, Y, N, nrhs, st);
    CK(cudaGetLastError());
    return finish();
  };
  std::vector<double> bnorm(nrhs, 1.0);
  // r <- r - A dx (dx: the correction just added to x) with an FP32 product.
  // Its rounding (~1e-6 of |A dx| ~ |r|) stays in the new residual and in x,
  // so it is used only while 1e-6 |r| is far below refine_tol; the new
  // residual goes to dx's buffer and the two buffers swap.
  auto residual_update32 = [&]() {
    dense_matvec32(F->dense_op, N, scaled(dX), N, Y, N, nrhs, st);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(norms, 0, 2 * nrhs * sizeof(double), st));
    residual64(R, Y, dX, N, nrhs, norms, st);
    std::swap(R, dX);
    CK(cudaMemcpyAsync(hn.data(), norms, 2 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double worst = 0;
    for (int r = 0; r < nrhs; ++r) worst = std::max(worst, std::sqrt(hn[2 * r]) / bnorm[r]);
    return worst;
  };
  auto precond = [&](const double2* rhs, double2* out, const std::vector<double>& colnorm) {
    for (int r = 0; r < nrhs; ++r) {
      double nr = colnorm[r] > 0 ? colnorm[r] : 1.0;
      hs[r] = 1.0 / nr;
      hs[nrhs + r] = nr;
    }
    run_planned(F, 1, rhs, nrhs, out, hs.data(), st);
  };
  // x0 = 0, r0 = b (no operator application needed)
  CK(cudaMemsetAsync(X, 0, sizeof(double2) * (size_t)N * nrhs, st));
  CK(cudaMemsetAsync(Y, 0, sizeof(double2) * (size_t)N * nrhs, st));
  double res = finish();
  std::vector<double> cn(nrhs);
  for (int r = 0; r < nrhs; ++r) {
    cn[r] = std::sqrt(hn[2 * r]);
    bnorm[r] = std::max(std::sqrt(hn[2 * r + 1]), 1e-300);
  }
  int it = 0;
  const double tolr = F->opts.refine_tol > 0 ? F->opts.refine_tol : 1e-10;
  const int maxit = F->opts.max_refine > 0 ? F->opts.max_refine : 10;
  std::vector<double> hist;
  double prev = -1;   // the residual before res (none yet)
  while (it < maxit) {
    precond(R, dX, cn);
    axpy64(X, dX, N, nrhs, st);
    ++it;
    bool exact = true;
    if (F->dense64) {
      // Refinement contracts the residual by a nearly constant factor; when
      // that trend says this step meets the tolerance, the residual is formed
      // in FP64 straight away (a wrong guess costs nothing: that residual
      // drives the next step).  Otherwise float-float or the FP32 update,
      // confirmed in FP64 once it meets the tolerance.
      // (factor 2 of margin: a wrong guess costs a second FP64 product)
      const double rate = prev > 0 ? res / prev : 1.0;
      exact = res * rate <= 0.5 * tolr;
    }
    double r_new;
    if (exact) r_new = residual(X);
    else if (prev < 0) {
      // first step (x0 = 0): its residual is ~1e-3 of b, far above the ~1e-6
      // error of an FP32 product; a smaller one is formed again in float-float
      r_new = residual_f32(X);
      if (r_new < 1e-4) r_new = residual_low(X);
    } else if (1e-6 * res <= 0.05 * tolr) r_new = residual_update32();
    else r_new = residual_low(X);
    if (!exact && r_new <= tolr) { r_new = residual(X); exact = true; }
    prev = res;
    res = r_new;
    hist.push_back(res);
    for (int r = 0; r < nrhs; ++r) cn[r] = std::sqrt(hn[2 * r]);
    if (exact && res <= tolr) break;
  }
  if (info) {
    info->iterations = it;
    info->residual = res;
    for (size_t i = 0; i < hist.size() && i < 16; ++i) info->history[i] = hist[i];
  }
  if (res > tolr) {
    int werr = 0;
    CK(cudaMemcpyAsync(&werr, F->d_wait_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (werr) return;   // reported as PM_ERR_TIMEOUT by the caller
    fail(PM_ERR_NOT_CONVERGED, "iterative refinement stopped at relative residual " + std::to_string(res));
  }
}

pm_status run_guarded(const char* where, const std::function<void()>& fn);

}  // namespace

namespace {
pm_status run_guarded(const char* where, const std::function<void()>& fn) {
  try {
    fn();
    return PM_OK;
  } catch (const PmError& e) {
    g_err = std::string(where) + ": " + e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    g_err = std::string(where) + ": host allocation failed";
    return PM_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = std::string(where) + ": " + e.what();
    return PM_ERR_INVALID_ARG;
  }
}

void check_device() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    fail(PM_ERR_CUDA, "no CUDA device available (this library has no CPU fallback)");
  }
}

// Device memory of the given device (or managed memory): anything else, such
// as a host pointer or another GPU's buffer, is rejected before a kernel could
// touch it.  cudaPointerGetAttributes allocates nothing.
void require_device_ptr(const void* p, int device, const char* what) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    fail(PM_ERR_INVALID_ARG, std::string(what) + " is not a CUDA pointer");
  }
  if (!(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged))
    fail(PM_ERR_INVALID_ARG, std::string(what) + " is not device memory (a host pointer?)");
  if (a.type == cudaMemoryTypeDevice && a.device != device)
    fail(PM_ERR_INVALID_ARG, std::string(what) + " lives on device " + std::to_string(a.device) + ", not on device " +
                                 std::to_string(device));
}

void require_current_device(int device, const char* what) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != device)
    fail(PM_ERR_INVALID_ARG, std::string(what) + ": the current device is " + std::to_string(dev) +
                                 ", the geometry was built on device " + std::to_string(device));
}

// Burton-Miller right-hand side from the PMCHWT one, per inclusion and column:
// [f_u + alpha f_q; 0] with f = [f_u; f_q] = [-u^I; -q^I], alpha = i / k+.
__global__ void k_bm_rhs(const InclDev* __restrict__ inc, const int* __restrict__ incl, int total, double k0,
                         const double2* __restrict__ f, double2* __restrict__ b, int N, int nrhs) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (q >= total || c >= nrhs) return;
  const InclDev d = inc[incl[q]];
  const int l = q - d.node_off;
  const double2 fu = f[d.row_off + l + (size_t)c * N], fq = f[d.row_off + d.n + l + (size_t)c * N];
  b[d.row_off + l + (size_t)c * N] = make_double2(fu.x - fq.y / k0, fu.y + fq.x / k0);
  b[d.row_off + d.n + l + (size_t)c * N] = make_double2(0.0, 0.0);
}

// [u; q] per inclusion (Burton-Miller unknowns) -> [q; u] (the PMCHWT order).
__global__ void k_bm_order(const InclDev* __restrict__ inc, const int* __restrict__ incl, int total,
                           const double2* __restrict__ x, double2* __restrict__ phi, int N, int nrhs) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (q >= total || c >= nrhs) return;
  const InclDev d = inc[incl[q]];
  const int l = q - d.node_off;
  const size_t o = (size_t)c * N + d.row_off;
  phi[o + l] = x[o + d.n + l];
  phi[o + d.n + l] = x[o + l];
}

// Sets *flag when any of the n doubles at x is NaN or infinite.
__global__ void k_flag_nonfinite(const double* __restrict__ x, size_t n, int* flag) {
  int bad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) *flag = 1;
}

// Rejects right-hand sides holding a NaN or an infinity (host or device data).
void require_finite_rhs(const pm_c64* rhs, size_t count, int on_device, Arena& ws, cudaStream_t st) {
  if (!on_device) {
    for (size_t i = 0; i < count; ++i)
      if (!std::isfinite(rhs[i].re) || !std::isfinite(rhs[i].im))
        fail(PM_ERR_INVALID_ARG, "right-hand side entry " + std::to_string(i) + " is not finite");
    return;
  }
  int* flag = ws.get<int>(1);
  CK(cudaMemsetAsync(flag, 0, sizeof(int), st));
  const size_t n = 2 * count;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
  k_flag_nonfinite<<<std::max(blocks, 1), 256, 0, st>>>((const double*)rhs, n, flag);
  pm_launch_count_add(1);
  CK(cudaGetLastError());
  int h = 0;
  CK(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h) fail(PM_ERR_INVALID_ARG, "a right-hand side entry is not finite");
}
}  // namespace

namespace {

// Option checks shared by pm_factorize and pm_factor_batch (sets g_err).
bool check_factor_opts(const pm_factor_opts* opts, const char* where) {
  const std::string w(where);
  if (!(opts->tol > 0 && opts->tol < 1)) { g_err = w + ": tol must be in (0, 1)"; return false; }
  if (opts->proxy_factor != 0 && !(opts->proxy_factor > 1)) { g_err = w + ": proxy_factor must be > 1"; return false; }
  if (opts->proxy_points < 0 || opts->proxy_points > 100000) { g_err = w + ": bad proxy_points"; return false; }
  if (opts->precision != PM_FP64 && opts->precision != PM_MIXED) { g_err = w + ": unsupported precision"; return false; }
  if (opts->precision == PM_MIXED && (opts->low_tol < 0 || opts->low_tol >= 1 || opts->refine_tol < 0 || opts->max_refine < 0)) {
    g_err = w + ": bad refinement options";
    return false;
  }
  if (opts->formulation < PM_FORM_OMIT || opts->formulation > PM_FORM_BM_SIMPLIFIED) {
    g_err = w + ": unknown formulation";
    return false;
  }
  if (!(opts->proxy_scale >= 0 && opts->proxy_scale <= 1)) { g_err = w + ": proxy_scale must be in [0, 1]"; return false; }
  return true;
}

// Options, tree and proxy plan of a new factorization; returns the ID threshold.
double setup_factor(pm_factor* F, const pm_geometry* g, const pm_factor_opts* opts) {
  if (opts->formulation != PM_FORM_OMIT) {
    if (opts->precision != PM_FP64) fail(PM_ERR_UNSUPPORTED, "PMCHWT (All) and Burton-Miller run in PM_FP64 only");
    for (const auto& c : g->inc)
      if (c.k_in.im != 0 || c.k_in.re != g->inc[0].k_in.re)
        fail(PM_ERR_UNSUPPORTED, "PMCHWT (All) and Burton-Miller need one real interior wavenumber for all inclusions");
  }
  F->g = g;
  F->opts = *opts;
  if (F->opts.proxy_factor == 0) F->opts.proxy_factor = 1.5;
  F->st = (cudaStream_t)opts->stream;
  F->L = g->L;
  F->precision = opts->precision;
  F->tree = g->levels;
  // the FP32 factorization of the mixed mode cannot resolve tolerances far below FP32 precision
  const double id_tol = F->precision == PM_MIXED ? std::max(opts->tol, opts->low_tol > 0 ? opts->low_tol : 5e-6)
                                                 : opts->tol;
  pm_factor_opts popts = F->opts;
  popts.tol = id_tol;
  plan_proxies(g, F->tree, &popts);
  F->stats.levels = F->L;
  F->stats.N = g->N;
  F->profiling = (opts->flags & 1u) != 0;
  if (F->precision == PM_FP64) F->lev64.assign(F->L + 1, {});
  else F->lev32.assign(F->L + 1, {});
  F->d_wait_err = F->arena.get<int>(1);
  CK(cudaMemsetAsync(F->d_wait_err, 0, sizeof(int), F->st));
  return id_tol;
}

// The levels of several factorizations (same precision and options) in shared
// launches: step s processes level L_i - s of every problem i that has one, so
// problems of different depths meet at their leaves first; then all top-level
// systems at once.  One factorization is the group of one.
// Scratch bytes a box's IDs take when its level runs (four inputs of W rows
// and about mb/2 candidates each, with the workspaces of the QR, the CPQR and
// the interpolation matrices), estimated before the level's active sets exist.
template <class C>
double box_scratch_bytes(pm_factor* F, int lev, int b) {
  auto mb_of = [&](int bb) -> double {
    const Box& x = F->tree[lev][bb];
    if (lev == F->L) return 2.0 * F->g->inc[x.leaves[0]].n_nodes;
    double m = 0;
    for (int c : x.children) m += levels_of<C>(F)[lev + 1][c].kb;
    return m;
  };
  const Box& box = F->tree[lev][b];
  double near = 0;
  for (int o : box.near) near += mb_of(o);
  const double W = near + (F->opts.formulation == PM_FORM_ALL ? 4.0 : 2.0) * box.p_rule;
  return 1.5 * sizeof(C) * 2.0 * W * mb_of(b);
}

// The jobs' boxes in consecutive chunks whose scratch estimates stay within
// budget bytes (a box larger than the budget runs alone).
template <class C>
std::vector<std::vector<LevelJob>> plan_chunks(const std::vector<LevelJob>& jobs, double budget) {
  std::vector<std::vector<LevelJob>> chunks(1);
  double acc = 0;
  for (const LevelJob& J : jobs) {
    const int nbj = (int)J.F->tree[J.lev].size();
    for (int b = 0; b < nbj; ++b) {
      const double bytes = box_scratch_bytes<C>(J.F, J.lev, b);
      if (acc > 0 && acc + bytes > budget) { chunks.emplace_back(); acc = 0; }
      auto& cur = chunks.back();
      if (!cur.empty() && cur.back().F == J.F && cur.back().b1 == b) cur.back().b1 = b + 1;
      else cur.push_back(LevelJob{J.F, J.lev, b, b + 1});
      acc += bytes;
    }
  }
  return chunks;
}

template <class C>
void factor_group_t(std::vector<pm_factor*>& Fs, double id_tol, Arena& scr, cudaStream_t st) {
  int Lmax = 0;
  for (pm_factor* F : Fs) Lmax = std::max(Lmax, F->L);
  for (int s = 0; s < Lmax; ++s) {
    std::vector<LevelJob> level_jobs;
    for (pm_factor* F : Fs)
      if (F->L - s >= 1) level_jobs.push_back(LevelJob{F, F->L - s});
    Timer tl(st);
    // scratch budget: opts.scratch_gb, else 35% of the device memory free now.
    // The scratch blocks of the previous step go back first: sized for its
    // boxes, they would otherwise stay allocated beside the larger ones the
    // next level's boxes need.
    if (s > 0) {
      CK(cudaStreamSynchronize(st));
      scr.release(Done::Idle);
    }
    double budget = Fs[0]->opts.scratch_gb * 1e9;
    if (!(budget > 0)) {
      size_t fr = 0, tot = 0;
      CK(cudaMemGetInfo(&fr, &tot));
      budget = 0.35 * (double)(fr + pool_cached_bytes(current_device()));
    }
    const auto chunks = plan_chunks<C>(level_jobs, budget);
    for (const auto& jobs : chunks) {
      std::vector<std::pair<int, int>> failed;
      std::vector<size_t> nx(jobs.size()), nt(jobs.size()), np(jobs.size());
      for (size_t j = 0; j < jobs.size(); ++j) {
        nx[j] = jobs[j].F->rank_X.size(); nt[j] = jobs[j].F->rank_T.size(); np[j] = jobs[j].F->proxy_ratio.size();
      }
      process_levels<C>(jobs, scr, st, id_tol, &failed);
      if (!failed.empty()) {
        // boxes whose learned proxy count failed the held-out check: the rule's
        // count from now on, and the level again (its samples recorded afresh)
        for (auto& fb : failed) {
          Box& box = jobs[fb.first].F->tree[jobs[fb.first].lev][fb.second];
          box.p = box.p_rule;
          box.locked = true;
          jobs[fb.first].F->stats.proxy_fallbacks++;
        }
        for (size_t j = 0; j < jobs.size(); ++j) {
          pm_factor* F = jobs[j].F;
          F->rank_X.resize(nx[j]); F->rank_T.resize(nt[j]);
          F->proxy_ratio.resize(np[j]); F->proxy_redone.resize(np[j]);
        }
        process_levels<C>(jobs, scr, st, id_tol, nullptr);
      }
    }
    const double ms = tl.stop();
    for (auto& J : level_jobs)
      if (J.lev < 16) J.F->stats.ms_level[J.lev] = ms;
    for (auto* F : Fs) F->stats.level_chunks += (int)chunks.size();
  }
  factor_tops<C>(Fs, scr, st);
}

void factor_group(std::vector<pm_factor*>& Fs, double id_tol, Arena& scr, cudaStream_t st) {
  if (Fs.empty()) return;
  if (Fs[0]->precision == PM_FP64) factor_group_t<double2>(Fs, id_tol, scr, st);
  else factor_group_t<float2>(Fs, id_tol, scr, st);
}

// Mixed mode, after the complex64 levels: the FP64 self blocks, index maps and
// (when it fits) the dense FP64 operator of the refinement residual.
// Average algorithmic FP64 flops of one Hankel pair (H0, H1) over the node
// pairs of a geometry (the square root, reciprocal square root, sincos and,
// below z = 8, CUDA's Bessel functions not counted): 64 for the 12-term
// expansion (z >= 60), 28 + 8 d for a degree-d fit (d = 5 on [20, 60), 7 on
// [12, 20), 8 on [8, 12)), none below 8; averaged over 65,536 pairs of
// nodes of different inclusions drawn with a fixed seed.  Used for the
// profiler's counts of the operator kernels.
double hankel_flops_per_pair(const pm_geometry* g) {
  const int T = g->total_nodes;
  if (T < 2 || g->m < 2) return 0.0;
  auto incl_of = [&](int q) {
    return (int)(std::upper_bound(g->node_off.begin(), g->node_off.begin() + g->m, q) - g->node_off.begin()) - 1;
  };
  uint64_t st = 0x9E3779B97F4A7C15ull;
  auto next = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (int)((st >> 33) % (uint64_t)T);
  };
  double sum = 0;
  int n = 0;
  while (n < 65536) {
    const int t = next(), q = next();
    if (incl_of(t) == incl_of(q)) continue;
    const double z = g->k0 * std::hypot(g->hx[t] - g->hx[q], g->hy[t] - g->hy[q]);
    if (z >= 60) sum += 64;
    else if (z >= 20) sum += 28 + 8 * 5;
    else if (z >= 12) sum += 28 + 8 * 7;
    else if (z >= 8) sum += 28 + 8 * 8;
    ++n;
  }
  return sum / n;
}

// Index maps, column scales and, when it fits, the dense FP64 operator of a
// mixed factorization (its self blocks are copied in by finish_mixed).
// beside: the assembly runs on a low-priority stream as the persistent
// kernel (one CTA of 128 threads per SM), concurrently with the
// factorization that follows: it is FP64-bound and the complex64
// factorization leaves the FP64 pipes idle; finish_mixed joins it.
void start_mixed_operator(pm_factor* F, bool beside) {
  const pm_geometry* g = F->g;
  const pm_factor_opts* opts = &F->opts;
  F->op_started = true;
  std::vector<int> iu(g->total_nodes), iq(g->total_nodes);
  for (int j = 0; j < g->m; ++j)
    for (int l = 0; l < g->inc[j].n_nodes; ++l) {
      iu[g->node_off[j] + l] = g->row_off[j] + l;
      iq[g->node_off[j] + l] = g->row_off[j] + g->inc[j].n_nodes + l;
    }
  F->d_iu = upload(F->arena, iu, F->st);
  F->d_iq = upload(F->arena, iq, F->st);
  // With room in HBM, write the FP64 operator out once: each refinement step
  // is then a skinny FP64 GEMM instead of a Hankel evaluation per node pair.
  // Budget: 60% of the free memory, and all dense operators held in the
  // process at most 40% of the device; otherwise (or if the allocation
  // fails) the refinement applies the operator on the fly.
  const size_t need = 2 * sizeof(float2) * (size_t)g->N * g->N;
  if (!(opts->flags & PM_FLAG_NO_DENSE_OPERATOR) && g->total_nodes <= 65535) {
    std::lock_guard<std::mutex> lk(g_dense_mu);
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    fr += pool_cached_bytes(current_device());   // cached blocks are free for this purpose
    if (need <= fr / 10 * 6 && g_dense_held + need <= tot / 10 * 4) {
      F->dense64 = (float2*)pool_malloc(need);
      if (F->dense64) {
        F->dense_op = SplitOp{F->dense64, F->dense64 + (size_t)g->N * g->N, (size_t)g->N};
        F->dense_bytes = need;
        g_dense_held += need;
      }
    }
  }
  if (!F->dense64) return;
  OpNodes nd{g->nodes.x, g->nodes.y, g->nodes.nx, g->nodes.ny, g->nodes.w, g->nodes.incl, F->d_iu, F->d_iq};
  F->d_colscale = F->arena.get<double>((size_t)g->N);
  dense_colscale(g->nodes.w, F->d_iu, F->d_iq, g->total_nodes, g->k0, F->d_colscale, F->st);
  if (beside) {
    int pr_lo = 0, pr_hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&pr_lo, &pr_hi));
    CK(cudaStreamCreateWithPriority(&F->op_st, cudaStreamNonBlocking, pr_lo));
    CK(cudaEventCreateWithFlags(&F->op_done, cudaEventDisableTiming));
    CK(cudaEventRecord(F->op_done, F->st));   // the index maps are on the device
    CK(cudaStreamWaitEvent(F->op_st, F->op_done, 0));
    int* counter = F->arena.get<int>(1);
    assemble_dense_offdiag64_rows(nd, g->total_nodes, g->k0, F->dense_op, counter, F->op_st);
    CK(cudaEventRecord(F->op_done, F->op_st));
  } else {
    assemble_dense_offdiag64(nd, g->total_nodes, g->k0, F->dense_op, F->st);
  }
  if (g_kprof) {
    double pairs = (double)g->total_nodes * g->total_nodes;
    for (int j = 0; j < g->m; ++j) pairs -= (double)g->inc[j].n_nodes * g->inc[j].n_nodes;
    // per unordered pair: 40 for the geometry and the eight entries of both
    // 2 x 2 blocks, plus the Hankel pair
    g_kprof->add_flops("dense_offdiag64", 0.5 * pairs * (40.0 + hankel_flops_per_pair(g)));
  }
  CK(cudaGetLastError());
}

void finish_mixed(pm_factor* F) {
  const pm_geometry* g = F->g;
  // FP64 self blocks and index maps for the refinement residual
  // (those of the leaves' inclusions were assembled with the leaf level)
  F->scratch.reset();
  std::vector<int> incl, lda;
  std::vector<double2*> A64;
  if (F->self64.size() != (size_t)g->m) F->self64.assign(g->m, nullptr);
  for (int j = 0; j < g->m; ++j) {
    if (F->self64[j]) continue;
    const int m2 = 2 * g->inc[j].n_nodes;
    F->self64[j] = F->arena.get<double2>((size_t)m2 * m2);
    incl.push_back(j); lda.push_back(m2); A64.push_back(F->self64[j]);
  }
  if (!incl.empty()) assemble_self<double2>(g, incl, A64, lda, F->scratch, F->st);
  if (!F->op_started) start_mixed_operator(F, false);
  if (F->dense64) {
    if (F->op_done) CK(cudaStreamWaitEvent(F->st, F->op_done, 0));
    for (int j = 0; j < g->m; ++j) {
      const int m2 = 2 * g->inc[j].n_nodes;
      split_copy(F->self64[j], m2, F->dense_op.at(g->row_off[j], g->row_off[j]), m2, m2, F->d_colscale + g->row_off[j],
                 F->st);
    }
    CK(cudaGetLastError());
  }
}

}  // namespace

extern "C" {

const char* pm_last_error(void) { return g_err.c_str(); }

pm_status pm_release_cached_memory(int64_t* bytes) {
  const size_t n = pool_trim(-1);
  if (bytes) *bytes = (int64_t)n;
  return PM_OK;
}

pm_status pm_build_geometry(const pm_problem* prob, pm_geometry** out) {
  if (!prob || !out) { g_err = "pm_build_geometry: NULL argument"; return PM_ERR_INVALID_ARG; }
  *out = nullptr;
  pm_geometry* g = nullptr;
  pm_status s = run_guarded("pm_build_geometry", [&] {
    if (prob->m < 1 || !prob->inc) fail(PM_ERR_INVALID_ARG, "need m >= 1 inclusions");
    if (!(prob->k_out > 0) || !std::isfinite(prob->k_out)) fail(PM_ERR_INVALID_ARG, "k_out must be positive");
    if (!(prob->spacing >= 0) || !std::isfinite(prob->spacing))
      fail(PM_ERR_INVALID_ARG, "spacing must be positive, or 0 for an arbitrary arrangement");
    for (int j = 0; j < prob->m; ++j) {
      const pm_inclusion& c = prob->inc[j];
      if (c.shape < 0 || c.shape > 3) fail(PM_ERR_INVALID_ARG, "unknown shape");
      if (c.n_nodes < 16 || c.n_nodes > 4096 || (c.n_nodes & 1)) fail(PM_ERR_INVALID_ARG, "n_nodes must be even in [16, 4096]");
      if (!std::isfinite(c.cx) || !std::isfinite(c.cy) || !std::isfinite(c.rot)) fail(PM_ERR_INVALID_ARG, "non-finite centre");
      for (int i = 0; i < 16; ++i) if (!std::isfinite(c.prm[i])) fail(PM_ERR_INVALID_ARG, "non-finite shape parameter");
      if (!(c.prm[0] > 0)) fail(PM_ERR_INVALID_ARG, "shape size must be positive");
      if (!(c.k_in.re > 0)) fail(PM_ERR_INVALID_ARG, "k_in must have positive real part");
      if (!(c.k_in.im >= 0) || !std::isfinite(c.k_in.im)) fail(PM_ERR_INVALID_ARG, "k_in must have Im >= 0");
    }
    check_device();
    g = new pm_geometry();
    CK(cudaGetDevice(&g->device));
    g->m = prob->m; g->k0 = prob->k_out; g->spacing = prob->spacing;
    g->general = prob->spacing == 0;
    g->gnx = prob->grid_nx; g->gny = prob->grid_ny;
    g->inc.assign(prob->inc, prob->inc + prob->m);
    g->node_off.assign(g->m + 1, 0); g->row_off.assign(g->m + 1, 0);
    for (int j = 0; j < g->m; ++j) {
      g->node_off[j + 1] = g->node_off[j] + g->inc[j].n_nodes;
      g->row_off[j + 1] = 2 * g->node_off[j + 1];
      g->maxn = std::max(g->maxn, g->inc[j].n_nodes);
    }
    g->total_nodes = g->node_off[g->m];
    g->N = 2 * g->total_nodes;
    upload_inclusions(g);
    cudaStream_t st = 0;
    g->d_inc = upload(g->arena, g->hinc, st);
    const size_t T = g->total_nodes;
    NodesDev& nd = g->nodes;
    nd.x = g->arena.get<double>(T); nd.y = g->arena.get<double>(T); nd.nx = g->arena.get<double>(T);
    nd.ny = g->arena.get<double>(T); nd.speed = g->arena.get<double>(T); nd.w = g->arena.get<double>(T);
    nd.curv = g->arena.get<double>(T); nd.kress = g->arena.get<double>(T);
    std::vector<int> incl(T);
    for (int j = 0; j < g->m; ++j) for (int q = g->node_off[j]; q < g->node_off[j + 1]; ++q) incl[q] = j;
    nd.incl = upload(g->arena, incl, st);
    geom_nodes(g->d_inc, nd, (int)T, g->hinc.data(), st);
    CK(cudaGetLastError());
    g->hx.resize(T); g->hy.resize(T); g->hnx.resize(T); g->hny.resize(T); g->hw.resize(T);
    CK(cudaMemcpy(g->hx.data(), nd.x, T * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(g->hy.data(), nd.y, T * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(g->hnx.data(), nd.nx, T * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(g->hny.data(), nd.ny, T * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(g->hw.data(), nd.w, T * 8, cudaMemcpyDeviceToHost));
    build_tree(g, nullptr);
  });
  if (s != PM_OK) { delete g; return s; }
  *out = g;
  return PM_OK;
}

pm_status pm_geometry_size(const pm_geometry* g, int32_t* N, int32_t* total_nodes) {
  if (!g) { g_err = "pm_geometry_size: NULL geometry"; return PM_ERR_INVALID_ARG; }
  if (N) *N = g->N;
  if (total_nodes) *total_nodes = g->total_nodes;
  return PM_OK;
}

pm_status pm_geometry_nodes(const pm_geometry* g, double* xy, double* nrm, double* w) {
  if (!g) { g_err = "pm_geometry_nodes: NULL geometry"; return PM_ERR_INVALID_ARG; }
  for (int q = 0; q < g->total_nodes; ++q) {
    if (xy) { xy[2 * q] = g->hx[q]; xy[2 * q + 1] = g->hy[q]; }
    if (nrm) { nrm[2 * q] = g->hnx[q]; nrm[2 * q + 1] = g->hny[q]; }
    if (w) w[q] = g->hw[q];
  }
  return PM_OK;
}

pm_status pm_plane_wave_rhs(const pm_geometry* g, const double* angles, int32_t nrhs, pm_c64* rhs, int32_t on_device) {
  if (!g || !angles || !rhs || nrhs < 1) { g_err = "pm_plane_wave_rhs: bad argument"; return PM_ERR_INVALID_ARG; }
  return run_guarded("pm_plane_wave_rhs", [&] {
    Arena ws;
    ws.min_block = 1 << 20;
    cudaStream_t st = 0;
    if (on_device) {
      require_current_device(g->device, "pm_plane_wave_rhs");
      require_device_ptr(rhs, g->device, "rhs");
    }
    std::vector<double> a(angles, angles + nrhs);
    double* da = upload(ws, a, st);
    Cd* F = on_device ? (Cd*)rhs : ws.get<Cd>((size_t)g->N * nrhs);
    plane_wave_rhs<Cd>(g->d_inc, g->nodes, g->total_nodes, g->k0, da, nrhs, F, g->N, st);
    CK(cudaGetLastError());
    if (!on_device) CK(cudaMemcpy(rhs, F, sizeof(Cd) * (size_t)g->N * nrhs, cudaMemcpyDeviceToHost));
    CK(cudaStreamSynchronize(st));
  });
}

pm_status pm_factorize(const pm_geometry* g, const pm_factor_opts* opts, pm_factor** out) {
  if (!g || !opts || !out) { g_err = "pm_factorize: NULL argument"; return PM_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!check_factor_opts(opts, "pm_factorize")) return opts->precision != PM_FP64 && opts->precision != PM_MIXED
                                                          ? PM_ERR_UNSUPPORTED : PM_ERR_INVALID_ARG;
  pm_factor* F = new pm_factor();
  pm_status s = run_guarded("pm_factorize", [&] {
    TuneScope ts((opts->flags & PM_FLAG_NO_AUTOTUNE) != 0);
    const double id_tol = setup_factor(F, g, opts);
    struct ProfScope {
      explicit ProfScope(KProf* p) { g_kprof = p; }
      ~ProfScope() { g_kprof = nullptr; }
    } scope(F->profiling ? &F->prof : nullptr);
    Timer tt(F->st);
    F->op_pending = F->precision == PM_MIXED && !(F->opts.flags & PM_FLAG_OPERATOR_AFTER);
    std::vector<pm_factor*> one{F};
    factor_group(one, id_tol, F->scratch, F->st);
    if (F->precision == PM_MIXED) finish_mixed(F);
    F->stats.ms_total = tt.stop();
    if (F->profiling) F->prof.collect();
    F->scratch.release(Done::Idle);   // tt.stop() waited for the stream
  });
  if (s != PM_OK) { delete F; return s; }
  *out = F;
  return PM_OK;
}

namespace {
pm_status solve_impl(const pm_factor* Fc, const pm_c64* rhs, int32_t nrhs, pm_c64* phi, int32_t on_device,
                     pm_solve_info* info, cudaStream_t st) {
  if (!Fc || !rhs || !phi || nrhs < 1) { g_err = "pm_solve: bad argument"; return PM_ERR_INVALID_ARG; }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->residual = -1;
  }
  pm_factor* F = const_cast<pm_factor*>(Fc);
  return run_guarded("pm_solve", [&] {
    TuneScope ts((F->opts.flags & PM_FLAG_NO_AUTOTUNE) != 0);
    Arena ws;
    ws.min_block = 1 << 20;
    const size_t bytes = sizeof(Cd) * (size_t)F->g->N * nrhs;
    if (on_device) {
      require_current_device(F->g->device, "pm_solve");
      require_device_ptr(rhs, F->g->device, "rhs");
      require_device_ptr(phi, F->g->device, "phi");
    }
    require_finite_rhs(rhs, (size_t)F->g->N * nrhs, on_device, ws, st);
    const Cd* drhs = (const Cd*)rhs;
    Cd* dphi = (Cd*)phi;
    if (!on_device) {
      Cd* a = ws.get<Cd>((size_t)F->g->N * nrhs);
      CK(cudaMemcpyAsync(a, rhs, bytes, cudaMemcpyHostToDevice, st));
      drhs = a;
      dphi = ws.get<Cd>((size_t)F->g->N * nrhs);
    } else if ((const void*)rhs == (const void*)phi) {
      Cd* a = ws.get<Cd>((size_t)F->g->N * nrhs);
      CK(cudaMemcpyAsync(a, rhs, bytes, cudaMemcpyDeviceToDevice, st));
      drhs = a;
    }
    struct ProfScope {
      explicit ProfScope(KProf* p) { g_kprof = p; }
      ~ProfScope() { g_kprof = nullptr; }
    } scope(F->profiling ? &F->prof : nullptr);
    std::lock_guard<std::mutex> plan_lock(F->plan_mu);   // solves of one factor share its graphs
    if (F->precision == PM_FP64 && F->opts.formulation >= PM_FORM_BM) {
      // Burton-Miller: its own right-hand side, then its [u; q] unknowns reordered
      const pm_geometry* g = F->g;
      Cd* b = ws.get<Cd>((size_t)g->N * nrhs);
      Cd* x = ws.get<Cd>((size_t)g->N * nrhs);
      const dim3 grid((g->total_nodes + 255) / 256, nrhs);
      k_bm_rhs<<<grid, 256, 0, st>>>(g->d_inc, g->nodes.incl, g->total_nodes, g->k0, drhs, b, g->N, nrhs);
      pm_launch_count_add(1);
      CK(cudaGetLastError());
      run_planned(F, 0, b, nrhs, x, nullptr, st);
      k_bm_order<<<grid, 256, 0, st>>>(g->d_inc, g->nodes.incl, g->total_nodes, x, dphi, g->N, nrhs);
      pm_launch_count_add(1);
      CK(cudaGetLastError());
    } else if (F->precision == PM_FP64) {
      run_planned(F, 0, drhs, nrhs, dphi, nullptr, st);
    } else {
      solve_refined(F, drhs, nrhs, dphi, ws, st, info);
    }
    if (!on_device) CK(cudaMemcpyAsync(phi, dphi, bytes, cudaMemcpyDeviceToHost, st));
    int werr = 0;
    CK(cudaMemcpyAsync(&werr, F->d_wait_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ws.release(Done::Idle);
    if (F->profiling) F->prof.collect();
    if (werr) {
      CK(cudaMemsetAsync(F->d_wait_err, 0, sizeof(int), st));
      CK(cudaStreamSynchronize(st));
      fail(PM_ERR_TIMEOUT, "a bounded wait of the chained top-level solve ran out");
    }
  });
}
}  // namespace

pm_status pm_solve_ex(const pm_factor* Fc, const pm_c64* rhs, int32_t nrhs, pm_c64* phi, int32_t on_device,
                      pm_solve_info* info) {
  return solve_impl(Fc, rhs, nrhs, phi, on_device, info, Fc ? Fc->st : nullptr);
}

pm_status pm_solve(const pm_factor* F, const pm_c64* rhs, int32_t nrhs, pm_c64* phi, int32_t on_device) {
  return pm_solve_ex(F, rhs, nrhs, phi, on_device, nullptr);
}

// Independent problems factored concurrently: `workers` host threads, each
// with its own CUDA stream, take problems from a shared counter.
namespace {
pm_status run_batch(int count, int workers, const std::function<pm_status(int, cudaStream_t)>& one) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { g_err = "batch: no CUDA device"; return PM_ERR_CUDA; }
  workers = std::max(1, std::min(workers, count));
  std::atomic<int> next{0};
  std::vector<pm_status> st(count, PM_OK);
  std::vector<std::string> msg(count);
  auto body = [&]() {
    cudaSetDevice(dev);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= count) break;
      st[i] = one(i, s);
      if (st[i] != PM_OK) msg[i] = g_err;
    }
    if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < workers; ++w) th.emplace_back(body);
  body();
  for (auto& t : th) t.join();
  for (int i = 0; i < count; ++i)
    if (st[i] != PM_OK) { g_err = "problem " + std::to_string(i) + ": " + msg[i]; return st[i]; }
  return PM_OK;
}
}  // namespace

pm_status pm_factor_batch(const pm_geometry* const* g, int32_t count, const pm_factor_opts* opts, pm_factor** out,
                          int32_t workers) {
  if (!g || !opts || !out || count < 1) { g_err = "pm_factor_batch: bad argument"; return PM_ERR_INVALID_ARG; }
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  for (int i = 0; i < count; ++i)
    if (!g[i]) { g_err = "pm_factor_batch: NULL geometry " + std::to_string(i); return PM_ERR_INVALID_ARG; }
  if (!check_factor_opts(opts, "pm_factor_batch"))
    return opts->precision != PM_FP64 && opts->precision != PM_MIXED ? PM_ERR_UNSUPPORTED : PM_ERR_INVALID_ARG;
  // groups: problems in descending order of work (~N^1.5), each to the group
  // with the least work so far; a group's levels share launches
  const int ng = std::max(1, std::min(workers > 0 ? workers : 4, count));
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  auto work = [&](int i) { return std::pow((double)g[i]->N, 1.5); };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
  std::vector<std::vector<int>> groups(ng);
  std::vector<double> load(ng, 0.0);
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    groups[k].push_back(i);
    load[k] += work(i);
  }
  for (auto& grp : groups) std::sort(grp.begin(), grp.end());
  pm_status s = run_batch(ng, ng, [&](int k, cudaStream_t st) {
    return run_guarded("pm_factor_batch", [&] {
      TuneScope ts((opts->flags & PM_FLAG_NO_AUTOTUNE) != 0);
      std::vector<pm_factor*> Fs;
      double id_tol = 0;
      pm_factor_opts o = *opts;
      o.stream = st;
      o.flags &= ~(uint32_t)PM_FLAG_PROFILE;   // per-kernel profiles are per factorization
      for (int i : groups[k]) {
        out[i] = new pm_factor();
        id_tol = setup_factor(out[i], g[i], &o);
        Fs.push_back(out[i]);
      }
      Timer tt(st);
      Arena scr;
      factor_group(Fs, id_tol, scr, st);
      scr.release(Done::Stream, st);
      for (pm_factor* F : Fs)
        if (F->precision == PM_MIXED) { finish_mixed(F); F->scratch.release(Done::Stream, st); }
      const double ms = tt.stop();
      for (pm_factor* F : Fs) {
        F->stats.ms_total = ms;
        F->st = nullptr;   // the worker streams end with the batch
      }
    });
  });
  if (s != PM_OK) {
    for (int i = 0; i < count; ++i) { delete out[i]; out[i] = nullptr; }
  }
  return s;
}

pm_status pm_solve_batch(const pm_factor* const* f, int32_t count, const pm_c64* const* rhs, int32_t nrhs,
                         pm_c64* const* phi, int32_t on_device, int32_t workers) {
  if (!f || !rhs || !phi || count < 1 || nrhs < 1) { g_err = "pm_solve_batch: bad argument"; return PM_ERR_INVALID_ARG; }
  return run_batch(count, workers > 0 ? workers : 8, [&](int i, cudaStream_t st) {
    return solve_impl(f[i], rhs[i], nrhs, phi[i], on_device, nullptr, st);
  });
}

pm_status pm_factor_stats(const pm_factor* F, pm_stats* out) {
  if (!F || !out) { g_err = "pm_factor_stats: NULL argument"; return PM_ERR_INVALID_ARG; }
  *out = F->stats;
  out->graph_captures = F->graph_captures;
  out->graph_launches = F->graph_launches;
  return PM_OK;
}

pm_status pm_factor_skeleton(const pm_factor* F, int32_t level, int32_t box, int32_t* rows, int32_t* cols,
                             int32_t cap, int32_t* k) {
  if (!F || !k || level < 1 || level > F->L) { g_err = "pm_factor_skeleton: bad argument"; return PM_ERR_INVALID_ARG; }
  const std::vector<int>* sr = nullptr;
  const std::vector<int>* sc = nullptr;
  int kb = 0;
  if (F->precision == PM_FP64) {
    if (box < 0 || box >= (int)F->lev64[level].size()) { g_err = "pm_factor_skeleton: bad box"; return PM_ERR_INVALID_ARG; }
    const auto& b = F->lev64[level][box];
    sr = &b.srows; sc = &b.scols; kb = b.kb;
  } else {
    if (box < 0 || box >= (int)F->lev32[level].size()) { g_err = "pm_factor_skeleton: bad box"; return PM_ERR_INVALID_ARG; }
    const auto& b = F->lev32[level][box];
    sr = &b.srows; sc = &b.scols; kb = b.kb;
  }
  *k = kb;
  for (int i = 0; i < std::min(cap, kb); ++i) {
    if (rows) rows[i] = (*sr)[i];
    if (cols) cols[i] = (*sc)[i];
  }
  return PM_OK;
}

pm_status pm_matrix_entries(const pm_geometry* g, const int32_t* rows, int32_t M, const int32_t* cols, int32_t Nc,
                            pm_c64* out) {
  if (!g || !rows || !cols || !out || M < 1 || Nc < 1) { g_err = "pm_matrix_entries: bad argument"; return PM_ERR_INVALID_ARG; }
  for (int i = 0; i < M; ++i) if (rows[i] < 0 || rows[i] >= g->N) { g_err = "pm_matrix_entries: row out of range"; return PM_ERR_INVALID_ARG; }
  for (int j = 0; j < Nc; ++j) if (cols[j] < 0 || cols[j] >= g->N) { g_err = "pm_matrix_entries: column out of range"; return PM_ERR_INVALID_ARG; }
  return run_guarded("pm_matrix_entries", [&] {
    Arena ws;
    cudaStream_t st = 0;
    std::vector<int> t(M), s(Nc);
    for (int i = 0; i < M; ++i) t[i] = g->code_of(rows[i]);
    for (int j = 0; j < Nc; ++j) s[j] = g->code_of(cols[j]);
    Cd* d = ws.get<Cd>((size_t)M * Nc);
    GatherBatch<Cd> gb;
    gb.add(d, M, M, Nc, t, s, 0);
    std::vector<int> dummy;
    PointsDev P = make_points(g, {}, ws, st, dummy);
    gb.run(ws, P, g->k0, st);
    CK(cudaMemcpy(out, d, sizeof(Cd) * (size_t)M * Nc, cudaMemcpyDeviceToHost));
    // same-inclusion pairs are not off-diagonal entries
    for (int i = 0; i < M; ++i) {
      int ji = int(std::upper_bound(g->row_off.begin(), g->row_off.end(), rows[i]) - g->row_off.begin()) - 1;
      for (int j = 0; j < Nc; ++j) {
        int jj = int(std::upper_bound(g->row_off.begin(), g->row_off.end(), cols[j]) - g->row_off.begin()) - 1;
        if (ji == jj) out[i + (size_t)j * M] = pm_c64{0, 0};
      }
    }
  });
}

namespace {
// Shared body of pm_far_field / pm_scattered_field: pts holds ndir angles
// (far) or npts points as x, y pairs (near).
pm_status field_impl(const char* where, bool far, const pm_geometry* g, const pm_c64* phi, int32_t nrhs,
                     int32_t on_device, const double* pts, int32_t npts, pm_c64* out) {
  if (!g || !phi || !pts || !out || nrhs < 1 || npts < 1) {
    g_err = std::string(where) + ": bad argument";
    return PM_ERR_INVALID_ARG;
  }
  const int nv = far ? npts : 2 * npts;
  for (int i = 0; i < nv; ++i)
    if (!std::isfinite(pts[i])) { g_err = std::string(where) + ": non-finite direction or point"; return PM_ERR_INVALID_ARG; }
  return run_guarded(where, [&] {
    Arena ws;
    ws.min_block = 1 << 20;
    cudaStream_t st = 0;
    const size_t nphi = (size_t)g->N * nrhs, nout = (size_t)npts * nrhs;
    const Cd* dphi = (const Cd*)phi;
    Cd* dout = (Cd*)out;
    if (on_device) {
      require_current_device(g->device, where);
      require_device_ptr(phi, g->device, "phi");
      require_device_ptr(out, g->device, "out");
    } else {
      Cd* a = ws.get<Cd>(nphi);
      CK(cudaMemcpyAsync(a, phi, nphi * sizeof(Cd), cudaMemcpyHostToDevice, st));
      dphi = a;
      dout = ws.get<Cd>(nout);
    }
    std::vector<double> hp(pts, pts + nv);
    double* dp = upload(ws, hp, st);
    if (far) far_field(g->d_inc, g->nodes, g->total_nodes, g->k0, dphi, g->N, nrhs, dp, npts, dout, st);
    else scattered_field(g->d_inc, g->nodes, g->total_nodes, g->k0, dphi, g->N, nrhs, dp, npts, dout, st);
    CK(cudaGetLastError());
    if (!on_device) CK(cudaMemcpyAsync(out, dout, nout * sizeof(Cd), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  });
}
}  // namespace

pm_status pm_far_field(const pm_geometry* g, const pm_c64* phi, int32_t nrhs, int32_t on_device, const double* angles,
                       int32_t ndir, pm_c64* out) {
  return field_impl("pm_far_field", true, g, phi, nrhs, on_device, angles, ndir, out);
}

pm_status pm_scattered_field(const pm_geometry* g, const pm_c64* phi, int32_t nrhs, int32_t on_device,
                             const double* xy, int32_t npts, pm_c64* out) {
  return field_impl("pm_scattered_field", false, g, phi, nrhs, on_device, xy, npts, out);
}

pm_status pm_self_block(const pm_geometry* g, int32_t j, pm_c64* out) {
  if (!g || !out || j < 0 || j >= g->m) { g_err = "pm_self_block: bad argument"; return PM_ERR_INVALID_ARG; }
  return run_guarded("pm_self_block", [&] {
    Arena ws;
    cudaStream_t st = 0;
    int n = g->inc[j].n_nodes;
    Cd* d = ws.get<Cd>((size_t)4 * n * n);
    assemble_self<Cd>(g, {j}, {d}, {2 * n}, ws, st);
    CK(cudaMemcpy(out, d, sizeof(Cd) * (size_t)4 * n * n, cudaMemcpyDeviceToHost));
  });
}

pm_status pm_factor_profile(const pm_factor* F, pm_kernel_stat* out, int32_t cap, int32_t* count) {
  if (!F || !count) { g_err = "pm_factor_profile: NULL argument"; return PM_ERR_INVALID_ARG; }
  int i = 0;
  for (const auto& kv : F->prof.agg) {
    if (out && i < cap) {
      pm_kernel_stat& o = out[i];
      std::memset(&o, 0, sizeof(o));
      std::strncpy(o.name, kv.first.c_str(), sizeof(o.name) - 1);
      o.launches = (int32_t)kv.second.launches;
      o.ms = kv.second.ms;
      o.work = kv.second.flops;
    }
    ++i;
  }
  *count = i;
  return PM_OK;
}

pm_status pm_factor_rank_data(const pm_factor* F, float* X, float* T, int32_t cap, int32_t* count) {
  if (!F || !count) { g_err = "pm_factor_rank_data: NULL argument"; return PM_ERR_INVALID_ARG; }
  const int n = (int)(F->rank_X.size() / MLP_IN);
  *count = n;
  for (int i = 0; i < std::min(cap, n); ++i) {
    if (X) std::memcpy(X + (size_t)i * MLP_IN, &F->rank_X[(size_t)i * MLP_IN], sizeof(float) * MLP_IN);
    if (T) std::memcpy(T + (size_t)i * MLP_OUT, &F->rank_T[(size_t)i * MLP_OUT], sizeof(float) * MLP_OUT);
  }
  return PM_OK;
}

pm_status pm_factor_proxy_data(const pm_factor* F, float* ratio, int32_t* redone, int32_t cap, int32_t* count) {
  if (!F || !count || cap < 0 || (cap > 0 && (!ratio || !redone))) {
    g_err = "pm_factor_proxy_data: bad argument";
    return PM_ERR_INVALID_ARG;
  }
  const int n = (int)F->proxy_ratio.size();
  *count = n;
  for (int i = 0; i < n && i < cap; ++i) { ratio[i] = F->proxy_ratio[i]; redone[i] = F->proxy_redone[i]; }
  return PM_OK;
}

pm_status pm_mlp_forward(int32_t dtype, const void* theta, int32_t B, const void* X, void* Y, void* stream) {
  if (!theta || !X || !Y || B < 0 || (dtype != 0 && dtype != 1)) { g_err = "pm_mlp_forward: bad argument"; return PM_ERR_INVALID_ARG; }
  return run_guarded("pm_mlp_forward", [&] {
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == 0) mlp_forward<float>((const float*)theta, B, (const float*)X, (float*)Y, st);
    else mlp_forward<double>((const double*)theta, B, (const double*)X, (double*)Y, st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  });
}

pm_status pm_mlp_loss_grad(int32_t dtype, const void* theta, int32_t B, const void* X, const void* T, double lam,
                           void* grad, void* loss, void* stream) {
  if (!theta || !X || !T || !grad || !loss || B < 1 || (dtype != 0 && dtype != 1)) {
    g_err = "pm_mlp_loss_grad: bad argument";
    return PM_ERR_INVALID_ARG;
  }
  return run_guarded("pm_mlp_loss_grad", [&] {
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == 0) {
      CK(cudaMemsetAsync(grad, 0, sizeof(float) * MLP_NPARAM, st));
      CK(cudaMemsetAsync(loss, 0, sizeof(float), st));
      mlp_loss_grad<float>((const float*)theta, B, (const float*)X, (const float*)T, lam, (float*)grad, (float*)loss, st);
    } else {
      CK(cudaMemsetAsync(grad, 0, sizeof(double) * MLP_NPARAM, st));
      CK(cudaMemsetAsync(loss, 0, sizeof(double), st));
      mlp_loss_grad<double>((const double*)theta, B, (const double*)X, (const double*)T, lam, (double*)grad,
                            (double*)loss, st);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  });
}

pm_status pm_mlp_adam_step(int32_t dtype, void* theta, const void* grad, void* m, void* v, int32_t t, double lr,
                           double b1, double b2, double eps, void* stream) {
  if (!theta || !grad || !m || !v || t < 1 || (dtype != 0 && dtype != 1)) { g_err = "pm_mlp_adam_step: bad argument"; return PM_ERR_INVALID_ARG; }
  return run_guarded("pm_mlp_adam_step", [&] {
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == 0) mlp_adam<float>((float*)theta, (const float*)grad, (float*)m, (float*)v, t, lr, b1, b2, eps, st);
    else mlp_adam<double>((double*)theta, (const double*)grad, (double*)m, (double*)v, t, lr, b1, b2, eps, st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  });
}

pm_status pm_mlp_train(void* theta, int32_t nsamples, const float* X, const float* T, int32_t epochs, int32_t batch,
                       double lr, double lam, uint64_t seed, double* loss_history, void* stream) {
  if (!theta || !X || !T || nsamples < 1 || epochs < 1 || batch < 1) { g_err = "pm_mlp_train: bad argument"; return PM_ERR_INVALID_ARG; }
  return run_guarded("pm_mlp_train", [&] {
    cudaStream_t st = (cudaStream_t)stream;
    Arena ws;
    ws.min_block = 1 << 20;
    float* th = (float*)theta;
    float* g = ws.get<float>(MLP_NPARAM);
    float* mm = ws.get<float>(MLP_NPARAM);
    float* vv = ws.get<float>(MLP_NPARAM);
    float* loss = ws.get<float>(1);
    float* xb = ws.get<float>((size_t)batch * MLP_IN);
    float* tb = ws.get<float>((size_t)batch * MLP_OUT);
    int* idx = ws.get<int>(nsamples);
    CK(cudaMemsetAsync(mm, 0, sizeof(float) * MLP_NPARAM, st));
    CK(cudaMemsetAsync(vv, 0, sizeof(float) * MLP_NPARAM, st));
    std::vector<int> perm(nsamples);
    uint64_t state = seed;
    auto next = [&]() {  // splitmix64
      uint64_t z = (state += 0x9E3779B97F4A7C15ull);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return z ^ (z >> 31);
    };
    int step = 0;
    for (int e = 0; e < epochs; ++e) {
      for (int i = 0; i < nsamples; ++i) perm[i] = i;
      for (int i = nsamples - 1; i > 0; --i) std::swap(perm[i], perm[(int)(next() % (uint64_t)(i + 1))]);
      CK(cudaMemcpyAsync(idx, perm.data(), sizeof(int) * nsamples, cudaMemcpyHostToDevice, st));
      double esum = 0;
      int nb = 0;
      for (int b0 = 0; b0 < nsamples; b0 += batch) {
        const int B = std::min(batch, nsamples - b0);
        mlp_gather_rows<float>(X, idx + b0, B, MLP_IN, xb, st);
        mlp_gather_rows<float>(T, idx + b0, B, MLP_OUT, tb, st);
        CK(cudaMemsetAsync(g, 0, sizeof(float) * MLP_NPARAM, st));
        CK(cudaMemsetAsync(loss, 0, sizeof(float), st));
        mlp_loss_grad<float>(th, B, xb, tb, lam, g, loss, st);
        mlp_adam<float>(th, g, mm, vv, ++step, lr, 0.9, 0.999, 1e-8, st);
        if (loss_history) {
          float hl = 0;
          CK(cudaMemcpyAsync(&hl, loss, sizeof(float), cudaMemcpyDeviceToHost, st));
          CK(cudaStreamSynchronize(st));
          esum += hl;
          ++nb;
        }
      }
      if (loss_history) loss_history[e] = nb ? esum / nb : 0;
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  });
}

pm_status pm_gemm_c32(int32_t m, int32_t n, int32_t k, const void* A, int32_t lda, int32_t conj_a, const void* B,
                      int32_t ldb, int32_t conj_b, void* C, int32_t ldc, const float* alpha, const float* beta,
                      void* stream) {
  if (m < 0 || n < 0 || k < 0 || !alpha || !beta || ((size_t)m * n > 0 && !C) ||
      ((size_t)m * n * k > 0 && (!A || !B)) || ldc < std::max(m, 1) || lda < std::max(conj_a ? k : m, 1) ||
      ldb < std::max(conj_b ? n : k, 1)) {
    g_err = "pm_gemm_c32: bad argument";
    return PM_ERR_INVALID_ARG;
  }
  if (m == 0 || n == 0) return PM_OK;
  return run_guarded("pm_gemm_c32", [&] {
    cudaStream_t st = (cudaStream_t)stream;
    Arena ws;
    TcGemmProb pr{(const float2*)A, lda, conj_a != 0, (const float2*)B, ldb, conj_b != 0, (float2*)C, ldc, m, n, k,
                  make_float2(alpha[0], alpha[1]), make_float2(beta[0], beta[1])};
    std::vector<TcGemmProb> v{pr};
    std::vector<int> off{0, tc_tiles(m, n)};
    auto* dp = upload(ws, v, st);
    int* doff = upload(ws, off, st);
    int* derr = ws.get<int>(1);
    CK(cudaMemsetAsync(derr, 0, sizeof(int), st));
    tc_gemm_batched(dp, doff, 1, off[1], derr, st);
    CK(cudaGetLastError());
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr) fail(PM_ERR_TIMEOUT, "a wait on the tensor cores ran out");
  });
}

pm_status pm_autotune_table(pm_tune_entry* out, int32_t cap, int32_t* count) {
  if (!count || cap < 0 || (cap > 0 && !out)) { g_err = "pm_autotune_table: bad argument"; return PM_ERR_INVALID_ARG; }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  int i = 0;
  for (const auto& kv : g_tune) {
    if (i < cap) {
      pm_tune_entry& e = out[i];
      std::memset(&e, 0, sizeof(e));
      e.device = kv.first.dev; e.complex_bytes = kv.first.bytes;
      e.log2_m = kv.first.lm; e.log2_n = kv.first.ln; e.log2_k = kv.first.lk; e.log2_count = kv.first.lc;
      e.tm = kGemmShapes[kv.second.shape].tm; e.tn = kGemmShapes[kv.second.shape].tn;
      for (int sh = 0; sh < GEMM_NSHAPES && sh < 8; ++sh) e.ms[sh] = kv.second.ms[sh];
      e.uses = kv.second.uses;
    }
    ++i;
  }
  *count = i;
  return PM_OK;
}

pm_status pm_launch_counter(uint64_t* out) {
  if (!out) { g_err = "pm_launch_counter: NULL argument"; return PM_ERR_INVALID_ARG; }
  *out = g_launches.load();
  return PM_OK;
}

void pm_factor_free(pm_factor* F) { delete F; }
void pm_geometry_free(pm_geometry* g) { delete g; }

}  // extern "C"

// ---------------------------------------------------------------------------------
// Allocation-free variant of pm_self_block.
//
// Some callers cannot let this library call cudaMalloc / cudaFree: those
// calls may synchronise the whole device (stalling work the caller has in
// flight on other streams), and a host application that runs under a fixed
// device-memory budget or its own memory manager may forbid allocations by
// libraries altogether.  pm_self_block_noalloc writes the self block into a
// caller-provided device buffer and keeps all of its scratch (the Maue
// factors and the launch descriptors) in the file-scope device array below.
namespace {

constexpr int NOALLOC_MAX_N = 256;                       // largest n_j accepted
constexpr size_t NOALLOC_DESC_BYTES = 64 * 1024;         // launch descriptors
constexpr size_t NOALLOC_MAT_BYTES = (size_t)NOALLOC_MAX_N * NOALLOC_MAX_N * sizeof(Cd);
constexpr size_t NOALLOC_BYTES = NOALLOC_DESC_BYTES + 4 * NOALLOC_MAT_BYTES;   // 4 MiB + 64 KiB

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mu;
char* g_noalloc_ptr[64] = {nullptr};

// Device address of the scratch array for the current device.  The host-side
// symbol is only a stand-in, so the address is looked up once per device with
// that device current (the first call on a device does this set-up).
char* noalloc_scratch() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) fail(PM_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = (char*)p;
  }
  return g_noalloc_ptr[dev];
}

}  // namespace

extern "C" pm_status pm_self_block_noalloc(const pm_geometry* g, int32_t j, pm_c64* out) {
  if (!g || !out || j < 0 || j >= g->m) { g_err = "pm_self_block_noalloc: bad argument"; return PM_ERR_INVALID_ARG; }
  const int n = g->inc[j].n_nodes;
  if (n > NOALLOC_MAX_N) {
    g_err = "pm_self_block_noalloc: n_j = " + std::to_string(n) + " exceeds the scratch limit of " +
            std::to_string(NOALLOC_MAX_N) + " nodes";
    return PM_ERR_INVALID_ARG;
  }
  return run_guarded("pm_self_block_noalloc", [&] {
    cudaStream_t st = 0;
    require_current_device(g->device, "pm_self_block_noalloc");
    require_device_ptr(out, g->device, "out");
    char* base = noalloc_scratch();
    Cd* A = (Cd*)out;
    const int lda = 2 * n;
    Cd* Cm = (Cd*)(base + NOALLOC_DESC_BYTES);
    Cd* DtS = (Cd*)(base + NOALLOC_DESC_BYTES + NOALLOC_MAT_BYTES);
    Cd* E = (Cd*)(base + NOALLOC_DESC_BYTES + 2 * NOALLOC_MAT_BYTES);
    Cd* Dt = (Cd*)(base + NOALLOC_DESC_BYTES + 3 * NOALLOC_MAT_BYTES);
    // descriptor area: fixed slots, every slot fully rewritten by each call
    struct Desc {
      GemmDesc<Cd> d1, d2;
      int off1[2], off2[2];
      Cd* Aptr[1];
      int ldA[1];
      Cd* Cptr[1];
      Cd* Dptr[1];
    } h;
    static_assert(sizeof(Desc) <= NOALLOC_DESC_BYTES, "descriptor area too small");
    h.d1 = GemmDesc<Cd>{n, n, n, Cm, n, Dt, n, E, n, make_double2(1, 0), make_double2(0, 0), 1};
    h.d2 = GemmDesc<Cd>{n, n, n, DtS, n, E, n, A + n + (size_t)n * lda, lda, make_double2(1, 0),
                        make_double2(1, 0), 0};
    h.off1[0] = 0; h.off1[1] = gemm_tiles(n, n);
    h.off2[0] = 0; h.off2[1] = gemm_tiles(n, n);
    h.Aptr[0] = A; h.ldA[0] = lda; h.Cptr[0] = Cm; h.Dptr[0] = DtS;
    Desc* d = (Desc*)base;
    CK(cudaMemcpyAsync(d, &h, sizeof(Desc), cudaMemcpyHostToDevice, st));
    const InclDev* dinc = g->d_inc + j;
    diff_matrices<Cd>(n, Dt, st);
    self_pointwise<Cd>(dinc, 1, n, g->nodes, g->k0, d->Aptr, d->ldA, d->Cptr, st);
    scaled_diff<Cd>(dinc, 1, n, g->nodes, d->Dptr, st);
    la_gemm_batched<Cd>(&d->d1, d->off1, 1, h.off1[1], st);
    la_gemm_batched<Cd>(&d->d2, d->off2, 1, h.off2[1], st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  });
}
