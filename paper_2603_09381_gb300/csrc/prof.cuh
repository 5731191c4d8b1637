// Optional per-kernel timing with CUDA events on the launching stream.
// Enabled per factorization (PM_FLAG_PROFILE); records one event pair per
// launch (or launch group) and the algorithmic flop count of that launch.
#pragma once
#include <cuda_runtime.h>
#include <map>
#include <string>
#include <vector>

struct KProf {
  struct Rec { cudaEvent_t a, b; std::string name; double flops; };
  struct Agg { long launches = 0; double ms = 0, flops = 0; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, Agg> agg;
  cudaEvent_t cur_a = nullptr;
  cudaEvent_t ev() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void begin(cudaStream_t st) { cur_a = ev(); cudaEventRecord(cur_a, st); }
  void end(cudaStream_t st, const char* name, double flops) {
    cudaEvent_t b = ev();
    cudaEventRecord(b, st);
    recs.push_back(Rec{cur_a, b, name, flops});
  }
  void add_flops(const char* name, double flops) { agg[name].flops += flops; }
  void collect() {
    for (auto& r : recs) {
      cudaEventSynchronize(r.b);
      float ms = 0;
      cudaEventElapsedTime(&ms, r.a, r.b);
      Agg& g = agg[r.name];
      g.launches += 1; g.ms += ms; g.flops += r.flops;
      pool.push_back(r.a); pool.push_back(r.b);
    }
    recs.clear();
  }
  ~KProf() {
    for (auto& r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// Profiler name of a kernel by arithmetic: FP32 variants carry a "32" suffix.
template <typename C> inline const char* kname(const char* base64, const char* base32);
template <> inline const char* kname<double2>(const char* b64, const char*) { return b64; }
template <> inline const char* kname<float2>(const char*, const char* b32) { return b32; }

// Process-wide count of kernel launches made by this library.
void pm_launch_count_add(long n);

// Set by the runtime around a profiled factorization (host thread-local).
extern thread_local KProf* g_kprof;

#define KPROF_BEGIN(st) do { if (g_kprof) g_kprof->begin(st); } while (0)
#define KPROF_END(st, name, flops) do { if (g_kprof) g_kprof->end(st, name, flops); } while (0)
