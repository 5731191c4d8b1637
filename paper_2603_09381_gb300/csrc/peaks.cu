// Peak FP64 and FP32 fused multiply-add rates of the current device,
// measured by a loop of independent FMA chains (the denominators of the
// roofline fractions that bench.py reports for the FP64- and FP32-bound
// kernels of the solver).
//
// Each thread runs CHAINS independent accumulator chains so that the FMA
// pipes never wait on a previous result; the grid covers every SM several
// times over.  The result is stored only when it equals a value it never
// reaches, so the compiler must keep every FMA while no memory traffic
// enters the timed loop.
#include <cuda_runtime.h>
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/pmchwt.h"
#include "prof.cuh"

namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;

template <typename R>
__global__ void __launch_bounds__(THREADS) k_fma_loop(int iters, const R* __restrict__ ab, R* sink,
                                                      long long* cycles) {
  const long long c0 = clock64();
  // multiplier and addend in registers (read from memory, not kernel
  // parameters), so every FMA has register operands only
  const R a = ab[0], b = ab[1];
  R x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = (R)(threadIdx.x + c) * (R)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
  }
  R s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  if (s == (R)-12345.0) *sink = s;   // never true for a in (0, 1), b > 0 (sink[0] is not an operand)
  __syncthreads();
  if (threadIdx.x == 0) cycles[blockIdx.x] = clock64() - c0;
}

// Returns TFLOP/s; *mhz receives the SM clock the loop ran at (cycles counted
// by the CTAs over the event time of the launch).
template <typename R>
double run(double ms_target, double* mhz) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8;
  R* sink = nullptr;
  long long* cyc = nullptr;
  if (cudaMalloc(&sink, 3 * sizeof(R)) != cudaSuccess) return -1;
  if (cudaMalloc(&cyc, sizeof(long long) * blocks) != cudaSuccess) { cudaFree(sink); return -1; }
  const R hab[2] = {(R)0.999999, (R)1e-7};
  cudaMemcpy(sink + 1, hab, 2 * sizeof(R), cudaMemcpyHostToDevice);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // calibrate the iteration count on a short run, then time one long launch
  int iters = 256;
  float ms = 0;
  for (int rep = 0; rep < 8; ++rep) {
    cudaEventRecord(e0);
    k_fma_loop<R><<<blocks, THREADS>>>(iters, sink + 1, sink, cyc);
    pm_launch_count_add(1);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms >= 0.5 * ms_target || iters >= (1 << 24)) break;
    iters = (int)std::min<double>(1 << 24, iters * std::max(2.0, 0.9 * ms_target / std::max(ms, 1e-3f)));
  }
  cudaEventRecord(e0);
  k_fma_loop<R><<<blocks, THREADS>>>(iters, sink + 1, sink, cyc);
  pm_launch_count_add(1);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  std::vector<long long> hc(blocks);
  cudaMemcpy(hc.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(cyc);
  if (err != cudaSuccess || ms <= 0) return -1;
  // the longest-running CTAs span the launch: their cycle count over its time is the clock
  long long mx = 0;
  for (long long c : hc) mx = std::max(mx, c);
  *mhz = (double)mx / (ms * 1e3);
  const double fmas = (double)blocks * THREADS * CHAINS * 16.0 * iters;
  return 2.0 * fmas / (ms * 1e-3) / 1e12;
}

}  // namespace

extern "C" pm_status pm_measure_peak(int32_t which, double ms_target, double* tflops, double* sm_mhz) {
  if (!tflops || (which != 0 && which != 1) || !(ms_target > 0 && ms_target <= 10000)) return PM_ERR_INVALID_ARG;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    return PM_ERR_CUDA;
  }
  double mhz = 0;
  const double r = which == 0 ? run<double>(ms_target, &mhz) : run<float>(ms_target, &mhz);
  if (!(r > 0)) return PM_ERR_CUDA;
  *tflops = r;
  if (sm_mhz) *sm_mhz = mhz;
  return PM_OK;
}
