// MLP kernels for the learned rank predictor.  Parameters are one flat array
// (row-major W1 64x8, b1, W2 64x64, b2, W3 2x64, b3).  One thread per sample;
// weights are staged in shared memory; the backward pass accumulates the
// gradient of a CTA's samples in shared memory before one global add per
// parameter and CTA.
//   loss = (1/B) sum (1 + lam [y < t]) (y - t)^2
#include "mlp.cuh"
#include "prof.cuh"
#include <cmath>

namespace {

constexpr int O_W1 = 0, O_B1 = O_W1 + MLP_H * MLP_IN, O_W2 = O_B1 + MLP_H, O_B2 = O_W2 + MLP_H * MLP_H,
              O_W3 = O_B2 + MLP_H, O_B3 = O_W3 + MLP_OUT * MLP_H;
constexpr int MLP_T = 64;   // samples per CTA

template <typename T> __device__ __forceinline__ T tanh_t(T x);
template <> __device__ __forceinline__ float tanh_t<float>(float x) { return tanhf(x); }
template <> __device__ __forceinline__ double tanh_t<double>(double x) { return tanh(x); }

template <typename T>
__device__ __forceinline__ void forward_one(const T* w, const T* x, T* h1, T* h2, T* y) {
  for (int j = 0; j < MLP_H; ++j) {
    T a = w[O_B1 + j];
    for (int i = 0; i < MLP_IN; ++i) a += w[O_W1 + j * MLP_IN + i] * x[i];
    h1[j] = tanh_t(a);
  }
  for (int j = 0; j < MLP_H; ++j) {
    T a = w[O_B2 + j];
    for (int i = 0; i < MLP_H; ++i) a += w[O_W2 + j * MLP_H + i] * h1[i];
    h2[j] = tanh_t(a);
  }
  for (int o = 0; o < MLP_OUT; ++o) {
    T a = w[O_B3 + o];
    for (int i = 0; i < MLP_H; ++i) a += w[O_W3 + o * MLP_H + i] * h2[i];
    y[o] = a;
  }
}

template <typename T>
__global__ void __launch_bounds__(MLP_T) k_forward(const T* __restrict__ theta, int B, const T* __restrict__ X,
                                                  T* __restrict__ Y) {
  extern __shared__ unsigned char smem_raw[];
  T* w = (T*)smem_raw;
  for (int p = threadIdx.x; p < MLP_NPARAM; p += blockDim.x) w[p] = theta[p];
  __syncthreads();
  const int s = blockIdx.x * MLP_T + threadIdx.x;
  if (s >= B) return;
  T x[MLP_IN], h1[MLP_H], h2[MLP_H], y[MLP_OUT];
  for (int i = 0; i < MLP_IN; ++i) x[i] = X[s * MLP_IN + i];
  forward_one(w, x, h1, h2, y);
  for (int o = 0; o < MLP_OUT; ++o) Y[s * MLP_OUT + o] = y[o];
}

template <typename T>
__global__ void __launch_bounds__(MLP_T) k_loss_grad(const T* __restrict__ theta, int B, const T* __restrict__ X,
                                                    const T* __restrict__ Tg, T lam, T* __restrict__ grad,
                                                    T* __restrict__ loss) {
  extern __shared__ unsigned char smem_raw[];
  T* w = (T*)smem_raw;
  T* g = w + MLP_NPARAM;
  __shared__ T sloss;
  for (int p = threadIdx.x; p < MLP_NPARAM; p += blockDim.x) { w[p] = theta[p]; g[p] = 0; }
  if (threadIdx.x == 0) sloss = 0;
  __syncthreads();
  const int s = blockIdx.x * MLP_T + threadIdx.x;
  if (s < B) {
    T x[MLP_IN], h1[MLP_H], h2[MLP_H], y[MLP_OUT], dy[MLP_OUT];
    for (int i = 0; i < MLP_IN; ++i) x[i] = X[s * MLP_IN + i];
    forward_one(w, x, h1, h2, y);
    T l = 0;
    for (int o = 0; o < MLP_OUT; ++o) {
      const T t = Tg[s * MLP_OUT + o];
      const T wt = (T)1 + (y[o] < t ? lam : (T)0);
      l += wt * (y[o] - t) * (y[o] - t);
      dy[o] = (T)2 * wt * (y[o] - t) / (T)B;
    }
    atomicAdd(&sloss, l / (T)B);
    // output layer
    for (int o = 0; o < MLP_OUT; ++o) {
      atomicAdd(&g[O_B3 + o], dy[o]);
      for (int i = 0; i < MLP_H; ++i) atomicAdd(&g[O_W3 + o * MLP_H + i], dy[o] * h2[i]);
    }
    // second hidden layer: dz2 = (W3^T dy) (1 - h2^2); reuse h2 for dz2
    for (int i = 0; i < MLP_H; ++i) {
      T a = 0;
      for (int o = 0; o < MLP_OUT; ++o) a += w[O_W3 + o * MLP_H + i] * dy[o];
      h2[i] = a * ((T)1 - h2[i] * h2[i]);
    }
    for (int j = 0; j < MLP_H; ++j) {
      atomicAdd(&g[O_B2 + j], h2[j]);
      for (int i = 0; i < MLP_H; ++i) atomicAdd(&g[O_W2 + j * MLP_H + i], h2[j] * h1[i]);
    }
    // first hidden layer: dz1 = (W2^T dz2) (1 - h1^2)
    T dz1[MLP_H];
    for (int i = 0; i < MLP_H; ++i) {
      T a = 0;
      for (int j = 0; j < MLP_H; ++j) a += w[O_W2 + j * MLP_H + i] * h2[j];
      dz1[i] = a * ((T)1 - h1[i] * h1[i]);
    }
    for (int j = 0; j < MLP_H; ++j) {
      atomicAdd(&g[O_B1 + j], dz1[j]);
      for (int i = 0; i < MLP_IN; ++i) atomicAdd(&g[O_W1 + j * MLP_IN + i], dz1[j] * x[i]);
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < MLP_NPARAM; p += blockDim.x) atomicAdd(&grad[p], g[p]);
  if (threadIdx.x == 0) atomicAdd(loss, sloss);
}

template <typename T>
__global__ void k_adam(T* __restrict__ theta, const T* __restrict__ grad, T* __restrict__ m, T* __restrict__ v,
                       T c1, T c2, T lr, T b1, T b2, T eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NPARAM) return;
  const T gp = grad[p];
  const T mp = b1 * m[p] + ((T)1 - b1) * gp;
  const T vp = b2 * v[p] + ((T)1 - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  theta[p] -= lr * (mp / c1) / (sqrt(vp / c2) + eps);
}

template <typename T>
__global__ void k_gather_rows(const T* __restrict__ src, const int* __restrict__ idx, int B, int width, T* __restrict__ dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * width) return;
  const int r = e / width, c = e % width;
  dst[e] = src[(size_t)idx[r] * width + c];
}

}  // namespace

template <typename T>
void mlp_forward(const T* theta, int B, const T* X, T* Y, cudaStream_t st) {
  if (B <= 0) return;
  const size_t sm = sizeof(T) * MLP_NPARAM;
  cudaFuncSetAttribute(k_forward<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_forward<T><<<(B + MLP_T - 1) / MLP_T, MLP_T, sm, st>>>(theta, B, X, Y);
  pm_launch_count_add(1);
}

template <typename T>
void mlp_loss_grad(const T* theta, int B, const T* X, const T* Tg, double lam, T* grad, T* loss, cudaStream_t st) {
  if (B <= 0) return;
  const size_t sm = 2 * sizeof(T) * MLP_NPARAM;
  cudaFuncSetAttribute(k_loss_grad<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_loss_grad<T><<<(B + MLP_T - 1) / MLP_T, MLP_T, sm, st>>>(theta, B, X, Tg, (T)lam, grad, loss);
  pm_launch_count_add(1);
}

template <typename T>
void mlp_adam(T* theta, const T* grad, T* m, T* v, int t, double lr, double b1, double b2, double eps, cudaStream_t st) {
  const double c1 = 1.0 - std::pow(b1, t), c2 = 1.0 - std::pow(b2, t);
  k_adam<T><<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(theta, grad, m, v, (T)c1, (T)c2, (T)lr, (T)b1, (T)b2, (T)eps);
  pm_launch_count_add(1);
}

template <typename T>
void mlp_gather_rows(const T* src, const int* idx, int B, int width, T* dst, cudaStream_t st) {
  if (B <= 0) return;
  k_gather_rows<T><<<(B * width + 255) / 256, 256, 0, st>>>(src, idx, B, width, dst);
  pm_launch_count_add(1);
}

template void mlp_forward<float>(const float*, int, const float*, float*, cudaStream_t);
template void mlp_forward<double>(const double*, int, const double*, double*, cudaStream_t);
template void mlp_loss_grad<float>(const float*, int, const float*, const float*, double, float*, float*, cudaStream_t);
template void mlp_loss_grad<double>(const double*, int, const double*, const double*, double, double*, double*, cudaStream_t);
template void mlp_adam<float>(float*, const float*, float*, float*, int, double, double, double, double, cudaStream_t);
template void mlp_adam<double>(double*, const double*, double*, double*, int, double, double, double, double, cudaStream_t);
template void mlp_gather_rows<float>(const float*, const int*, int, int, float*, cudaStream_t);
template void mlp_gather_rows<double>(const double*, const int*, int, int, double*, cudaStream_t);
