// Small MLP (8 -> 64 -> 64 -> 2, tanh) that predicts interpolative-decomposition
// ranks, with hand-written forward, backward and Adam kernels.
#pragma once
#include <cuda_runtime.h>

constexpr int MLP_IN = 8, MLP_H = 64, MLP_OUT = 2;
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT;   // 4866

template <typename T>
void mlp_forward(const T* theta, int B, const T* X, T* Y, cudaStream_t st);
// loss (1 value, accumulated) and gradient (MLP_NPARAM, accumulated): callers zero them
template <typename T>
void mlp_loss_grad(const T* theta, int B, const T* X, const T* Tg, double lam, T* grad, T* loss, cudaStream_t st);
template <typename T>
void mlp_adam(T* theta, const T* grad, T* m, T* v, int t, double lr, double b1, double b2, double eps, cudaStream_t st);
template <typename T>
void mlp_gather_rows(const T* src, const int* idx, int B, int width, T* dst, cudaStream_t st);
