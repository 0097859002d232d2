// Element-wise kernels of the reconstruction solvers built on the products
// with U and U^*: the fused FISTA proximal step with momentum and its
// vector-Jacobian product, and FP64-accumulated inner products (the only
// FP64 arithmetic of the solver loop on the GPU).  FISTA (Beck-Teboulle) for
// min 1/2 ||P_Omega U x - y||^2 + lam ||x||_1, the l1-regularised recovery
// problem of the paper's compressive-sensing setting (Sec. 1.2, Remark 4.2).
#include <cuda_runtime.h>

#include <cstdint>

#include "uw_internal.h"

namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

// sum of a double over the block, added to *out by one atomic per block
__device__ __forceinline__ void block_add(double v, double* out) {
  __shared__ double part[kThreads / 32];
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) part[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) atomicAdd(out, v);
  }
}

// v = z - tau (G - B); x1 = soft(v, tau lam); z1 = x1 + beta (x1 - x0)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fista_step(int64_t n, const T* __restrict__ z, const T* __restrict__ G,
                                                         const T* __restrict__ B, const T* __restrict__ x0, T tau,
                                                         T lam, T beta, T* __restrict__ x1, T* __restrict__ z1) {
  const T thr = tau * lam;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T v = z[i] - tau * (G[i] - B[i]);
    const T x = v > thr ? v - thr : (v < -thr ? v + thr : T(0));
    x1[i] = x;
    z1[i] = x + beta * (x - x0[i]);
  }
}

// vector-Jacobian product of k_fista_step: w = gx1 + (1 + beta) gz1 reaches
// v through the active set |v| > tau lam; d x1 / d lam = -tau sign(v) there
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fista_step_bwd(int64_t n, const T* __restrict__ z,
                                                             const T* __restrict__ G, const T* __restrict__ B, T tau,
                                                             T lam, T beta, const T* __restrict__ gx1,
                                                             const T* __restrict__ gz1, T* __restrict__ gz,
                                                             T* __restrict__ gG, T* __restrict__ gB,
                                                             T* __restrict__ gx0, double* glam) {
  const T thr = tau * lam;
  double dl = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T gzi = gz1 ? gz1[i] : T(0);
    const T w = (gx1 ? gx1[i] : T(0)) + (T(1) + beta) * gzi;
    const T v = z[i] - tau * (G[i] - B[i]);
    const bool act = v > thr || v < -thr;
    const T gv = act ? w : T(0);
    gz[i] = gv;
    gG[i] = -tau * gv;
    gB[i] = tau * gv;
    if (gx0) gx0[i] = -beta * gzi;
    if (act) dl -= (double)tau * (double)(v > T(0) ? w : -w);
  }
  block_add(dl, glam);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_dot(int64_t n, const T* __restrict__ a, const T* __restrict__ b,
                                                  double* out) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)a[i] * (double)b[i];
  block_add(s, out);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_axpby(int64_t n, T alpha, const T* __restrict__ a, T beta,
                                                    const T* __restrict__ b, T* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = alpha * a[i] + (b ? beta * b[i] : T(0));
}

int check_prec(int prec, int64_t n) {
  if (prec != UW_F64 && prec != UW_F32) {
    uw::set_error(UW_ERR_INVALID_ARG, "solver kernels take UW_F64 or UW_F32 data");
    return UW_ERR_INVALID_ARG;
  }
  if (n < 0) {
    uw::set_error(UW_ERR_INVALID_ARG, "negative length");
    return UW_ERR_INVALID_ARG;
  }
  return UW_OK;
}

int finish(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    uw::set_error(UW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return UW_ERR_CUDA;
  }
  return UW_OK;
}

}  // namespace

extern "C" {

int uw_fista_step(int prec, int64_t n, const void* z, const void* G, const void* B, const void* x0, double tau,
                  double lam, double beta, void* x1, void* z1, void* stream) {
  int st = check_prec(prec, n);
  if (st != UW_OK) return st;
  if (n == 0) return UW_OK;
  if (!z || !G || !B || !x0 || !x1 || !z1) {
    uw::set_error(UW_ERR_INVALID_ARG, "null buffer");
    return UW_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == UW_F64)
    k_fista_step<double><<<blocks_for(n), kThreads, 0, s>>>(n, (const double*)z, (const double*)G, (const double*)B,
                                                            (const double*)x0, tau, lam, beta, (double*)x1,
                                                            (double*)z1);
  else
    k_fista_step<float><<<blocks_for(n), kThreads, 0, s>>>(n, (const float*)z, (const float*)G, (const float*)B,
                                                           (const float*)x0, (float)tau, (float)lam, (float)beta,
                                                           (float*)x1, (float*)z1);
  return finish("uw_fista_step");
}

int uw_fista_step_backward(int prec, int64_t n, const void* z, const void* G, const void* B, double tau, double lam,
                           double beta, const void* gx1, const void* gz1, void* gz, void* gG, void* gB, void* gx0,
                           double* glam, void* stream) {
  int st = check_prec(prec, n);
  if (st != UW_OK) return st;
  if (n == 0) return UW_OK;
  if (!z || !G || !B || !gz || !gG || !gB || !glam) {
    uw::set_error(UW_ERR_INVALID_ARG, "null buffer");
    return UW_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == UW_F64)
    k_fista_step_bwd<double><<<blocks_for(n), kThreads, 0, s>>>(
        n, (const double*)z, (const double*)G, (const double*)B, tau, lam, beta, (const double*)gx1,
        (const double*)gz1, (double*)gz, (double*)gG, (double*)gB, (double*)gx0, glam);
  else
    k_fista_step_bwd<float><<<blocks_for(n), kThreads, 0, s>>>(
        n, (const float*)z, (const float*)G, (const float*)B, (float)tau, (float)lam, (float)beta, (const float*)gx1,
        (const float*)gz1, (float*)gz, (float*)gG, (float*)gB, (float*)gx0, glam);
  return finish("uw_fista_step_backward");
}

int uw_dot(int prec, int64_t n, const void* a, const void* b, double* out, void* stream) {
  int st = check_prec(prec, n);
  if (st != UW_OK) return st;
  if (!out || (n > 0 && (!a || !b))) {
    uw::set_error(UW_ERR_INVALID_ARG, "null buffer");
    return UW_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(out, 0, sizeof(double), s) != cudaSuccess) return finish("uw_dot");
  if (n == 0) return UW_OK;
  if (prec == UW_F64) k_dot<double><<<blocks_for(n), kThreads, 0, s>>>(n, (const double*)a, (const double*)b, out);
  else k_dot<float><<<blocks_for(n), kThreads, 0, s>>>(n, (const float*)a, (const float*)b, out);
  return finish("uw_dot");
}

int uw_axpby(int prec, int64_t n, double alpha, const void* a, double beta, const void* b, void* out, void* stream) {
  int st = check_prec(prec, n);
  if (st != UW_OK) return st;
  if (n == 0) return UW_OK;
  if (!a || !out) {
    uw::set_error(UW_ERR_INVALID_ARG, "null buffer");
    return UW_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == UW_F64)
    k_axpby<double><<<blocks_for(n), kThreads, 0, s>>>(n, alpha, (const double*)a, beta, (const double*)b,
                                                       (double*)out);
  else
    k_axpby<float><<<blocks_for(n), kThreads, 0, s>>>(n, (float)alpha, (const float*)a, (float)beta,
                                                      (const float*)b, (float*)out);
  return finish("uw_axpby");
}

}  // extern "C"
