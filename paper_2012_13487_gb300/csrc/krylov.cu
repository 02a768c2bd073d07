// Device vector kernels of the implicit solver (see krylov.h).
#include "krylov.h"

namespace fedbm {
namespace krylov {
namespace {

int grid_of(int64_t n) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  return int(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

__global__ void axpby_kernel(int64_t n, double a, const double* x, double b, const double* y, double* out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = a * x[i] + b * y[i];
}

__global__ void combination_kernel(int64_t n, int m, const double* V, const double* c, double* y, double sign) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < m; ++j) acc += c[j] * V[size_t(j) * n + i];
    y[i] += sign * acc;
  }
}

// partial[j][block] = sum over this block's grid-stride share of V_j[i] w[i]
__global__ void dot_partial_kernel(int64_t n, const double* V, const double* w, double* partial) {
  __shared__ double red[kThreads / 32];
  const int j = blockIdx.y;
  const double* v = V + size_t(j) * n;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * int64_t(kThreads) + threadIdx.x; i < n; i += int64_t(kDotBlocks) * kThreads)
    acc += v[i] * w[i];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    partial[size_t(j) * kDotBlocks + blockIdx.x] = t;
  }
}

// h[j] = sum of partial[j][*], one block per j
__global__ void dot_final_kernel(const double* partial, double* h) {
  __shared__ double red[kThreads / 32];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int q = threadIdx.x; q < kDotBlocks; q += kThreads) acc += partial[size_t(j) * kDotBlocks + q];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    h[j] = t;
  }
}

__global__ void to_f32_kernel(int64_t n, const double* x, float* y) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = float(x[i]);
}
__global__ void to_f64_kernel(int64_t n, const float* x, double* y) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = double(x[i]);
}

template <typename R>
__global__ void set_geo_dt_kernel(int64_t K, int stride, int slot, double value, R* geo) {
  for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < K; k += int64_t(gridDim.x) * blockDim.x)
    geo[k * stride + slot] = R(value);
}

}  // namespace

cudaError_t axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t st) {
  axpby_kernel<<<grid_of(n), kThreads, 0, st>>>(n, a, x, b, y, out);
  return cudaGetLastError();
}

cudaError_t sub_combination(int64_t n, int m, const double* V, const double* c_dev, double* y, cudaStream_t st) {
  if (m < 1) return cudaSuccess;
  combination_kernel<<<grid_of(n), kThreads, 0, st>>>(n, m, V, c_dev, y, -1.0);
  return cudaGetLastError();
}

cudaError_t add_combination(int64_t n, int m, const double* V, const double* c_dev, double* out, cudaStream_t st) {
  if (m < 1) return cudaSuccess;
  combination_kernel<<<grid_of(n), kThreads, 0, st>>>(n, m, V, c_dev, out, 1.0);
  return cudaGetLastError();
}

cudaError_t multi_dot(int64_t n, int m, const double* V, const double* w, double* partial, double* h, cudaStream_t st) {
  if (m < 1) return cudaSuccess;
  dot_partial_kernel<<<dim3(kDotBlocks, m), kThreads, 0, st>>>(n, V, w, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dot_final_kernel<<<m, kThreads, 0, st>>>(partial, h);
  return cudaGetLastError();
}

cudaError_t to_f32(int64_t n, const double* x, float* y, cudaStream_t st) {
  to_f32_kernel<<<grid_of(n), kThreads, 0, st>>>(n, x, y);
  return cudaGetLastError();
}

cudaError_t to_f64(int64_t n, const float* x, double* y, cudaStream_t st) {
  to_f64_kernel<<<grid_of(n), kThreads, 0, st>>>(n, x, y);
  return cudaGetLastError();
}

cudaError_t set_geo_dt(int64_t K, int stride, int slot, double value, void* geo, int real_bytes, cudaStream_t st) {
  const int grid = grid_of(K);
  if (real_bytes == 8) set_geo_dt_kernel<double><<<grid, kThreads, 0, st>>>(K, stride, slot, value, static_cast<double*>(geo));
  else set_geo_dt_kernel<float><<<grid, kThreads, 0, st>>>(K, stride, slot, value, static_cast<float*>(geo));
  return cudaGetLastError();
}

}  // namespace krylov
}  // namespace fedbm
