// Device vector kernels of the implicit solver (see krylov.h).
#include "krylov.h"

#include <type_traits>

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

// ---- element-and-velocity block-Jacobi preconditioner --------------------------
// For element k and velocity i the block of (I - dtg J) that couples the
// element's own nodes at velocity i is
//   M = (1 + dtg / tau_k) I + dtg (a_r Dr + a_s Ds) - dtg LIFT diag(c) E,
// where a_r = e_x r_x + e_y r_y, a_s = e_x s_x + e_y s_y, E picks the face
// nodes out of the element's nodes, and c = Fscale (e.n - ab |e.n|) / 2 is the
// numerical flux's coefficient of the element's own trace on each face (the
// strong-form residual of eq. byparts).  Neighbour traces, wall reflection and
// the equilibrium's dependence on the other velocities are left out.  M is
// inverted by Gauss-Jordan elimination with partial pivoting, one thread per
// (element, velocity).
namespace fedbm {
namespace krylov {
namespace {

constexpr int kMaxNp = 28;  // degree 6

template <typename R, int NPT>
__global__ void bj_build_kernel(int64_t K, int Np, int Nfp, int Qp, const R* geo, const double* vel64,
                                const double* ops, const int* fmask, double dtg, double ab, double* minv) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= K * Qp) return;
  const int64_t k = t / Qp;
  const int i = int(t % Qp);
  const R* g = geo + k * 16;
  const double ex = vel64[i], ey = vel64[Qp + i];
  const double ar = ex * double(g[0]) + ey * double(g[2]);
  const double as = ex * double(g[1]) + ey * double(g[3]);
  const double itau = double(g[15]);
  const double* Dr = ops;
  const double* Ds = ops + Np * Np;
  const double* LIFT = ops + 2 * Np * Np;
  const int NF = 3 * Nfp;
  double A[NPT * NPT], B[NPT * NPT];  // Np <= NPT
  for (int n = 0; n < Np; ++n)
    for (int m = 0; m < Np; ++m) {
      A[n * Np + m] = (n == m ? 1.0 + dtg * itau : 0.0) + dtg * (ar * Dr[n * Np + m] + as * Ds[n * Np + m]);
      B[n * Np + m] = n == m ? 1.0 : 0.0;
    }
  for (int f = 0; f < 3; ++f) {
    const double en = ex * double(g[4 + 3 * f]) + ey * double(g[5 + 3 * f]);
    const double c = 0.5 * (en - ab * fabs(en)) * double(g[6 + 3 * f]);
    if (c == 0.0) continue;
    for (int a = 0; a < Nfp; ++a) {
      const int j = f * Nfp + a, m = fmask[j];
      for (int n = 0; n < Np; ++n) A[n * Np + m] -= dtg * LIFT[n * NF + j] * c;
    }
  }
  // Gauss-Jordan with partial pivoting: B <- A^-1
  for (int col = 0; col < Np; ++col) {
    int piv = col;
    for (int r = col + 1; r < Np; ++r)
      if (fabs(A[r * Np + col]) > fabs(A[piv * Np + col])) piv = r;
    if (piv != col)
      for (int q = 0; q < Np; ++q) {
        double x = A[col * Np + q]; A[col * Np + q] = A[piv * Np + q]; A[piv * Np + q] = x;
        x = B[col * Np + q]; B[col * Np + q] = B[piv * Np + q]; B[piv * Np + q] = x;
      }
    const double d = 1.0 / A[col * Np + col];
    for (int q = 0; q < Np; ++q) {
      A[col * Np + q] *= d;
      B[col * Np + q] *= d;
    }
    for (int r = 0; r < Np; ++r) {
      if (r == col) continue;
      const double fct = A[r * Np + col];
      if (fct == 0.0) continue;
      for (int q = 0; q < Np; ++q) {
        A[r * Np + q] -= fct * A[col * Np + q];
        B[r * Np + q] -= fct * B[col * Np + q];
      }
    }
  }
  for (int n = 0; n < Np; ++n)
    for (int m = 0; m < Np; ++m) minv[((k * Np + n) * Np + m) * Qp + i] = B[n * Np + m];
}

__global__ void bj_apply_kernel(int64_t K, int Np, int Qp, const double* minv, const double* v, double* z) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= K * Qp) return;
  const int64_t k = t / Qp;
  const int i = int(t % Qp);
  double x[kMaxNp];
  for (int m = 0; m < Np; ++m) x[m] = v[(k * Np + m) * Qp + i];
  for (int n = 0; n < Np; ++n) {
    double acc = 0.0;
    for (int m = 0; m < Np; ++m) acc += minv[((k * Np + n) * Np + m) * Qp + i] * x[m];
    z[(k * Np + n) * Qp + i] = acc;
  }
}

}  // namespace

cudaError_t block_jacobi_build(int64_t K, int Np, int Nfp, int Qp, const void* geo, int real_bytes,
                               const double* vel64, const double* ops, const int* fmask, double dtg, double ab,
                               double* minv, cudaStream_t st) {
  if (Np > kMaxNp) return cudaErrorInvalidValue;
  const int64_t n = K * Qp;
  const int blocks = int((n + 127) / 128);
  // the block size rounded up to a degree's node count keeps the per-thread
  // work arrays (local memory) small at low degree
  auto run = [&](auto npt) {
    constexpr int NPT = decltype(npt)::value;
    if (real_bytes == 8)
      bj_build_kernel<double, NPT><<<blocks, 128, 0, st>>>(K, Np, Nfp, Qp, static_cast<const double*>(geo), vel64,
                                                           ops, fmask, dtg, ab, minv);
    else
      bj_build_kernel<float, NPT><<<blocks, 128, 0, st>>>(K, Np, Nfp, Qp, static_cast<const float*>(geo), vel64,
                                                          ops, fmask, dtg, ab, minv);
  };
  if (Np <= 6) run(std::integral_constant<int, 6>{});
  else if (Np <= 15) run(std::integral_constant<int, 15>{});
  else run(std::integral_constant<int, kMaxNp>{});
  return cudaGetLastError();
}

cudaError_t block_jacobi_apply(int64_t K, int Np, int Qp, const double* minv, const double* v, double* z,
                               cudaStream_t st) {
  const int64_t n = K * Qp;
  bj_apply_kernel<<<int((n + 255) / 256), 256, 0, st>>>(K, Np, Qp, minv, v, z);
  return cudaGetLastError();
}

}  // namespace krylov
}  // namespace fedbm
