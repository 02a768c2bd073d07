// Device vector kernels of the implicit solver (Newton-GMRES): FP64 vectors
// of the solver's internal layout [K][Np][Qp], reductions in a fixed order
// (the same result on every run).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fedbm {
namespace krylov {

// Blocks of the partial-sum reductions (one partial sum per block).
constexpr int kDotBlocks = 512;
constexpr int kThreads = 256;

// out = a x + b y (out may alias x or y)
cudaError_t axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t st);
// y -= sum_i c[i] V_i for i < m; V holds m vectors of n values each, c is host memory
cudaError_t sub_combination(int64_t n, int m, const double* V, const double* c_dev, double* y, cudaStream_t st);
// out = sum_i c[i] V_i + b out (i < m); c in device memory
cudaError_t add_combination(int64_t n, int m, const double* V, const double* c_dev, double* out, cudaStream_t st);
// h[i] = <V_i, w> for i < m, through partial[m][kDotBlocks] (device); h in device memory
cudaError_t multi_dot(int64_t n, int m, const double* V, const double* w, double* partial, double* h, cudaStream_t st);
// FP64 <-> FP32 copies
cudaError_t to_f32(int64_t n, const double* x, float* y, cudaStream_t st);
cudaError_t to_f64(int64_t n, const float* x, double* y, cudaStream_t st);
// geo[k][dt slot] = value for every element (a copy of the geometry with a unit time step)
cudaError_t set_geo_dt(int64_t K, int stride, int slot, double value, void* geo, int real_bytes, cudaStream_t st);

}  // namespace krylov
}  // namespace fedbm

namespace fedbm {
namespace krylov {

// Element-and-velocity block-Jacobi preconditioner of (I - dtg J) (see
// krylov.cu): the inverse of every (element, velocity) block, stored
// [K][Np][Np][Qp], built from the FP64 reference operators ops = [Dr | Ds |
// LIFT] (row-major, Np*Np, Np*Np, Np*3Nfp), fmask [3][Nfp], the velocity table
// vel64 [3][Qp] and the element geometry (real_bytes 8 or 4).
cudaError_t block_jacobi_build(int64_t K, int Np, int Nfp, int Qp, const void* geo, int real_bytes,
                               const double* vel64, const double* ops, const int* fmask, double dtg, double ab,
                               double* minv, cudaStream_t st);
// z = M^-1 v, blockwise
cudaError_t block_jacobi_apply(int64_t K, int Np, int Qp, const double* minv, const double* v, double* z,
                               cudaStream_t st);

}  // namespace krylov
}  // namespace fedbm
