// Allocation-free variant of the FP64 mass diagnostic.
//
// fedbm_mass() keeps its per-block partial sums in device memory that the
// solver allocates with cudaMalloc.  This file offers the same reduction to
// callers that must not allocate device memory after start-up -- for example
// an application whose device memory is owned by another allocator (a
// framework's caching allocator or a fixed pre-reserved pool), or a real-time
// loop that cannot afford cudaMalloc's latency and implicit synchronisation.
// Its scratch lives in one file-scope __device__ array of fixed size that the
// CUDA runtime places in every device's memory when the library is loaded and
// that stays there until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "fedbm.h"

namespace fedbm {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 8192;                                   // one partial sum per block
constexpr int64_t kMaxNodes = int64_t(kMaxBlocks) * kThreads;      // 2,097,152 nodes
constexpr size_t kScratchBytes = size_t(kMaxBlocks) * sizeof(double) + 256;  // partials + status word

// The shared scratch: block partial sums followed by a status word.  In host
// code this name is only a stand-in for the symbol; the device address comes
// from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_mass_scratch[kScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once per device).
int scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    fedbm::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return FEDBM_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    fedbm::set_last_error("device ordinal out of range");
    return FEDBM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_mass_scratch);
    if (e != cudaSuccess || p == nullptr) {
      fedbm::set_last_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      return FEDBM_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return FEDBM_OK;
}

// One thread per node: rho = sum_i f_i in FP64, contribution J_k (1^T M)_n rho.
__global__ void noalloc_mass_partial(const double* __restrict__ f, const double* __restrict__ jac,
                                     const double* __restrict__ colsum, int64_t K, int Np, int Q,
                                     double* partial, int* status) {
  __shared__ double red[kThreads / 32];
  const int64_t node = int64_t(blockIdx.x) * kThreads + threadIdx.x;
  double acc = 0.0;
  if (node < K * Np) {
    const double* row = f + node * Q;
    double rho = 0.0;
    for (int i = 0; i < Q; ++i) rho += row[i];
    if (!(rho > 0.0) || !isfinite(rho)) atomicOr(status, 1);
    acc = jac[node / Np] * colsum[node % Np] * rho;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int j = 0; j < kThreads / 32; ++j) t += red[j];
    partial[blockIdx.x] = t;
  }
}

// Deterministic sum of the partials (fixed order), then copy the status word.
__global__ void noalloc_mass_final(const double* partial, int nblocks, const int* status_in, double* total,
                                   int32_t* status_out) {
  __shared__ double red[kThreads / 32];
  double acc = 0.0;
  for (int j = threadIdx.x; j < nblocks; j += kThreads) acc += partial[j];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int j = 0; j < kThreads / 32; ++j) t += red[j];
    total[0] = t;
    status_out[0] = status_in[0];
  }
}

}  // namespace

extern "C" int fedbm_mass_noalloc(const double* f, const double* jac, const double* mass_colsum, int64_t K,
                                  int32_t Np, int32_t Q, double* total, int32_t* status, void* cuda_stream) {
  if (!f || !jac || !mass_colsum || !total || !status) {
    fedbm::set_last_error("fedbm_mass_noalloc: null pointer argument");
    return FEDBM_EINVAL;
  }
  if (K < 1 || Np < 1 || Q < 1) {
    fedbm::set_last_error("fedbm_mass_noalloc: K, Np and Q must be positive");
    return FEDBM_EINVAL;
  }
  if (K * Np > kMaxNodes) {
    fedbm::set_last_error("fedbm_mass_noalloc: K*Np = " + std::to_string(K * Np) +
                          " nodes exceeds the fixed scratch capacity of " + std::to_string(kMaxNodes) +
                          " nodes; use fedbm_mass on a solver instead");
    return FEDBM_EINVAL;
  }
  unsigned char* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != FEDBM_OK) return rc;
  double* partial = reinterpret_cast<double*>(scratch);
  int* flag = reinterpret_cast<int*>(scratch + size_t(kMaxBlocks) * sizeof(double));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nblocks = int((K * Np + kThreads - 1) / kThreads);
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);  // the status word must start at zero
  if (e == cudaSuccess) {
    noalloc_mass_partial<<<nblocks, kThreads, 0, st>>>(f, jac, mass_colsum, K, Np, Q, partial, flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    noalloc_mass_final<<<1, kThreads, 0, st>>>(partial, nblocks, flag, total, status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    fedbm::set_last_error(std::string("fedbm_mass_noalloc: ") + cudaGetErrorString(e));
    return FEDBM_ECUDA;
  }
  return FEDBM_OK;
}
