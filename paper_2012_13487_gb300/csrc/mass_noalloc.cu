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
#include <cuda.h>  // driver API types only; the functions come from cudaGetDriverEntryPointByVersion
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

// The symbol's device address belongs to a CUDA context (the module is loaded
// once per context), not to a device ordinal: cudaDeviceReset or a driver-API
// context of its own gives the same device another copy of the array.  The
// address is therefore cached per context, keyed by the context's unique ID
// (cuCtxGetId; a context created after a reset gets a new ID even if its
// handle value repeats).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

constexpr int kCacheSlots = 64;
struct ScratchSlot {
  unsigned long long ctx_id = 0;
  unsigned char* addr = nullptr;
};
std::mutex g_mutex;
ScratchSlot g_cache[kCacheSlots];
int g_next_slot = 0;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

int cuda_fail(const char* what, cudaError_t e) {
  fedbm::set_last_error(std::string("fedbm_mass_noalloc: ") + what + ": " + cudaGetErrorString(e));
  return FEDBM_ECUDA;
}

// Unique ID of the calling thread's current context (0 if none is current).
int current_context_id(unsigned long long* id) {
  *id = 0;
  if (!g_ctx_get_current || !g_ctx_get_id) {
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return cuda_fail("driver entry points", e);
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
      fedbm::set_last_error("fedbm_mass_noalloc: the driver has no cuCtxGetCurrent/cuCtxGetId");
      return FEDBM_ECUDA;
    }
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) {
    fedbm::set_last_error("fedbm_mass_noalloc: cuCtxGetCurrent failed");
    return FEDBM_ECUDA;
  }
  if (ctx && g_ctx_get_id(ctx, id) != CUDA_SUCCESS) {
    fedbm::set_last_error("fedbm_mass_noalloc: cuCtxGetId failed");
    return FEDBM_ECUDA;
  }
  return FEDBM_OK;
}

// Device address of the scratch in the current context, looked up with
// cudaGetSymbolAddress the first time a context calls and cached for it.
int scratch_address(unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  unsigned long long id = 0;
  int rc = current_context_id(&id);
  if (rc != FEDBM_OK) return rc;
  if (id != 0) {
    for (const ScratchSlot& sl : g_cache)
      if (sl.ctx_id == id && sl.addr) {
        *out = sl.addr;
        return FEDBM_OK;
      }
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_mass_scratch);  // makes the device's primary context current if none is
  if (e != cudaSuccess || p == nullptr) return cuda_fail("cudaGetSymbolAddress(scratch)", e);
  if (id == 0 && (rc = current_context_id(&id)) != FEDBM_OK) return rc;
  ScratchSlot& sl = g_cache[g_next_slot];
  g_next_slot = (g_next_slot + 1) % kCacheSlots;
  sl.ctx_id = id;
  sl.addr = static_cast<unsigned char*>(p);
  *out = sl.addr;
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
