// C ABI of the solver: set-up, state transfer, LSRK stepping (CUDA graphs of
// the fused stage kernel), moments and the FP64 mass diagnostic.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "fedbm.h"
#include "host_setup.h"
#include "krylov.h"
#include "stage_dispatch.h"

namespace {
// NVTX range over one library call (shown by Nsight timelines; a no-op when no
// tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

namespace fedbm {
namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

const char* g_last_error_c() { return g_last_error.c_str(); }

#define FEDBM_CK(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? FEDBM_ENOMEM : FEDBM_ECUDA,          \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

// Carpenter & Kennedy (1994) LSRK(5,4) 2N-storage coefficients.
const double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kRkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};

StageEntry stage_entry(int p) {
  switch (p) {
    case 0: return stage_entry_p0();
    case 1: return stage_entry_p1();
    case 2: return stage_entry_p2();
    case 3: return stage_entry_p3();
    case 4: return stage_entry_p4();
    case 5: return stage_entry_p5();
    default: return stage_entry_p6();
  }
}

std::mutex g_upload_mutex;
bool g_uploaded[256] = {};

// Reference operators of every degree go to constant memory once per device.
int ensure_ops_uploaded(int dev) {
  std::lock_guard<std::mutex> lock(g_upload_mutex);
  if (dev < 0 || dev >= 256) return fail(FEDBM_EINVAL, "device ordinal out of range");
  if (g_uploaded[dev]) return FEDBM_OK;
  for (int p = 0; p <= kMaxOrder; ++p) {
    RefOps o;
    std::string err;
    if (!build_ref_ops(p, o, err)) return fail(FEDBM_EINVAL, err);
    cudaError_t e = stage_entry(p).upload(o.Dr.data(), o.Ds.data(), o.LIFT.data());
    if (e != cudaSuccess) return fail(FEDBM_ECUDA, std::string("operator upload: ") + cudaGetErrorString(e));
  }
  g_uploaded[dev] = true;
  return FEDBM_OK;
}

size_t store_bytes(int kind) { return kind == kStoreF64 ? 8 : kind == kStoreF32 ? 4 : 2; }

// Largest dynamic shared memory of one CTA (227 KB on sm_103a).
constexpr size_t kMaxSmem = 227 * 1024;
size_t real_bytes(int kind) { return kind == kStoreF64 ? 8 : 4; }

// ---------------------------------------------------------------- aux kernels
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// canonical f = f^eq(rho0, u0) (1 + amp u(seed, index)) in FP64
// (vel64 in the internal velocity order, iperm[c] = internal index of
// canonical velocity c)
__global__ void equilibrium_kernel(double* out, const double* vel64, const int32_t* iperm, int64_t K, int Np,
                                   int Q, int Qp, double rho0, double ux0, double uy0, double amp, uint64_t seed,
                                   int eq_order) {
  const int64_t n = K * Np * Q;
  for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < n;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int i = iperm[int(idx % Q)];
    const double ex = vel64[i], ey = vel64[Qp + i], w = vel64[2 * Qp + i];
    const double eu = ex * ux0 + ey * uy0, uu = ux0 * ux0 + uy0 * uy0;
    double poly = 1.0 + eu + 0.5 * (eu * eu - uu);
    if (eq_order == 3) poly = poly + eu * eu * eu / 6.0 - 0.5 * eu * uu;
    const double feq = w * rho0 * poly;
    const uint64_t z = splitmix64(seed ^ uint64_t(idx));
    const double u = 2.0 * (double(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    out[idx] = feq * (1.0 + amp * u);
  }
}

// canonical FP64 or FP32 [K][Np][Q] -> internal storage [K][Np][Qp], canonical
// velocity c at internal index iperm[c], the padding velocities zero (one CTA
// per element; the deviation forms compute their scale and codes in FP64)
template <class ST, typename TIn>
__global__ void encode_kernel(const TIn* in, void* out, float* scale, const double* vel64, const int32_t* iperm,
                              int Np, int Q, int Qp) {
  using S = typename ST::S;
  const int64_t k = blockIdx.x;
  const TIn* src = in + k * Np * Q;
  S* dst = static_cast<S*>(out) + k * Np * Qp;
  const double* w = vel64 + 2 * Qp;
  if constexpr (ST::dev) {
    __shared__ float red[32];
    float m = 0.f;
    for (int j = threadIdx.x; j < Np * Q; j += blockDim.x) {
      const int i = iperm[j % Q];
      if (w[i] > 0) m = fmaxf(m, float(fabs((double(src[j]) - w[i]) / w[i])));
    }
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      float mm = 0.f;
      for (int j = 0; j < int(blockDim.x + 31) / 32; ++j) mm = fmaxf(mm, red[j]);
      float sc = 1.0f;
      if (mm > 0.f) {
        int e2;
        frexpf(mm, &e2);
        sc = ldexpf(1.0f, e2 - ST::qmax_log2);
      }
      red[0] = sc;
      scale[k] = sc;
    }
    __syncthreads();
    const double inv_s = 1.0 / double(red[0]);
    for (int j = threadIdx.x; j < Np * Q; j += blockDim.x) {
      const int n = j / Q, i = iperm[j % Q];
      float q = 0.f;
      if (w[i] > 0) q = float((double(src[j]) - w[i]) / w[i] * inv_s);
      dst[n * Qp + i] = ST::from_r(q);
    }
  } else {
    (void)scale;
    (void)w;
    for (int j = threadIdx.x; j < Np * Q; j += blockDim.x) dst[(j / Q) * Qp + iperm[j % Q]] = S(double(src[j]));
  }
  for (int j = threadIdx.x; j < Np * (Qp - Q); j += blockDim.x)
    dst[(j / (Qp - Q)) * Qp + Q + j % (Qp - Q)] = S(0.0f);
}

template <class ST>
__device__ __forceinline__ double decode64(const typename ST::S v, double w, double s) {
  if constexpr (ST::dev) return w + w * s * double(ST::to_r(v));
  else return double(v);
}

// internal state -> canonical FP64 (canonical velocity c from internal index iperm[c])
template <class ST>
__global__ void decode_kernel(const void* in, const float* scale, double* out, const double* vel64,
                              const int32_t* iperm, int64_t K, int Np, int Q, int Qp) {
  using S = typename ST::S;
  const int64_t n = K * Np * Q;
  const double* w = vel64 + 2 * Qp;
  for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < n;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int i = iperm[int(idx % Q)];
    const int64_t kn = idx / Q;
    const int64_t k = kn / Np;
    const double s = ST::dev ? double(scale[k]) : 0.0;
    out[idx] = decode64<ST>(static_cast<const S*>(in)[kn * Qp + i], w[i], s);
  }
}

template <typename R>
__global__ void decode_residual_kernel(const R* in, const int32_t* iperm, double* out, int64_t K, int Np, int Q,
                                       int Qp) {
  const int64_t n = K * Np * Q;
  for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < n;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int i = iperm[int(idx % Q)];
    const int64_t kn = idx / Q;
    out[idx] = double(in[kn * Qp + i]);
  }
}

// One value of a node row in the state's compute precision R (FP64 state:
// double; FP32 and 16-bit states: float, f = w + (w s) q for the latter).
template <class ST>
__device__ __forceinline__ typename ST::R decode_r(const typename ST::S v, typename ST::R w, typename ST::R ws) {
  if constexpr (ST::dev) return fmaf(ws, ST::to_r(v), w);
  else return typename ST::R(v);
}

// Sums over one node row: one warp per node, lanes on consecutive velocities
// (coalesced), partial sums and the warp reduction in the state's compute
// precision R (FP64 for the FP64 state), returned as FP64.
template <class ST>
__device__ __forceinline__ void node_sums(const typename ST::S* row, const typename ST::R* vel, int Qp,
                                          typename ST::R s, int lane, typename ST::R& d0, typename ST::R& d1,
                                          typename ST::R& d2) {
  using R = typename ST::R;
  using S = typename ST::S;
  constexpr int V = 16 / sizeof(S);  // values per 16-byte load (Qp is a multiple of 8)
  R m0 = 0, m1 = 0, m2 = 0;
  // 16-byte loads, several in flight per lane: one 128-byte load per warp at a
  // time leaves HBM latency-bound
#pragma unroll 4
  for (int i = lane * V; i < Qp; i += 32 * V) {
    __align__(16) S q[V];
    *reinterpret_cast<uint4*>(q) = *reinterpret_cast<const uint4*>(row + i);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      const R w = vel[kVelW * Qp + i + j];
      const R f = decode_r<ST>(q[j], w, w * s);
      m0 += f;
      m1 = fma(vel[kVelEx * Qp + i + j], f, m1);
      m2 = fma(vel[kVelEy * Qp + i + j], f, m2);
    }
  }
  // the warp reduction in R as well (FP64 throughput is low on this part; for
  // the FP32 and 16-bit states the lane sums are FP32 already)
  for (int off = 16; off > 0; off >>= 1) {
    m0 += __shfl_xor_sync(0xffffffffu, m0, off);
    m1 += __shfl_xor_sync(0xffffffffu, m1, off);
    m2 += __shfl_xor_sync(0xffffffffu, m2, off);
  }
  d0 = m0;
  d1 = m1;
  d2 = m2;
}

// node moments rho, u_x, u_y (FP64 outputs), one warp per node
template <class ST>
__global__ void moments_kernel(const void* in, const float* scale, const typename ST::R* vel, int64_t K, int Np,
                               int Qp, double* rho, double* ux, double* uy) {
  using S = typename ST::S;
  using R = typename ST::R;
  const int lane = threadIdx.x & 31;
  const int64_t nodes = K * Np;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t kn = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; kn < nodes; kn += nw) {
    const S* row = static_cast<const S*>(in) + kn * Qp;
    const R s = ST::dev ? R(scale[kn / Np]) : R(0);
    R m0, m1, m2;
    node_sums<ST>(row, vel, Qp, s, lane, m0, m1, m2);
    if (lane == 0) {
      // the quotients in R too: FP64 division is slow here, and the FP32 and
      // 16-bit states carry FP32 precision
      rho[kn] = double(m0);
      ux[kn] = double(m1 / m0);
      uy[kn] = double(m2 / m0);
    }
  }
}

// rho of one node row summed in FP64 over its velocities: one warp per node,
// 16-byte loads, every stored value decoded to FP64 (exact for FP32 state; for
// the deviation forms f = w + (w s) q with w from the FP64 velocity table),
// FP64 lane sums and an FP64 warp reduction.  The mass diagnostic resolves
// conservation drift far below FP32 rounding of a velocity sum this way.
template <class ST>
__device__ __forceinline__ double node_rho64(const typename ST::S* row, const double* w64, int Qp, double s,
                                             int lane) {
  using S = typename ST::S;
  constexpr int V = 16 / sizeof(S);  // values per 16-byte load (Qp is a multiple of 8)
  double m0 = 0.0;
#pragma unroll 4
  for (int i = lane * V; i < Qp; i += 32 * V) {
    __align__(16) S q[V];
    *reinterpret_cast<uint4*>(q) = *reinterpret_cast<const uint4*>(row + i);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      if constexpr (ST::dev) {
        const double w = w64[i + j];
        m0 += w + w * s * double(ST::to_r(q[j]));
      } else {
        m0 += double(q[j]);
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) m0 += __shfl_xor_sync(0xffffffffu, m0, off);
  return m0;
}

// mass partial sums: sum over nodes of J_k mw_n rho, all in FP64; flags
// non-finite / rho <= 0
template <class ST>
__global__ void mass_partial_kernel(const void* in, const float* scale, const double* w64, const double* Jk,
                                    const double* mw, int64_t K, int Np, int Qp, double* partial, int* flag) {
  using S = typename ST::S;
  __shared__ double red[32];
  const int lane = threadIdx.x & 31;
  const int64_t nodes = K * Np;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  double acc = 0.0;
  for (int64_t kn = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; kn < nodes; kn += nw) {
    const S* row = static_cast<const S*>(in) + kn * Qp;
    const int64_t k = kn / Np;
    const double s = ST::dev ? double(scale[k]) : 0.0;
    const double rho = node_rho64<ST>(row, w64, Qp, s, lane);
    if (lane == 0) {
      if (!(rho > 0.0) || !isfinite(rho)) atomicOr(flag, 1);
      acc += Jk[k] * mw[kn % Np] * rho;
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int j = 0; j < int(blockDim.x + 31) / 32; ++j) t += red[j];
    partial[blockIdx.x] = t;
  }
}

__global__ void mass_final_kernel(const double* partial, int n, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) acc += partial[j];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int j = 0; j < int(blockDim.x + 31) / 32; ++j) t += red[j];
    out[0] = t;
  }
}

constexpr int kMassBlocks = 1024;
constexpr int kMassThreads = 256;

// SM count of the current device (queried once per device; 152 on GB300).
int sm_count() {
  static std::mutex mu;
  static int cache[256] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return 152;
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[dev] && cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    cache[dev] = 152;
  return cache[dev];
}

// Grid of a grid-stride elementwise kernel: enough blocks for n threads, at
// most 32 resident blocks per SM.
int grid_for(int64_t n, int block) {
  return int(std::max<int64_t>(1, std::min<int64_t>((n + block - 1) / block, int64_t(sm_count()) * 32)));
}



// ---------------------------------------------------------------- batch and solver objects

// One case: its descriptors, its element range inside its group and its clock.
struct Case {
  fedbm_mesh_desc md{};
  fedbm_velset_desc vd{};
  fedbm_params prm{};
  int group = 0;
  int local = 0;        // index of the case inside its group (wall slots 4*local .. 4*local+3)
  int64_t k_off = 0;    // first element inside the group
  int64_t K = 0;
  double dt = 0, tau = 0;
};

// Cases that share degree, velocity set, precision and kernel options run as
// one concatenated element list: one stage-kernel launch covers all of them.
struct Group {
  int p = 0, store = kStoreF32, Q = 0, Qp = 0, Np = 0, Nfp = 0;
  fedbm_velset_desc vd{};
  int collision = 1, reduction = 0;
  double beta = 1.0;
  int test_wait_timeout = 0;
  int tc_mode = 0;  // fedbm_params.tensor_cores of the group's cases
  int tc = 0;       // 1: the stage kernel is the tensor-core form
  int vsplit = 0;   // fedbm_params.velocity_split of the group's cases
  int rounding = 0; // fedbm_params.rounding: 1 = stochastic BF16 encode
  uint32_t* sr_step = nullptr;  // stochastic rounding: steps taken since the state load
  int ncl = 0;      // > 1: the velocity-split form with clusters of ncl CTAs
  int64_t K = 0;
  std::vector<int> cases;
  int epc = 0, tpb = 0, nstages = 1, grid = 0;
  size_t smem = 0;
  RefOps ops;
  VelocitySet vs;
  void* f[2] = {nullptr, nullptr};
  void* res = nullptr;
  float* scale[2] = {nullptr, nullptr};
  int32_t* nbr = nullptr;
  void* geo = nullptr;          // [K][16] compute precision
  void* vel = nullptr;          // [kVelRows][Qp]
  double* vel64 = nullptr;      // [3][Qp]
  int32_t* iperm = nullptr;     // [Q] internal index of canonical velocity c
  void* wall_feq = nullptr;     // [4 * ncases][Qp]
  void* wall_den_inv = nullptr; // [4 * ncases]
  double* Jk = nullptr;         // [K]
  double* mw = nullptr;         // [Np]
  double* partial = nullptr;    // mass partial sums [kMassBlocks + 1]
  int* flag = nullptr;          // [0] mass diagnostic, [1] stage-kernel wait timeout
  int wall_any = 0;
  double W0 = 0, W1x = 0, W1y = 0;
  cudaStream_t branch = nullptr;  // graph-capture branch of this group
};

struct Batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;
  std::vector<Case> cases;
  std::vector<Group> groups;
  int cur = 0;                   // state buffer holding the current f (all groups step together)
  double time = 0;               // time advanced by implicit steps since the last state load
  int64_t steps = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  double* staging = nullptr;     // canonical FP64 buffer of the largest case (lazy)
  size_t staging_elems = 0;
  double* mom = nullptr;         // [3][K*Np] of the largest case (lazy)
  size_t mom_elems = 0;
  struct Implicit* implicit = nullptr;  // Newton-GMRES work space (lazy, single solvers)
};

bool same_group(const Group& g, const fedbm_mesh_desc& md, const fedbm_velset_desc& vd, const fedbm_params& prm) {
  return g.p == md.order && g.store == prm.precision && g.vd.kind == vd.kind && g.vd.n == vd.n &&
         g.vd.nc_extent == vd.nc_extent && g.vd.nc_sqrt2 == vd.nc_sqrt2 && g.vd.eq_order == vd.eq_order &&
         g.collision == prm.collision && g.reduction == prm.reduction && g.beta == prm.beta &&
         g.epc == prm.elems_per_cta && g.tpb == prm.threads_per_cta && g.nstages == prm.pipeline_stages &&
         g.test_wait_timeout == prm.test_wait_timeout && g.tc_mode == prm.tensor_cores &&
         g.vsplit == prm.velocity_split && g.rounding == prm.rounding;
}

template <typename R>
void fill_stage_args(const Group& g, int stage, int from, StageArgs<R>& a) {
  a.f_in = g.f[from];
  a.f_out = g.f[1 - from];
  a.res = static_cast<R*>(g.res);
  a.scale_in = g.scale[from];
  a.scale_out = g.scale[1 - from];
  a.nbr = g.nbr;
  a.geo = static_cast<const R*>(g.geo);
  a.vel = static_cast<const R*>(g.vel);
  a.wall_feq = static_cast<const R*>(g.wall_feq);
  a.wall_den_inv = static_cast<const R*>(g.wall_den_inv);
  a.wall_any = g.wall_any;
  a.W0 = R(g.W0);
  a.W1x = R(g.W1x);
  a.W1y = R(g.W1y);
  a.K = g.K;
  a.Qp = g.Qp;
  a.epc = g.epc;
  a.nstages = g.nstages;
  a.rkA = R(kRkA[stage]);
  a.rkB = R(kRkB[stage]);
  a.ab = R(2.0 * g.beta - 1.0);
  a.collision = g.collision;
  a.eq_order = g.vd.eq_order;
  a.red = g.reduction;
  a.err = g.flag + 1;
  a.extra_tx = g.test_wait_timeout ? 16u : 0u;
  a.sr_step = g.sr_step;
  a.sr_stage = stage;
}

// one more step for the stochastic-rounding draws (a graph node after each step)
__global__ void sr_step_kernel(uint32_t* step) { step[0] += 1u; }

// Launch the group's configured stage-kernel form with these arguments.
cudaError_t launch_args(const Group& g, const void* args, cudaStream_t st, int grid = 0) {
  const StageEntry e = stage_entry(g.p);
  if (grid <= 0) grid = g.grid;
  if (g.ncl > 1) return e.launch_cl(g.store, args, g.grid / g.ncl, g.ncl, g.smem, st);
  if (g.tc) return e.launch_tc(g.store, args, grid, g.smem, st);
  if (g.nstages == 3) return e.launch_ws(g.store, args, grid, g.smem, st);
  return e.launch(g.store, args, grid, g.tpb, g.smem, st);
}

cudaError_t launch_stage(const Group& g, int stage, int from, cudaStream_t st, int grid = 0) {
  if (g.store == kStoreF64) {
    StageArgs<double> a;
    fill_stage_args(g, stage, from, a);
    return launch_args(g, &a, st, grid);
  }
  StageArgs<float> a;
  fill_stage_args(g, stage, from, a);
  return launch_args(g, &a, st, grid);
}


void drop_graphs(Batch& b) {
  for (int c = 0; c < 2; ++c)
    if (b.graph[c]) {
      cudaGraphExecDestroy(b.graph[c]);
      b.graph[c] = nullptr;
    }
}

// The tensor-core form of a group: one element per CTA, 128 threads, one
// velocity per thread in each 128-velocity pass.  Each CTA holds tc_tmem_cols tensor-memory columns for its whole
// life; the resident CTAs of an SM must fit in its 512 columns so that an
// allocation never waits on another CTA of the same kernel.
int configure_tc(Batch& b, Group& g) {
  const StageEntry e = stage_entry(g.p);
  size_t smem = e.tc_smem(g.store, g.Qp);
  if (g.tc_mode < 0 || smem == 0) return fail(FEDBM_EINVAL, "this form has no tensor-core stage kernel");
  int nsm = 0;
  FEDBM_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b.device));
  int smem_sm = 0;
  FEDBM_CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, b.device));
  // small tiles: reserve enough shared memory that no more CTAs fit on an SM
  // than its tensor memory serves
  const int max_ctas = 512 / e.tc_tmem_cols(g.Qp);
  smem = std::max(smem, size_t(smem_sm) / size_t(max_ctas + 1) + 1024);
  FEDBM_CK(e.set_smem_tc(g.store, g.Qp, kMaxSmem));
  const int per_sm = e.occupancy_tc(g.store, g.Qp, smem);
  const int by_smem = int(size_t(smem_sm) / smem);
  if (per_sm < 1 || std::max(per_sm, by_smem) * e.tc_tmem_cols(g.Qp) > 512)
    return fail(FEDBM_EINVAL, "tensor-core stage kernel cannot be resident within tensor memory");
  g.tc = 1;
  g.ncl = 0;
  g.epc = g.Qp < 128 ? 128 / g.Qp : 1;  // stacked elements per tile below 128 velocities
  g.tpb = 128;                          // one 128-row MMA tile per pass
  g.nstages = 1;
  g.smem = smem;
  g.grid = int(std::min<int64_t>((g.K + g.epc - 1) / g.epc, int64_t(per_sm) * nsm));
  drop_graphs(b);
  return FEDBM_OK;
}

bool tc_available(const Group& g) { return g.tc_mode >= 0 && stage_entry(g.p).tc_smem(g.store, g.Qp) > 0; }

// The velocity-split form of a group: clusters of ncl CTAs, each CTA one
// slice of Qp / ncl velocities of one element per tile, 256 threads; the
// persistent grid holds as many clusters as can be resident at once.
int configure_cluster(Batch& b, Group& g, int ncl) {
  const StageEntry e = stage_entry(g.p);
  const size_t smem = e.cl_smem(g.store, g.Qp, ncl, 1);
  if (smem == 0) return fail(FEDBM_EINVAL, "no velocity-split form for this precision or cluster size "
                                           "(FP64, FP32 or BF16 state; clusters of 2, 4 or 8 CTAs dividing the "
                                           "padded velocity count into multiples of 8)");
  if (smem > kMaxSmem) return fail(FEDBM_EINVAL, "velocity-split tile does not fit in shared memory");
  FEDBM_CK(e.set_smem_cl(g.store, kMaxSmem));
  const int nclusters_max = e.occupancy_cl(g.store, ncl, smem);
  if (nclusters_max < 1) return fail(FEDBM_EINVAL, "velocity-split clusters cannot be resident");
  g.tc = 0;
  g.ncl = ncl;
  g.epc = 1;
  g.tpb = 256;
  g.nstages = 1;
  g.smem = smem;
  g.grid = int(std::min<int64_t>(g.K, int64_t(nclusters_max))) * ncl;
  drop_graphs(b);
  return FEDBM_OK;
}

// Cluster size of the automatic velocity-split form: the one that keeps the
// most CTAs resident on the device (smaller slices let more CTAs share an SM),
// the smaller one on a tie; 0 if no slice fits shared memory.
int auto_cluster(const Group& g) {
  const StageEntry e = stage_entry(g.p);
  int best = 0, best_ctas = 0;
  for (int ncl : {2, 4, 8}) {
    const size_t smem = e.cl_smem(g.store, g.Qp, ncl, 1);
    if (smem == 0 || smem > kMaxSmem) continue;
    if (e.set_smem_cl(g.store, kMaxSmem) != cudaSuccess) continue;
    const int ctas = e.occupancy_cl(g.store, ncl, smem) * ncl;
    if (ctas > best_ctas) {
      best = ncl;
      best_ctas = ctas;
    }
  }
  return best;
}

// The warp-specialised form of a group: one element per ring stage, eight
// consumer warps (one velocity per thread) and one producer warp.
bool ws_available(const Group& g) { return stage_entry(g.p).ws_smem(g.store, g.Qp) > 0; }

// The untuned default takes the warp-specialised form where it measured
// faster than the FMA kernel's default tile on the 256-velocity cavities of
// about 30M DOF: FP32 state at degree 1-4 (x1.04-1.12), BF16 at degree 3-5
// (x1.21-1.41, the volume contractions on tensor cores).  FP32 at degree 5
// holds one CTA per SM (three 39 KB stages) and BF16 at degree 1-2 loses to
// the FMA kernel's two velocities per thread.
bool ws_default(const Group& g) {
  if (!ws_available(g)) return false;
  return (g.store == kStoreF32 && g.p >= 1 && g.p <= 4) || (g.store == kStoreBF16 && g.p >= 3);
}

int configure_ws(Batch& b, Group& g) {
  const StageEntry e = stage_entry(g.p);
  const size_t smem = e.ws_smem(g.store, g.Qp);
  if (smem == 0)
    return fail(FEDBM_EINVAL, "pipeline_stages = 3 (the warp-specialised stage kernel) needs FP32 or BF16 state, "
                              "256 padded velocities and degree <= 5");
  if (smem > kMaxSmem) return fail(FEDBM_EINVAL, "warp-specialised ring does not fit in shared memory");
  FEDBM_CK(e.set_smem_ws(g.store, kMaxSmem));
  int nsm = 0;
  FEDBM_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b.device));
  const int per_sm = e.occupancy_ws(g.store, smem);
  if (per_sm < 1) return fail(FEDBM_EINVAL, "warp-specialised stage kernel cannot be resident on an SM");
  g.tc = 0;
  g.ncl = 0;
  g.epc = 1;
  g.tpb = 288;
  g.nstages = 3;
  g.smem = smem;
  g.grid = int(std::min<int64_t>(g.K, int64_t(per_sm) * nsm));
  drop_graphs(b);
  return FEDBM_OK;
}

// Tile shape, pipeline depth and persistent grid of a group's stage kernel.
int configure_tiles(Batch& b, Group& g, int epc, int tpb, int stages) {
  if (stages == 3) return configure_ws(b, g);  // tile and threads are the form's own
  // the group is changed only once the whole configuration is valid
  int e_pc = epc > 0 ? epc : (g.Qp < 128 ? std::max(1, 128 / g.Qp) : 1);
  int t_pb = tpb > 0 ? tpb : std::min(128, std::max(32, (e_pc * g.Qp + 31) / 32 * 32));
  if (epc == 0 && tpb == 0 && g.Qp == 16 && (g.store == kStoreF32 || g.store == kStoreBF16)) {
    // 16 velocities: the autotuner's picks on ~20-45M-DOF Couette cases (FP32
    // x1.4 at degree 1, x1.15 at 2; BF16 x1.9, 1.8, 1.6, 1.25, 1.04 at 1..5):
    // 16 elements per tile up to degree 2, else 8; 64 threads for BF16 state
    // (one item per thread where two velocities share a thread)
    e_pc = g.p <= 2 ? 16 : 8;
    t_pb = g.store == kStoreBF16 ? 64 : 128;
  }
  if (t_pb % 32 || t_pb > 256) return fail(FEDBM_EINVAL, "threads_per_cta must be a multiple of 32, <= 256");
  if (stages < 0 || stages > 3) return fail(FEDBM_EINVAL, "pipeline_stages must be 0, 1, 2 or 3");
  int nst = stages == 2 ? 2 : 1;
  size_t smem = stage_smem_bytes(g.p, g.store, e_pc, g.Qp, nst);
  if (smem > kMaxSmem && nst == 2) {
    nst = 1;
    smem = stage_smem_bytes(g.p, g.store, e_pc, g.Qp, 1);
  }
  if (smem > kMaxSmem) return fail(FEDBM_EINVAL, "stage tile does not fit in shared memory");
  const StageEntry e = stage_entry(g.p);
  // the kernel's dynamic shared-memory limit stays at the maximum, so that
  // groups of one batch sharing this kernel with other tiles keep launching
  FEDBM_CK(e.set_smem(g.store, g.Qp, kMaxSmem));
  int nsm = 0;
  FEDBM_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b.device));
  const int per_sm = e.occupancy(g.store, g.Qp, t_pb, smem);
  if (per_sm < 1) return fail(FEDBM_EINVAL, "stage tile cannot be resident on an SM");
  const int64_t ntiles = (g.K + e_pc - 1) / e_pc;
  g.tc = 0;
  g.ncl = 0;
  g.epc = e_pc;
  g.tpb = t_pb;
  g.nstages = nst;
  g.smem = smem;
  g.grid = int(std::min<int64_t>(ntiles, int64_t(per_sm) * nsm));
  drop_graphs(b);
  return FEDBM_OK;
}

// ---- tile autotuner ------------------------------------------------------------
// For every group, time each candidate (elements per CTA, threads per CTA,
// pipeline stages, kernel form) on `trials` step-shaped rounds (RK stage 1,
// which reads no residual, then four launches of stage 2, which does) and keep
// the fastest.  Every launch reads f[cur] and writes f[1-cur] and the
// residual, so the current state is untouched; the residual's contents are
// overwritten by the next step's first stage, which does not read it.
// Results are cached per (device, degree, velocity count, precision,
// element count) in a flat JSON object, one entry per line.
struct TuneEntry {
  int epc = 0, tpb = 0, stages = 0, tc = 0;
  int ncl = 0;  // > 1: the velocity-split form with clusters of ncl CTAs
  double us = 0;
};

int apply_tune(Batch& b, Group& g, const TuneEntry& t) {
  if (t.ncl > 1) return configure_cluster(b, g, t.ncl);
  return t.tc ? configure_tc(b, g) : configure_tiles(b, g, t.epc, t.tpb, t.stages);
}

// The velocity-split form can serve this group with clusters of ncl CTAs.
bool cluster_available(const Group& g, int ncl) {
  if (g.vsplit == 1) return false;  // the caller ruled the form out
  const size_t smem = stage_entry(g.p).cl_smem(g.store, g.Qp, ncl, 1);
  return smem > 0 && smem <= kMaxSmem;
}

std::string tune_key(const Batch& b, const Group& g) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, b.device);
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s|p%d|Q%d|store%d|red%d|K%lld", prop.name, g.p, g.Qp, g.store, g.reduction,
                static_cast<long long>(g.K));
  return buf;
}

std::vector<std::pair<std::string, TuneEntry>> read_tune_cache(const char* path) {
  std::vector<std::pair<std::string, TuneEntry>> out;
  if (!path || !*path) return out;
  FILE* fp = std::fopen(path, "r");
  if (!fp) return out;
  char line[1024];
  while (std::fgets(line, sizeof(line), fp)) {
    char key[512];
    TuneEntry t;
    if (std::sscanf(line, " \"%511[^\"]\": {\"epc\": %d, \"tpb\": %d, \"stages\": %d, \"tc\": %d, \"ncl\": %d, \"us\": %lf}",
                    key, &t.epc, &t.tpb, &t.stages, &t.tc, &t.ncl, &t.us) == 7)
      out.emplace_back(key, t);
  }
  std::fclose(fp);
  return out;
}

void write_tune_cache(const char* path, const std::vector<std::pair<std::string, TuneEntry>>& entries) {
  if (!path || !*path) return;
  FILE* fp = std::fopen(path, "w");
  if (!fp) return;
  std::fprintf(fp, "{\n");
  for (size_t j = 0; j < entries.size(); ++j)
    std::fprintf(fp, "\"%s\": {\"epc\": %d, \"tpb\": %d, \"stages\": %d, \"tc\": %d, \"ncl\": %d, \"us\": %.3f}%s\n",
                 entries[j].first.c_str(), entries[j].second.epc, entries[j].second.tpb, entries[j].second.stages,
                 entries[j].second.tc, entries[j].second.ncl, entries[j].second.us,
                 j + 1 < entries.size() ? "," : "");
  std::fprintf(fp, "}\n");
  std::fclose(fp);
}

int autotune(Batch& b, const char* cache_path, int trials) {
  NvtxRange nvtx("fedbm autotune");
  if (trials < 1) trials = 5;
  auto cache = read_tune_cache(cache_path);
  bool dirty = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FEDBM_CK(cudaEventCreate(&e0));
  FEDBM_CK(cudaEventCreate(&e1));
  int rc = FEDBM_OK;
  for (Group& g : b.groups) {
    if (g.ncl > 1) continue;  // the velocity-split form has a single configuration
    if (g.tc_mode > 0) {  // tensor cores required: nothing to choose
      if ((rc = configure_tc(b, g)) != FEDBM_OK) break;
      continue;
    }
    const std::string key = tune_key(b, g);
    const TuneEntry* hit = nullptr;
    for (auto& kv : cache)
      if (kv.first == key) hit = &kv.second;
    if (hit && (!hit->tc || tc_available(g)) && (hit->ncl < 2 || cluster_available(g, hit->ncl)) &&
        (hit->stages != 3 || ws_available(g))) {
      if ((rc = apply_tune(b, g, *hit)) != FEDBM_OK) break;
      continue;
    }
    TuneEntry best;
    best.us = 1e300;
    // a trial is one step's mix: stage 0 (no residual read) and four
    // residual-reading launches, all from f[cur]
    auto time_current = [&](TuneEntry cand) {
      if (launch_stage(g, 1, b.cur, b.stream) != cudaSuccess) return;  // warm-up
      cudaEventRecord(e0, b.stream);
      for (int t = 0; t < trials; ++t) {
        launch_stage(g, 0, b.cur, b.stream);
        for (int r = 0; r < 4; ++r) launch_stage(g, 1, b.cur, b.stream);
      }
      cudaEventRecord(e1, b.stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) return;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      cand.us = 1e3 * double(ms) / trials;
      if (cand.us < best.us) best = cand;
    };
    const int epcs[] = {1, 2, 4, 8, 16, 32};
    const int tpbs[] = {64, 128, 256};
    for (int epc : epcs) {
      if (epc * g.Qp > 4096 || epc > g.K) continue;
      for (int tpb : tpbs) {
        if (tpb > 32 * ((epc * g.Qp + 31) / 32) * 2) continue;  // at most half the threads idle
        for (int stages = 1; stages <= 2; ++stages) {
          if (configure_tiles(b, g, epc, tpb, stages) != FEDBM_OK || g.nstages != stages) continue;
          TuneEntry cand;
          cand.epc = epc;
          cand.tpb = tpb;
          cand.stages = stages;
          time_current(cand);
        }
      }
    }
    if (ws_available(g) && configure_ws(b, g) == FEDBM_OK) {
      TuneEntry cand;
      cand.epc = 1;
      cand.tpb = 288;
      cand.stages = 3;
      time_current(cand);
    }
    if (tc_available(g) && configure_tc(b, g) == FEDBM_OK) {
      TuneEntry cand;
      cand.epc = 1;
      cand.tpb = g.Qp;
      cand.stages = 1;
      cand.tc = 1;
      time_current(cand);
    }
    // the velocity-split form where the velocity count is large enough that
    // a smaller per-CTA slice may let more CTAs share an SM
    for (int ncl : {2, 4}) {
      if (g.Qp < 256 || !cluster_available(g, ncl) || configure_cluster(b, g, ncl) != FEDBM_OK) continue;
      TuneEntry cand;
      cand.epc = 1;
      cand.tpb = 256;
      cand.stages = 1;
      cand.ncl = ncl;
      time_current(cand);
    }
    cudaGetLastError();
    if (best.epc == 0) {
      rc = fail(FEDBM_ECUDA, "autotune: no tile candidate could run");
      break;
    }
    if ((rc = apply_tune(b, g, best)) != FEDBM_OK) break;
    cache.emplace_back(key, best);
    dirty = true;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == FEDBM_OK && dirty) write_tune_cache(cache_path, cache);
  return rc;
}

// One RK step of every group, captured once per buffer parity; groups are
// independent branches of the graph so that small groups run side by side.
int build_graphs(Batch& b) {
  for (int c = 0; c < 2; ++c) {
    if (b.graph[c]) continue;
    cudaGraph_t graph = nullptr;
    FEDBM_CK(cudaStreamBeginCapture(b.capture, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    std::vector<cudaEvent_t> evs;
    cudaEvent_t fork = nullptr;
    const bool branches = b.groups.size() > 1;
    if (branches) {
      le = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
      if (le == cudaSuccess) le = cudaEventRecord(fork, b.capture);
    }
    for (Group& g : b.groups) {
      if (le != cudaSuccess) break;
      cudaStream_t st = b.capture;
      if (branches) {
        st = g.branch;
        le = cudaStreamWaitEvent(st, fork, 0);
      }
      int from = c;
      for (int s = 0; s < 5 && le == cudaSuccess; ++s) {
        le = launch_stage(g, s, from, st);
        from = 1 - from;
      }
      if (g.sr_step && le == cudaSuccess) {
        sr_step_kernel<<<1, 1, 0, st>>>(g.sr_step);
        le = cudaGetLastError();
      }
      if (branches && le == cudaSuccess) {
        cudaEvent_t done = nullptr;
        le = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
        if (le == cudaSuccess) le = cudaEventRecord(done, st);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(b.capture, done, 0);
        evs.push_back(done);
      }
    }
    cudaError_t ee = cudaStreamEndCapture(b.capture, &graph);
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (le != cudaSuccess) return fail(FEDBM_ECUDA, std::string("stage launch in capture: ") + cudaGetErrorString(le));
    if (ee != cudaSuccess) return fail(FEDBM_ECUDA, std::string("end capture: ") + cudaGetErrorString(ee));
    cudaError_t ie = cudaGraphInstantiate(&b.graph[c], graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return fail(FEDBM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
  }
  return FEDBM_OK;
}

template <typename T>
int upload_vec(const std::vector<T>& h, void** d) {
  FEDBM_CK(cudaMalloc(d, std::max<size_t>(1, h.size() * sizeof(T))));
  FEDBM_CK(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FEDBM_OK;
}

template <typename R>
int upload_real(const std::vector<double>& h, void** d) {
  std::vector<R> v(h.begin(), h.end());
  return upload_vec(v, d);
}

// Relaxation time from Kn (Sec. II.A.4, theta = RT = c_s^2 = 1):
//   FEDBM_TAU_KN:          eq. KnTau, mean free path lambda = sqrt(3) tau c_s,
//                          tau = Kn L / (sqrt(3) c_s);
//   FEDBM_TAU_KIM_PITSCH:  the kinetic-theory mean free path of Kim and Pitsch,
//                          which puts a factor sqrt(pi/6) into Kn:
//                          Kn = sqrt(pi/6) sqrt(3) tau c_s / L, i.e.
//                          tau = Kn L / (sqrt(pi/2) c_s);
//   FEDBM_TAU_PSI:         eq. KnTau scaled by the Kn-dependent function
//                          psi(Kn) = (2/pi) arctan(sqrt(2) Kn^(-3/4)) (Zhang).
double relaxation_time(double kn, double L, int model) {
  const double pi = 3.14159265358979323846;
  switch (model) {
    case FEDBM_TAU_KIM_PITSCH: return kn * L / std::sqrt(pi / 2.0);
    case FEDBM_TAU_PSI: return kn * L / std::sqrt(3.0) * (2.0 / pi) * std::atan(std::sqrt(2.0) * std::pow(kn, -0.75));
    default: return kn * L / std::sqrt(3.0);
  }
}

// Internal velocity order: by direction (half-plane, then the sign of the
// cross product), then speed, so that the 32 velocities of a warp point into a
// narrow range of directions and mostly leave or enter an element through the
// same faces (the warp-specialised kernel skips faces with no inflow for a
// whole warp).  Exact comparisons of IEEE products: the same order on every
// host.  order[j] = canonical index of internal velocity j.
std::vector<int> direction_order(const VelocitySet& vs) {
  std::vector<int> order(vs.Q);
  for (int i = 0; i < vs.Q; ++i) order[i] = i;
  auto half = [&](int i) { return vs.ey[i] < 0 || (vs.ey[i] == 0 && vs.ex[i] < 0) ? 1 : 0; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const int ha = half(a), hb = half(b);
    if (ha != hb) return ha < hb;
    const double cr = vs.ex[a] * vs.ey[b] - vs.ey[a] * vs.ex[b];
    if (cr != 0) return cr > 0;
    return vs.ex[a] * vs.ex[a] + vs.ey[a] * vs.ey[a] < vs.ex[b] * vs.ex[b] + vs.ey[b] * vs.ey[b];
  });
  return order;
}

// Host set-up of a group in FP64 (meshes, walls, geometry) and device upload.
int build_group(Batch& b, Group& g) {
  std::string err;
  if (!build_velocity_set(g.vd, g.vs, err)) return fail(FEDBM_EINVAL, err);
  // the device tables, state and residual hold the velocities in the internal
  // order; set/get state and residual map the canonical order through iperm
  const std::vector<int> order = direction_order(g.vs);
  std::vector<int32_t> iperm(g.vs.Q);
  {
    VelocitySet canon = g.vs;
    for (int j = 0; j < g.vs.Q; ++j) {
      g.vs.ex[j] = canon.ex[order[j]];
      g.vs.ey[j] = canon.ey[order[j]];
      g.vs.w[j] = canon.w[order[j]];
      iperm[order[j]] = j;
    }
  }
  if (!build_ref_ops(g.p, g.ops, err)) return fail(FEDBM_EINVAL, err);
  g.Np = g.ops.Np;
  g.Nfp = g.ops.Nfp;
  g.Q = g.vs.Q;
  // padded velocity count: a multiple of 8 (16-byte vectors of the 16-bit
  // forms); above 512 velocities a multiple of 32, so that the velocity-split
  // form can give clusters of 2 or 4 CTAs slices of whole vectors
  g.Qp = g.Q > 512 ? (g.Q + 31) / 32 * 32 : (g.Q + 7) / 8 * 8;
  const int Np = g.Np, Qp = g.Qp, Q = g.Q;
  const int nslots = 4 * int(g.cases.size());
  std::vector<int32_t> nbr;
  std::vector<double> geo, Jk, wfeq(size_t(nslots) * Qp, 0.0), wden(nslots, 0.0);
  const double nrm[4][2] = {{0, -1}, {1, 0}, {0, 1}, {-1, 0}};
  for (int lc = 0; lc < int(g.cases.size()); ++lc) {
    Case& cs = b.cases[g.cases[lc]];
    Mesh m;
    if (!build_mesh(cs.md, m, err)) return fail(FEDBM_EINVAL, err);
    // an unstructured mesh's caller arrays are read only during creation
    cs.md.vert_xy = nullptr;
    cs.md.tri = nullptr;
    cs.local = lc;
    cs.k_off = g.K;
    cs.K = m.K;
    const double L = cs.prm.length > 0 ? cs.prm.length : 1.0;
    cs.tau = relaxation_time(cs.prm.kn, L, cs.prm.tau_model);
    cs.dt = cs.prm.dt > 0 ? cs.prm.dt : time_step(m, g.vs, g.p, cs.prm.cfl);
    const double itau = g.collision ? 1.0 / cs.tau : 0.0;
    for (int64_t k = 0; k < m.K; ++k) {
      for (int f = 0; f < 3; ++f) {
        const int32_t code = m.nbr[k * 3 + f];
        nbr.push_back(code >= 0 ? encode_face((code >> 3) + cs.k_off, (code >> 1) & 3, code & 1)
                                : int32_t(-(4 * lc + (-code - 1) + 1)));
      }
      for (int j = 0; j < kGeoStride; ++j) geo.push_back(m.geo[k * kGeoStride + j]);
      geo[geo.size() - kGeoStride + kGeoDt] = cs.dt;
      geo[geo.size() - kGeoStride + kGeoInvTau] = itau;
      Jk.push_back(m.geo[k * kGeoStride + kGeoJ]);
    }
    for (int sd = 0; sd < 4; ++sd) {
      const int slot = 4 * lc + sd;
      double den = 0.0;
      for (int i = 0; i < Q; ++i) {
        const double fb = equilibrium(g.vs.w[i], g.vs.ex[i], g.vs.ey[i], 1.0, cs.md.wall_ux[sd], cs.md.wall_uy[sd],
                                      g.vd.eq_order);
        wfeq[size_t(slot) * Qp + i] = fb;
        const double en = g.vs.ex[i] * nrm[sd][0] + g.vs.ey[i] * nrm[sd][1];
        if (en < 0) den -= en * fb;
      }
      if (cs.md.bc[sd] == FEDBM_BC_WALL_DIFFUSE && den > 0) {
        wden[slot] = 1.0 / den;
        g.wall_any = 1;
      }
    }
    g.K += m.K;
  }
  // velocity table, padded with zero-weight zero-speed velocities
  std::vector<double> vel(size_t(kVelRows) * Qp, 0.0), v64(size_t(3) * Qp, 0.0), mw(Np, 0.0);
  for (int i = 0; i < Q; ++i) {
    vel[kVelEx * Qp + i] = g.vs.ex[i];
    vel[kVelEy * Qp + i] = g.vs.ey[i];
    vel[kVelW * Qp + i] = g.vs.w[i];
    vel[kVelInvW * Qp + i] = g.vs.w[i] > 0 ? 1.0 / g.vs.w[i] : 0.0;
    vel[kVelWex * Qp + i] = g.vs.w[i] * g.vs.ex[i];
    vel[kVelWey * Qp + i] = g.vs.w[i] * g.vs.ey[i];
    v64[i] = g.vs.ex[i];
    v64[Qp + i] = g.vs.ey[i];
    v64[2 * Qp + i] = g.vs.w[i];
    g.W0 += g.vs.w[i];
    g.W1x += g.vs.w[i] * g.vs.ex[i];
    g.W1y += g.vs.w[i] * g.vs.ey[i];
  }
  for (int j = 0; j < Np; ++j)
    for (int n = 0; n < Np; ++n) mw[n] += g.ops.M[size_t(j) * Np + n];
  const size_t dofp = size_t(g.K) * Np * Qp;
  for (int c = 0; c < 2; ++c) {
    FEDBM_CK(cudaMalloc(&g.f[c], dofp * store_bytes(g.store)));
    FEDBM_CK(cudaMemset(g.f[c], 0, dofp * store_bytes(g.store)));
    if (g.store >= kStoreBF16) {
      FEDBM_CK(cudaMalloc(&g.scale[c], size_t(g.K) * sizeof(float)));
      FEDBM_CK(cudaMemset(g.scale[c], 0, size_t(g.K) * sizeof(float)));
    }
  }
  FEDBM_CK(cudaMalloc(&g.res, dofp * real_bytes(g.store)));
  FEDBM_CK(cudaMemset(g.res, 0, dofp * real_bytes(g.store)));
  int rc;
  if ((rc = upload_vec(nbr, reinterpret_cast<void**>(&g.nbr))) != FEDBM_OK) return rc;
  if ((rc = upload_vec(v64, reinterpret_cast<void**>(&g.vel64))) != FEDBM_OK) return rc;
  if ((rc = upload_vec(iperm, reinterpret_cast<void**>(&g.iperm))) != FEDBM_OK) return rc;
  if ((rc = upload_vec(Jk, reinterpret_cast<void**>(&g.Jk))) != FEDBM_OK) return rc;
  if ((rc = upload_vec(mw, reinterpret_cast<void**>(&g.mw))) != FEDBM_OK) return rc;
  if (g.store == kStoreF64) {
    if ((rc = upload_real<double>(geo, &g.geo)) != FEDBM_OK) return rc;
    if ((rc = upload_real<double>(vel, &g.vel)) != FEDBM_OK) return rc;
    if ((rc = upload_real<double>(wfeq, &g.wall_feq)) != FEDBM_OK) return rc;
    if ((rc = upload_real<double>(wden, &g.wall_den_inv)) != FEDBM_OK) return rc;
  } else {
    if ((rc = upload_real<float>(geo, &g.geo)) != FEDBM_OK) return rc;
    if ((rc = upload_real<float>(vel, &g.vel)) != FEDBM_OK) return rc;
    if ((rc = upload_real<float>(wfeq, &g.wall_feq)) != FEDBM_OK) return rc;
    if ((rc = upload_real<float>(wden, &g.wall_den_inv)) != FEDBM_OK) return rc;
  }
  FEDBM_CK(cudaMalloc(&g.partial, (kMassBlocks + 1) * sizeof(double)));
  FEDBM_CK(cudaMalloc(&g.flag, 2 * sizeof(int)));
  FEDBM_CK(cudaMemset(g.flag, 0, 2 * sizeof(int)));
  if (g.rounding == 1) {
    FEDBM_CK(cudaMalloc(&g.sr_step, sizeof(uint32_t)));
    FEDBM_CK(cudaMemset(g.sr_step, 0, sizeof(uint32_t)));
  }
  FEDBM_CK(cudaStreamCreateWithFlags(&g.branch, cudaStreamNonBlocking));
  return FEDBM_OK;
}

void free_implicit_of(Batch* b);

void free_batch(Batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int c = 0; c < 2; ++c)
    if (b->graph[c]) cudaGraphExecDestroy(b->graph[c]);
  for (Group& g : b->groups) {
    for (int c = 0; c < 2; ++c) {
      cudaFree(g.f[c]);
      cudaFree(g.scale[c]);
    }
    void* bufs[] = {g.res, g.nbr, g.geo, g.vel, g.vel64, g.iperm, g.wall_feq, g.wall_den_inv, g.Jk, g.mw, g.partial,
                    g.flag, g.sr_step};
    for (void* p : bufs) cudaFree(p);
    if (g.branch) cudaStreamDestroy(g.branch);
  }
  cudaFree(b->staging);
  cudaFree(b->mom);
  free_implicit_of(b);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

int create_batch(const fedbm_case_desc* cd, int ncases, void* stream, Batch** out) {
  if (!cd || ncases < 1 || !out) return fail(FEDBM_EINVAL, "need at least one case and an output pointer");
  *out = nullptr;
  Batch* b = new Batch();
  b->stream = static_cast<cudaStream_t>(stream);
  auto bail = [&](int code) {
    free_batch(b);
    return code;
  };
  for (int c = 0; c < ncases; ++c) {
    const fedbm_params& prm = cd[c].params;
    if (prm.precision < FEDBM_FP64 || prm.precision > FEDBM_FP16_DEV) return bail(fail(FEDBM_EINVAL, "unknown precision"));
    if (prm.reduction < FEDBM_RED_DEFAULT || prm.reduction > FEDBM_RED_COMP_FP32)
      return bail(fail(FEDBM_EINVAL, "unknown reduction mode"));
    if (!(prm.kn > 0)) return bail(fail(FEDBM_EINVAL, "kn must be > 0"));
    if (prm.tau_model < FEDBM_TAU_KN || prm.tau_model > FEDBM_TAU_PSI)
      return bail(fail(FEDBM_EINVAL, "unknown tau_model"));
    if (prm.tensor_cores < -1 || prm.tensor_cores > 1) return bail(fail(FEDBM_EINVAL, "tensor_cores must be -1, 0 or 1"));
    if (prm.velocity_split != 0 && prm.velocity_split != 1 && prm.velocity_split != 2 && prm.velocity_split != 4 &&
        prm.velocity_split != 8)
      return bail(fail(FEDBM_EINVAL, "velocity_split must be 0, 1, 2, 4 or 8"));
    if (prm.rounding != 0 && !(prm.rounding == 1 && prm.precision == FEDBM_BF16_DEV))
      return bail(fail(FEDBM_EINVAL, "rounding: 0 (nearest even), or 1 (stochastic) for BF16 deviation state"));
    if (!(prm.beta >= 0.5 && prm.beta <= 1.0)) return bail(fail(FEDBM_EINVAL, "beta must be in [0.5, 1]"));
    if (!(prm.dt > 0) && !(prm.cfl > 0)) return bail(fail(FEDBM_EINVAL, "need dt > 0 or cfl > 0"));
    if (cd[c].mesh.order < 0 || cd[c].mesh.order > kMaxOrder) return bail(fail(FEDBM_EINVAL, "order must be in 0..6"));
    Case cs;
    cs.md = cd[c].mesh;
    cs.vd = cd[c].velset;
    cs.prm = prm;
    int gi = -1;
    for (int j = 0; j < int(b->groups.size()); ++j)
      if (same_group(b->groups[j], cs.md, cs.vd, cs.prm)) gi = j;
    if (gi < 0) {
      Group g;
      g.p = cs.md.order;
      g.store = prm.precision;
      g.vd = cs.vd;
      g.collision = prm.collision;
      g.reduction = prm.reduction;
      g.beta = prm.beta;
      g.epc = prm.elems_per_cta;
      g.tpb = prm.threads_per_cta;
      g.nstages = prm.pipeline_stages;
      g.test_wait_timeout = prm.test_wait_timeout;
      g.tc_mode = prm.tensor_cores;
      g.vsplit = prm.velocity_split;
      g.rounding = prm.rounding;
      b->groups.push_back(g);
      gi = int(b->groups.size()) - 1;
    }
    cs.group = gi;
    b->groups[gi].cases.push_back(c);
    b->cases.push_back(cs);
  }
  int rc = FEDBM_OK;
  if ((rc = [&]() -> int {
         FEDBM_CK(cudaGetDevice(&b->device));
         int r = ensure_ops_uploaded(b->device);
         if (r != FEDBM_OK) return r;
         FEDBM_CK(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
         for (Group& g : b->groups) {
           const int epc = g.epc, tpb = g.tpb, st = g.nstages;
           if ((r = build_group(*b, g)) != FEDBM_OK) return r;
           // default: the FMA kernel for every form, as its warp-specialised
           // variant where ws_default says so (with its compile-time operator
           // tables it measured faster than the tensor-core form on FP32 state
           // too, 2.52e11 vs 2.04e11-2.20e11 DOF-stage/s at 256 velocities;
           // the 16-bit forms, 1024 velocities, stacked 16-velocity tiles and
           // degree 5 likewise); tensor cores on request (tensor_cores = 1) or
           // when the autotuner times them faster
           const bool want_tc = g.tc_mode > 0;
           // the velocity-split form on request, or when one CTA cannot hold
           // an element's velocities (automatic mode)
           const bool too_big = stage_smem_bytes(g.p, g.store, std::max(1, epc), g.Qp, 1) > kMaxSmem;
           const int ncl = g.vsplit >= 2 ? g.vsplit : (g.vsplit == 0 && too_big && !want_tc ? auto_cluster(g) : 0);
           if (ncl >= 2) {
             if ((r = configure_cluster(*b, g, ncl)) != FEDBM_OK) return r;
           } else if (want_tc) {
             if ((r = configure_tc(*b, g)) != FEDBM_OK) return r;
           } else if (epc == 0 && tpb == 0 && st == 0 && g.vsplit <= 1 && ws_default(g)) {
             if ((r = configure_ws(*b, g)) != FEDBM_OK) return r;
           } else if ((r = configure_tiles(*b, g, epc, tpb, st)) != FEDBM_OK) {
             return r;
           }
         }
         return FEDBM_OK;
       }()) != FEDBM_OK)
    return bail(rc);
  *out = b;
  return FEDBM_OK;
}

int check_batch(const Batch* b, int c) {
  if (!b) return fail(FEDBM_EINVAL, "null handle");
  if (c < 0 || c >= int(b->cases.size())) return fail(FEDBM_EINVAL, "case index out of range");
  FEDBM_CK(cudaSetDevice(b->device));
  return FEDBM_OK;
}

int ensure_staging(Batch& b, size_t elems) {
  if (b.staging_elems < elems) {
    cudaFree(b.staging);
    b.staging = nullptr;
    b.staging_elems = 0;
    FEDBM_CK(cudaMalloc(&b.staging, elems * sizeof(double)));
    b.staging_elems = elems;
  }
  return FEDBM_OK;
}

// Queue a copy of the group's stage-kernel timeout word into *word (host);
// read it after the stream has been synchronised.
int queue_timeout_read(const Batch& b, const Group& g, int* word) {
  FEDBM_CK(cudaMemcpyAsync(word, g.flag + 1, sizeof(int), cudaMemcpyDeviceToHost, b.stream));
  return FEDBM_OK;
}

int timeout_status(int word) {
  return word ? fail(FEDBM_ETIMEOUT, "a stage kernel's bounded wait for its tile copies gave up; the state is "
                                     "partly updated (load a new state to clear this)")
              : FEDBM_OK;
}

// canonical FP64 (device) -> internal state of case c
template <typename TIn>
int encode_case(Batch& b, int c, const TIn* src) {
  const Case& cs = b.cases[c];
  const Group& g = b.groups[cs.group];
  const size_t off = size_t(cs.k_off) * g.Np * g.Qp;
  float* sc = g.scale[b.cur] ? g.scale[b.cur] + cs.k_off : nullptr;
  const int blk = 256;
  switch (g.store) {
    case kStoreF64: encode_kernel<StoreF64, TIn><<<int(cs.K), blk, 0, b.stream>>>(src, static_cast<double*>(g.f[b.cur]) + off, nullptr, g.vel64, g.iperm, g.Np, g.Q, g.Qp); break;
    case kStoreF32: encode_kernel<StoreF32, TIn><<<int(cs.K), blk, 0, b.stream>>>(src, static_cast<float*>(g.f[b.cur]) + off, nullptr, g.vel64, g.iperm, g.Np, g.Q, g.Qp); break;
    case kStoreBF16: encode_kernel<StoreBF16, TIn><<<int(cs.K), blk, 0, b.stream>>>(src, static_cast<__nv_bfloat16*>(g.f[b.cur]) + off, sc, g.vel64, g.iperm, g.Np, g.Q, g.Qp); break;
    default: encode_kernel<StoreF16, TIn><<<int(cs.K), blk, 0, b.stream>>>(src, static_cast<__half*>(g.f[b.cur]) + off, sc, g.vel64, g.iperm, g.Np, g.Q, g.Qp); break;
  }
  FEDBM_CK(cudaGetLastError());
  // a new state starts with a clear stage-kernel timeout word (and the
  // stochastic-rounding draws from step 0)
  FEDBM_CK(cudaMemsetAsync(g.flag + 1, 0, sizeof(int), b.stream));
  if (g.sr_step) FEDBM_CK(cudaMemsetAsync(g.sr_step, 0, sizeof(uint32_t), b.stream));
  b.time = 0;
  b.steps = 0;
  return FEDBM_OK;
}

// canonical state (FP64, or FP32 for fedbm_set_state_f32) -> internal state
template <typename TIn>
int set_state(Batch& b, int c, const TIn* f, int on_device) {
  NvtxRange nvtx("fedbm set_state");
  if (!f) return fail(FEDBM_EINVAL, "null state pointer");
  const Case& cs = b.cases[c];
  const Group& g = b.groups[cs.group];
  const size_t n = size_t(cs.K) * g.Np * g.Q;
  const TIn* src = f;
  if (!on_device) {
    int rc = ensure_staging(b, n);  // n doubles hold n values of either type
    if (rc) return rc;
    FEDBM_CK(cudaMemcpyAsync(b.staging, f, n * sizeof(TIn), cudaMemcpyHostToDevice, b.stream));
    src = reinterpret_cast<const TIn*>(b.staging);
  }
  int rc = encode_case(b, c, src);
  if (rc) return rc;
  if (!on_device) FEDBM_CK(cudaStreamSynchronize(b.stream));
  return FEDBM_OK;
}

int set_equilibrium(Batch& b, int c, double rho0, double ux0, double uy0, double amp, uint64_t seed) {
  const Case& cs = b.cases[c];
  const Group& g = b.groups[cs.group];
  const int64_t n = cs.K * g.Np * g.Q;
  int rc = ensure_staging(b, size_t(n));
  if (rc) return rc;
  equilibrium_kernel<<<grid_for(n, 256), 256, 0, b.stream>>>(b.staging, g.vel64, g.iperm, cs.K, g.Np, g.Q, g.Qp, rho0, ux0, uy0,
                                                             amp, seed, g.vd.eq_order);
  FEDBM_CK(cudaGetLastError());
  return encode_case(b, c, static_cast<const double*>(b.staging));
}

template <class ST>
void launch_decode(const Group& g, int cur, const Case& cs, double* dst, cudaStream_t st) {
  using S = typename ST::S;
  const int64_t n = cs.K * g.Np * g.Q;
  const S* in = static_cast<const S*>(g.f[cur]) + size_t(cs.k_off) * g.Np * g.Qp;
  const float* sc = g.scale[cur] ? g.scale[cur] + cs.k_off : nullptr;
  decode_kernel<ST><<<grid_for(n, 256), 256, 0, st>>>(in, sc, dst, g.vel64, g.iperm, cs.K, g.Np, g.Q, g.Qp);
}

int get_state(Batch& b, int c, double* f, int on_device) {
  NvtxRange nvtx("fedbm get_state");
  if (!f) return fail(FEDBM_EINVAL, "null output");
  const Case& cs = b.cases[c];
  const Group& g = b.groups[cs.group];
  const size_t n = size_t(cs.K) * g.Np * g.Q;
  double* dst = f;
  if (!on_device) {
    int rc = ensure_staging(b, n);
    if (rc) return rc;
    dst = b.staging;
  }
  switch (g.store) {
    case kStoreF64: launch_decode<StoreF64>(g, b.cur, cs, dst, b.stream); break;
    case kStoreF32: launch_decode<StoreF32>(g, b.cur, cs, dst, b.stream); break;
    case kStoreBF16: launch_decode<StoreBF16>(g, b.cur, cs, dst, b.stream); break;
    default: launch_decode<StoreF16>(g, b.cur, cs, dst, b.stream); break;
  }
  FEDBM_CK(cudaGetLastError());
  if (!on_device) {
    int word = 0;
    FEDBM_CK(cudaMemcpyAsync(f, dst, n * sizeof(double), cudaMemcpyDeviceToHost, b.stream));
    int rc = queue_timeout_read(b, g, &word);
    if (rc) return rc;
    FEDBM_CK(cudaStreamSynchronize(b.stream));
    return timeout_status(word);
  }
  return FEDBM_OK;
}

int get_residual(Batch& b, int c, double* r, int on_device) {
  if (!r) return fail(FEDBM_EINVAL, "null output");
  const Case& cs = b.cases[c];
  const Group& g = b.groups[cs.group];
  const int64_t n = cs.K * g.Np * g.Q;
  double* dst = r;
  if (!on_device) {
    int rc = ensure_staging(b, size_t(n));
    if (rc) return rc;
    dst = b.staging;
  }
  const size_t off = size_t(cs.k_off) * g.Np * g.Qp;
  if (g.store == kStoreF64)
    decode_residual_kernel<double><<<grid_for(n, 256), 256, 0, b.stream>>>(static_cast<const double*>(g.res) + off, g.iperm, dst, cs.K, g.Np, g.Q, g.Qp);
  else
    decode_residual_kernel<float><<<grid_for(n, 256), 256, 0, b.stream>>>(static_cast<const float*>(g.res) + off, g.iperm, dst, cs.K, g.Np, g.Q, g.Qp);
  FEDBM_CK(cudaGetLastError());
  if (!on_device) {
    FEDBM_CK(cudaMemcpyAsync(r, dst, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, b.stream));
    FEDBM_CK(cudaStreamSynchronize(b.stream));
  }
  return FEDBM_OK;
}

template <class ST>
void launch_moments(const Group& g, int cur, const Case& cs, double* r, double* x, double* y, cudaStream_t st) {
  using S = typename ST::S;
  const int64_t nodes = cs.K * g.Np;
  const S* in = static_cast<const S*>(g.f[cur]) + size_t(cs.k_off) * g.Np * g.Qp;
  const float* sc = g.scale[cur] ? g.scale[cur] + cs.k_off : nullptr;
  using R = typename ST::R;
  moments_kernel<ST><<<grid_for(nodes * 32, 256), 256, 0, st>>>(in, sc, static_cast<const R*>(g.vel), cs.K, g.Np,
                                                                  g.Qp, r, x, y);
}

int get_moments(Batch& b, int c, double* rho, double* ux, double* uy, int on_device) {
  NvtxRange nvtx("fedbm get_moments");
  const Case& cs = b.cases[c];
  const Group& g = b.groups[cs.group];
  const int64_t nodes = cs.K * g.Np;
  double *dr = rho, *dx = ux, *dy = uy;
  if (!on_device) {
    if (b.mom_elems < size_t(3 * nodes)) {
      cudaFree(b.mom);
      b.mom = nullptr;
      b.mom_elems = 0;
      FEDBM_CK(cudaMalloc(&b.mom, size_t(3) * nodes * sizeof(double)));
      b.mom_elems = size_t(3) * nodes;
    }
    dr = b.mom;
    dx = b.mom + nodes;
    dy = b.mom + 2 * nodes;
  } else if (!rho || !ux || !uy) {
    return fail(FEDBM_EINVAL, "device moments need three output pointers");
  }
  switch (g.store) {
    case kStoreF64: launch_moments<StoreF64>(g, b.cur, cs, dr, dx, dy, b.stream); break;
    case kStoreF32: launch_moments<StoreF32>(g, b.cur, cs, dr, dx, dy, b.stream); break;
    case kStoreBF16: launch_moments<StoreBF16>(g, b.cur, cs, dr, dx, dy, b.stream); break;
    default: launch_moments<StoreF16>(g, b.cur, cs, dr, dx, dy, b.stream); break;
  }
  FEDBM_CK(cudaGetLastError());
  if (!on_device) {
    const size_t bytes = size_t(nodes) * sizeof(double);
    if (rho) FEDBM_CK(cudaMemcpyAsync(rho, dr, bytes, cudaMemcpyDeviceToHost, b.stream));
    if (ux) FEDBM_CK(cudaMemcpyAsync(ux, dx, bytes, cudaMemcpyDeviceToHost, b.stream));
    if (uy) FEDBM_CK(cudaMemcpyAsync(uy, dy, bytes, cudaMemcpyDeviceToHost, b.stream));
    int word = 0;
    int rc = queue_timeout_read(b, g, &word);
    if (rc) return rc;
    FEDBM_CK(cudaStreamSynchronize(b.stream));
    return timeout_status(word);
  }
  return FEDBM_OK;
}

template <class ST>
void launch_mass(const Group& g, int cur, const Case& cs, int blocks, cudaStream_t st) {
  using S = typename ST::S;
  const S* in = static_cast<const S*>(g.f[cur]) + size_t(cs.k_off) * g.Np * g.Qp;
  const float* sc = g.scale[cur] ? g.scale[cur] + cs.k_off : nullptr;
  mass_partial_kernel<ST><<<blocks, kMassThreads, 0, st>>>(in, sc, g.vel64 + 2 * g.Qp, g.Jk + cs.k_off, g.mw, cs.K,
                                                           g.Np, g.Qp, g.partial, g.flag);
}

int mass(Batch& b, int c, double* total) {
  NvtxRange nvtx("fedbm mass");
  if (!total) return fail(FEDBM_EINVAL, "null output");
  const Case& cs = b.cases[c];
  const Group& g = b.groups[cs.group];
  FEDBM_CK(cudaMemsetAsync(g.flag, 0, sizeof(int), b.stream));
  const int64_t nodes = cs.K * g.Np;
  const int blocks = int(std::min<int64_t>(kMassBlocks, (nodes * 32 + kMassThreads - 1) / kMassThreads));
  switch (g.store) {
    case kStoreF64: launch_mass<StoreF64>(g, b.cur, cs, blocks, b.stream); break;
    case kStoreF32: launch_mass<StoreF32>(g, b.cur, cs, blocks, b.stream); break;
    case kStoreBF16: launch_mass<StoreBF16>(g, b.cur, cs, blocks, b.stream); break;
    default: launch_mass<StoreF16>(g, b.cur, cs, blocks, b.stream); break;
  }
  FEDBM_CK(cudaGetLastError());
  mass_final_kernel<<<1, 256, 0, b.stream>>>(g.partial, blocks, g.partial + kMassBlocks);
  FEDBM_CK(cudaGetLastError());
  int flag[2] = {0, 0};
  FEDBM_CK(cudaMemcpyAsync(total, g.partial + kMassBlocks, sizeof(double), cudaMemcpyDeviceToHost, b.stream));
  FEDBM_CK(cudaMemcpyAsync(flag, g.flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, b.stream));
  FEDBM_CK(cudaStreamSynchronize(b.stream));
  if (flag[1]) return timeout_status(flag[1]);
  if (flag[0]) return fail(FEDBM_ENONFINITE, "state has a non-finite value or a node with rho <= 0");
  return FEDBM_OK;
}

int rk_step(Batch& b, int nsteps) {
  NvtxRange nvtx("fedbm rk_step");
  if (nsteps < 0) return fail(FEDBM_EINVAL, "nsteps must be >= 0");
  int rc = build_graphs(b);
  if (rc) return rc;
  for (int n = 0; n < nsteps; ++n) {
    FEDBM_CK(cudaGraphLaunch(b.graph[b.cur], b.stream));
    b.cur = 1 - b.cur;  // five stages: the state ends in the other buffer
    b.steps += 1;
  }
  return FEDBM_OK;
}

int info(const Batch& b, int c, fedbm_info_t* out) {
  if (!out) return fail(FEDBM_EINVAL, "null output");
  const Case& cs = b.cases[c];
  const Group& g = b.groups[cs.group];
  out->K = cs.K;
  out->Np = g.Np;
  out->Nfp = g.Nfp;
  out->Q = g.Q;
  out->Q_padded = g.Qp;
  out->dt = cs.dt;
  out->tau = cs.tau;
  out->time = cs.dt * double(b.steps) + b.time;
  out->steps = b.steps;
  out->precision = g.store;
  out->reduction = g.reduction;
  out->order = g.p;
  out->eq_order = g.vd.eq_order;
  out->elems_per_cta = g.epc;
  out->threads_per_cta = g.tpb;
  out->pipeline_stages = g.nstages;
  out->grid = g.grid;
  out->group = cs.group;
  out->ngroups = int32_t(b.groups.size());
  out->tensor_cores = g.tc;
  out->velocity_split = g.ncl > 1 ? g.ncl : 1;
  out->state_bytes = cs.K * g.Np * g.Qp * int64_t(store_bytes(g.store));
  out->residual_bytes = cs.K * g.Np * g.Qp * int64_t(real_bytes(g.store));
  return FEDBM_OK;
}

// ---------------------------------------------------------------- implicit time marching
// SDIRK methods with matrix-free Newton-GMRES (Sec. II.B.3: the paper marches
// with SDIRK, a four-stage fourth-order scheme for the Couette order study and
// backward Euler for the cavities, each stage linearised by Newton and solved
// by GMRES).  Every residual evaluation R(Y) is one launch of the fused stage
// kernel with A = B = 0 and a unit time step in its geometry copy (so that its
// residual register receives R(Y) itself); Jacobian-vector products are finite
// differences of R; all vectors are FP64 in the internal layout [K][Np][Qp].

struct Tableau {
  int s = 0;
  double A[6][6] = {};
  double b[6] = {};
};

bool make_tableau(const fedbm_implicit_params& ip, Tableau& t, std::string& err) {
  switch (ip.scheme) {
    case FEDBM_IMPLICIT_BE:  // backward Euler: one stage, first order
      t.s = 1;
      t.A[0][0] = 1.0;
      t.b[0] = 1.0;
      return true;
    case FEDBM_IMPLICIT_SDIRK3_O4: {
      // Crouzeix (1975) / Norsett: three stages, fourth order, A-stable,
      // gamma = 1/2 + cos(pi/18)/sqrt(3), delta = 1 / (6 (2 gamma - 1)^2)
      const double g = 0.5 + std::cos(3.14159265358979323846 / 18.0) / std::sqrt(3.0);
      const double d = 1.0 / (6.0 * (2.0 * g - 1.0) * (2.0 * g - 1.0));
      t.s = 3;
      t.A[0][0] = g;
      t.A[1][0] = 0.5 - g;
      t.A[1][1] = g;
      t.A[2][0] = 2.0 * g;
      t.A[2][1] = 1.0 - 4.0 * g;
      t.A[2][2] = g;
      t.b[0] = d;
      t.b[1] = 1.0 - 2.0 * d;
      t.b[2] = d;
      return true;
    }
    case FEDBM_IMPLICIT_SDIRK5_O4: {
      // Hairer & Wanner (Solving ODEs II, Sec. IV.6): five stages, fourth
      // order, L-stable, gamma = 1/4, stiffly accurate (b = last row)
      const double A[5][5] = {{1.0 / 4, 0, 0, 0, 0},
                              {1.0 / 2, 1.0 / 4, 0, 0, 0},
                              {17.0 / 50, -1.0 / 25, 1.0 / 4, 0, 0},
                              {371.0 / 1360, -137.0 / 2720, 15.0 / 544, 1.0 / 4, 0},
                              {25.0 / 24, -49.0 / 48, 125.0 / 16, -85.0 / 12, 1.0 / 4}};
      t.s = 5;
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) t.A[i][j] = A[i][j];
      for (int j = 0; j < 5; ++j) t.b[j] = A[4][j];
      return true;
    }
    case FEDBM_IMPLICIT_CUSTOM: {
      if (ip.stages < 1 || ip.stages > 6) {
        err = "custom tableau: stages must be 1..6";
        return false;
      }
      t.s = ip.stages;
      const double gam = ip.A[0];
      if (!(gam > 0)) {
        err = "custom tableau: the diagonal must be positive";
        return false;
      }
      for (int i = 0; i < t.s; ++i) {
        for (int j = 0; j < t.s; ++j) {
          const double v = ip.A[i * 6 + j];
          if (j > i && v != 0.0) {
            err = "custom tableau: A must be lower triangular";
            return false;
          }
          if (j == i && v != gam) {
            err = "custom tableau: every diagonal entry must equal A[0][0] (singly diagonally implicit)";
            return false;
          }
          t.A[i][j] = v;
        }
        t.b[i] = ip.b[i];
      }
      return true;
    }
  }
  err = "unknown implicit scheme";
  return false;
}

// Device work space of the implicit solver of a single-group solver.
struct Implicit {
  int64_t n = 0;        // K * Np * Qp
  int m = 0, s = 0;     // GMRES restart length, stages
  double* u0 = nullptr;     // state at the start of the step
  double* Y = nullptr;      // stage value (Newton iterate)
  double* base = nullptr;   // u0 + dt sum_{j<i} a_ij k_j
  double* RY = nullptr;     // R(Y)
  double* G = nullptr;      // Newton residual, then the GMRES right-hand side -G
  double* d = nullptr;      // Newton update
  double* w = nullptr;      // GMRES work vector
  double* Yp = nullptr;     // Y + eps v
  double* Rp = nullptr;     // R(Y + eps v)
  double* V = nullptr;      // GMRES basis [m+1][n]
  double* k = nullptr;      // stage derivatives [s][n]
  double* partial = nullptr;  // [m+1][kDotBlocks]
  double* hdev = nullptr;     // [m+2] dot results / combination coefficients
  void* x32 = nullptr;        // FP32 state: FP32 copy of the input of R
  void* r32 = nullptr;        // FP32 state: FP32 residual register
  void* scratch = nullptr;    // stage-kernel state output (unused values)
  void* geo_unit = nullptr;   // geometry with dt = 1
  // element-and-velocity block-Jacobi preconditioner (right preconditioning)
  double* minv = nullptr;     // [K][Np][Np][Qp] block inverses of (I - dt gamma J)
  double* z = nullptr;        // M^-1 v
  double* ops = nullptr;      // FP64 Dr | Ds | LIFT of the degree
  int* fmask = nullptr;       // [3][Nfp]
  double minv_dtg = 0;        // dt gamma the inverses were built for (0 = none)
};

void free_implicit(Implicit& im) {
  void* bufs[] = {im.u0, im.Y, im.base, im.RY, im.G, im.d, im.w, im.Yp, im.Rp, im.V, im.k, im.partial, im.hdev,
                  im.x32, im.r32, im.scratch, im.geo_unit, im.minv, im.z, im.ops, im.fmask};
  for (void* p : bufs) cudaFree(p);
  im = Implicit();
}

int ensure_implicit(const Batch& b, const Group& g, Implicit& im, int m, int s) {
  const int64_t n = g.K * g.Np * g.Qp;
  if (im.n == n && im.m >= m && im.s >= s) return FEDBM_OK;
  free_implicit(im);
  im.n = n;
  im.m = m;
  im.s = s;
  const size_t vb = size_t(n) * sizeof(double);
  double** vecs[] = {&im.u0, &im.Y, &im.base, &im.RY, &im.G, &im.d, &im.w, &im.Yp, &im.Rp};
  for (double** v : vecs) FEDBM_CK(cudaMalloc(v, vb));
  FEDBM_CK(cudaMalloc(&im.V, vb * size_t(m + 1)));
  FEDBM_CK(cudaMalloc(&im.k, vb * size_t(s)));
  FEDBM_CK(cudaMalloc(&im.partial, size_t(m + 1) * krylov::kDotBlocks * sizeof(double)));
  FEDBM_CK(cudaMalloc(&im.hdev, size_t(m + 2) * sizeof(double)));
  const size_t rb = real_bytes(g.store);
  FEDBM_CK(cudaMalloc(&im.scratch, size_t(n) * rb));
  if (g.store == kStoreF32) {
    FEDBM_CK(cudaMalloc(&im.x32, size_t(n) * 4));
    FEDBM_CK(cudaMalloc(&im.r32, size_t(n) * 4));
  }
  FEDBM_CK(cudaMalloc(&im.geo_unit, size_t(g.K) * kGeoStrideDev * rb));
  FEDBM_CK(cudaMemcpyAsync(im.geo_unit, g.geo, size_t(g.K) * kGeoStrideDev * rb, cudaMemcpyDeviceToDevice, b.stream));
  FEDBM_CK(krylov::set_geo_dt(g.K, kGeoStrideDev, kGeoDt, 1.0, im.geo_unit, int(rb), b.stream));
  return FEDBM_OK;
}

// The block-Jacobi inverses for this dt gamma (built on first use, rebuilt
// when dt gamma changes).
int ensure_block_jacobi(const Batch& b, const Group& g, Implicit& im, double dtg) {
  if (im.minv && im.minv_dtg == dtg) return FEDBM_OK;
  if (!im.minv) {
    FEDBM_CK(cudaMalloc(&im.minv, size_t(im.n) * g.Np * sizeof(double)));
    FEDBM_CK(cudaMalloc(&im.z, size_t(im.n) * sizeof(double)));
    std::vector<double> ops(g.ops.Dr);
    ops.insert(ops.end(), g.ops.Ds.begin(), g.ops.Ds.end());
    ops.insert(ops.end(), g.ops.LIFT.begin(), g.ops.LIFT.end());
    int rc = upload_vec(ops, reinterpret_cast<void**>(&im.ops));
    if (rc) return rc;
    if ((rc = upload_vec(g.ops.fmask, reinterpret_cast<void**>(&im.fmask))) != FEDBM_OK) return rc;
  }
  FEDBM_CK(krylov::block_jacobi_build(g.K, g.Np, g.Nfp, g.Qp, g.geo, int(real_bytes(g.store)), g.vel64, im.ops,
                                      im.fmask, dtg, 2.0 * g.beta - 1.0, im.minv, b.stream));
  im.minv_dtg = dtg;
  return FEDBM_OK;
}

// r = R(x): one fused stage-kernel launch with A = B = 0 and unit time step
int implicit_rhs(const Batch& b, const Group& g, Implicit& im, const double* x, double* r) {
  if (g.store == kStoreF64) {
    StageArgs<double> a;
    fill_stage_args(g, 0, b.cur, a);
    a.f_in = x;
    a.f_out = im.scratch;
    a.res = r;
    a.geo = static_cast<const double*>(im.geo_unit);
    a.rkA = 0.0;
    a.rkB = 0.0;
    FEDBM_CK(launch_args(g, &a, b.stream));
    return FEDBM_OK;
  }
  FEDBM_CK(krylov::to_f32(im.n, x, static_cast<float*>(im.x32), b.stream));
  StageArgs<float> a;
  fill_stage_args(g, 0, b.cur, a);
  a.f_in = im.x32;
  a.f_out = im.scratch;
  a.res = static_cast<float*>(im.r32);
  a.geo = static_cast<const float*>(im.geo_unit);
  a.rkA = 0.f;
  a.rkB = 0.f;
  FEDBM_CK(launch_args(g, &a, b.stream));
  FEDBM_CK(krylov::to_f64(im.n, static_cast<const float*>(im.r32), r, b.stream));
  return FEDBM_OK;
}

// 2-norm of x (synchronous)
int implicit_norm(const Batch& b, Implicit& im, const double* x, double* out) {
  FEDBM_CK(krylov::multi_dot(im.n, 1, x, x, im.partial, im.hdev, b.stream));
  double h = 0;
  FEDBM_CK(cudaMemcpyAsync(&h, im.hdev, sizeof(double), cudaMemcpyDeviceToHost, b.stream));
  FEDBM_CK(cudaStreamSynchronize(b.stream));
  *out = std::sqrt(std::max(0.0, h));
  return FEDBM_OK;
}

struct ImplicitCounters {
  int newton = 0, gmres = 0, rhs = 0;
  double residual = 0;
  bool converged = true;
};

// Restarted GMRES(m) for (I - dt gamma J) d = rhs (rhs in im.G), x0 = 0,
// classical Gram-Schmidt with one re-orthogonalisation; J v is taken as
// (R(Y + eps v) - R(Y)) / eps.  Stops when the residual is <= tol.
int implicit_gmres(const Batch& b, const Group& g, Implicit& im, double dtg, double eps, double tol, int max_iter,
                   bool precond, ImplicitCounters& cnt) {
  const int64_t n = im.n;
  const int m = im.m;
  cudaStream_t st = b.stream;
  FEDBM_CK(cudaMemsetAsync(im.d, 0, size_t(n) * sizeof(double), st));
  std::vector<double> H(size_t(m + 1) * m, 0.0), cs(m), sn(m), gv(m + 1), y(m), h1(m + 1), h2(m + 1);
  int total = 0;
  bool first = true;
  while (total < max_iter) {
    // r = rhs - A d  (d = 0 on the first cycle)
    double* v0 = im.V;
    if (first) {
      FEDBM_CK(cudaMemcpyAsync(v0, im.G, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      // A d = d - dtg (R(Y + e d) - R(Y)) / e, e = eps / |d| (a unit-size difference)
      double dn = 0;
      int rc = implicit_norm(b, im, im.d, &dn);
      if (rc) return rc;
      const double ed = dn > 0 ? eps / dn : eps;
      FEDBM_CK(krylov::axpby(n, 1.0, im.Y, ed, im.d, im.Yp, st));
      if ((rc = implicit_rhs(b, g, im, im.Yp, im.Rp)) != FEDBM_OK) return rc;
      ++cnt.rhs;
      FEDBM_CK(krylov::axpby(n, 1.0, im.Rp, -1.0, im.RY, im.w, st));
      FEDBM_CK(krylov::axpby(n, 1.0, im.d, -dtg / ed, im.w, im.w, st));
      FEDBM_CK(krylov::axpby(n, 1.0, im.G, -1.0, im.w, v0, st));
    }
    first = false;
    double beta = 0;
    int rc = implicit_norm(b, im, v0, &beta);
    if (rc) return rc;
    if (beta <= tol) return FEDBM_OK;
    FEDBM_CK(krylov::axpby(n, 1.0 / beta, v0, 0.0, v0, v0, st));
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int jend = 0;
    double resid = beta;
    for (int j = 0; j < m && total < max_iter; ++j, ++total) {
      double* vj = im.V + size_t(j) * n;
      // w = A M^-1 v_j (right preconditioning; M = I without a preconditioner)
      const double* xj = vj;
      double ex = eps;
      if (precond) {
        FEDBM_CK(krylov::block_jacobi_apply(g.K, g.Np, g.Qp, im.minv, vj, im.z, st));
        double zn = 0;
        if ((rc = implicit_norm(b, im, im.z, &zn)) != FEDBM_OK) return rc;
        xj = im.z;
        ex = zn > 0 ? eps / zn : eps;
      }
      FEDBM_CK(krylov::axpby(n, 1.0, im.Y, ex, xj, im.Yp, st));
      if ((rc = implicit_rhs(b, g, im, im.Yp, im.Rp)) != FEDBM_OK) return rc;
      ++cnt.rhs;
      FEDBM_CK(krylov::axpby(n, 1.0, im.Rp, -1.0, im.RY, im.w, st));
      FEDBM_CK(krylov::axpby(n, 1.0, xj, -dtg / ex, im.w, im.w, st));
      // two passes of classical Gram-Schmidt against v_0 .. v_j
      for (int pass = 0; pass < 2; ++pass) {
        std::vector<double>& hh = pass == 0 ? h1 : h2;
        FEDBM_CK(krylov::multi_dot(n, j + 1, im.V, im.w, im.partial, im.hdev, st));
        FEDBM_CK(krylov::sub_combination(n, j + 1, im.V, im.hdev, im.w, st));
        FEDBM_CK(cudaMemcpyAsync(hh.data(), im.hdev, size_t(j + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
      }
      double hn = 0;
      if ((rc = implicit_norm(b, im, im.w, &hn)) != FEDBM_OK) return rc;  // synchronises: h1, h2 are valid
      ++cnt.gmres;
      for (int i = 0; i <= j; ++i) H[size_t(i) * m + j] = h1[i] + h2[i];
      H[size_t(j + 1) * m + j] = hn;
      if (j + 1 <= m && hn > 0)
        FEDBM_CK(krylov::axpby(n, 1.0 / hn, im.w, 0.0, im.w, im.V + size_t(j + 1) * n, st));
      // Givens rotations
      for (int i = 0; i < j; ++i) {
        const double a0 = H[size_t(i) * m + j], a1 = H[size_t(i + 1) * m + j];
        H[size_t(i) * m + j] = cs[i] * a0 + sn[i] * a1;
        H[size_t(i + 1) * m + j] = -sn[i] * a0 + cs[i] * a1;
      }
      const double a0 = H[size_t(j) * m + j], a1 = H[size_t(j + 1) * m + j];
      const double r = std::hypot(a0, a1);
      cs[j] = r > 0 ? a0 / r : 1.0;
      sn[j] = r > 0 ? a1 / r : 0.0;
      H[size_t(j) * m + j] = r;
      H[size_t(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      resid = std::fabs(gv[j + 1]);
      jend = j + 1;
      if (resid <= tol || hn == 0.0) {
        ++total;
        break;
      }
    }
    // y = H^-1 g (upper triangular jend x jend), d += V y
    for (int i = jend - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int q = i + 1; q < jend; ++q) acc -= H[size_t(i) * m + q] * y[q];
      y[i] = H[size_t(i) * m + i] != 0.0 ? acc / H[size_t(i) * m + i] : 0.0;
    }
    FEDBM_CK(cudaMemcpyAsync(im.hdev, y.data(), size_t(jend) * sizeof(double), cudaMemcpyHostToDevice, st));
    if (precond) {  // d += M^-1 (V y)
      FEDBM_CK(cudaMemsetAsync(im.w, 0, size_t(n) * sizeof(double), st));
      FEDBM_CK(krylov::add_combination(n, jend, im.V, im.hdev, im.w, st));
      FEDBM_CK(krylov::block_jacobi_apply(g.K, g.Np, g.Qp, im.minv, im.w, im.z, st));
      FEDBM_CK(krylov::axpby(n, 1.0, im.d, 1.0, im.z, im.d, st));
    } else {
      FEDBM_CK(krylov::add_combination(n, jend, im.V, im.hdev, im.d, st));
    }
    FEDBM_CK(cudaStreamSynchronize(st));  // y (host) is reused by the next cycle
    if (resid <= tol) return FEDBM_OK;
  }
  return FEDBM_OK;  // the caller's Newton loop judges the outcome
}

void free_implicit_of(Batch* b) {
  if (b->implicit) {
    free_implicit(*b->implicit);
    delete b->implicit;
    b->implicit = nullptr;
  }
}

int implicit_step(Batch& b, const fedbm_implicit_params& ip, int nsteps, fedbm_implicit_stats* stats) {
  NvtxRange nvtx("fedbm implicit_step");
  if (b.groups.size() != 1 || b.cases.size() != 1)
    return fail(FEDBM_EINVAL, "implicit stepping serves single solvers (one case)");
  Group& g = b.groups[0];
  if (g.store != kStoreF64 && g.store != kStoreF32)
    return fail(FEDBM_EINVAL, "implicit stepping needs FP64 or FP32 state");
  if (nsteps < 0) return fail(FEDBM_EINVAL, "nsteps must be >= 0");
  if (!(ip.dt > 0)) return fail(FEDBM_EINVAL, "implicit dt must be > 0");
  Tableau tb;
  std::string err;
  if (!make_tableau(ip, tb, err)) return fail(FEDBM_EINVAL, err);
  const int m = ip.gmres_restart > 0 ? std::min(ip.gmres_restart, 200) : 30;
  const int gmax = ip.gmres_max_iter > 0 ? ip.gmres_max_iter : 1000;
  const int nmax = ip.newton_max_iter > 0 ? ip.newton_max_iter : 20;
  const double rtol = ip.newton_rtol > 0 ? ip.newton_rtol : 1e-10;
  const double atol = ip.newton_atol > 0 ? ip.newton_atol : 0.0;
  const double eta = ip.gmres_rtol > 0 ? ip.gmres_rtol : 1e-4;
  if (!b.implicit) b.implicit = new Implicit();
  Implicit* im = b.implicit;
  int rc = ensure_implicit(b, g, *im, m, tb.s);
  if (rc) return rc;
  const int64_t n = im->n;
  cudaStream_t st = b.stream;
  const double eps_mach = g.store == kStoreF64 ? 2.220446049250313e-16 : 1.1920929e-07;
  const double dt = ip.dt;
  const double dtg = dt * tb.A[0][0];
  if (ip.preconditioner < 0 || ip.preconditioner > 1) return fail(FEDBM_EINVAL, "unknown preconditioner");
  const bool precond = ip.preconditioner == 1;
  if (precond && (rc = ensure_block_jacobi(b, g, *im, dtg)) != FEDBM_OK) return rc;
  ImplicitCounters cnt;
  const size_t vb = size_t(n) * sizeof(double);
  for (int step = 0; step < nsteps; ++step) {
    // u0 = current state in FP64
    if (g.store == kStoreF64) FEDBM_CK(cudaMemcpyAsync(im->u0, g.f[b.cur], vb, cudaMemcpyDeviceToDevice, st));
    else FEDBM_CK(krylov::to_f64(n, static_cast<const float*>(g.f[b.cur]), im->u0, st));
    for (int i = 0; i < tb.s; ++i) {
      // base = u0 + dt sum_{j<i} a_ij k_j
      FEDBM_CK(cudaMemcpyAsync(im->base, im->u0, vb, cudaMemcpyDeviceToDevice, st));
      if (i > 0) {
        std::vector<double> c(i);
        for (int j = 0; j < i; ++j) c[j] = dt * tb.A[i][j];
        FEDBM_CK(cudaMemcpyAsync(im->hdev, c.data(), size_t(i) * sizeof(double), cudaMemcpyHostToDevice, st));
        FEDBM_CK(krylov::add_combination(n, i, im->k, im->hdev, im->base, st));
        FEDBM_CK(cudaStreamSynchronize(st));
      }
      // initial guess: the previous stage value (or u0)
      if (i == 0) FEDBM_CK(cudaMemcpyAsync(im->Y, im->u0, vb, cudaMemcpyDeviceToDevice, st));
      double g0 = -1, gn = 0;
      bool ok = false;
      for (int it = 0; it <= nmax; ++it) {
        if ((rc = implicit_rhs(b, g, *im, im->Y, im->RY)) != FEDBM_OK) return rc;
        ++cnt.rhs;
        // G = Y - base - dtg R(Y)
        FEDBM_CK(krylov::axpby(n, 1.0, im->Y, -1.0, im->base, im->G, st));
        FEDBM_CK(krylov::axpby(n, 1.0, im->G, -dtg, im->RY, im->G, st));
        if ((rc = implicit_norm(b, *im, im->G, &gn)) != FEDBM_OK) return rc;
        if (g0 < 0) g0 = gn;
        if (!std::isfinite(gn)) return fail(FEDBM_ENONFINITE, "implicit step: non-finite Newton residual");
        if (gn <= std::max(rtol * g0, atol)) {
          ok = true;
          break;
        }
        if (it == nmax) break;
        ++cnt.newton;
        // solve (I - dtg J) d = -G
        FEDBM_CK(krylov::axpby(n, -1.0, im->G, 0.0, im->G, im->G, st));
        double ynorm = 0;
        if ((rc = implicit_norm(b, *im, im->Y, &ynorm)) != FEDBM_OK) return rc;
        const double eps = std::sqrt(eps_mach) * (1.0 + ynorm);
        if ((rc = implicit_gmres(b, g, *im, dtg, eps, eta * gn, gmax, precond, cnt)) != FEDBM_OK) return rc;
        FEDBM_CK(krylov::axpby(n, 1.0, im->Y, 1.0, im->d, im->Y, st));
      }
      cnt.residual = gn;
      if (!ok) cnt.converged = false;
      // k_i = (Y - base) / (dt gamma), consistent with the solved stage equation
      FEDBM_CK(krylov::axpby(n, 1.0 / dtg, im->Y, -1.0 / dtg, im->base, im->k + size_t(i) * n, st));
    }
    // u1 = u0 + dt sum_i b_i k_i, into the current state buffer
    std::vector<double> c(tb.s);
    for (int j = 0; j < tb.s; ++j) c[j] = dt * tb.b[j];
    FEDBM_CK(cudaMemcpyAsync(im->hdev, c.data(), size_t(tb.s) * sizeof(double), cudaMemcpyHostToDevice, st));
    FEDBM_CK(krylov::add_combination(n, tb.s, im->k, im->hdev, im->u0, st));
    if (g.store == kStoreF64) FEDBM_CK(cudaMemcpyAsync(g.f[b.cur], im->u0, vb, cudaMemcpyDeviceToDevice, st));
    else FEDBM_CK(krylov::to_f32(n, im->u0, static_cast<float*>(g.f[b.cur]), st));
    FEDBM_CK(cudaStreamSynchronize(st));
    b.time += dt;
    if (!cnt.converged) break;
  }
  {
    int word = 0;  // a residual launch whose bounded wait gave up invalidates the step
    rc = queue_timeout_read(b, g, &word);
    if (rc) return rc;
    FEDBM_CK(cudaStreamSynchronize(b.stream));
    if (word) return timeout_status(word);
  }
  if (stats) {
    stats->newton_iters = cnt.newton;
    stats->gmres_iters = cnt.gmres;
    stats->rhs_evals = cnt.rhs;
    stats->converged = cnt.converged ? 1 : 0;
    stats->residual = cnt.residual;
  }
  if (!cnt.converged) return fail(FEDBM_ENOCONV, "implicit step: Newton did not reach its tolerance");
  return FEDBM_OK;
}

}  // namespace

void set_last_error(const std::string& msg) { g_last_error = msg; }

}  // namespace fedbm

using namespace fedbm;

// Opaque handles of the C ABI: a solver is a batch of one case.
struct fedbm_batch {
  Batch* b = nullptr;
};
struct fedbm_solver {
  Batch* b = nullptr;
};

// ---------------------------------------------------------------- host-only queries
extern "C" const char* fedbm_last_error(void) { return g_last_error_c(); }

extern "C" int fedbm_velset(const fedbm_velset_desc* d, double* ex, double* ey, double* w, int32_t* q) {
  if (!d) return fail(FEDBM_EINVAL, "null descriptor");
  VelocitySet v;
  std::string err;
  if (!build_velocity_set(*d, v, err)) return fail(FEDBM_EINVAL, err);
  if (q) *q = v.Q;
  if (ex) std::memcpy(ex, v.ex.data(), v.Q * sizeof(double));
  if (ey) std::memcpy(ey, v.ey.data(), v.Q * sizeof(double));
  if (w) std::memcpy(w, v.w.data(), v.Q * sizeof(double));
  return FEDBM_OK;
}

extern "C" int fedbm_ref_operators(int32_t p, double* r, double* s, double* Dr, double* Ds, double* LIFT,
                                   double* M, int32_t* fmask) {
  RefOps o;
  std::string err;
  if (!build_ref_ops(p, o, err)) return fail(FEDBM_EINVAL, err);
  auto cp = [](double* dst, const std::vector<double>& v) {
    if (dst) std::memcpy(dst, v.data(), v.size() * sizeof(double));
  };
  cp(r, o.r);
  cp(s, o.s);
  cp(Dr, o.Dr);
  cp(Ds, o.Ds);
  cp(LIFT, o.LIFT);
  cp(M, o.M);
  if (fmask) std::memcpy(fmask, o.fmask.data(), o.fmask.size() * sizeof(int32_t));
  return FEDBM_OK;
}

extern "C" int fedbm_mesh_nodes(const fedbm_mesh_desc* md, const fedbm_velset_desc* vd, const fedbm_params* prm,
                                double* x, double* y, double* dt) {
  if (!md) return fail(FEDBM_EINVAL, "null mesh descriptor");
  Mesh m;
  RefOps o;
  std::string err;
  if (!build_mesh(*md, m, err)) return fail(FEDBM_EINVAL, err);
  if (!build_ref_ops(md->order, o, err)) return fail(FEDBM_EINVAL, err);
  if (x || y) {
    std::vector<double> xx, yy;
    node_coordinates(m, o, xx, yy);
    if (x) std::memcpy(x, xx.data(), xx.size() * sizeof(double));
    if (y) std::memcpy(y, yy.data(), yy.size() * sizeof(double));
  }
  if (dt) {
    if (!vd || !prm) return fail(FEDBM_EINVAL, "dt needs velocity set and params");
    VelocitySet v;
    if (!build_velocity_set(*vd, v, err)) return fail(FEDBM_EINVAL, err);
    *dt = prm->dt > 0 ? prm->dt : time_step(m, v, md->order, prm->cfl);
  }
  return FEDBM_OK;
}

extern "C" int fedbm_mesh_connectivity(const fedbm_mesh_desc* md, int32_t* nbr) {
  if (!md || !nbr) return fail(FEDBM_EINVAL, "null argument");
  Mesh m;
  std::string err;
  if (!build_mesh(*md, m, err)) return fail(FEDBM_EINVAL, err);
  std::memcpy(nbr, m.nbr.data(), m.nbr.size() * sizeof(int32_t));
  return FEDBM_OK;
}

// ---------------------------------------------------------------- single solver
extern "C" int fedbm_create(const fedbm_mesh_desc* md, const fedbm_velset_desc* vd, const fedbm_params* prm,
                            void* cuda_stream, fedbm_solver** out) {
  if (!md || !vd || !prm || !out) return fail(FEDBM_EINVAL, "null argument");
  *out = nullptr;
  fedbm_case_desc cd;
  cd.mesh = *md;
  cd.velset = *vd;
  cd.params = *prm;
  Batch* b = nullptr;
  int rc = create_batch(&cd, 1, cuda_stream, &b);
  if (rc) return rc;
  fedbm_solver* s = new fedbm_solver();
  s->b = b;
  *out = s;
  return FEDBM_OK;
}

extern "C" void fedbm_destroy(fedbm_solver* s) {
  if (!s) return;
  free_batch(s->b);
  delete s;
}

#define FEDBM_SOLVER(s)                                         \
  if (!(s)) return fail(FEDBM_EINVAL, "null solver");            \
  Batch& B = *(s)->b;                                           \
  do {                                                          \
    int rc_ = check_batch(&B, 0);                               \
    if (rc_) return rc_;                                        \
  } while (0)

extern "C" int fedbm_set_state(fedbm_solver* s, const double* f, int32_t on_device) {
  FEDBM_SOLVER(s);
  return set_state(B, 0, f, on_device);
}

extern "C" int fedbm_set_state_f32(fedbm_solver* s, const float* f, int32_t on_device) {
  FEDBM_SOLVER(s);
  return set_state(B, 0, f, on_device);
}

extern "C" int fedbm_set_equilibrium(fedbm_solver* s, double rho0, double ux0, double uy0, double amp,
                                     uint64_t seed) {
  FEDBM_SOLVER(s);
  return set_equilibrium(B, 0, rho0, ux0, uy0, amp, seed);
}

extern "C" int fedbm_rk_step(fedbm_solver* s, int32_t nsteps) {
  FEDBM_SOLVER(s);
  return rk_step(B, nsteps);
}

extern "C" int fedbm_rk_stage(fedbm_solver* s, int32_t stage) {
  FEDBM_SOLVER(s);
  if (stage < 0 || stage > 4) return fail(FEDBM_EINVAL, "stage must be in 0..4");
  FEDBM_CK(launch_stage(B.groups[0], stage, B.cur, B.stream));
  B.cur = 1 - B.cur;
  return FEDBM_OK;
}

extern "C" int fedbm_implicit_step(fedbm_solver* s, const fedbm_implicit_params* ip, int32_t nsteps,
                                   fedbm_implicit_stats* stats) {
  FEDBM_SOLVER(s);
  if (!ip) return fail(FEDBM_EINVAL, "null implicit parameters");
  return implicit_step(B, *ip, nsteps, stats);
}

extern "C" int fedbm_get_moments(fedbm_solver* s, double* rho, double* ux, double* uy, int32_t on_device) {
  FEDBM_SOLVER(s);
  return get_moments(B, 0, rho, ux, uy, on_device);
}

extern "C" int fedbm_get_state(fedbm_solver* s, double* f, int32_t on_device) {
  FEDBM_SOLVER(s);
  return get_state(B, 0, f, on_device);
}

extern "C" int fedbm_get_residual(fedbm_solver* s, double* r, int32_t on_device) {
  FEDBM_SOLVER(s);
  return get_residual(B, 0, r, on_device);
}

extern "C" int fedbm_mass(fedbm_solver* s, double* total) {
  FEDBM_SOLVER(s);
  return mass(B, 0, total);
}

extern "C" int fedbm_info(const fedbm_solver* s, fedbm_info_t* out) {
  if (!s || !s->b) return fail(FEDBM_EINVAL, "null solver");
  return info(*s->b, 0, out);
}

// ---------------------------------------------------------------- batch
extern "C" int fedbm_batch_create(const fedbm_case_desc* cases, int32_t ncases, void* cuda_stream,
                                  fedbm_batch** out) {
  if (!out) return fail(FEDBM_EINVAL, "null output");
  *out = nullptr;
  Batch* b = nullptr;
  int rc = create_batch(cases, ncases, cuda_stream, &b);
  if (rc) return rc;
  fedbm_batch* h = new fedbm_batch();
  h->b = b;
  *out = h;
  return FEDBM_OK;
}

extern "C" void fedbm_batch_destroy(fedbm_batch* h) {
  if (!h) return;
  free_batch(h->b);
  delete h;
}

#define FEDBM_BATCH(h, c)                                       \
  if (!(h)) return fail(FEDBM_EINVAL, "null batch");             \
  Batch& B = *(h)->b;                                           \
  do {                                                          \
    int rc_ = check_batch(&B, (c));                             \
    if (rc_) return rc_;                                        \
  } while (0)

extern "C" int fedbm_batch_set_state(fedbm_batch* h, int32_t c, const double* f, int32_t on_device) {
  FEDBM_BATCH(h, c);
  return set_state(B, c, f, on_device);
}

extern "C" int fedbm_batch_set_state_f32(fedbm_batch* h, int32_t c, const float* f, int32_t on_device) {
  FEDBM_BATCH(h, c);
  return set_state(B, c, f, on_device);
}

extern "C" int fedbm_batch_set_equilibrium(fedbm_batch* h, int32_t c, double rho0, double ux0, double uy0,
                                           double amp, uint64_t seed) {
  FEDBM_BATCH(h, c);
  return set_equilibrium(B, c, rho0, ux0, uy0, amp, seed);
}

extern "C" int fedbm_batch_rk_step(fedbm_batch* h, int32_t nsteps) {
  FEDBM_BATCH(h, 0);
  return rk_step(B, nsteps);
}

extern "C" int fedbm_batch_get_state(fedbm_batch* h, int32_t c, double* f, int32_t on_device) {
  FEDBM_BATCH(h, c);
  return get_state(B, c, f, on_device);
}

extern "C" int fedbm_batch_get_moments(fedbm_batch* h, int32_t c, double* rho, double* ux, double* uy,
                                       int32_t on_device) {
  FEDBM_BATCH(h, c);
  return get_moments(B, c, rho, ux, uy, on_device);
}

extern "C" int fedbm_batch_mass(fedbm_batch* h, int32_t c, double* total) {
  FEDBM_BATCH(h, c);
  return mass(B, c, total);
}

extern "C" int fedbm_batch_info(const fedbm_batch* h, int32_t c, fedbm_info_t* out) {
  if (!h || !h->b) return fail(FEDBM_EINVAL, "null batch");
  if (c < 0 || c >= int(h->b->cases.size())) return fail(FEDBM_EINVAL, "case index out of range");
  return info(*h->b, c, out);
}

extern "C" int fedbm_batch_set_tiles(fedbm_batch* h, int32_t group, int32_t elems_per_cta, int32_t threads_per_cta,
                                     int32_t pipeline_stages) {
  FEDBM_BATCH(h, 0);
  if (group < 0 || group >= int(B.groups.size())) return fail(FEDBM_EINVAL, "group index out of range");
  return configure_tiles(B, B.groups[group], elems_per_cta, threads_per_cta, pipeline_stages);
}

extern "C" int fedbm_batch_set_tensor_cores(fedbm_batch* h, int32_t group, int32_t on) {
  FEDBM_BATCH(h, 0);
  if (group < 0 || group >= int(B.groups.size())) return fail(FEDBM_EINVAL, "group index out of range");
  Group& g = B.groups[group];
  if (on) return configure_tc(B, g);
  return ws_default(g) && g.vsplit <= 1 ? configure_ws(B, g) : configure_tiles(B, g, 0, 0, 0);
}

extern "C" int fedbm_batch_autotune(fedbm_batch* h, const char* cache_path, int32_t trials) {
  FEDBM_BATCH(h, 0);
  return autotune(B, cache_path, trials);
}

extern "C" int fedbm_autotune(fedbm_solver* s, const char* cache_path, int32_t trials) {
  FEDBM_SOLVER(s);
  return autotune(B, cache_path, trials);
}
