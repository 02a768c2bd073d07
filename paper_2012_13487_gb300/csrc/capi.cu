// C ABI of the solver: set-up, state transfer, LSRK stepping (CUDA graphs of
// the fused stage kernel), moments and the FP64 mass diagnostic.
#include <cuda_runtime.h>

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
#include "stage_dispatch.h"

namespace fedbm {
namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

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
size_t real_bytes(int kind) { return kind == kStoreF64 ? 8 : 4; }

// ---------------------------------------------------------------- aux kernels
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// canonical f = f^eq(rho0, u0) (1 + amp u(seed, index)) in FP64
__global__ void equilibrium_kernel(double* out, const double* vel64, int64_t K, int Np, int Q, int Qp,
                                   double rho0, double ux0, double uy0, double amp, uint64_t seed,
                                   int eq_order) {
  const int64_t n = K * Np * Q;
  for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < n;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(idx % Q);
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

// canonical FP64 [K][Np][Q] -> internal storage [K][Np][Qp] (one CTA per element)
template <class ST>
__global__ void encode_kernel(const double* in, void* out, float* scale, const double* vel64, int Np, int Q,
                              int Qp) {
  using S = typename ST::S;
  const int64_t k = blockIdx.x;
  const double* src = in + k * Np * Q;
  S* dst = static_cast<S*>(out) + k * Np * Qp;
  const double* w = vel64 + 2 * Qp;
  if constexpr (ST::dev) {
    __shared__ float red[32];
    float m = 0.f;
    for (int j = threadIdx.x; j < Np * Q; j += blockDim.x) {
      const int i = j % Q;
      if (w[i] > 0) m = fmaxf(m, float(fabs((src[j] - w[i]) / w[i])));
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
    for (int j = threadIdx.x; j < Np * Qp; j += blockDim.x) {
      const int n = j / Qp, i = j % Qp;
      float q = 0.f;
      if (i < Q && w[i] > 0) q = float((src[n * Q + i] - w[i]) / w[i] * inv_s);
      dst[j] = ST::from_r(q);
    }
  } else {
    (void)scale;
    (void)w;
    for (int j = threadIdx.x; j < Np * Qp; j += blockDim.x) {
      const int n = j / Qp, i = j % Qp;
      dst[j] = S(i < Q ? src[n * Q + i] : 0.0);
    }
  }
}

template <class ST>
__device__ __forceinline__ double decode64(const typename ST::S v, double w, double s) {
  if constexpr (ST::dev) return w + w * s * double(ST::to_r(v));
  else return double(v);
}

// internal state -> canonical FP64
template <class ST>
__global__ void decode_kernel(const void* in, const float* scale, double* out, const double* vel64, int64_t K,
                              int Np, int Q, int Qp) {
  using S = typename ST::S;
  const int64_t n = K * Np * Q;
  const double* w = vel64 + 2 * Qp;
  for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < n;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(idx % Q);
    const int64_t kn = idx / Q;
    const int64_t k = kn / Np;
    const double s = ST::dev ? double(scale[k]) : 0.0;
    out[idx] = decode64<ST>(static_cast<const S*>(in)[kn * Qp + i], w[i], s);
  }
}

template <typename R>
__global__ void decode_residual_kernel(const R* in, double* out, int64_t K, int Np, int Q, int Qp) {
  const int64_t n = K * Np * Q;
  for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < n;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(idx % Q);
    const int64_t kn = idx / Q;
    out[idx] = double(in[kn * Qp + i]);
  }
}

// node moments in FP64 (one thread per node)
template <class ST>
__global__ void moments_kernel(const void* in, const float* scale, const double* vel64, int64_t K, int Np,
                               int Qp, double* rho, double* ux, double* uy) {
  using S = typename ST::S;
  const int64_t nodes = K * Np;
  for (int64_t kn = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; kn < nodes;
       kn += int64_t(gridDim.x) * blockDim.x) {
    const S* row = static_cast<const S*>(in) + kn * Qp;
    const double s = ST::dev ? double(scale[kn / Np]) : 0.0;
    double m0 = 0, m1 = 0, m2 = 0;
    for (int i = 0; i < Qp; ++i) {
      const double f = decode64<ST>(row[i], vel64[2 * Qp + i], s);
      m0 += f;
      m1 += vel64[i] * f;
      m2 += vel64[Qp + i] * f;
    }
    rho[kn] = m0;
    ux[kn] = m1 / m0;
    uy[kn] = m2 / m0;
  }
}

// mass partial sums: sum over nodes of J_k mw_n rho; flags non-finite / rho <= 0
template <class ST>
__global__ void mass_partial_kernel(const void* in, const float* scale, const double* vel64, const double* Jk,
                                    const double* mw, int64_t K, int Np, int Qp, double* partial, int* flag) {
  using S = typename ST::S;
  __shared__ double red[32];
  const int64_t nodes = K * Np;
  double acc = 0.0;
  for (int64_t kn = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; kn < nodes;
       kn += int64_t(gridDim.x) * blockDim.x) {
    const S* row = static_cast<const S*>(in) + kn * Qp;
    const int64_t k = kn / Np;
    const double s = ST::dev ? double(scale[k]) : 0.0;
    double rho = 0.0;
    for (int i = 0; i < Qp; ++i) rho += decode64<ST>(row[i], vel64[2 * Qp + i], s);
    if (!(rho > 0.0) || !isfinite(rho)) atomicOr(flag, 1);
    acc += Jk[k] * mw[kn % Np] * rho;
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

int grid_for(int64_t n, int block) {
  return int(std::min<int64_t>((n + block - 1) / block, 152 * 32));
}

}  // namespace

void set_last_error(const std::string& msg) { g_last_error = msg; }

}  // namespace fedbm

using namespace fedbm;

// ---------------------------------------------------------------- solver object
struct fedbm_solver {
  int device = 0;
  cudaStream_t stream = nullptr;     // caller's stream
  cudaStream_t capture = nullptr;    // private stream for graph capture
  fedbm_mesh_desc mesh_desc{};
  fedbm_velset_desc vs_desc{};
  fedbm_params prm{};
  Mesh mesh;
  VelocitySet vs;
  RefOps ops;
  int store = kStoreF32;
  int64_t K = 0;
  int Np = 0, Nfp = 0, Q = 0, Qp = 0;
  int epc = 0, tpb = 0;
  size_t smem = 0;
  double dt = 0, tau = 0, time = 0;
  int64_t steps = 0;
  int cur = 0;                       // state buffer holding the current f
  // device memory
  void* f[2] = {nullptr, nullptr};
  void* res = nullptr;
  float* scale[2] = {nullptr, nullptr};
  int32_t* nbr = nullptr;
  void* geo = nullptr;               // [K][16] in the compute precision
  void* vel = nullptr;               // [kVelRows][Qp] in the compute precision
  double* vel64 = nullptr;           // [3][Qp] ex, ey, w in FP64
  void* wall_feq = nullptr;          // [4][Qp]
  void* wall_den_inv = nullptr;      // [4]
  double* Jk = nullptr;              // [K]
  double* mw = nullptr;              // [Np] column sums of M
  double* staging = nullptr;         // canonical FP64 [K][Np][Q] (lazy)
  double* mom = nullptr;             // [3][K][Np] (lazy)
  double* partial = nullptr;         // [kMassBlocks + 1]
  int* flag = nullptr;               // [0]: mass diagnostic flag, [1]: stage-kernel wait timeout
  int wall_diffuse_mask = 0;
  double W0 = 0, W1x = 0, W1y = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
};

namespace {

template <typename R>
void fill_stage_args(const fedbm_solver* s, int stage, int from, StageArgs<R>& a) {
  a.f_in = s->f[from];
  a.f_out = s->f[1 - from];
  a.res = static_cast<R*>(s->res);
  a.scale_in = s->scale[from];
  a.scale_out = s->scale[1 - from];
  a.nbr = s->nbr;
  a.geo = static_cast<const R*>(s->geo);
  a.vel = static_cast<const R*>(s->vel);
  a.wall_feq = static_cast<const R*>(s->wall_feq);
  a.wall_den_inv = static_cast<const R*>(s->wall_den_inv);
  a.wall_diffuse_mask = s->wall_diffuse_mask;
  a.W0 = R(s->W0);
  a.W1x = R(s->W1x);
  a.W1y = R(s->W1y);
  a.K = s->K;
  a.Qp = s->Qp;
  a.epc = s->epc;
  a.dt = R(s->dt);
  a.rkA = R(kRkA[stage]);
  a.rkB = R(kRkB[stage]);
  a.inv_tau = R(1.0 / s->tau);
  a.ab = R(2.0 * s->prm.beta - 1.0);
  a.collision = s->prm.collision;
  a.eq_order = s->vs_desc.eq_order;
  a.red = s->prm.reduction;
  a.err = s->flag + 1;
}

cudaError_t launch_stage(const fedbm_solver* s, int stage, int from, cudaStream_t st) {
  const int grid = int((s->K + s->epc - 1) / s->epc);
  const StageEntry e = stage_entry(s->ops.p);
  if (s->store == kStoreF64) {
    StageArgs<double> a;
    fill_stage_args(s, stage, from, a);
    return e.launch(s->store, &a, grid, s->tpb, s->smem, st);
  }
  StageArgs<float> a;
  fill_stage_args(s, stage, from, a);
  return e.launch(s->store, &a, grid, s->tpb, s->smem, st);
}

int build_graphs(fedbm_solver* s) {
  for (int c = 0; c < 2; ++c) {
    if (s->graph[c]) continue;
    cudaGraph_t g = nullptr;
    FEDBM_CK(cudaStreamBeginCapture(s->capture, cudaStreamCaptureModeThreadLocal));
    int from = c;
    cudaError_t le = cudaSuccess;
    for (int st = 0; st < 5 && le == cudaSuccess; ++st) {
      le = launch_stage(s, st, from, s->capture);
      from = 1 - from;
    }
    cudaError_t ee = cudaStreamEndCapture(s->capture, &g);
    if (le != cudaSuccess) return fail(FEDBM_ECUDA, std::string("stage launch in capture: ") + cudaGetErrorString(le));
    if (ee != cudaSuccess) return fail(FEDBM_ECUDA, std::string("end capture: ") + cudaGetErrorString(ee));
    cudaError_t ie = cudaGraphInstantiate(&s->graph[c], g, 0);
    cudaGraphDestroy(g);
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

int ensure_staging(fedbm_solver* s) {
  if (!s->staging) FEDBM_CK(cudaMalloc(&s->staging, size_t(s->K) * s->Np * s->Q * sizeof(double)));
  return FEDBM_OK;
}

int encode_from_staging(fedbm_solver* s) {
  const int b = 256;
  switch (s->store) {
    case kStoreF64: encode_kernel<StoreF64><<<int(s->K), b, 0, s->stream>>>(s->staging, s->f[s->cur], nullptr, s->vel64, s->Np, s->Q, s->Qp); break;
    case kStoreF32: encode_kernel<StoreF32><<<int(s->K), b, 0, s->stream>>>(s->staging, s->f[s->cur], nullptr, s->vel64, s->Np, s->Q, s->Qp); break;
    case kStoreBF16: encode_kernel<StoreBF16><<<int(s->K), b, 0, s->stream>>>(s->staging, s->f[s->cur], s->scale[s->cur], s->vel64, s->Np, s->Q, s->Qp); break;
    default: encode_kernel<StoreF16><<<int(s->K), b, 0, s->stream>>>(s->staging, s->f[s->cur], s->scale[s->cur], s->vel64, s->Np, s->Q, s->Qp); break;
  }
  FEDBM_CK(cudaGetLastError());
  s->time = 0;
  s->steps = 0;
  return FEDBM_OK;
}

int check_solver(const fedbm_solver* s) {
  if (!s) return fail(FEDBM_EINVAL, "null solver");
  FEDBM_CK(cudaSetDevice(s->device));
  return FEDBM_OK;
}

}  // namespace

// ---------------------------------------------------------------- host-only queries
extern "C" const char* fedbm_last_error(void) { return g_last_error.c_str(); }

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

// ---------------------------------------------------------------- lifecycle
extern "C" void fedbm_destroy(fedbm_solver* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (int c = 0; c < 2; ++c) {
    if (s->graph[c]) cudaGraphExecDestroy(s->graph[c]);
    cudaFree(s->f[c]);
    cudaFree(s->scale[c]);
  }
  void* bufs[] = {s->res, s->nbr, s->geo, s->vel, s->vel64, s->wall_feq, s->wall_den_inv,
                  s->Jk, s->mw, s->staging, s->mom, s->partial, s->flag};
  for (void* b : bufs) cudaFree(b);
  if (s->capture) cudaStreamDestroy(s->capture);
  delete s;
}

extern "C" int fedbm_create(const fedbm_mesh_desc* md, const fedbm_velset_desc* vd, const fedbm_params* prm,
                            void* cuda_stream, fedbm_solver** out) {
  if (!md || !vd || !prm || !out) return fail(FEDBM_EINVAL, "null argument");
  *out = nullptr;
  fedbm_solver* s = new fedbm_solver();
  s->mesh_desc = *md;
  s->vs_desc = *vd;
  s->prm = *prm;
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  int rc = FEDBM_OK;
  auto bail = [&](int code) {
    fedbm_destroy(s);
    return code;
  };
  std::string err;
  if (prm->precision < FEDBM_FP64 || prm->precision > FEDBM_FP16_DEV)
    return bail(fail(FEDBM_EINVAL, "unknown precision"));
  if (prm->reduction < FEDBM_RED_DEFAULT || prm->reduction > FEDBM_RED_COMP_FP32)
    return bail(fail(FEDBM_EINVAL, "unknown reduction mode"));
  if (!(prm->kn > 0)) return bail(fail(FEDBM_EINVAL, "kn must be > 0"));
  if (!(prm->beta >= 0.5 && prm->beta <= 1.0)) return bail(fail(FEDBM_EINVAL, "beta must be in [0.5, 1]"));
  if (!(prm->dt > 0) && !(prm->cfl > 0)) return bail(fail(FEDBM_EINVAL, "need dt > 0 or cfl > 0"));
  if (!build_velocity_set(*vd, s->vs, err)) return bail(fail(FEDBM_EINVAL, err));
  if (!build_mesh(*md, s->mesh, err)) return bail(fail(FEDBM_EINVAL, err));
  if (!build_ref_ops(md->order, s->ops, err)) return bail(fail(FEDBM_EINVAL, err));
  s->store = prm->precision;  // enum values coincide with StoreKind
  s->K = s->mesh.K;
  s->Np = s->ops.Np;
  s->Nfp = s->ops.Nfp;
  s->Q = s->vs.Q;
  s->Qp = (s->Q + 7) / 8 * 8;
  const double L = prm->length > 0 ? prm->length : 1.0;
  s->tau = prm->kn * L / std::sqrt(3.0);
  s->dt = prm->dt > 0 ? prm->dt : time_step(s->mesh, s->vs, md->order, prm->cfl);
  // stage tile: elements per CTA and threads per CTA
  s->epc = prm->elems_per_cta > 0 ? prm->elems_per_cta : (s->Qp < 128 ? std::max(1, 128 / s->Qp) : 1);
  if (prm->threads_per_cta > 0) {
    s->tpb = prm->threads_per_cta;
  } else {
    s->tpb = std::min(256, std::max(32, (s->epc * s->Qp + 31) / 32 * 32));
  }
  if (s->tpb % 32 || s->tpb > 256) return bail(fail(FEDBM_EINVAL, "threads_per_cta must be a multiple of 32, <= 256"));
  s->smem = stage_smem_bytes(md->order, s->store, s->epc, s->Qp);
  if (s->smem > 227 * 1024) return bail(fail(FEDBM_EINVAL, "stage tile does not fit in shared memory"));

  if ((rc = [&]() -> int {
         FEDBM_CK(cudaGetDevice(&s->device));
         if ((rc = ensure_ops_uploaded(s->device)) != FEDBM_OK) return rc;
         FEDBM_CK(cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking));
         const StageEntry e = stage_entry(md->order);
         FEDBM_CK(e.set_smem(s->store, s->smem));
         const size_t dofp = size_t(s->K) * s->Np * s->Qp;
         for (int c = 0; c < 2; ++c) {
           FEDBM_CK(cudaMalloc(&s->f[c], dofp * store_bytes(s->store)));
           FEDBM_CK(cudaMemset(s->f[c], 0, dofp * store_bytes(s->store)));
           if (s->store >= kStoreBF16) {
             FEDBM_CK(cudaMalloc(&s->scale[c], size_t(s->K) * sizeof(float)));
             FEDBM_CK(cudaMemset(s->scale[c], 0, size_t(s->K) * sizeof(float)));
           }
         }
         FEDBM_CK(cudaMalloc(&s->res, dofp * real_bytes(s->store)));
         FEDBM_CK(cudaMemset(s->res, 0, dofp * real_bytes(s->store)));
         // velocity table, padded with zero-weight zero-speed velocities
         const int Qp = s->Qp, Q = s->Q;
         std::vector<double> vel(size_t(kVelRows) * Qp, 0.0), v64(size_t(3) * Qp, 0.0);
         for (int i = 0; i < Q; ++i) {
           vel[kVelEx * Qp + i] = s->vs.ex[i];
           vel[kVelEy * Qp + i] = s->vs.ey[i];
           vel[kVelW * Qp + i] = s->vs.w[i];
           vel[kVelInvW * Qp + i] = s->vs.w[i] > 0 ? 1.0 / s->vs.w[i] : 0.0;
           vel[kVelWex * Qp + i] = s->vs.w[i] * s->vs.ex[i];
           vel[kVelWey * Qp + i] = s->vs.w[i] * s->vs.ey[i];
           v64[i] = s->vs.ex[i];
           v64[Qp + i] = s->vs.ey[i];
           v64[2 * Qp + i] = s->vs.w[i];
           s->W0 += s->vs.w[i];
           s->W1x += s->vs.w[i] * s->vs.ex[i];
           s->W1y += s->vs.w[i] * s->vs.ey[i];
         }
         // walls: f^eq(1, u_b) per side and the eq. FullBC denominators
         const double nrm[4][2] = {{0, -1}, {1, 0}, {0, 1}, {-1, 0}};
         std::vector<double> wfeq(size_t(4) * Qp, 0.0), wden(4, 0.0);
         for (int sd = 0; sd < 4; ++sd) {
           if (md->bc[sd] == FEDBM_BC_WALL_DIFFUSE) s->wall_diffuse_mask |= 1 << sd;
           double den = 0.0;
           for (int i = 0; i < Q; ++i) {
             const double fb = equilibrium(s->vs.w[i], s->vs.ex[i], s->vs.ey[i], 1.0, md->wall_ux[sd],
                                           md->wall_uy[sd], vd->eq_order);
             wfeq[size_t(sd) * Qp + i] = fb;
             const double en = s->vs.ex[i] * nrm[sd][0] + s->vs.ey[i] * nrm[sd][1];
             if (en < 0) den -= en * fb;
           }
           wden[sd] = den > 0 ? 1.0 / den : 0.0;
         }
         std::vector<double> Jk(s->K), mw(s->Np, 0.0);
         for (int64_t k = 0; k < s->K; ++k) Jk[k] = s->mesh.geo[k * kGeoStride + 13];
         for (int j = 0; j < s->Np; ++j)
           for (int n = 0; n < s->Np; ++n) mw[n] += s->ops.M[size_t(j) * s->Np + n];
         if ((rc = upload_vec(s->mesh.nbr, reinterpret_cast<void**>(&s->nbr))) != FEDBM_OK) return rc;
         if ((rc = upload_vec(v64, reinterpret_cast<void**>(&s->vel64))) != FEDBM_OK) return rc;
         if ((rc = upload_vec(Jk, reinterpret_cast<void**>(&s->Jk))) != FEDBM_OK) return rc;
         if ((rc = upload_vec(mw, reinterpret_cast<void**>(&s->mw))) != FEDBM_OK) return rc;
         if (s->store == kStoreF64) {
           if ((rc = upload_real<double>(s->mesh.geo, &s->geo)) != FEDBM_OK) return rc;
           if ((rc = upload_real<double>(vel, &s->vel)) != FEDBM_OK) return rc;
           if ((rc = upload_real<double>(wfeq, &s->wall_feq)) != FEDBM_OK) return rc;
           if ((rc = upload_real<double>(wden, &s->wall_den_inv)) != FEDBM_OK) return rc;
         } else {
           if ((rc = upload_real<float>(s->mesh.geo, &s->geo)) != FEDBM_OK) return rc;
           if ((rc = upload_real<float>(vel, &s->vel)) != FEDBM_OK) return rc;
           if ((rc = upload_real<float>(wfeq, &s->wall_feq)) != FEDBM_OK) return rc;
           if ((rc = upload_real<float>(wden, &s->wall_den_inv)) != FEDBM_OK) return rc;
         }
         FEDBM_CK(cudaMalloc(&s->partial, (kMassBlocks + 1) * sizeof(double)));
         FEDBM_CK(cudaMalloc(&s->flag, 2 * sizeof(int)));
         FEDBM_CK(cudaMemset(s->flag, 0, 2 * sizeof(int)));
         return FEDBM_OK;
       }()) != FEDBM_OK)
    return bail(rc);
  *out = s;
  return FEDBM_OK;
}

// ---------------------------------------------------------------- state
extern "C" int fedbm_set_state(fedbm_solver* s, const double* f, int32_t on_device) {
  int rc = check_solver(s);
  if (rc) return rc;
  if (!f) return fail(FEDBM_EINVAL, "null state pointer");
  if ((rc = ensure_staging(s))) return rc;
  const size_t bytes = size_t(s->K) * s->Np * s->Q * sizeof(double);
  FEDBM_CK(cudaMemcpyAsync(s->staging, f, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           s->stream));
  if ((rc = encode_from_staging(s))) return rc;
  if (!on_device) FEDBM_CK(cudaStreamSynchronize(s->stream));
  return FEDBM_OK;
}

extern "C" int fedbm_set_equilibrium(fedbm_solver* s, double rho0, double ux0, double uy0, double amp,
                                     uint64_t seed) {
  int rc = check_solver(s);
  if (rc) return rc;
  if ((rc = ensure_staging(s))) return rc;
  const int64_t n = s->K * s->Np * s->Q;
  equilibrium_kernel<<<grid_for(n, 256), 256, 0, s->stream>>>(s->staging, s->vel64, s->K, s->Np, s->Q, s->Qp, rho0,
                                                              ux0, uy0, amp, seed, s->vs_desc.eq_order);
  FEDBM_CK(cudaGetLastError());
  return encode_from_staging(s);
}

extern "C" int fedbm_get_state(fedbm_solver* s, double* f, int32_t on_device) {
  int rc = check_solver(s);
  if (rc) return rc;
  if (!f) return fail(FEDBM_EINVAL, "null output");
  double* dst = f;
  if (!on_device) {
    if ((rc = ensure_staging(s))) return rc;
    dst = s->staging;
  }
  const int64_t n = s->K * s->Np * s->Q;
  const int g = grid_for(n, 256);
  switch (s->store) {
    case kStoreF64: decode_kernel<StoreF64><<<g, 256, 0, s->stream>>>(s->f[s->cur], nullptr, dst, s->vel64, s->K, s->Np, s->Q, s->Qp); break;
    case kStoreF32: decode_kernel<StoreF32><<<g, 256, 0, s->stream>>>(s->f[s->cur], nullptr, dst, s->vel64, s->K, s->Np, s->Q, s->Qp); break;
    case kStoreBF16: decode_kernel<StoreBF16><<<g, 256, 0, s->stream>>>(s->f[s->cur], s->scale[s->cur], dst, s->vel64, s->K, s->Np, s->Q, s->Qp); break;
    default: decode_kernel<StoreF16><<<g, 256, 0, s->stream>>>(s->f[s->cur], s->scale[s->cur], dst, s->vel64, s->K, s->Np, s->Q, s->Qp); break;
  }
  FEDBM_CK(cudaGetLastError());
  if (!on_device) {
    FEDBM_CK(cudaMemcpyAsync(f, dst, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    FEDBM_CK(cudaStreamSynchronize(s->stream));
  }
  return FEDBM_OK;
}

extern "C" int fedbm_get_residual(fedbm_solver* s, double* r, int32_t on_device) {
  int rc = check_solver(s);
  if (rc) return rc;
  if (!r) return fail(FEDBM_EINVAL, "null output");
  double* dst = r;
  if (!on_device) {
    if ((rc = ensure_staging(s))) return rc;
    dst = s->staging;
  }
  const int64_t n = s->K * s->Np * s->Q;
  const int g = grid_for(n, 256);
  if (s->store == kStoreF64)
    decode_residual_kernel<double><<<g, 256, 0, s->stream>>>(static_cast<const double*>(s->res), dst, s->K, s->Np, s->Q, s->Qp);
  else
    decode_residual_kernel<float><<<g, 256, 0, s->stream>>>(static_cast<const float*>(s->res), dst, s->K, s->Np, s->Q, s->Qp);
  FEDBM_CK(cudaGetLastError());
  if (!on_device) {
    FEDBM_CK(cudaMemcpyAsync(r, dst, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    FEDBM_CK(cudaStreamSynchronize(s->stream));
  }
  return FEDBM_OK;
}

// ---------------------------------------------------------------- stepping
extern "C" int fedbm_rk_step(fedbm_solver* s, int32_t nsteps) {
  int rc = check_solver(s);
  if (rc) return rc;
  if (nsteps < 0) return fail(FEDBM_EINVAL, "nsteps must be >= 0");
  if ((rc = build_graphs(s))) return rc;
  for (int n = 0; n < nsteps; ++n) {
    FEDBM_CK(cudaGraphLaunch(s->graph[s->cur], s->stream));
    s->cur = 1 - s->cur;  // five stages: the state ends in the other buffer
    s->time += s->dt;
    s->steps += 1;
  }
  return FEDBM_OK;
}

extern "C" int fedbm_rk_stage(fedbm_solver* s, int32_t stage) {
  int rc = check_solver(s);
  if (rc) return rc;
  if (stage < 0 || stage > 4) return fail(FEDBM_EINVAL, "stage must be in 0..4");
  FEDBM_CK(launch_stage(s, stage, s->cur, s->stream));
  s->cur = 1 - s->cur;
  return FEDBM_OK;
}

// ---------------------------------------------------------------- diagnostics
extern "C" int fedbm_get_moments(fedbm_solver* s, double* rho, double* ux, double* uy, int32_t on_device) {
  int rc = check_solver(s);
  if (rc) return rc;
  const int64_t nodes = s->K * s->Np;
  double *dr = rho, *dx = ux, *dy = uy;
  if (!on_device) {
    if (!s->mom) FEDBM_CK(cudaMalloc(&s->mom, size_t(3) * nodes * sizeof(double)));
    dr = s->mom;
    dx = s->mom + nodes;
    dy = s->mom + 2 * nodes;
  } else if (!rho || !ux || !uy) {
    return fail(FEDBM_EINVAL, "device moments need three output pointers");
  }
  const int g = grid_for(nodes, 256);
  switch (s->store) {
    case kStoreF64: moments_kernel<StoreF64><<<g, 256, 0, s->stream>>>(s->f[s->cur], nullptr, s->vel64, s->K, s->Np, s->Qp, dr, dx, dy); break;
    case kStoreF32: moments_kernel<StoreF32><<<g, 256, 0, s->stream>>>(s->f[s->cur], nullptr, s->vel64, s->K, s->Np, s->Qp, dr, dx, dy); break;
    case kStoreBF16: moments_kernel<StoreBF16><<<g, 256, 0, s->stream>>>(s->f[s->cur], s->scale[s->cur], s->vel64, s->K, s->Np, s->Qp, dr, dx, dy); break;
    default: moments_kernel<StoreF16><<<g, 256, 0, s->stream>>>(s->f[s->cur], s->scale[s->cur], s->vel64, s->K, s->Np, s->Qp, dr, dx, dy); break;
  }
  FEDBM_CK(cudaGetLastError());
  if (!on_device) {
    const size_t b = size_t(nodes) * sizeof(double);
    if (rho) FEDBM_CK(cudaMemcpyAsync(rho, dr, b, cudaMemcpyDeviceToHost, s->stream));
    if (ux) FEDBM_CK(cudaMemcpyAsync(ux, dx, b, cudaMemcpyDeviceToHost, s->stream));
    if (uy) FEDBM_CK(cudaMemcpyAsync(uy, dy, b, cudaMemcpyDeviceToHost, s->stream));
    FEDBM_CK(cudaStreamSynchronize(s->stream));
  }
  return FEDBM_OK;
}

extern "C" int fedbm_mass(fedbm_solver* s, double* total) {
  int rc = check_solver(s);
  if (rc) return rc;
  if (!total) return fail(FEDBM_EINVAL, "null output");
  FEDBM_CK(cudaMemsetAsync(s->flag, 0, sizeof(int), s->stream));
  const int64_t nodes = s->K * s->Np;
  const int g = int(std::min<int64_t>(kMassBlocks, (nodes + kMassThreads - 1) / kMassThreads));
  switch (s->store) {
    case kStoreF64: mass_partial_kernel<StoreF64><<<g, kMassThreads, 0, s->stream>>>(s->f[s->cur], nullptr, s->vel64, s->Jk, s->mw, s->K, s->Np, s->Qp, s->partial, s->flag); break;
    case kStoreF32: mass_partial_kernel<StoreF32><<<g, kMassThreads, 0, s->stream>>>(s->f[s->cur], nullptr, s->vel64, s->Jk, s->mw, s->K, s->Np, s->Qp, s->partial, s->flag); break;
    case kStoreBF16: mass_partial_kernel<StoreBF16><<<g, kMassThreads, 0, s->stream>>>(s->f[s->cur], s->scale[s->cur], s->vel64, s->Jk, s->mw, s->K, s->Np, s->Qp, s->partial, s->flag); break;
    default: mass_partial_kernel<StoreF16><<<g, kMassThreads, 0, s->stream>>>(s->f[s->cur], s->scale[s->cur], s->vel64, s->Jk, s->mw, s->K, s->Np, s->Qp, s->partial, s->flag); break;
  }
  FEDBM_CK(cudaGetLastError());
  mass_final_kernel<<<1, 256, 0, s->stream>>>(s->partial, g, s->partial + kMassBlocks);
  FEDBM_CK(cudaGetLastError());
  int flag[2] = {0, 0};
  FEDBM_CK(cudaMemcpyAsync(total, s->partial + kMassBlocks, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  FEDBM_CK(cudaMemcpyAsync(flag, s->flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  FEDBM_CK(cudaStreamSynchronize(s->stream));
  if (flag[1]) return fail(FEDBM_ETIMEOUT, "a stage kernel's bounded wait for its tile copies gave up");
  if (flag[0]) return fail(FEDBM_ENONFINITE, "state has a non-finite value or a node with rho <= 0");
  return FEDBM_OK;
}

extern "C" int fedbm_info(const fedbm_solver* s, fedbm_info_t* info) {
  if (!s || !info) return fail(FEDBM_EINVAL, "null argument");
  info->K = s->K;
  info->Np = s->Np;
  info->Nfp = s->Nfp;
  info->Q = s->Q;
  info->Q_padded = s->Qp;
  info->dt = s->dt;
  info->tau = s->tau;
  info->time = s->time;
  info->steps = s->steps;
  info->precision = s->prm.precision;
  info->reduction = s->prm.reduction;
  info->order = s->ops.p;
  info->eq_order = s->vs_desc.eq_order;
  info->elems_per_cta = s->epc;
  info->threads_per_cta = s->tpb;
  info->state_bytes = int64_t(s->K) * s->Np * s->Qp * int64_t(store_bytes(s->store));
  info->residual_bytes = int64_t(s->K) * s->Np * s->Qp * int64_t(real_bytes(s->store));
  return FEDBM_OK;
}
