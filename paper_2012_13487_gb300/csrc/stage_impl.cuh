// Fused LSRK(5,4) stage kernel for polynomial degree FEDBM_P.
//
// One CTA owns a tile of `epc` consecutive elements and every velocity of
// them.  Per stage it computes, for each element, node and velocity,
//   rhs_i = -(e_i . grad) f_i                       volume term (Dr, Ds)
//           + LIFT (Fscale (F^- - F^*) . n)         upwind/central surface flux
//           - (f_i - f_i^eq(rho, u)) / tau          BGK collision, eq. feq
// which is the strong form of eq. byparts (Sec. II.B.1); neighbour traces come
// from the input state (an L2-resident re-read), wall traces from eq. FullBC
// or eq. UsedBC (Sec. II.A.4).  It then applies the 2N-storage update
//   res <- A res + dt rhs ; f <- f + B res
// and writes the new state to the other state buffer (neighbours still read
// the old one).  The reference operators Dr, Ds, LIFT live in constant memory
// and every loop over nodes is unrolled, so they are immediate operands of
// the FMAs.
//
// Phases of a CTA:
//   1. copy the element tile f[k0:k0+epc][Np][Qp] to shared memory (16-byte
//      vectors), plus geometry, face codes and (deviation forms) scales;
//   2. node moments rho, u (Sec. II.A.2) by a G-lane reduction per node;
//   3. wall numerators sum_{e.n>0} (e.n) f^- of eq. FullBC per wall node;
//   4. per (element, velocity) item: residual, update and store;
//   5. deviation forms only: per-element scale from max |f/w - 1|, encode.
#include "device_common.cuh"
#include "stage_dispatch.h"

#ifndef FEDBM_P
#error "FEDBM_P must be defined"
#endif

namespace fedbm {
namespace {

constexpr int P = FEDBM_P;
constexpr int NP = np_of(P);
constexpr int NFP = P + 1;
constexpr int NF = 3 * NFP;
constexpr int OFF_DR = 0;
constexpr int OFF_DS = NP * NP;
constexpr int OFF_LIFT = 2 * NP * NP;
constexpr int OPS_N = 2 * NP * NP + NP * NF;

static __constant__ float c_ops32[OPS_N];
static __constant__ double c_ops64[OPS_N];

template <typename R>
__device__ __forceinline__ R opv(int idx);
template <>
__device__ __forceinline__ float opv<float>(int idx) { return c_ops32[idx]; }
template <>
__device__ __forceinline__ double opv<double>(int idx) { return c_ops64[idx]; }

// Node index of face node a on face f (rows of the reference triangle start at
// a(P+1) - a(a-1)/2; face 0 is row 0, face 1 the row ends, face 2 the row starts).
__host__ __device__ constexpr int face_node(int f, int a) {
  return f == 0 ? a : (f == 1 ? a * (P + 1) - a * (a - 1) / 2 + (P - a) : a * (P + 1) - a * (a - 1) / 2);
}

constexpr unsigned kFull = 0xffffffffu;

// ---- moment accumulators ----------------------------------------------------
struct AccD {
  double s = 0.0;
  __device__ void add(double v) { s += v; }
  __device__ void reduce(int G) {
    for (int off = G >> 1; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
  }
  __device__ double value() const { return s; }
};
struct AccF {
  float s = 0.f;
  __device__ void add(float v) { s += v; }
  __device__ void reduce(int G) {
    for (int off = G >> 1; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
  }
  __device__ float value() const { return s; }
};
// Neumaier's compensated summation (Neumaier 1974) in FP32.
struct AccN {
  float s = 0.f, c = 0.f;
  __device__ void add(float v) {
    const float t = s + v;
    c += (fabsf(s) >= fabsf(v)) ? (s - t) + v : (v - t) + s;
    s = t;
  }
  __device__ void reduce(int G) {
    for (int off = G >> 1; off > 0; off >>= 1) {
      const float s2 = __shfl_xor_sync(kFull, s, off);
      const float c2 = __shfl_xor_sync(kFull, c, off);
      const float t = s + s2;
      const float e = (fabsf(s) >= fabsf(s2)) ? (s - t) + s2 : (s2 - t) + s;
      c = c + c2 + e;
      s = t;
    }
  }
  __device__ float value() const { return s + c; }
};

__device__ __forceinline__ int pow2_floor_32(int g) {
  return g >= 32 ? 32 : g >= 16 ? 16 : g >= 8 ? 8 : g >= 4 ? 4 : g >= 2 ? 2 : 1;
}

template <class ST>
__device__ __forceinline__ typename ST::R decode(const typename ST::S v, typename ST::R w, typename ST::R ws) {
  if constexpr (ST::dev) {
    return fmaf(ws, ST::to_r(v), w);
  } else {
    (void)w;
    (void)ws;
    return typename ST::R(v);
  }
}

// Phase 2: rho, u_x, u_y of every node of the tile into s_mom.
template <class ST, class Acc>
__device__ void tile_moments(const StageArgs<typename ST::R>& a, const typename ST::S* s_f,
                             const typename ST::R* s_scale, typename ST::R* s_mom, int ne) {
  using R = typename ST::R;
  const int Qp = a.Qp, tid = threadIdx.x, nth = blockDim.x;
  const int G = pow2_floor_32(nth / (a.epc * NP));
  const int ngroups = nth / G, grp = tid / G, lane = tid % G;
  const int npair = ne * NP;
  const R* ex = a.vel + kVelEx * Qp;
  const R* ey = a.vel + kVelEy * Qp;
  const R* wv = a.vel + kVelW * Qp;
  const R* wex = a.vel + kVelWex * Qp;
  const R* wey = a.vel + kVelWey * Qp;
  for (int base = 0; base < npair; base += ngroups) {
    const int pair = base + grp;
    const bool valid = pair < npair;
    Acc m0, m1, m2;
    if (valid) {
      const typename ST::S* row = s_f + size_t(pair) * Qp;
      for (int i = lane; i < Qp; i += G) {
        if constexpr (ST::dev) {
          const float q = ST::to_r(row[i]);
          m0.add(wv[i] * q);
          m1.add(wex[i] * q);
          m2.add(wey[i] * q);
        } else {
          const R f = row[i];
          m0.add(f);
          m1.add(ex[i] * f);
          m2.add(ey[i] * f);
        }
      }
    }
    m0.reduce(G);
    m1.reduce(G);
    m2.reduce(G);
    if (valid && lane == 0) {
      double rho, jx, jy;
      if constexpr (ST::dev) {
        const double sc = s_scale[pair / NP];
        rho = double(a.W0) + sc * double(m0.value());
        jx = double(a.W1x) + sc * double(m1.value());
        jy = double(a.W1y) + sc * double(m2.value());
      } else {
        rho = m0.value();
        jx = m1.value();
        jy = m2.value();
      }
      R* mm = s_mom + size_t(pair) * 4;
      mm[0] = R(rho);
      mm[1] = R(jx / rho);
      mm[2] = R(jy / rho);
    }
  }
}

// Phase 3: numerators of eq. FullBC, sum over outgoing velocities of (e.n) f^-.
template <class ST>
__device__ void tile_wall_numerators(const StageArgs<typename ST::R>& a, const typename ST::S* s_f,
                                     const typename ST::R* s_geo, const int* s_nbr,
                                     const typename ST::R* s_scale, typename ST::R* s_wn, int ne) {
  using R = typename ST::R;
  const int Qp = a.Qp, tid = threadIdx.x, nth = blockDim.x;
  const int G = pow2_floor_32(nth / (a.epc * NF));
  const int ngroups = nth / G, grp = tid / G, lane = tid % G;
  const int ntrip = ne * NF;
  const R* ex = a.vel + kVelEx * Qp;
  const R* ey = a.vel + kVelEy * Qp;
  const R* wv = a.vel + kVelW * Qp;
  for (int base = 0; base < ntrip; base += ngroups) {
    const int trip = base + grp;
    const int e = trip / NF, fc = (trip % NF) / NFP, aa = trip % NFP;
    bool active = false;
    if (trip < ntrip) {
      const int code = s_nbr[e * 3 + fc];
      active = code < 0 && ((a.wall_diffuse_mask >> (-code - 1)) & 1);
    }
    typename ST::R acc = 0;
    if (active) {
      const R nxf = s_geo[e * kGeoStrideDev + 4 + 3 * fc];
      const R nyf = s_geo[e * kGeoStrideDev + 5 + 3 * fc];
      const int node = (fc == 0) ? aa : (fc == 1 ? aa * (P + 1) - aa * (aa - 1) / 2 + (P - aa)
                                                 : aa * (P + 1) - aa * (aa - 1) / 2);
      const typename ST::S* row = s_f + (size_t(e) * NP + node) * Qp;
      const R sc = ST::dev ? s_scale[e] : R(0);
      for (int i = lane; i < Qp; i += G) {
        const R en = ex[i] * nxf + ey[i] * nyf;
        if (en > 0) acc += en * decode<ST>(row[i], wv[i], wv[i] * sc);
      }
    }
    for (int off = G >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    if (active && lane == 0) s_wn[trip] = acc;
  }
}

template <class ST>
__global__ void __launch_bounds__(512) stage_kernel(const StageArgs<typename ST::R> a) {
  using R = typename ST::R;
  using S = typename ST::S;
  extern __shared__ __align__(16) unsigned char smem[];
  const int epc = a.epc, Qp = a.Qp;
  const int64_t k0 = int64_t(blockIdx.x) * epc;
  const int ne = int(min(int64_t(epc), a.K - k0));
  const int tid = threadIdx.x, nth = blockDim.x;

  unsigned char* p = smem;
  S* s_f = reinterpret_cast<S*>(p);
  p += align16(size_t(epc) * NP * Qp * sizeof(S));
  R* s_geo = reinterpret_cast<R*>(p);
  p += align16(size_t(epc) * kGeoStrideDev * sizeof(R));
  int* s_nbr = reinterpret_cast<int*>(p);
  p += align16(size_t(epc) * 3 * 4);
  R* s_scale = reinterpret_cast<R*>(p);
  p += align16(size_t(epc) * 4 * sizeof(R));
  R* s_mom = reinterpret_cast<R*>(p);
  p += align16(size_t(epc) * NP * 4 * sizeof(R));
  R* s_wn = reinterpret_cast<R*>(p);
  p += align16(size_t(epc) * NF * sizeof(R));
  float* s_fnew = nullptr;
  unsigned* s_max = nullptr;
  if constexpr (ST::dev) {
    s_fnew = reinterpret_cast<float*>(p);
    p += align16(size_t(epc) * NP * Qp * 4);
    s_max = reinterpret_cast<unsigned*>(p);
  }

  // ---- 1. tile load --------------------------------------------------------
  {
    const S* fin = static_cast<const S*>(a.f_in);
    const size_t nvec = size_t(ne) * NP * Qp * sizeof(S) / 16;
    const uint4* src = reinterpret_cast<const uint4*>(fin + k0 * NP * Qp);
    uint4* dst = reinterpret_cast<uint4*>(s_f);
    for (size_t v = tid; v < nvec; v += nth) dst[v] = __ldg(src + v);
    for (int v = tid; v < ne * kGeoStrideDev; v += nth) s_geo[v] = a.geo[k0 * kGeoStrideDev + v];
    for (int v = tid; v < ne * 3; v += nth) s_nbr[v] = a.nbr[k0 * 3 + v];
    if constexpr (ST::dev) {
      for (int v = tid; v < ne; v += nth) {
        s_scale[v] = a.scale_in[k0 + v];
        s_max[v] = 0u;
      }
    }
  }
  __syncthreads();

  // ---- 2. node moments ---------------------------------------------------------
  if (a.collision) {
    if constexpr (sizeof(R) == 8) {
      tile_moments<ST, AccD>(a, s_f, s_scale, s_mom, ne);
    } else {
      if (a.red == kRedFP64) tile_moments<ST, AccD>(a, s_f, s_scale, s_mom, ne);
      else if (a.red == kRedCompFP32) tile_moments<ST, AccN>(a, s_f, s_scale, s_mom, ne);
      else tile_moments<ST, AccF>(a, s_f, s_scale, s_mom, ne);
    }
  }
  // ---- 3. wall numerators ------------------------------------------------------
  if (a.wall_diffuse_mask) tile_wall_numerators<ST>(a, s_f, s_geo, s_nbr, s_scale, s_wn, ne);
  __syncthreads();

  // ---- 4. residual and update per (element, velocity) ---------------------------
  const R dt = a.dt, rkA = a.rkA, rkB = a.rkB, ab = a.ab, inv_tau = a.inv_tau;
  const S* fin = static_cast<const S*>(a.f_in);
  float dmax = 0.f;
  int emax = -1;
  for (int item = tid; item < epc * Qp; item += nth) {
    const int e = item / Qp;
    const int i = item - e * Qp;
    if (e >= ne) break;
    const int64_t k = k0 + e;
    const R ex = a.vel[kVelEx * Qp + i], ey = a.vel[kVelEy * Qp + i], w = a.vel[kVelW * Qp + i];
    const R* g = s_geo + e * kGeoStrideDev;
    const R ar = ex * g[0] + ey * g[2];
    const R as = ex * g[1] + ey * g[3];
    R ws = 0;
    if constexpr (ST::dev) ws = w * s_scale[e];

    R fr[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) fr[m] = decode<ST>(s_f[(size_t(e) * NP + m) * Qp + i], w, ws);

    R flux[NF];
#pragma unroll
    for (int fc = 0; fc < 3; ++fc) {
      const R en = ex * g[4 + 3 * fc] + ey * g[5 + 3 * fc];
      const R c = R(0.5) * (en - ab * fabs(en)) * g[6 + 3 * fc];
      const int code = s_nbr[e * 3 + fc];
      if (c != R(0) && code >= 0) {
        const int64_t kn = code >> 3;
        const int fn = (code >> 1) & 3;
        const int rv = code & 1;
        const S* nb = fin + kn * NP * Qp + i;
        R wsn = 0;
        if constexpr (ST::dev) wsn = w * __ldg(a.scale_in + kn);
#pragma unroll
        for (int aa = 0; aa < NFP; ++aa) {
          const int a2 = rv ? NFP - 1 - aa : aa;
          const int rs = a2 * (P + 1) - a2 * (a2 - 1) / 2;
          const int node = fn == 0 ? a2 : (fn == 1 ? rs + (P - a2) : rs);
          const R fp = decode<ST>(__ldg(nb + size_t(node) * Qp), w, wsn);
          flux[fc * NFP + aa] = c * (fr[face_node(fc, aa)] - fp);
        }
      } else if (c != R(0) && en < R(0)) {
        const int side = -code - 1;
        const R fb = a.wall_feq[side * Qp + i];
        const bool diffuse = (a.wall_diffuse_mask >> side) & 1;
        const R scale = diffuse ? a.wall_den_inv[side] * fb : R(0);
#pragma unroll
        for (int aa = 0; aa < NFP; ++aa) {
          const R fp = diffuse ? s_wn[e * NF + fc * NFP + aa] * scale : fb;
          flux[fc * NFP + aa] = c * (fr[face_node(fc, aa)] - fp);
        }
      } else {
#pragma unroll
        for (int aa = 0; aa < NFP; ++aa) flux[fc * NFP + aa] = R(0);
      }
    }

    const int64_t gbase = k * NP * Qp + i;
    float dloc = 0.f;
    const R invw = ST::dev ? a.vel[kVelInvW * Qp + i] : R(0);
#pragma unroll
    for (int n = 0; n < NP; ++n) {
      R dr = 0, ds = 0;
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        dr = fma(opv<R>(OFF_DR + n * NP + m), fr[m], dr);
        ds = fma(opv<R>(OFF_DS + n * NP + m), fr[m], ds);
      }
      R lf = 0;
#pragma unroll
      for (int j = 0; j < NF; ++j) lf = fma(opv<R>(OFF_LIFT + n * NF + j), flux[j], lf);
      R rhs = lf - (ar * dr + as * ds);
      if (a.collision) {
        const R* mm = s_mom + (size_t(e) * NP + n) * 4;
        const R rho = mm[0], ux = mm[1], uy = mm[2];
        const R eu = ex * ux + ey * uy, uu = ux * ux + uy * uy;
        R poly = R(1) + eu + R(0.5) * (eu * eu - uu);
        if (a.eq_order == 3) poly += eu * (eu * eu * R(1.0 / 6.0) - R(0.5) * uu);
        rhs -= (fr[n] - w * rho * poly) * inv_tau;
      }
      const int64_t gi = gbase + int64_t(n) * Qp;
      R r = dt * rhs;
      if (rkA != R(0)) r = fma(rkA, a.res[gi], r);
      a.res[gi] = r;
      const R fnew = fma(rkB, r, fr[n]);
      if constexpr (ST::dev) {
        s_fnew[(size_t(e) * NP + n) * Qp + i] = fnew;
        dloc = fmaxf(dloc, fabsf((fnew - w) * invw));
      } else {
        static_cast<S*>(a.f_out)[gi] = S(fnew);
      }
    }
    if constexpr (ST::dev) {
      if (e != emax) {
        if (emax >= 0) atomicMax(&s_max[emax], __float_as_uint(dmax));
        emax = e;
        dmax = 0.f;
      }
      dmax = fmaxf(dmax, dloc);
    }
  }

  // ---- 5. deviation forms: new per-element scale and encoding ------------------
  if constexpr (ST::dev) {
    if (emax >= 0) atomicMax(&s_max[emax], __float_as_uint(dmax));
    __syncthreads();
    for (int e = tid; e < ne; e += nth) {
      const float md = __uint_as_float(s_max[e]);
      float sc = 1.0f;
      if (md > 0.f) {
        int ex2;
        frexpf(md, &ex2);
        sc = ldexpf(1.0f, ex2 - ST::qmax_log2);
      }
      s_scale[e] = sc;
      a.scale_out[k0 + e] = sc;
    }
    __syncthreads();
    const int nvec = ne * NP * Qp / 8;
    S* fout = static_cast<S*>(a.f_out) + k0 * NP * Qp;
    for (int v = tid; v < nvec; v += nth) {
      const int idx = v * 8;
      const int e = idx / (NP * Qp);
      const int i0 = idx % Qp;
      const float inv_s = 1.0f / s_scale[e];
      __align__(16) S q[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float w = a.vel[kVelW * Qp + i0 + j];
        const float invw = a.vel[kVelInvW * Qp + i0 + j];
        q[j] = ST::from_r((s_fnew[idx + j] - w) * invw * inv_s);
      }
      reinterpret_cast<uint4*>(fout)[v] = *reinterpret_cast<const uint4*>(q);
    }
  }
}

template <class ST>
cudaError_t launch_one(const void* args, int grid, int block, size_t smem, cudaStream_t st) {
  const auto& a = *static_cast<const StageArgs<typename ST::R>*>(args);
  stage_kernel<ST><<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

template <class ST>
cudaError_t set_smem_one(size_t smem) {
  return cudaFuncSetAttribute(stage_kernel<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

cudaError_t launch(int store_kind, const void* args, int grid, int block, size_t smem, cudaStream_t st) {
  switch (store_kind) {
    case kStoreF64: return launch_one<StoreF64>(args, grid, block, smem, st);
    case kStoreF32: return launch_one<StoreF32>(args, grid, block, smem, st);
    case kStoreBF16: return launch_one<StoreBF16>(args, grid, block, smem, st);
    case kStoreF16: return launch_one<StoreF16>(args, grid, block, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t set_smem(int store_kind, size_t smem) {
  switch (store_kind) {
    case kStoreF64: return set_smem_one<StoreF64>(smem);
    case kStoreF32: return set_smem_one<StoreF32>(smem);
    case kStoreBF16: return set_smem_one<StoreBF16>(smem);
    case kStoreF16: return set_smem_one<StoreF16>(smem);
  }
  return cudaErrorInvalidValue;
}

cudaError_t upload(const double* Dr, const double* Ds, const double* LIFT) {
  double h64[OPS_N];
  float h32[OPS_N];
  for (int j = 0; j < NP * NP; ++j) {
    h64[OFF_DR + j] = Dr[j];
    h64[OFF_DS + j] = Ds[j];
  }
  for (int j = 0; j < NP * NF; ++j) h64[OFF_LIFT + j] = LIFT[j];
  for (int j = 0; j < OPS_N; ++j) h32[j] = float(h64[j]);
  cudaError_t e = cudaMemcpyToSymbol(c_ops64, h64, sizeof(h64));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_ops32, h32, sizeof(h32));
}

}  // namespace

StageEntry FEDBM_STAGE_ENTRY_NAME() {
  StageEntry s;
  s.launch = &launch;
  s.set_smem = &set_smem;
  s.upload = &upload;
  return s;
}

}  // namespace fedbm
