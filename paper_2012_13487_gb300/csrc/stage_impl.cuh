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
// the old one).
//
// Phases of a CTA:
//   1. bulk-copy (TMA) the element tile f[k0:k0+epc][Np][Qp] and its geometry
//      (first barrier), the residual tile and every neighbour face row (second
//      barrier) into shared memory;
//   2. node moments rho, u (Sec. II.A.2) by a G-lane reduction per node, kept
//      as the coefficients of f^eq/tau per node, while the second part lands;
//   3. wall numerators sum_{e.n>0} (e.n) f^- of eq. FullBC per wall node;
//   4. residual and update, one thread per (element, velocity) item, with
//      Dr, Ds, LIFT as instruction immediates (compile-time tables) or
//      constant-memory operands of unrolled FMAs (the 16-bit forms up to
//      degree 3 take two velocities per thread as packed FP32 pairs,
//      fma.rn.f32x2);
//   5. deviation forms only: per-element scale from max |f/w - 1|, encode;
//   6. bulk-store the new state and residual tiles.
#include "device_common.cuh"
#include "stage_dispatch.h"

#include <cstring>

// Largest degree whose 16-bit forms take two velocities per thread (and the
// FP32 state too when FEDBM_VPT2_FP32_STATE is 1); FEDBM_PACKED_FMA = 1 runs
// the two velocities' contractions as packed FP32 pairs.  Measured on the BF16
// cavities: two velocities per thread are faster at degree 3, one at degree 4.
#ifndef FEDBM_VPT2_MAX_P
#define FEDBM_VPT2_MAX_P 3
#endif
#ifndef FEDBM_VPT2_FP32_STATE
#define FEDBM_VPT2_FP32_STATE 0
#endif
#ifndef FEDBM_PACKED_FMA
#define FEDBM_PACKED_FMA 1
#endif
// FEDBM_FACE_SKIP = 0: the FMA kernel evaluates every face's flux and lift
// columns also where a whole warp leaves an element through the face
#ifndef FEDBM_FACE_SKIP
#define FEDBM_FACE_SKIP 1
#endif

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
// every FP32 coefficient twice, as the broadcast operand of a packed FMA
static __constant__ unsigned long long c_ops32x2[OPS_N];

#include "ops_tables.inc"

// Dr, Ds, LIFT entry idx in the compute precision.  kImm: the FP32 operators
// of this degree as a compile-time table (the operators depend only on the
// degree, and with the node loops unrolled every entry becomes an instruction
// immediate instead of a constant-memory load; the table holds the runtime
// upload's values, which a CPU test checks); otherwise constant memory.
template <typename R, bool kImm>
__device__ __forceinline__ R opv(int idx);
template <>
__device__ __forceinline__ float opv<float, false>(int idx) { return c_ops32[idx]; }
template <>
__device__ __forceinline__ double opv<double, false>(int idx) { return c_ops64[idx]; }
#ifdef FEDBM_OPS32_TABLE
constexpr bool kHaveOpsTable = true;
template <>
__device__ __forceinline__ float opv<float, true>(int idx) {
  constexpr float t[] = {FEDBM_OPS32_TABLE};
  static_assert(sizeof(t) / sizeof(t[0]) == OPS_N, "operator table of another degree");
  return t[idx];
}
#else
constexpr bool kHaveOpsTable = false;
template <>
__device__ __forceinline__ float opv<float, true>(int idx) { return c_ops32[idx]; }
#endif
template <>
__device__ __forceinline__ double opv<double, true>(int idx) { return c_ops64[idx]; }

// Which FMA kernels take the operators as immediates: every FP32-arithmetic
// kernel up to degree 4; at degree 5 (1,260 operator entries) only the
// compile-time velocity counts of the FP32 and BF16 states, which keeps that
// translation unit's compile time within a few minutes.
template <class ST, int QT>
__host__ __device__ constexpr bool ops_immediate() {
  return kHaveOpsTable && sizeof(typename ST::R) == 4 &&
         (P <= 4 || (QT > 0 && (ST::kind == kStoreF32 || ST::kind == kStoreBF16)));
}

// Node index of face node a on face f (rows of the reference triangle start at
// a(P+1) - a(a-1)/2; face 0 is row 0, face 1 the row ends, face 2 the row starts).
__host__ __device__ constexpr int face_node(int f, int a) {
  return f == 0 ? a : (f == 1 ? a * (P + 1) - a * (a - 1) / 2 + (P - a) : a * (P + 1) - a * (a - 1) / 2);
}

constexpr unsigned kFull = 0xffffffffu;

// Packed FP32 pairs (two velocities of one node in a 64-bit register pair):
// fma.rn.f32x2 rounds each half exactly like fmaf.
__device__ __forceinline__ unsigned long long f2pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2unpack(unsigned long long p, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p));
}
__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

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

__host__ __device__ constexpr int pow2_floor_32(int g) {
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

// ---- asynchronous bulk copies (TMA, non-tensor) and their mbarrier -----------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// try_wait with a suspend-time hint: a thread whose phase is not complete is
// suspended until the phase completes or about hint_ns pass, instead of
// returning at once, so that waiting warps do not take issue slots from the
// warps that compute.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of the barrier for at most about `limit_ns` (each
// suspended try_wait lasts at most 20 us past the limit); false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (!mbar_try_wait_suspend(bar, parity, 20000u)) {
    if (global_timer_ns() - t0 > limit_ns) return false;
  }
  return true;
}
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst_smem)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src_smem)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until every committed bulk store of this thread has finished reading shared memory
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Vector of the storage type covering 16 bytes.
template <class ST>
struct Vec16 {
  static constexpr int N = 16 / int(sizeof(typename ST::S));
};

// Phase 2: rho, u_x, u_y of every node of the tile into s_mom.  G lanes share a
// node; each lane reduces 16-byte chunks of the node's velocity row.
// Lanes per node group: the largest power of two <= 32 that gives every node
// of the tile a group and no lane more than one chunk fewer than another.
__host__ __device__ constexpr int moment_lanes(int nth, int epc, int nchunk) {
  int G = pow2_floor_32(nth / (epc * NP));
  while (G > 1 && G > nchunk) G >>= 1;
  return G;
}

// NTH > 0: a CTA of NTH threads and EPC elements per tile (the tensor-core
// kernel), so the lane grouping and the chunk loop are compile-time.
template <class ST, class Acc, int QT, int NTH = 0, int EPC = 1>
__device__ void tile_moments(const StageArgs<typename ST::R>& a, const typename ST::S* s_f,
                             const float* s_scale, const typename ST::R* s_geo, typename ST::R* s_mom, int ne,
                             const typename ST::R* s_vel) {
  using R = typename ST::R;
  using S = typename ST::S;
  constexpr int V = Vec16<ST>::N;
  static_assert(NTH == 0 || QT > 0, "a compile-time CTA needs a compile-time velocity count");
  const int Qp = QT > 0 ? QT : a.Qp, tid = threadIdx.x, nth = NTH > 0 ? NTH : blockDim.x;
  const int nchunk = Qp / V;
  const int G = NTH > 0 ? moment_lanes(NTH, EPC, (QT > 0 ? QT : 1) / V) : moment_lanes(nth, a.epc, nchunk);
  const int ngroups = nth / G, grp = tid / G, lane = tid % G;
  const int npair = ne * NP;
  const R* ex = s_vel + kVelEx * Qp;  // shared-memory copy of the velocity rows
  const R* ey = s_vel + kVelEy * Qp;
  const R* wv = s_vel + kVelW * Qp;
  for (int base = 0; base < npair; base += ngroups) {
    const int pair = base + grp;
    const bool valid = pair < npair;
    Acc m0, m1, m2;
    if (valid) {
      const S* row = s_f + size_t(pair) * Qp;
      auto chunk = [&](int c) {
        __align__(16) S v[V];
        __align__(16) R exv[V], eyv[V], wvv[V];
        *reinterpret_cast<uint4*>(v) = *reinterpret_cast<const uint4*>(row + c * V);
#pragma unroll
        for (int j = 0; j < V * int(sizeof(R)) / 16; ++j) {
          reinterpret_cast<uint4*>(exv)[j] = reinterpret_cast<const uint4*>(ex + c * V)[j];
          reinterpret_cast<uint4*>(eyv)[j] = reinterpret_cast<const uint4*>(ey + c * V)[j];
          if constexpr (ST::dev) reinterpret_cast<uint4*>(wvv)[j] = reinterpret_cast<const uint4*>(wv + c * V)[j];
        }
        // sums over the chunk in the compute precision, then one accumulator
        // update per chunk (FP64 or compensated across chunks)
        R c0 = 0, c1 = 0, c2 = 0;
#pragma unroll
        for (int j = 0; j < V; ++j) {
          R f;
          if constexpr (ST::dev) f = wvv[j] * ST::to_r(v[j]);
          else f = v[j];
          c0 += f;
          c1 = fma(exv[j], f, c1);
          c2 = fma(eyv[j], f, c2);
        }
        m0.add(c0);
        m1.add(c1);
        m2.add(c2);
      };
      if constexpr (NTH > 0) {
        constexpr int GC = moment_lanes(NTH > 0 ? NTH : 1, EPC, (QT > 0 ? QT : V) / V);
#pragma unroll 8
        for (int c = 0; c < (QT > 0 ? QT : V) / V; c += GC) chunk(c + lane);
      } else {
        for (int c = lane; c < nchunk; c += G) chunk(c);
      }
    }
    m0.reduce(G);
    m1.reduce(G);
    m2.reduce(G);
    if (valid && lane == 0) {
      // in the compute precision R: FP64 arithmetic is kept out of the FP32 paths
      R rho, jx, jy;
      if constexpr (ST::dev) {
        const R sc = s_scale[pair / NP];
        rho = a.W0 + sc * R(m0.value());
        jx = a.W1x + sc * R(m1.value());
        jy = a.W1y + sc * R(m2.value());
      } else {
        rho = R(m0.value());
        jx = R(m1.value());
        jy = R(m2.value());
      }
      // f^eq_i / tau = w_i [m0 + e_x m1 + e_y m2 + m3 (e.u)^2 + (e.u)(m6 (e.u)^2 - m7)]
      // with e.u = e_x m4 + e_y m5 (eq. feq; the m6, m7 terms are the third
      // Hermite order of eq. Herm3a and vanish for eq_order 2)
      const R irho = R(1) / rho;
      const R it = s_geo[(pair / NP) * kGeoStrideDev + kGeoInvTau];  // 1/tau of the element's case
      const R ux = jx * irho, uy = jy * irho, uu = ux * ux + uy * uy;
      const bool third = a.eq_order == 3;
      R* mm = s_mom + size_t(pair) * 8;
      mm[0] = rho * (R(1) - R(0.5) * uu) * it;
      mm[1] = jx * it;
      mm[2] = jy * it;
      mm[3] = R(0.5) * rho * it;
      mm[4] = ux;
      mm[5] = uy;
      mm[6] = third ? rho * it * R(1.0 / 6.0) : R(0);
      mm[7] = third ? R(0.5) * rho * uu * it : R(0);
    }
  }
}

// Phase 3: numerators of eq. FullBC, sum over outgoing velocities of (e.n) f^-.
template <class ST, int QT>
__device__ void tile_wall_numerators(const StageArgs<typename ST::R>& a, const typename ST::S* s_f,
                                     const typename ST::R* s_geo, const int* s_nbr,
                                     const float* s_scale, typename ST::R* s_wn, int ne,
                                     const typename ST::R* s_vel) {
  using R = typename ST::R;
  const int Qp = QT > 0 ? QT : a.Qp, tid = threadIdx.x, nth = blockDim.x;
  const int G = pow2_floor_32(nth / (a.epc * NF));
  const int ngroups = nth / G, grp = tid / G, lane = tid % G;
  const int ntrip = ne * NF;
  const R* ex = s_vel + kVelEx * Qp;  // shared-memory copy of the velocity rows
  const R* ey = s_vel + kVelEy * Qp;
  const R* wv = s_vel + kVelW * Qp;
  for (int base = 0; base < ntrip; base += ngroups) {
    const int trip = base + grp;
    const int e = trip / NF, fc = (trip % NF) / NFP, aa = trip % NFP;
    bool active = false;
    if (trip < ntrip) {
      const int code = s_nbr[e * 3 + fc];
      active = code < 0 && __ldg(a.wall_den_inv + (-code - 1)) > R(0);
    }
    R acc = 0;
    if (active) {
      const R nxf = s_geo[e * kGeoStrideDev + 4 + 3 * fc];
      const R nyf = s_geo[e * kGeoStrideDev + 5 + 3 * fc];
      const int rs = aa * (P + 1) - aa * (aa - 1) / 2;
      const int node = (fc == 0) ? aa : (fc == 1 ? rs + (P - aa) : rs);
      const typename ST::S* row = s_f + (size_t(e) * NP + node) * Qp;
      const R sc = ST::dev ? s_scale[e] : R(0);
      for (int i = lane; i < Qp; i += G) {
        const R en = ex[i] * nxf + ey[i] * nyf;
        const R w = ST::dev ? wv[i] : R(0);  // the plain forms do not use (or hold) the w row
        if (en > 0) acc += en * decode<ST>(row[i], w, w * sc);
      }
    }
    for (int off = G >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    if (active && lane == 0) s_wn[trip] = acc;
  }
}

// new f of one value: decode, then f + B res (shared by the update and the
// encoding pass of the deviation forms so both see the same rounding)
template <class ST>
__device__ __forceinline__ typename ST::R new_f(typename ST::R fold, typename ST::R rkB, typename ST::R r) {
  return fma(rkB, r, fold);
}

// tau-scaled collision term w f^eq(rho, u)/tau - f/tau of one value, from the
// node record written by tile_moments (all zero when collision is off)
template <typename R>
__device__ __forceinline__ R collision(const R* mm, R ex, R ey, R w, R f, R inv_tau, bool third) {
  const R eu = ex * mm[4] + ey * mm[5];
  R feq = fma(ey, mm[2], fma(ex, mm[1], mm[0]));
  feq = fma(eu, mm[3] * eu, feq);
  if (third) feq = fma(eu, fma(mm[6], eu * eu, -mm[7]), feq);
  return fma(w, feq, -inv_tau * f);
}

// Deviation form whose 16-bit format has FP32's exponent range (BF16): a
// power-of-two element scale changes neither the rounding of q nor the decoded
// f = w (1 + s q), so the element keeps the scale it was encoded with and the
// new state is encoded where it is computed.  FP16 (|q| < 2^15) must rescale.
template <class ST>
__host__ __device__ constexpr bool keeps_scale() {
  if constexpr (ST::dev) return ST::qmax_log2 == 0;
  else return false;
}

// Adjacent velocities handled by one thread in phase 4: two for the
// specialised 16-bit-state kernels up to degree 3 (each operator constant then
// feeds two FMAs and the per-item set-up is shared), else one.
template <class ST, int QT>
__host__ __device__ constexpr int items_vpt() {
  return (QT > 0 && sizeof(typename ST::R) == 4 && (ST::dev || FEDBM_VPT2_FP32_STATE) && P <= FEDBM_VPT2_MAX_P)
             ? 2
             : 1;
}

template <typename T, int N>
struct alignas(N * sizeof(T)) Vec {
  T v[N];
};

// Phase 4: residual, 2N-storage update and write-back of every (element,
// velocity) value of the tile; each thread owns VPT adjacent velocities of one
// element.  Plain forms and BF16 (kept element scale) update f in place in
// shared memory; FP16 only tracks max |f/w - 1| per element (the encoding pass
// recomputes f with the new scale).
template <class ST, int QT, int VPT>
__device__ __forceinline__ void item_update(const StageArgs<typename ST::R>& a,
                                            StageSmem<typename ST::R, typename ST::S>& sm, int64_t k0, int ne,
                                            bool read_res, float& dmax, int& emax) {
  using R = typename ST::R;
  using S = typename ST::S;
  using SV = Vec<S, VPT>;
  using RV = Vec<R, VPT>;
  const int Qp = QT > 0 ? QT : a.Qp;
  const int Qv = Qp / VPT;
  const int tid = threadIdx.x, nth = blockDim.x;
  const R rkA = a.rkA, rkB = a.rkB, ab = a.ab;
  const bool third = a.eq_order == 3;
  constexpr bool kPacked = FEDBM_PACKED_FMA && sizeof(R) == 4 && VPT == 2;
  constexpr bool kImm = ops_immediate<ST, QT>();
  // outflow faces skipped per warp where a warp's items belong to one element
  // (one velocity per thread: with two, the packed lift accumulators measured
  // slower, 2.26e11 vs 2.37e11 on the BF16 NC 32x32 cavity)
  constexpr bool kSkip = FEDBM_FACE_SKIP && QT >= 128 && VPT == 1;
  constexpr bool kKeep = keeps_scale<ST>();
  constexpr bool kTrack = ST::dev && !kKeep;
  // stochastic rounding of the BF16 encode: the step counter is read once
  const bool sr = kKeep && a.sr_step != nullptr;
  const uint32_t sr_step = sr ? __ldg(a.sr_step) : 0u;
  for (int item = tid; item < ne * Qv; item += nth) {
    const int e = item / Qv;
    const int i = (item - e * Qv) * VPT;
    const RV exv = *reinterpret_cast<const RV*>(a.vel + kVelEx * Qp + i);
    const RV eyv = *reinterpret_cast<const RV*>(a.vel + kVelEy * Qp + i);
    const RV wv = *reinterpret_cast<const RV*>(a.vel + kVelW * Qp + i);
    const R* g = sm.geo + e * kGeoStrideDev;
    const R dt = g[kGeoDt], inv_tau = g[kGeoInvTau];  // per element: cases of a batch differ
    R ar[VPT], as[VPT], ws[VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      ar[v] = exv.v[v] * g[0] + eyv.v[v] * g[2];
      as[v] = exv.v[v] * g[1] + eyv.v[v] * g[3];
      ws[v] = ST::dev ? wv.v[v] * R(sm.scale[e]) : R(0);
    }
    S* frow = sm.f + size_t(e) * NP * Qp + i;
    R* rrow = sm.res + size_t(e) * NP * Qp + i;

    R fr[VPT][NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      const SV x = *reinterpret_cast<const SV*>(frow + m * Qp);
#pragma unroll
      for (int v = 0; v < VPT; ++v) fr[v][m] = decode<ST>(x.v[v], wv.v[v], ws[v]);
    }

    R flux[VPT][NF];
    // kSkip: face fc carries flux for some velocity of the lanes running this
    // iteration together (an outflow face's upwind jump term is zero), else
    // its traces and lift columns are skipped
    bool on[3];
#pragma unroll
    for (int fc = 0; fc < 3; ++fc) {
      R c[VPT], en[VPT];
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        en[v] = exv.v[v] * g[4 + 3 * fc] + eyv.v[v] * g[5 + 3 * fc];
        c[v] = R(0.5) * (en[v] - ab * fabs(en[v])) * g[6 + 3 * fc];
      }
      const int code = sm.nbr[e * 3 + fc];
      on[fc] = true;
      if constexpr (kSkip) {
        bool nz = false;
#pragma unroll
        for (int v = 0; v < VPT; ++v) nz = nz || (c[v] != R(0) && (code >= 0 || en[v] < R(0)));
        on[fc] = __any_sync(__activemask(), nz);
#pragma unroll
        for (int v = 0; v < VPT; ++v)
#pragma unroll
          for (int aa = 0; aa < NFP; ++aa) flux[v][fc * NFP + aa] = R(0);
        if (!on[fc]) continue;
      }
      if (code >= 0) {
        R wsn[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) wsn[v] = ST::dev ? wv.v[v] * R(sm.nscale[e * 3 + fc]) : R(0);
        const S* trow = sm.tr + size_t(e * NF + fc * NFP) * Qp + i;
#pragma unroll
        for (int aa = 0; aa < NFP; ++aa) {
          const SV x = *reinterpret_cast<const SV*>(trow + aa * Qp);
#pragma unroll
          for (int v = 0; v < VPT; ++v)
            flux[v][fc * NFP + aa] = c[v] * (fr[v][face_node(fc, aa)] - decode<ST>(x.v[v], wv.v[v], wsn[v]));
        }
      } else {
        const int slot = -code - 1;  // wall slot: 4 * case + side
        const RV fbv = *reinterpret_cast<const RV*>(a.wall_feq + slot * Qp + i);
        const R den_inv = __ldg(a.wall_den_inv + slot);
        const bool diffuse = den_inv > R(0);
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          // incoming velocities take the wall state; outgoing ones have no jump
          const R scale = diffuse ? den_inv * fbv.v[v] : R(0);
#pragma unroll
          for (int aa = 0; aa < NFP; ++aa) {
            const R fp = diffuse ? sm.wn[e * NF + fc * NFP + aa] * scale : fbv.v[v];
            flux[v][fc * NFP + aa] = en[v] < R(0) ? c[v] * (fr[v][face_node(fc, aa)] - fp) : R(0);
          }
        }
      }
    }

    // kSkip: the lift contraction by faces, the faces without flux skipped
    // (the same accumulation order as the node loop's)
    R lfa[VPT][kSkip ? NP : 1];
    unsigned long long lfp2[kSkip && kPacked ? NP : 1];
    if constexpr (kSkip) {
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        if constexpr (kPacked) lfp2[n] = 0ull;
#pragma unroll
        for (int v = 0; v < VPT; ++v) lfa[v][n] = R(0);
      }
#pragma unroll
      for (int fc = 0; fc < 3; ++fc) {
        if (!on[fc]) continue;
#pragma unroll
        for (int aa = 0; aa < NFP; ++aa) {
          const int j = fc * NFP + aa;
          if constexpr (kPacked) {
            const unsigned long long x = f2pack(flux[0][j], flux[1][j]);
#pragma unroll
            for (int n = 0; n < NP; ++n) lfp2[n] = f2fma(c_ops32x2[OFF_LIFT + n * NF + j], x, lfp2[n]);
          } else {
#pragma unroll
            for (int n = 0; n < NP; ++n) {
              const R cl = opv<R, kImm>(OFF_LIFT + n * NF + j);
#pragma unroll
              for (int v = 0; v < VPT; ++v) lfa[v][n] = fma(cl, flux[v][j], lfa[v][n]);
            }
          }
        }
      }
    }
    float dloc = 0.f;
    R invw[VPT];
    if constexpr (ST::dev) {
      const RV iw = *reinterpret_cast<const RV*>(a.vel + kVelInvW * Qp + i);
#pragma unroll
      for (int v = 0; v < VPT; ++v) invw[v] = iw.v[v] * (kKeep ? R(1) / R(sm.scale[e]) : R(1));
    }
#pragma unroll
    for (int n = 0; n < NP; ++n) {
      RV rold;
      if (read_res) rold = *reinterpret_cast<const RV*>(rrow + n * Qp);
      R dr[VPT], ds[VPT], lf[VPT];
      if constexpr (kPacked) {
        // two velocities per packed FMA; the same rounding as the scalar form
        unsigned long long drp = 0ull, dsp = 0ull, lfp = 0ull;
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          const unsigned long long x = f2pack(fr[0][m], fr[1][m]);
          drp = f2fma(c_ops32x2[OFF_DR + n * NP + m], x, drp);
          dsp = f2fma(c_ops32x2[OFF_DS + n * NP + m], x, dsp);
        }
        if constexpr (kSkip) {
          lfp = lfp2[n];
        } else {
#pragma unroll
          for (int j = 0; j < NF; ++j)
            lfp = f2fma(c_ops32x2[OFF_LIFT + n * NF + j], f2pack(flux[0][j], flux[1][j]), lfp);
        }
        f2unpack(drp, dr[0], dr[VPT - 1]);
        f2unpack(dsp, ds[0], ds[VPT - 1]);
        f2unpack(lfp, lf[0], lf[VPT - 1]);
      } else {
#pragma unroll
        for (int v = 0; v < VPT; ++v) dr[v] = ds[v] = lf[v] = R(0);
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          const R cr = opv<R, kImm>(OFF_DR + n * NP + m), cs = opv<R, kImm>(OFF_DS + n * NP + m);
#pragma unroll
          for (int v = 0; v < VPT; ++v) {
            dr[v] = fma(cr, fr[v][m], dr[v]);
            ds[v] = fma(cs, fr[v][m], ds[v]);
          }
        }
        if constexpr (kSkip) {
#pragma unroll
          for (int v = 0; v < VPT; ++v) lf[v] = lfa[v][n];
        } else {
#pragma unroll
          for (int j = 0; j < NF; ++j) {
            const R cl = opv<R, kImm>(OFF_LIFT + n * NF + j);
#pragma unroll
            for (int v = 0; v < VPT; ++v) lf[v] = fma(cl, flux[v][j], lf[v]);
          }
        }
      }
      const R* mm = sm.mom + (size_t(e) * NP + n) * 8;
      RV rr;
      SV fnew_s;
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        R rhs = fma(-ar[v], dr[v], fma(-as[v], ds[v], lf[v]));
        rhs += collision<R>(mm, exv.v[v], eyv.v[v], wv.v[v], fr[v][n], inv_tau, third);
        R r = dt * rhs;
        if (read_res) r = fma(rkA, rold.v[v], r);
        rr.v[v] = r;
        const R fnew = new_f<ST>(fr[v][n], rkB, r);
        if constexpr (kTrack) {
          dloc = fmaxf(dloc, fabsf((fnew - wv.v[v]) * invw[v]));
        } else if constexpr (kKeep) {
          const float qv = (fnew - wv.v[v]) * invw[v];
          if (sr) {
            const uint64_t gi = (uint64_t(k0 + e) * NP + n) * uint64_t(Qp) + uint64_t(i + v);
            fnew_s.v[v] = bf16_round_stochastic(qv, sr_hash(gi, sr_step, uint32_t(a.sr_stage)));
          } else {
            fnew_s.v[v] = ST::from_r(qv);
          }
        } else {
          fnew_s.v[v] = S(fnew);
        }
      }
      *reinterpret_cast<RV*>(rrow + n * Qp) = rr;
      if constexpr (!kTrack) *reinterpret_cast<SV*>(frow + n * Qp) = fnew_s;
    }
    if constexpr (kTrack) {
      if (e != emax) {
        if (emax >= 0) atomicMax(&sm.dmax[emax], __float_as_uint(dmax));
        emax = e;
        dmax = 0.f;
      }
      dmax = fmaxf(dmax, dloc);
    }
  }
}

// Minimum resident CTAs of 256 threads per SM: bounds the registers per thread
// (65536 / (256 * min)) so that the unrolled node loop does not spill.  At
// degree 4 the shared memory of the usual 128-thread tile already limits an SM
// to four CTAs, so 128 registers cost no occupancy there (measured +4 %); at
// degree 5, 128 registers measured slower than 85.
template <class ST, int QT>
__host__ __device__ constexpr int stage_min_blocks() {
  return sizeof(typename ST::R) == 8 ? 2 : items_vpt<ST, QT>() == 2 ? 2 : (P <= 3 || P == 5 ? 3 : 2);
}


// Bulk copies (TMA) of one tile into a shared-memory stage, issued by warp 0:
// element tile, residual tile (stages 2..5), geometry and every neighbour face
// row, all completing on the stage's mbarrier; the lanes also store the face
// codes (and for the deviation forms the scales) of the tile.
template <class ST, int QT>
__device__ void issue_tile_loads(const StageArgs<typename ST::R>& a, StageSmem<typename ST::R, typename ST::S>& sm,
                                 int64_t k0, int ne, bool read_res) {
  using R = typename ST::R;
  using S = typename ST::S;
  const int lane = threadIdx.x & 31;
  const int Qp = QT > 0 ? QT : a.Qp;
  const size_t row_bytes = size_t(Qp) * sizeof(S);
  const S* fin = static_cast<const S*>(a.f_in);
  const uint32_t tile_bytes = uint32_t(size_t(ne) * NP * row_bytes);
  const uint32_t res_bytes = uint32_t(size_t(ne) * NP * Qp * sizeof(R));
  const uint32_t geo_bytes = uint32_t(size_t(ne) * kGeoStrideDev * sizeof(R));
  // plain shared-memory stores first: the release of the arrive below makes
  // them visible to every thread that waits on the barrier
  for (int v = lane; v < ne * 3; v += 32) {
    const int code = __ldg(a.nbr + k0 * 3 + v);
    sm.nbr[v] = code;
    if constexpr (ST::dev) sm.nscale[v] = code >= 0 ? __ldg(a.scale_in + (code >> 3)) : 0.f;
  }
  if constexpr (ST::dev) {
    for (int v = lane; v < ne; v += 32) {
      sm.scale[v] = __ldg(a.scale_in + k0 + v);
      sm.dmax[v] = 0u;
    }
  }
  // two barriers: bar[0] for the element tile and geometry (needed first, by
  // the moment and wall-numerator reductions), bar[1] for the residual tile
  // and the neighbour traces (needed only by the update), so the reductions
  // start while the larger second part is still in flight
  uint64_t* bar_rt = sm.bar + 1;
  uint32_t bytes = 0;
  if (lane == 0) bytes += (read_res ? res_bytes : 0u);
  for (int row = lane; row < ne * NF; row += 32) {
    const int code = __ldg(a.nbr + (k0 + row / NF) * 3 + (row % NF) / NFP);
    if (code >= 0) bytes += uint32_t(row_bytes);
  }
  mbar_arrive_expect_tx(sm.bar, lane == 0 ? tile_bytes + geo_bytes + a.extra_tx : 0u);
  mbar_arrive_expect_tx(bar_rt, bytes);
  if (lane == 0) {
    bulk_load(sm.f, fin + k0 * NP * Qp, tile_bytes, sm.bar);
    bulk_load(sm.geo, a.geo + k0 * kGeoStrideDev, geo_bytes, sm.bar);
    if (read_res) bulk_load(sm.res, a.res + k0 * NP * Qp, res_bytes, bar_rt);
  }
  for (int row = lane; row < ne * NF; row += 32) {
    const int e = row / NF, fc = (row % NF) / NFP, aa = row % NFP;
    const int code = __ldg(a.nbr + (k0 + e) * 3 + fc);
    if (code >= 0) {
      const int64_t kn = code >> 3;
      const int fn = (code >> 1) & 3;
      const int a2 = (code & 1) ? NFP - 1 - aa : aa;
      const int rs = a2 * (P + 1) - a2 * (a2 - 1) / 2;
      const int node = fn == 0 ? a2 : (fn == 1 ? rs + (P - a2) : rs);
      bulk_load(sm.tr + size_t(row) * Qp, fin + (kn * NP + node) * Qp, uint32_t(row_bytes), bar_rt);
    }
  }
}

// Persistent kernel: CTA b handles tiles b, b + gridDim.x, ... through two
// shared-memory stages, loading tile j+1 while it computes tile j.
// QT > 0: the padded velocity count is the compile-time constant QT (all
// shared-memory strides become immediate offsets); QT = 0: taken from a.Qp.
template <class ST, int QT>
__global__ void __launch_bounds__(256, stage_min_blocks<ST, QT>()) stage_kernel(const StageArgs<typename ST::R> a) {
  using R = typename ST::R;
  using S = typename ST::S;
  extern __shared__ __align__(128) unsigned char smem[];
  const int epc = a.epc, Qp = QT > 0 ? QT : a.Qp;
  const int tid = threadIdx.x, nth = blockDim.x;
  const R rkA = a.rkA;
  const bool read_res = rkA != R(0);
  const int64_t ntiles = (a.K + epc - 1) / epc;
  const size_t stage_bytes = stage_smem_stride(NP, NF, epc, Qp, sizeof(S), sizeof(R));
  auto stage = [&](int sidx) { return carve_stage_smem<R, S>(smem + sidx * stage_bytes, NP, NF, epc, Qp); };
  const size_t row_bytes = size_t(Qp) * sizeof(S);

  const bool two = a.nstages == 2;
  // velocity rows e_x, e_y, w into every stage's copy (read by the moment and
  // wall-numerator reductions)
  for (int sidx = 0; sidx < (two ? 2 : 1); ++sidx) {
    R* sv = stage(sidx).vel;
    for (int v = tid; v < 3 * Qp; v += nth) sv[v] = a.vel[v];
  }
  if (tid == 0) {
    mbar_init(stage(0).bar, 32);
    mbar_init(stage(0).bar + 1, 32);
    if (two) {  // the second stage exists only when nstages == 2
      mbar_init(stage(1).bar, 32);
      mbar_init(stage(1).bar + 1, 32);
    }
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  __syncthreads();

  int64_t tile = blockIdx.x;
  if (tid < 32 && tile < ntiles) {
    StageSmem<R, S> s0 = stage(0);
    issue_tile_loads<ST, QT>(a, s0, tile * epc, int(min(int64_t(epc), a.K - tile * epc)), read_res);
  }

  for (int j = 0; tile < ntiles; ++j, tile += gridDim.x) {
    StageSmem<R, S> sm = stage(two ? (j & 1) : 0);
    const uint32_t parity = uint32_t((two ? (j >> 1) : j) & 1);
    const int64_t k0 = tile * epc;
    const int ne = int(min(int64_t(epc), a.K - k0));
    const int64_t next = tile + gridDim.x;
    if (tid < 32) {
      if (two && next < ntiles) {
        // prefetch the next tile into the other stage once its bulk store has read it
        if (tid == 0) bulk_wait_read();
        __syncwarp();
        StageSmem<R, S> sn = stage((j + 1) & 1);
        issue_tile_loads<ST, QT>(a, sn, next * epc, int(min(int64_t(epc), a.K - next * epc)), read_res);
      } else if (!two && j > 0) {
        // single stage: load this tile once the previous tile's store has read it
        if (tid == 0) bulk_wait_read();
        __syncwarp();
        issue_tile_loads<ST, QT>(a, sm, k0, ne, read_res);
      }
    }
    // warp 0 waits for the tile (suspended in try_wait); the other warps
    // wait at the block barrier, where they take no issue slots
    bool ok = true;
    if (tid < 32) ok = mbar_wait_bounded(sm.bar, parity, 2000000000ull);
    if (__syncthreads_or(!ok)) {
      if (tid == 0 && a.err) atomicExch(a.err, 1);
      // let copies still in flight land before the CTA exits
      if (tid < 32) mbar_wait_bounded(sm.bar + 1, parity, 1000000000ull);
      if (tid < 32 && two && next < ntiles) {
        mbar_wait_bounded(stage((j + 1) & 1).bar, uint32_t(((j + 1) >> 1) & 1), 1000000000ull);
        mbar_wait_bounded(stage((j + 1) & 1).bar + 1, uint32_t(((j + 1) >> 1) & 1), 1000000000ull);
      }
      if (tid == 0) bulk_wait_read();
      return;
    }
    // the phase is complete: one try_wait gives every other thread its own
    // acquire of the copied data
    if (tid >= 32) mbar_try_wait(sm.bar, parity);

    // ---- 2. node moments ---------------------------------------------------------
    if (!a.collision) {
      for (int v = tid; v < ne * NP * 8; v += nth) sm.mom[v] = R(0);
    } else {
      // the usual large-Q tiles (one element, 128 or 256 threads) take the
      // moment reduction with compile-time lane groups and an unrolled loop
      auto moments = [&](auto acc) {
        using Acc = decltype(acc);
        constexpr int kBig = QT >= 128 ? 1 : 0;
        if (kBig && epc == 1 && nth == 128)
          tile_moments<ST, Acc, QT, kBig * 128, 1>(a, sm.f, sm.scale, sm.geo, sm.mom, ne, sm.vel);
        else if (kBig && epc == 1 && nth == 256)
          tile_moments<ST, Acc, QT, kBig * 256, 1>(a, sm.f, sm.scale, sm.geo, sm.mom, ne, sm.vel);
        else
          tile_moments<ST, Acc, QT>(a, sm.f, sm.scale, sm.geo, sm.mom, ne, sm.vel);
      };
      if constexpr (sizeof(R) == 8) {
        moments(AccD{});
      } else {
        if (a.red == kRedFP64) moments(AccD{});
        else if (a.red == kRedCompFP32) moments(AccN{});
        else moments(AccF{});
      }
    }
    // ---- 3. wall numerators ------------------------------------------------------
    if (a.wall_any) tile_wall_numerators<ST, QT>(a, sm.f, sm.geo, sm.nbr, sm.scale, sm.wn, ne, sm.vel);
    // the residual tile and the neighbour traces (bar[1]), as for bar[0]
    ok = true;
    if (tid < 32) ok = mbar_wait_bounded(sm.bar + 1, parity, 2000000000ull);
    if (__syncthreads_or(!ok)) {
      if (tid == 0 && a.err) atomicExch(a.err, 1);
      if (tid < 32 && two && next < ntiles)
        mbar_wait_bounded(stage((j + 1) & 1).bar + 1, uint32_t(((j + 1) >> 1) & 1), 1000000000ull);
      if (tid == 0) bulk_wait_read();
      return;
    }
    if (tid >= 32) mbar_try_wait(sm.bar + 1, parity);

    // ---- 4. residual and update ----------------------------------------------------
    float dmax = 0.f;  // deviation forms: running max |f/w - 1| of element emax
    int emax = -1;
    item_update<ST, QT, items_vpt<ST, QT>()>(a, sm, k0, ne, read_res, dmax, emax);

    // ---- 5. deviation forms: the kept scale (BF16), or the new per-element
    // scale and the encoding in place (FP16) ------------------------------------
    if constexpr (keeps_scale<ST>()) {
      for (int e = tid; e < ne; e += nth) a.scale_out[k0 + e] = sm.scale[e];
    } else if constexpr (ST::dev) {
      if (emax >= 0) atomicMax(&sm.dmax[emax], __float_as_uint(dmax));
      __syncthreads();
      for (int e = tid; e < ne; e += nth) {
        const float md = __uint_as_float(sm.dmax[e]);
        float sc = 1.0f;
        if (md > 0.f) {
          int ex2;
          frexpf(md, &ex2);
          sc = ldexpf(1.0f, ex2 - ST::qmax_log2);
        }
        sm.nscale[e] = sc;  // face scales are no longer needed
        a.scale_out[k0 + e] = sc;
      }
      __syncthreads();
      constexpr int V = Vec16<ST>::N;
      const int nvec = ne * NP * Qp / V;
      for (int v = tid; v < nvec; v += nth) {
        const int idx = v * V;
        const int e = idx / (NP * Qp);
        const int i0 = idx % Qp;
        const float sold = sm.scale[e];
        const float inv_s = 1.0f / sm.nscale[e];
        __align__(16) S q[V];
        *reinterpret_cast<uint4*>(q) = *reinterpret_cast<const uint4*>(sm.f + idx);
  #pragma unroll
        for (int j = 0; j < V; ++j) {
          const float w = __ldg(a.vel + kVelW * Qp + i0 + j);
          const float invw = __ldg(a.vel + kVelInvW * Qp + i0 + j);
          const float fold = decode<ST>(q[j], w, w * sold);
          const float fnew = new_f<ST>(fold, a.rkB, sm.res[idx + j]);
          q[j] = ST::from_r((fnew - w) * invw * inv_s);
        }
        *reinterpret_cast<uint4*>(sm.f + idx) = *reinterpret_cast<const uint4*>(q);
      }
    }


    // ---- 6. bulk store of the new state and residual tiles -----------------------
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      bulk_store(static_cast<S*>(a.f_out) + k0 * NP * Qp, sm.f, uint32_t(size_t(ne) * NP * row_bytes));
      bulk_store(a.res + k0 * NP * Qp, sm.res, uint32_t(size_t(ne) * NP * Qp * sizeof(R)));
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait_read();
}

#include "stage_tc.cuh"
#include "stage_cluster.cuh"
#include "stage_ws.cuh"

template <class ST, int QT>
cudaError_t launch_one(const void* args, int grid, int block, size_t smem, cudaStream_t st) {
  const auto& a = *static_cast<const StageArgs<typename ST::R>*>(args);
  stage_kernel<ST, QT><<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

// Velocity counts with a specialised kernel (the GH D2Q16 and NC 16x16 /
// 32x32 sets; the larger sets only at the degrees their workloads use, which
// keeps the high-degree translation units quick to compile); other counts use
// the runtime-stride kernel.
constexpr bool specialised_q(int Qp) {
  return (Qp == 16 && P <= 5) || (Qp == 256 && P <= 5) || (Qp == 1024 && P <= 4);
}

template <class ST>
cudaError_t launch_q(int Qp, const void* args, int grid, int block, size_t smem, cudaStream_t st) {
  if constexpr (ST::kind != kStoreF64) {
    if constexpr (specialised_q(16))
      if (Qp == 16) return launch_one<ST, 16>(args, grid, block, smem, st);
    if constexpr (specialised_q(256))
      if (Qp == 256) return launch_one<ST, 256>(args, grid, block, smem, st);
    if constexpr (specialised_q(1024))
      if (Qp == 1024) return launch_one<ST, 1024>(args, grid, block, smem, st);
  }
  return launch_one<ST, 0>(args, grid, block, smem, st);
}

template <class ST>
int occupancy_q(int Qp, int block, size_t smem) {
  int n = 0;
  auto occ = [&](auto kernel) { cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem); };
  if constexpr (ST::kind != kStoreF64) {
    if constexpr (specialised_q(16))
      if (Qp == 16) { occ(stage_kernel<ST, 16>); return n; }
    if constexpr (specialised_q(256))
      if (Qp == 256) { occ(stage_kernel<ST, 256>); return n; }
    if constexpr (specialised_q(1024))
      if (Qp == 1024) { occ(stage_kernel<ST, 1024>); return n; }
  }
  occ(stage_kernel<ST, 0>);
  return n;
}

// resident CTAs per SM of the kernel a launch with these parameters uses
int occupancy(int store_kind, int Qp, int block, size_t smem) {
  switch (store_kind) {
    case kStoreF64: return occupancy_q<StoreF64>(Qp, block, smem);
    case kStoreF32: return occupancy_q<StoreF32>(Qp, block, smem);
    case kStoreBF16: return occupancy_q<StoreBF16>(Qp, block, smem);
    case kStoreF16: return occupancy_q<StoreF16>(Qp, block, smem);
  }
  return 0;
}

template <class ST>
cudaError_t set_smem_q(int Qp, size_t smem) {
  auto set = [smem](auto kernel) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  };
  if constexpr (ST::kind != kStoreF64) {
    if constexpr (specialised_q(16))
      if (Qp == 16) return set(stage_kernel<ST, 16>);
    if constexpr (specialised_q(256))
      if (Qp == 256) return set(stage_kernel<ST, 256>);
    if constexpr (specialised_q(1024))
      if (Qp == 1024) return set(stage_kernel<ST, 1024>);
  }
  return set(stage_kernel<ST, 0>);
}

cudaError_t launch(int store_kind, const void* args, int grid, int block, size_t smem, cudaStream_t st) {
  const int Qp = store_kind == kStoreF64 ? static_cast<const StageArgs<double>*>(args)->Qp
                                         : static_cast<const StageArgs<float>*>(args)->Qp;
  switch (store_kind) {
    case kStoreF64: return launch_q<StoreF64>(Qp, args, grid, block, smem, st);
    case kStoreF32: return launch_q<StoreF32>(Qp, args, grid, block, smem, st);
    case kStoreBF16: return launch_q<StoreBF16>(Qp, args, grid, block, smem, st);
    case kStoreF16: return launch_q<StoreF16>(Qp, args, grid, block, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t set_smem(int store_kind, int Qp, size_t smem) {
  switch (store_kind) {
    case kStoreF64: return set_smem_q<StoreF64>(Qp, smem);
    case kStoreF32: return set_smem_q<StoreF32>(Qp, smem);
    case kStoreBF16: return set_smem_q<StoreBF16>(Qp, smem);
    case kStoreF16: return set_smem_q<StoreF16>(Qp, smem);
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
  unsigned long long h32x2[OPS_N];
  for (int j = 0; j < OPS_N; ++j) {
    h32[j] = float(h64[j]);
    uint32_t bits;
    std::memcpy(&bits, &h32[j], 4);
    h32x2[j] = (static_cast<unsigned long long>(bits) << 32) | bits;
  }
  cudaError_t e = cudaMemcpyToSymbol(c_ops64, h64, sizeof(h64));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_ops32x2, h32x2, sizeof(h32x2));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_ops32, h32, sizeof(h32));
}

}  // namespace

StageEntry FEDBM_STAGE_ENTRY_NAME() {
  StageEntry s;
  s.launch = &launch;
  s.set_smem = &set_smem;
  s.upload = &upload;
  s.occupancy = &occupancy;
  s.tc_smem = &tc_smem;
  s.tc_tmem_cols = &tc_tmem_cols;
  s.launch_tc = &launch_tc;
  s.set_smem_tc = &set_smem_tc;
  s.occupancy_tc = &occupancy_tc;
  s.cl_smem = &cl_smem;
  s.launch_cl = &launch_cl;
  s.set_smem_cl = &set_smem_cl;
  s.occupancy_cl = &occupancy_cl;
  s.ws_smem = &ws_smem;
  s.launch_ws = &launch_ws;
  s.set_smem_ws = &set_smem_ws;
  s.occupancy_ws = &occupancy_ws;
  return s;
}

}  // namespace fedbm
