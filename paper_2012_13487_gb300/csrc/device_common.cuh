// Shared device-side definitions of the fused LSRK stage kernel.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fedbm {

// Storage forms of the distribution state.  Plain forms store f itself; the
// deviation forms store q with f_i = w_i (1 + s_k q_i), s_k a per-element
// power-of-two scale, and compute in FP32.
enum StoreKind { kStoreF64 = 0, kStoreF32 = 1, kStoreBF16 = 2, kStoreF16 = 3 };

struct StoreF64 {
  using S = double;
  using R = double;
  static constexpr bool dev = false;
  static constexpr int kind = kStoreF64;
};
struct StoreF32 {
  using S = float;
  using R = float;
  static constexpr bool dev = false;
  static constexpr int kind = kStoreF32;
};
struct StoreBF16 {
  using S = __nv_bfloat16;
  using R = float;
  static constexpr bool dev = true;
  static constexpr int kind = kStoreBF16;
  static constexpr int qmax_log2 = 0;  // |q| <= 1 (BF16 keeps its exponent range)
  __device__ static float to_r(S q) { return __bfloat162float(q); }
  __device__ static S from_r(float v) { return __float2bfloat16_rn(v); }
};
struct StoreF16 {
  using S = __half;
  using R = float;
  static constexpr bool dev = true;
  static constexpr int kind = kStoreF16;
  static constexpr int qmax_log2 = 15;  // |q| <= 2^15 < 65504
  __device__ static float to_r(S q) { return __half2float(q); }
  __device__ static S from_r(float v) { return __float2half_rn(v); }
};

// Per-velocity constant rows of the velocity table [kVelRows][Qp].
enum VelRow { kVelEx = 0, kVelEy = 1, kVelW = 2, kVelInvW = 3, kVelWex = 4, kVelWey = 5, kVelRows = 6 };

// Reduction modes for the velocity moments (enum fedbm_reduction).
enum RedMode { kRedDefault = 0, kRedFP64 = 1, kRedCompFP32 = 2 };

// Per-element record [kGeoStrideDev]: r_x, s_x, r_y, s_y, then (n_x, n_y, Fscale)
// for faces 0..2, the Jacobian J, the time step and 1/tau of the element's case
// (1/tau = 0 switches the collision term off).
constexpr int kGeoStrideDev = 16;
constexpr int kGeoJ = 13, kGeoDt = 14, kGeoInvTau = 15;

// Kernel arguments (by value).  Pointers are device pointers of the solver.
template <typename R>
struct StageArgs {
  const void* f_in;         // state read by this stage  [K][Np][Qp] storage type
  void* f_out;              // state written             [K][Np][Qp]
  R* res;                   // LSRK residual register     [K][Np][Qp]
  const float* scale_in;    // deviation forms: per-element scale read  [K]
  float* scale_out;         // deviation forms: per-element scale written
  const int32_t* nbr;       // [K][3] face codes
  const R* geo;             // [K][16] geometry
  const R* vel;             // [kVelRows][Qp]
  const R* wall_feq;        // [slots][Qp] f^eq(1, u_b) per wall slot (4 * case + side)
  const R* wall_den_inv;    // [slots] 1 / sum_{e.n<0} |e.n| f^eq(1,u_b); 0 for eq. UsedBC walls
  int32_t wall_any;         // 1 if some slot is an eq. FullBC wall
  R W0, W1x, W1y;           // sum w, sum w ex, sum w ey (deviation moments)
  int64_t K;
  int32_t Qp;
  int32_t epc;              // elements per CTA tile
  int32_t nstages;          // 2: double-buffered tile pipeline, 1: single buffer
  R rkA, rkB, ab;
  int32_t collision, eq_order, red;
  int* err;                 // set to 1 if a bounded wait of a CTA gave up
  uint32_t extra_tx;        // test hook: bytes expected on top of the copies (0)
  const uint32_t* sr_step;  // BF16 stochastic rounding: the step counter (nullptr = nearest-even)
  int32_t sr_stage;         // RK stage index mixed into the rounding draws
};

// Stochastic rounding of an FP32 value to BF16: a uniform 16-bit draw is
// added to the 16 bits that BF16 drops, then they are cut off, so x rounds
// away from zero with probability (dropped bits) / 2^16 and the stored value
// is x in expectation (|x| <= 1 here: no overflow).  The draw comes from a
// counter-based hash of the value's index, the step and the stage
// (the 32-bit finaliser of MurmurHash3, Appleby).
__device__ __forceinline__ uint32_t sr_hash(uint64_t idx, uint32_t step, uint32_t stage) {
  uint32_t h = uint32_t(idx) ^ uint32_t(idx >> 32) * 0x9E3779B1u ^ (step * 0x85EBCA77u) ^ (stage * 0xC2B2AE3Du);
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}
__device__ __forceinline__ __nv_bfloat16 bf16_round_stochastic(float x, uint32_t draw) {
  const uint32_t b = (__float_as_uint(x) + (draw & 0xFFFFu)) & 0xFFFF0000u;
  return __ushort_as_bfloat16(static_cast<unsigned short>(b >> 16));
}

__host__ __device__ constexpr int np_of(int p) { return (p + 1) * (p + 2) / 2; }

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Shared-memory layout of one stage CTA (offsets in bytes); the host sizes the
// launch with it and the kernel carves its buffers with it.
enum SmemPart { kSmBar, kSmF, kSmRes, kSmTr, kSmGeo, kSmNbr, kSmScale, kSmNScale, kSmDmax, kSmMom, kSmWn, kSmVel, kSmEnd };

__host__ __device__ inline size_t stage_smem_layout(int Np, int NF, int epc, int Qp, size_t s_bytes, size_t r_bytes,
                                                    size_t off[kSmEnd + 1]) {
  size_t b = 0;
  off[kSmBar] = b;    b += 16;
  off[kSmF] = b;      b += align16(size_t(epc) * Np * Qp * s_bytes);   // element tile (updated in place)
  off[kSmRes] = b;    b += align16(size_t(epc) * Np * Qp * r_bytes);   // residual tile (updated in place)
  off[kSmTr] = b;     b += align16(size_t(epc) * NF * Qp * s_bytes);   // neighbour face traces
  off[kSmGeo] = b;    b += align16(size_t(epc) * kGeoStrideDev * r_bytes);
  off[kSmNbr] = b;    b += align16(size_t(epc) * 3 * 4);
  off[kSmScale] = b;  b += align16(size_t(epc) * 4);                  // element scale (deviation forms)
  off[kSmNScale] = b; b += align16(size_t(epc) * 3 * 4);              // neighbour scales, then new scale
  off[kSmDmax] = b;   b += align16(size_t(epc) * 4);
  off[kSmMom] = b;    b += align16(size_t(epc) * Np * 8 * r_bytes);   // f^eq/tau coefficients per node
  off[kSmWn] = b;     b += align16(size_t(epc) * NF * r_bytes);        // wall numerators
  off[kSmVel] = b;    b += align16(size_t(3) * Qp * r_bytes);          // e_x, e_y, w rows (copied once)
  off[kSmEnd] = b;
  return b;
}

template <typename R, typename S>
struct StageSmem {
  uint64_t* bar;
  S* f;
  R* res;
  S* tr;
  R* geo;
  int* nbr;
  float* scale;
  float* nscale;
  unsigned* dmax;
  R* mom;
  R* wn;
  R* vel;  // e_x, e_y, w: three rows of Qp
};

template <typename R, typename S>
__device__ inline StageSmem<R, S> carve_stage_smem(unsigned char* base, int Np, int NF, int epc, int Qp) {
  size_t off[kSmEnd + 1];
  stage_smem_layout(Np, NF, epc, Qp, sizeof(S), sizeof(R), off);
  StageSmem<R, S> s;
  s.bar = reinterpret_cast<uint64_t*>(base + off[kSmBar]);
  s.f = reinterpret_cast<S*>(base + off[kSmF]);
  s.res = reinterpret_cast<R*>(base + off[kSmRes]);
  s.tr = reinterpret_cast<S*>(base + off[kSmTr]);
  s.geo = reinterpret_cast<R*>(base + off[kSmGeo]);
  s.nbr = reinterpret_cast<int*>(base + off[kSmNbr]);
  s.scale = reinterpret_cast<float*>(base + off[kSmScale]);
  s.nscale = reinterpret_cast<float*>(base + off[kSmNScale]);
  s.dmax = reinterpret_cast<unsigned*>(base + off[kSmDmax]);
  s.mom = reinterpret_cast<R*>(base + off[kSmMom]);
  s.wn = reinterpret_cast<R*>(base + off[kSmWn]);
  s.vel = reinterpret_cast<R*>(base + off[kSmVel]);
  return s;
}

// Bytes between the two pipeline stages of a CTA (one stage, 128-byte aligned).
__host__ __device__ inline size_t stage_smem_stride(int Np, int NF, int epc, int Qp, size_t s_bytes, size_t r_bytes) {
  size_t off[kSmEnd + 1];
  return (stage_smem_layout(Np, NF, epc, Qp, s_bytes, r_bytes, off) + 127) & ~size_t(127);
}

// Dynamic shared memory of one stage CTA with `nstages` pipeline stages.
__host__ inline size_t stage_smem_bytes(int p, int store_kind, int epc, int Qp, int nstages) {
  const size_t s_bytes = store_kind == kStoreF64 ? 8 : store_kind == kStoreF32 ? 4 : 2;
  const size_t r_bytes = store_kind == kStoreF64 ? 8 : 4;
  return size_t(nstages) * stage_smem_stride(np_of(p), 3 * (p + 1), epc, Qp, s_bytes, r_bytes);
}

}  // namespace fedbm
