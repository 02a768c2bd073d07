// Warp-specialised form of the FMA stage kernel for 256 velocities (the NC
// 16 x 16 sets), FP32 or BF16 deviation state.  Included by stage_impl.cuh
// inside its namespace; the arithmetic of a stage is that of the FMA kernel.
//
// A CTA has eight consumer warps (one thread per velocity of an element) and
// one producer warp.  The producer keeps a ring of kWsStages shared-memory
// stages filled with the next elements' state tiles, geometry and neighbour
// face rows (bulk copies, one "full" mbarrier per stage); the consumers take
// the elements in order, reduce the node moments and wall numerators from the
// stage, read their own residual column straight from global memory (issued
// before the reductions, so that its latency is covered), evaluate volume,
// flux, lift, collision and the update, write the new state and residual
// columns straight to global memory, and release the stage on its "empty"
// mbarrier.  So the consumers do not wait for copies while the ring is ahead
// of them, which the single-buffered kernel does once per tile.
//
// BF16 state: the volume contractions run on the tensor cores.  With
// f_m = w (1 + s q_m) and Dr 1 = Ds 1 = 0 (the derivative of a constant),
//   sum_m Dr[n][m] f_m = w s sum_m Dr[n][m] q_m,
// and the stored q is an exact BF16 operand.  Each thread writes its velocity's
// q column as one row of a K-major operand (two 16-byte stores at degree <= 4),
// one thread issues tcgen05 MMAs (kind::f16, BF16 inputs, FP32 accumulators in
// tensor memory) of the 256 x Np q block against [Dr; Ds] split into three
// BF16 pieces (8 + 8 + 8 significant bits, so the operators keep FP32
// precision), and the lift contraction runs on FMAs while the MMAs are in
// flight.
//
// Every wait is bounded by %globaltimer.  Consumer warp 0 waits on the full
// barrier and the consumers agree on the outcome with a reducing named
// barrier; on a timeout the consumers record it and leave, the producer stops
// issuing and, before it leaves, waits (bounded) for the copies it issued.

namespace ws {

// FEDBM_WS_MMA = 0 keeps the BF16 volume contractions on FMAs.
#ifndef FEDBM_WS_MMA
#define FEDBM_WS_MMA 1
#endif
// FEDBM_WS_SKIP = 0 evaluates every face's flux and lift columns
#ifndef FEDBM_WS_SKIP
#define FEDBM_WS_SKIP 1
#endif
constexpr int kWsStages = 3;
constexpr int kWsQ = 256;                  // velocities (one per consumer thread)
constexpr int kWsConsumers = kWsQ;         // eight warps
constexpr int kWsThreads = kWsConsumers + 32;

// named barrier 1 over the consumer threads, OR-reducing a predicate
__device__ __forceinline__ bool consumers_sync_or(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbarrier.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(pred ? 1u : 0u), "n"(kWsConsumers)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void consumers_sync() {
  asm volatile("barrier.sync 1, %0;" ::"n"(kWsConsumers) : "memory");
}
// plain arrive (release) of this thread on a barrier
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// ---- tensor-core volume contractions of the BF16 form --------------------------
template <class ST>
__host__ __device__ constexpr bool ws_mma() {
  return FEDBM_WS_MMA != 0 && ST::kind == kStoreBF16;
}
constexpr int MK = (NP + 15) / 16 * 16;   // K of the MMAs: input nodes, padded
constexpr int MKC = MK / 8;               // 16-byte chunks (8 BF16) per operand row
constexpr int MND = (NP + 15) / 16 * 16;  // accumulator columns of one operator
constexpr int MN = 2 * MND;               // N of the MMAs: [Dr; Ds]
constexpr int kPieces = 3;                // BF16 pieces per operator entry
constexpr int kMmaCols = 2 * MN <= 64 ? 64 : 128;  // two 128-velocity halves
static_assert(2 * MN <= 128, "tensor-memory columns of the BF16 form");

// byte offset of (row r, column k) in a K-major BF16 operand without swizzle:
// 8 rows x 16 bytes per core matrix, core matrices along K at 128 bytes, 8-row
// groups at KC * 128 bytes
__host__ __device__ constexpr int bidx(int r, int k, int KC) {
  return ((r >> 3) * KC + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
// instruction descriptor: D F32, A and B BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

// Shared-memory layout: per stage the state tile [NP][256], the neighbour face
// rows [NF][256], the geometry, face codes and scales, two barriers; once per
// CTA the velocity rows and two alternating sets of node records and wall
// numerators.
struct Layout {
  size_t stage, f, tr, geo, nbr, scale, nscale, bars, end_stage;
  size_t vel, mom, wn, mA, mB, mbar, end;
};
// mma: the BF16 form's q operand [256][MK], the operator pieces
// [kPieces][MN][MK], the MMA barrier and the tensor-memory address
__host__ __device__ inline Layout layout(int s_bytes, bool mma) {
  Layout o;
  size_t b = 0;
  o.f = b;      b += align16(size_t(NP) * kWsQ * s_bytes);
  o.tr = b;     b += align16(size_t(NF) * kWsQ * s_bytes);
  o.geo = b;    b += align16(size_t(kGeoStrideDev) * 4);
  o.nbr = b;    b += 16;
  o.scale = b;  b += 16;
  o.nscale = b; b += 16;
  o.bars = b;   b += 16;                   // full, empty
  o.end_stage = b;
  o.stage = (b + 127) / 128 * 128;
  b = o.stage * kWsStages;
  o.vel = b;    b += align16(size_t(3) * kWsQ * 4);
  o.mom = b;    b += align16(size_t(2) * NP * 8 * 4);
  o.wn = b;     b += align16(size_t(2) * NF * 4);
  b = (b + 127) / 128 * 128;
  o.mA = b;     b += mma ? size_t(kWsQ) * MK * 2 : 0;
  o.mB = b;     b += mma ? size_t(kPieces) * MN * MK * 2 : 0;
  o.mbar = b;   b += mma ? 16 : 0;
  o.end = b;
  return o;
}

template <class ST>
__global__ void __launch_bounds__(kWsThreads, 2) stage_kernel_ws(const StageArgs<float> a) {
  using S = typename ST::S;
  constexpr bool kMma = ws_mma<ST>();
  extern __shared__ __align__(128) unsigned char smem[];
  const Layout o = layout(int(sizeof(S)), kMma);
  const int tid = threadIdx.x;
  const bool producer = tid >= kWsConsumers;
  const int64_t K = a.K;
  const bool read_res = a.rkA != 0.f;
  const bool third = a.eq_order == 3;
  const S* fin = static_cast<const S*>(a.f_in);
  S* fout = static_cast<S*>(a.f_out);
  float* s_vel = reinterpret_cast<float*>(smem + o.vel);
  auto st_f = [&](int s) { return reinterpret_cast<S*>(smem + s * o.stage + o.f); };
  auto st_tr = [&](int s) { return reinterpret_cast<S*>(smem + s * o.stage + o.tr); };
  auto st_geo = [&](int s) { return reinterpret_cast<float*>(smem + s * o.stage + o.geo); };
  auto st_nbr = [&](int s) { return reinterpret_cast<int*>(smem + s * o.stage + o.nbr); };
  auto st_scale = [&](int s) { return reinterpret_cast<float*>(smem + s * o.stage + o.scale); };
  auto st_nscale = [&](int s) { return reinterpret_cast<float*>(smem + s * o.stage + o.nscale); };
  auto full = [&](int s) { return reinterpret_cast<uint64_t*>(smem + s * o.stage + o.bars); };
  auto empty = [&](int s) { return reinterpret_cast<uint64_t*>(smem + s * o.stage + o.bars) + 1; };

  unsigned char* sA = smem + o.mA;
  unsigned char* sB = smem + o.mB;
  uint64_t* mma_bar = reinterpret_cast<uint64_t*>(smem + o.mbar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + o.mbar + 8);

  for (int v = tid; v < 3 * kWsQ; v += kWsThreads) s_vel[v] = a.vel[v];
  if (tid == 0) {
    for (int s = 0; s < kWsStages; ++s) {
      mbar_init(full(s), 32);               // the producer's 32 lanes
      mbar_init(empty(s), kWsConsumers);    // every consumer thread
    }
    if constexpr (kMma) mbar_init(mma_bar, 1);  // one commit per element
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  if constexpr (kMma) {
    if (tid < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                   "n"(kMmaCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // [Dr; Ds] (rows n, then MND + n; columns: input nodes) from the FP64
    // operators as three BF16 pieces x = p0 + p1 + p2 + O(2^-24 |x|)
    for (int v = tid; v < MN * MK; v += kWsThreads) {
      const int n = v / MK, m = v % MK;
      const int nn = n < MND ? n : n - MND;
      double x = 0.0;
      if (nn < NP && m < NP) x = c_ops64[(n < MND ? OFF_DR : OFF_DS) + nn * NP + m];
#pragma unroll
      for (int q = 0; q < kPieces; ++q) {
        const __nv_bfloat16 pc = __float2bfloat16_rn(float(x));
        *reinterpret_cast<__nv_bfloat16*>(sB + size_t(q) * MN * MK * 2 + bidx(n, m, MKC)) = pc;
        x -= double(__bfloat162float(pc));
      }
    }
    fence_proxy_async_smem();
    tc::fence_before_sync();
  }
  __syncthreads();

  if (producer) {
    // ---- producer warp: element k = blockIdx.x + j gridDim.x into stage j % kWsStages
    const int lane = tid - kWsConsumers;
    const size_t row_bytes = size_t(kWsQ) * sizeof(S);
    int issued = 0;  // elements issued
    for (int64_t k = blockIdx.x; k < K; k += gridDim.x, ++issued) {
      const int s = issued % kWsStages;
      if (issued >= kWsStages) {
        // the consumers released element issued - kWsStages from this stage
        const uint32_t ph = uint32_t((issued / kWsStages - 1) & 1);
        bool ok = true;
        if (lane == 0) ok = mbar_wait_bounded(empty(s), ph, 2000000000ull);
        ok = __shfl_sync(kFull, ok ? 1 : 0, 0) != 0;
        if (!ok) break;  // the consumers gave up (or a release never came)
        if (lane != 0) mbar_try_wait(empty(s), ph);
      }
      int* nb = st_nbr(s);
      for (int v = lane; v < 3; v += 32) {
        const int code = __ldg(a.nbr + k * 3 + v);
        nb[v] = code;
        if constexpr (ST::dev) st_nscale(s)[v] = code >= 0 ? __ldg(a.scale_in + (code >> 3)) : 0.f;
      }
      if constexpr (ST::dev)
        if (lane == 0) st_scale(s)[0] = __ldg(a.scale_in + k);
      uint32_t bytes = lane == 0 ? uint32_t(NP * row_bytes + kGeoStrideDev * 4) + a.extra_tx : 0u;
      for (int row = lane; row < NF; row += 32)
        if (__ldg(a.nbr + k * 3 + row / NFP) >= 0) bytes += uint32_t(row_bytes);
      mbar_arrive_expect_tx(full(s), bytes);
      if (lane == 0) {
        bulk_load(st_f(s), fin + size_t(k) * NP * kWsQ, uint32_t(NP * row_bytes), full(s));
        bulk_load(st_geo(s), a.geo + k * kGeoStrideDev, uint32_t(kGeoStrideDev * 4), full(s));
      }
      for (int row = lane; row < NF; row += 32) {
        const int fc = row / NFP, aa = row % NFP;
        const int code = __ldg(a.nbr + k * 3 + fc);
        if (code >= 0) {
          const int64_t kn = code >> 3;
          const int fn = (code >> 1) & 3;
          const int a2 = (code & 1) ? NFP - 1 - aa : aa;
          bulk_load(st_tr(s) + size_t(row) * kWsQ, fin + (size_t(kn) * NP + face_node(fn, a2)) * kWsQ,
                    uint32_t(row_bytes), full(s));
        }
      }
    }
    // let every copy this warp issued land before the CTA can leave: the last
    // min(issued, stages) elements' full barriers (complete long since on a
    // normal exit; after a timeout the bound is short, copies take microseconds)
    if (lane == 0) {
      for (int q = 0; q < kWsStages && q < issued; ++q) {
        const int e = issued - 1 - q;
        mbar_wait_bounded(full(e % kWsStages), uint32_t((e / kWsStages) & 1), 100000000ull);
      }
    }
    return;
  }

  // ---- consumers: thread = velocity i of each element of this CTA -----------------
  const int i = tid;
  uint32_t ta = 0;  // BF16 form: this thread's accumulator row (lane i % 128, half i / 128)
  if constexpr (kMma) {
    tc::fence_after_sync();
    ta = *tslot + (uint32_t(32 * ((tid >> 5) & 3)) << 16) + uint32_t((tid >> 7) * MN);
  }
  // leave with the tensor memory released (warp 0 allocated it); nmma MMA
  // groups were committed, the last one is waited for (bounded) first
  auto release_tmem = [&](int nmma) {
    if constexpr (kMma) {
      tc::fence_before_sync();
      consumers_sync();
      if (tid < 32) {
        if (nmma > 0) mbar_wait_bounded(mma_bar, uint32_t((nmma - 1) & 1), 100000000ull);
        __syncwarp();
        tc::fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "n"(kMmaCols));
      }
    }
  };
  const float ex = s_vel[kVelEx * kWsQ + i], ey = s_vel[kVelEy * kWsQ + i], w = s_vel[kVelW * kWsQ + i];
  const float iw = ST::dev ? __ldg(a.vel + kVelInvW * kWsQ + i) : 0.f;
  const float rkA = a.rkA, rkB = a.rkB, ab = a.ab;
  const uint32_t sr_step = (ST::dev && a.sr_step) ? __ldg(a.sr_step) : 0u;
  int j = 0;
  for (int64_t k = blockIdx.x; k < K; k += gridDim.x, ++j) {
    const int s = j % kWsStages;
    const uint32_t ph = uint32_t((j / kWsStages) & 1);
    // the residual column of this element (before the wait: its latency
    // overlaps the copies and the reductions)
    float rold[NP];
    if (read_res) {
#pragma unroll
      for (int n = 0; n < NP; ++n) rold[n] = a.res[(size_t(k) * NP + n) * kWsQ + i];
    }
    bool ok = true;
    if (tid < 32) ok = mbar_wait_bounded(full(s), ph, 2000000000ull);
    if (consumers_sync_or(!ok)) {
      if (tid == 0 && a.err) atomicExch(a.err, 1);
      release_tmem(j);
      return;  // the producer waits for its copies in flight before it leaves
    }
    if (tid >= 32) mbar_try_wait(full(s), ph);
    const S* sf = st_f(s);
    const float* g = st_geo(s);
    const int* nb = st_nbr(s);
    float* mom = reinterpret_cast<float*>(smem + o.mom) + (j & 1) * NP * 8;
    float* wn = reinterpret_cast<float*>(smem + o.wn) + (j & 1) * NF;
    const float sc = ST::dev ? st_scale(s)[0] : 0.f;
    const float ws = ST::dev ? w * sc : 0.f;
    float fr[NP];  // this velocity's state at the element's nodes
    if constexpr (kMma) {
      // this velocity's q column, once: row i of the MMA operand (K-major; the
      // previous element's MMAs have completed, so the operand is free), and
      // decoded
      uint32_t qb[MK];
#pragma unroll
      for (int m = 0; m < MK; ++m) {
        if (m < NP) {
          const S q = sf[m * kWsQ + i];
          qb[m] = uint32_t(__bfloat16_as_ushort(q));
          fr[m] = decode<ST>(q, w, ws);
        } else {
          qb[m] = 0u;
        }
      }
#pragma unroll
      for (int c = 0; c < MKC; ++c)
        *reinterpret_cast<uint4*>(sA + bidx(i, 8 * c, MKC)) =
            make_uint4(qb[8 * c] | (qb[8 * c + 1] << 16), qb[8 * c + 2] | (qb[8 * c + 3] << 16),
                       qb[8 * c + 4] | (qb[8 * c + 5] << 16), qb[8 * c + 6] | (qb[8 * c + 7] << 16));
    }

    // one thread issues the element's MMAs: D[h] = q[h] [Dr; Ds]^T summed over
    // the operator pieces, h = velocities 128 h .. 128 h + 127
    auto issue_mma = [&]() {
      if (tid == 0) {
        tc::fence_after_sync();
        const uint64_t dA = tc::sdesc(smem_u32(sA), 128, MKC * 128), dB = tc::sdesc(smem_u32(sB), 128, MKC * 128);
        constexpr uint32_t id = idesc_bf16(128, MN);
        const uint32_t tm = *tslot;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int ks = 0; ks < MK / 16; ++ks)
#pragma unroll
            for (int q = 0; q < kPieces; ++q) {
              const uint64_t ao = uint64_t(h * 16 * MKC * 128 + ks * 256) >> 4;
              const uint64_t bo = uint64_t(q * MN * MK * 2 + ks * 256) >> 4;
              mma_bf16(tm + uint32_t(h * MN), dA + ao, dB + bo, id, (ks | q) != 0);
            }
        tc::mma_commit(mma_bar);
      }
    };

    // ---- node moments (as in the FMA kernel) and wall numerators -----------
    if (!a.collision) {
      for (int v = tid; v < NP * 8; v += kWsConsumers) mom[v] = 0.f;
    } else if (a.red == kRedFP64) {
      tile_moments<ST, AccD, kWsQ, kWsConsumers, 1>(a, sf, st_scale(s), g, mom, 1, s_vel);
    } else if (a.red == kRedCompFP32) {
      tile_moments<ST, AccN, kWsQ, kWsConsumers, 1>(a, sf, st_scale(s), g, mom, 1, s_vel);
    } else {
      tile_moments<ST, AccF, kWsQ, kWsConsumers, 1>(a, sf, st_scale(s), g, mom, 1, s_vel);
    }
    if (a.wall_any) {
      // one warp per wall face node: sum over outgoing velocities of (e.n) f^-
      const int lane = tid & 31, warp = tid >> 5;
      for (int trip = warp; trip < NF; trip += kWsConsumers / 32) {
        const int fc = trip / NFP, aa = trip % NFP;
        const int code = nb[fc];
        if (!(code < 0 && __ldg(a.wall_den_inv + (-code - 1)) > 0.f)) continue;
        const float nxf = g[4 + 3 * fc], nyf = g[5 + 3 * fc];
        const S* row = sf + face_node(fc, aa) * kWsQ;
        float acc = 0.f;
        for (int v = lane; v < kWsQ; v += 32) {
          const float en = s_vel[kVelEx * kWsQ + v] * nxf + s_vel[kVelEy * kWsQ + v] * nyf;
          const float wv = ST::dev ? s_vel[kVelW * kWsQ + v] : 0.f;
          if (en > 0) acc += en * decode<ST>(row[v], wv, wv * sc);
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
        if (lane == 0) wn[trip] = acc;
      }
    }
    if constexpr (kMma) {
      fence_proxy_async_smem();  // the operand rows, for the tensor cores
      tc::fence_before_sync();
    }
    consumers_sync();
    // the MMAs run while the fluxes and the lift contraction are computed
    if constexpr (kMma) issue_mma();


    // ---- residual and update of velocity i, all nodes ---------------------
    const float dt = g[kGeoDt], inv_tau = g[kGeoInvTau];
    const float ar = ex * g[0] + ey * g[2], as = ex * g[1] + ey * g[3];
    if constexpr (!kMma) {
#pragma unroll
      for (int m = 0; m < NP; ++m) fr[m] = decode<ST>(sf[m * kWsQ + i], w, ws);
    }
    float flux[NF];
    // face fc carries flux for some velocity of this warp (warp-uniform; with
    // the upwind flux an outflow face's jump term is zero, so a face that is
    // outflow for all 32 velocities skips its traces and lift columns)
    bool on[3];
#pragma unroll
    for (int fc = 0; fc < 3; ++fc) {
      const float en = ex * g[4 + 3 * fc] + ey * g[5 + 3 * fc];
      const float c = 0.5f * (en - ab * fabsf(en)) * g[6 + 3 * fc];
      const int code = nb[fc];
      on[fc] = FEDBM_WS_SKIP ? __any_sync(kFull, c != 0.f && (code >= 0 || en < 0.f)) : true;
#pragma unroll
      for (int aa = 0; aa < NFP; ++aa) flux[fc * NFP + aa] = 0.f;
      if (!on[fc]) continue;
      if (code >= 0) {
        const float wsn = ST::dev ? w * st_nscale(s)[fc] : 0.f;
        const S* trow = st_tr(s) + fc * NFP * kWsQ + i;
#pragma unroll
        for (int aa = 0; aa < NFP; ++aa)
          flux[fc * NFP + aa] = c * (fr[face_node(fc, aa)] - decode<ST>(trow[aa * kWsQ], w, wsn));
      } else {
        const int slot = -code - 1;
        const float fb = a.wall_feq[slot * kWsQ + i];
        const float den_inv = __ldg(a.wall_den_inv + slot);
        const bool diffuse = den_inv > 0.f;
#pragma unroll
        for (int aa = 0; aa < NFP; ++aa) {
          const float fp = diffuse ? wn[fc * NFP + aa] * (den_inv * fb) : fb;
          flux[fc * NFP + aa] = en < 0.f ? c * (fr[face_node(fc, aa)] - fp) : 0.f;
        }
      }
    }
    // the stage's shared data are read: release it to the producer
    mbar_arrive(empty(s));
    // BF16 keeps the element's power-of-two scale: q = (f - w) / (w s)
    const float invw = ST::dev ? iw * (1.0f / sc) : 0.f;
    // rhs, update and write-back of node n from its advection term
    // -(e . grad) f + LIFT (flux)
    auto finish = [&](int n, float adv) {
      float rhs = adv;
      rhs += collision<float>(mom + n * 8, ex, ey, w, fr[n], inv_tau, third);
      float r = dt * rhs;
      if (read_res) r = fmaf(rkA, rold[n], r);
      const size_t gi = (size_t(k) * NP + n) * kWsQ + i;
      a.res[gi] = r;
      const float fnew = new_f<ST>(fr[n], rkB, r);
      if constexpr (ST::dev) {
        const float qv = (fnew - w) * invw;
        fout[gi] = a.sr_step ? bf16_round_stochastic(qv, sr_hash(gi, sr_step, uint32_t(a.sr_stage)))
                             : ST::from_r(qv);
      } else {
        fout[gi] = fnew;
      }
    };
    constexpr bool kImm = ops_immediate<ST, kWsQ>();
    if constexpr (kMma) {
      // lift on FMAs while the MMAs run, then the accumulators in groups of 8 nodes
      float lf[NP];
#pragma unroll
      for (int n = 0; n < NP; ++n) lf[n] = 0.f;
#pragma unroll
      for (int fc = 0; fc < 3; ++fc) {
        if (!on[fc]) continue;
#pragma unroll
        for (int n = 0; n < NP; ++n)
#pragma unroll
          for (int aa = 0; aa < NFP; ++aa) {
            const int q = fc * NFP + aa;
            lf[n] = fmaf(opv<float, kImm>(OFF_LIFT + n * NF + q), flux[q], lf[n]);
          }
      }
      const float arw = ar * ws, asw = as * ws;  // Dr f = w s (Dr q)
      if (!mbar_wait_bounded(mma_bar, uint32_t(j & 1), 2000000000ull) && a.err) atomicExch(a.err, 1);
      __syncwarp();
      tc::fence_after_sync();
      constexpr int NG = (NP + 7) / 8;
#pragma unroll
      for (int c = 0; c < NG; ++c) {
        float V[8], W[8];
        tc::tmem_ld8(ta + 8 * c, V);
        tc::tmem_ld8(ta + MND + 8 * c, W);
        tc::tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (8 * c + q < NP) finish(8 * c + q, fmaf(-arw, V[q], fmaf(-asw, W[q], lf[8 * c + q])));
      }
    } else if (FEDBM_WS_SKIP) {
      // lift by faces (the faces without flux skipped), then volume and update
      float lf[NP];
#pragma unroll
      for (int n = 0; n < NP; ++n) lf[n] = 0.f;
#pragma unroll
      for (int fc = 0; fc < 3; ++fc) {
        if (!on[fc]) continue;
#pragma unroll
        for (int n = 0; n < NP; ++n)
#pragma unroll
          for (int aa = 0; aa < NFP; ++aa) {
            const int q = fc * NFP + aa;
            lf[n] = fmaf(opv<float, kImm>(OFF_LIFT + n * NF + q), flux[q], lf[n]);
          }
      }
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        float dr = 0.f, ds = 0.f;
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          dr = fmaf(opv<float, kImm>(OFF_DR + n * NP + m), fr[m], dr);
          ds = fmaf(opv<float, kImm>(OFF_DS + n * NP + m), fr[m], ds);
        }
        finish(n, fmaf(-ar, dr, fmaf(-as, ds, lf[n])));
      }
    } else {
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        float dr = 0.f, ds = 0.f, lf = 0.f;
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          dr = fmaf(opv<float, kImm>(OFF_DR + n * NP + m), fr[m], dr);
          ds = fmaf(opv<float, kImm>(OFF_DS + n * NP + m), fr[m], ds);
        }
#pragma unroll
        for (int q = 0; q < NF; ++q) lf = fmaf(opv<float, kImm>(OFF_LIFT + n * NF + q), flux[q], lf);
        finish(n, fmaf(-ar, dr, fmaf(-as, ds, lf)));
      }
    }
    if constexpr (ST::dev)
      if (tid == 0) a.scale_out[k] = sc;
  }
  release_tmem(j);
}

}  // namespace ws

// ---- host-side entry points of the form ---------------------------------------
template <class ST>
constexpr bool ws_form() {
  return P <= 5 && (ST::kind == kStoreF32 || ST::kind == kStoreBF16);
}

size_t ws_smem(int store_kind, int Qp) {
  if (P > 5 || Qp != ws::kWsQ || (store_kind != kStoreF32 && store_kind != kStoreBF16)) return 0;
  return ws::layout(store_kind == kStoreF32 ? 4 : 2, store_kind == kStoreBF16 && FEDBM_WS_MMA != 0).end;
}

template <class ST>
cudaError_t launch_ws_as(const void* args, int grid, size_t smem, cudaStream_t st) {
  if constexpr (ws_form<ST>()) {
    ws::stage_kernel_ws<ST><<<grid, ws::kWsThreads, smem, st>>>(*static_cast<const StageArgs<float>*>(args));
    return cudaGetLastError();
  } else {
    (void)args; (void)grid; (void)smem; (void)st;
    return cudaErrorInvalidValue;
  }
}

cudaError_t launch_ws(int store_kind, const void* args, int grid, size_t smem, cudaStream_t st) {
  if (store_kind == kStoreF32) return launch_ws_as<StoreF32>(args, grid, smem, st);
  if (store_kind == kStoreBF16) return launch_ws_as<StoreBF16>(args, grid, smem, st);
  return cudaErrorInvalidValue;
}

template <class ST>
cudaError_t set_smem_ws_as(size_t smem) {
  if constexpr (ws_form<ST>())
    return cudaFuncSetAttribute(ws::stage_kernel_ws<ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  (void)smem;
  return cudaErrorInvalidValue;
}
cudaError_t set_smem_ws(int store_kind, size_t smem) {
  if (store_kind == kStoreF32) return set_smem_ws_as<StoreF32>(smem);
  if (store_kind == kStoreBF16) return set_smem_ws_as<StoreBF16>(smem);
  return cudaErrorInvalidValue;
}

// Resident CTAs per SM from the kernel's registers, its shared memory (with
// the per-block reservation), the thread limit and, for the BF16 form, the
// SM's 512 tensor-memory columns (computed here rather than by the occupancy
// calculator, which does not know the tensor memory).
template <class ST>
int occupancy_ws_as(size_t smem) {
  if constexpr (ws_form<ST>()) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, ws::stage_kernel_ws<ST>) != cudaSuccess) return 0;
    int dev = 0, regs_sm = 0, smem_sm = 0, thr_sm = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    // registers are allocated per warp in units of 256, from the register file
    // of the warp's SM sub-partition (a quarter of the SM's): count warps per
    // sub-partition, then CTAs of nine warps
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = 4 * ((regs_sm / 4) / regs_warp) / (ws::kWsThreads / 32);
    const int by_smem = int(size_t(smem_sm) / (smem + fa.sharedSizeBytes + size_t(reserved)));
    const int by_thr = thr_sm / ws::kWsThreads;
    const int by_tmem = ws::ws_mma<ST>() ? 512 / ws::kMmaCols : by_thr;
    return std::min(std::min(by_regs, by_smem), std::min(by_thr, by_tmem));
  } else {
    (void)smem;
    return 0;
  }
}
int occupancy_ws(int store_kind, size_t smem) {
  if (store_kind == kStoreF32) return occupancy_ws_as<StoreF32>(smem);
  if (store_kind == kStoreBF16) return occupancy_ws_as<StoreBF16>(smem);
  return 0;
}
