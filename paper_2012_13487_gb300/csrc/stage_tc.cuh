// Tensor-core form of the stage kernel: FP32 state or BF16/FP16 deviation
// state, FP32 arithmetic; 128 threads per CTA.  QT = 128, 256 or 1024
// velocities run in 128-velocity passes (one velocity per thread); QT = 16
// stacks eight elements into one 128-row tile.  Included by stage_impl.cuh
// inside its namespace: it reuses the tile loads, node moments, wall numerators
// and collision term of the FMA kernel and replaces the element-local
// contractions of phase 4,
//   V = (f - f_0 1) Dr^T,  W = (f - f_0 1) Ds^T,  Lf = flux LIFT^T,
// by tcgen05 MMAs (kind::tf32, M = 128 rows per MMA, accumulators in tensor
// memory).  Subtracting the first node's value f_0 changes nothing in exact
// arithmetic (Dr 1 = Ds 1 = 0, the derivative of a constant) and keeps the
// operands small.  Each FP32 operand x is split into x_hi = tf32(x) and
// x_lo = x - x_hi (read by the MMA as TF32) and every product is taken as
// a_hi b_hi + a_lo b_hi + a_hi b_lo (three MMAs), which keeps the contraction
// error near FP32 rounding of the operands.
//
// Operands live in shared memory K-major without swizzle: a row of K values is
// split into 16-byte chunks of 4 values; the 8 rows x 16 bytes of one chunk
// column form a contiguous 128-byte core matrix; core matrix (row group g,
// chunk c) sits at byte (g * KC + c) * 128.  In the matrix descriptor the
// leading-dimension offset (next chunk along K) is 128 bytes and the stride
// offset (next 8-row group) is KC * 128 bytes.

namespace tc {

constexpr int KD = (NP + 7) / 8 * 8;      // K of the derivative MMAs (nodes)
constexpr int ND = (NP + 15) / 16 * 16;   // N of one derivative operator (nodes)
constexpr int KL = (NF + 7) / 8 * 8;      // K of the lift MMA (face nodes)
constexpr int NL = ND;                    // N of the lift MMA
constexpr int KCD = KD / 4, KCL = KL / 4; // 16-byte chunks per operand row
constexpr int CPM = 2 * ND + NL;          // accumulator columns of one 128-velocity pass
constexpr int kTcThreads = 128;           // one MMA tile of (element, velocity) rows per pass

// elements per tile: one for 128 or more velocities (in 128-velocity passes),
// else 128 / QT elements stacked into one MMA tile (the operators are the same
// for every element; the geometric factors enter per row in the epilogue)
__host__ __device__ constexpr int elems_per_tile(int QT) { return QT >= kTcThreads ? 1 : kTcThreads / QT; }

// tensor-memory columns of one CTA: a power of two >= 32
constexpr int kTcCols = CPM <= 32 ? 32 : CPM <= 64 ? 64 : CPM <= 128 ? 128 : 256;

// float index of (row r, column k) in a K-major operand with KC chunks per row
__host__ __device__ constexpr int kidx(int r, int k, int KC) {
  return ((r >> 3) * KC + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

// Shared-memory layout (byte offsets) of one CTA.  Only the element's state
// tile comes through shared memory (the node moments are reductions over all
// velocities); each thread loads its own residual and neighbour-trace columns
// into registers and writes its outputs from registers.  s_bytes is the state
// element size; the velocity rows are e_x, e_y (and w for the deviation forms).
struct Layout {
  size_t bar, f, A, F, B, L, geo, nbr, sc, mom, wn, vel, end;
};
__host__ __device__ inline size_t al(size_t x, size_t a) { return (x + a - 1) / a * a; }
__host__ __device__ inline Layout layout(int QT, int s_bytes, int vel_rows) {
  Layout o;
  size_t b = 0;
  o.bar = b;  b += 32;                                       // tile barrier, MMA barrier, TMEM address
  b = al(b, 128);
  const int EPT = elems_per_tile(QT);
  o.f = b;    b += size_t(EPT) * NP * QT * s_bytes;           // state tile
  b = al(b, 128);
  o.A = b;    b += 2 * size_t(kTcThreads) * KD * 4;           // (f - f_0) hi|lo of one pass
  o.F = b;    b += 2 * size_t(kTcThreads) * KL * 4;           // face fluxes hi|lo of one pass
  o.B = b;    b += 2 * size_t(2 * ND) * KD * 4;               // [Dr; Ds] hi|lo
  o.L = b;    b += 2 * size_t(NL) * KL * 4;                   // LIFT hi|lo
  o.geo = b;  b += al(size_t(EPT) * kGeoStrideDev * 4, 16);
  o.nbr = b;  b += al(size_t(EPT) * 3 * 4, 16);
  o.sc = b;   b += al(size_t(EPT + 2) * 4, 16);              // element scales, new scale, max deviation
  o.mom = b;  b += al(size_t(EPT) * NP * 8 * 4, 16);
  o.wn = b;   b += al(size_t(EPT) * NF * 4, 16);
  o.vel = b;  b += al(size_t(vel_rows) * QT * 4, 16);
  o.end = b;
  return o;
}

// x rounded to the 10 explicit mantissa bits of TF32 (nearest, ties away from
// zero in magnitude) by integer arithmetic on its bit pattern: add half a TF32
// unit in the last place, clear the 13 low bits.  Finite |x| < 2^127 only.
__device__ __forceinline__ uint32_t tf32_round_bits(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}
// x = hi + lo: hi in TF32, lo = x - hi exact in FP32 (|lo| <= 2^-11 |x|).  The
// MMA reads the top 19 bits of lo, so the pair carries x to about 2^-21 |x|.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_round_bits(x);
  lo = __float_as_uint(x - __uint_as_float(hi));
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = uint64_t((saddr >> 4) & 0x3FFF);
  d |= uint64_t((lbo >> 4) & 0x3FFF) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFF) << 32;
  d |= uint64_t(1) << 46;  // descriptor version of tcgen05; no swizzle, base offset 0
  return d;
}
// instruction descriptor: D F32, A and B TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Writes row r (KC chunks of 4 values) of a K-major hi|lo operand pair:
// x[k] - shift for k < LEN, zero beyond.
template <int KC, int LEN>
__device__ __forceinline__ void put_row(float* hi, float* lo, int r, const float (&x)[LEN], float shift) {
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 4 * c + q;
      const float v = k < LEN ? x[k] - shift : 0.f;
      split_tf32(v, h[q], l[q]);
    }
    const int o = kidx(r, 4 * c, KC);
    *reinterpret_cast<uint4*>(hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

}  // namespace tc

// Bulk copies of one tile's state and geometry (warp 0): elements k0 ..
// k0 + ne - 1; the lanes also store their face codes (and, for the deviation
// forms, their scales and a zero running maximum).  Every lane arrives on the
// barrier, so the plain stores are visible to the threads that wait on it.
template <class ST>
__device__ __forceinline__ void tc_issue_tile(const StageArgs<float>& a, StageSmem<float, typename ST::S>& sm,
                                              int QT, int64_t k0, int ne) {
  using S = typename ST::S;
  const int lane = threadIdx.x & 31;
  for (int v = lane; v < 3 * ne; v += 32) sm.nbr[v] = __ldg(a.nbr + k0 * 3 + v);
  if constexpr (ST::dev) {
    for (int v = lane; v < ne; v += 32) sm.scale[v] = __ldg(a.scale_in + k0 + v);
    if (lane == 0) sm.dmax[0] = 0u;
  }
  const uint32_t tile_bytes = uint32_t(size_t(ne) * NP * QT * sizeof(S));
  const uint32_t geo_bytes = uint32_t(ne * kGeoStrideDev * 4);
  mbar_arrive_expect_tx(sm.bar, lane == 0 ? tile_bytes + geo_bytes + a.extra_tx : 0u);
  if (lane == 0) {
    bulk_load(sm.f, static_cast<const S*>(a.f_in) + k0 * NP * QT, tile_bytes, sm.bar);
    bulk_load(sm.geo, a.geo + k0 * kGeoStrideDev, geo_bytes, sm.bar);
  }
}

// Persistent tensor-core stage kernel: CTA b handles elements b, b + gridDim.x,
// ...  Per element: wait for the state tile; node moments and wall numerators
// from it; then, for each pass of 128 velocities (thread t owns velocity
// 128 pass + t), each thread gathers its state, residual and neighbour traces,
// forms its face fluxes and writes its operand rows, one thread issues the
// MMAs, and the epilogue reads the accumulators and writes the new state and
// residual from registers.  Once the last pass has read the state tile, the
// next element's copy starts and overlaps that pass's MMAs and epilogue.
template <class ST, int QT>
__global__ void __launch_bounds__(tc::kTcThreads, 4) stage_kernel_tc(const StageArgs<float> a) {
  using S = typename ST::S;
  using namespace tc;
  constexpr int VROWS = ST::dev ? 3 : 2;
  // BF16 keeps FP32's exponent range: a power-of-two element scale changes
  // neither the rounding of q nor the decoded f = w (1 + s q), so the element
  // keeps its scale and the new state is encoded straight from registers.
  // FP16 (|q| < 2^15) needs the new scale of the element's largest deviation,
  // found after every velocity is done, and a second encoding sweep.
  constexpr bool kKeepScale = keeps_scale<ST>();
  constexpr bool kRescale = ST::dev && !kKeepScale;
  static_assert(QT % kTcThreads == 0 || kTcThreads % QT == 0, "whole passes or whole stacked elements");
  constexpr int EPT = elems_per_tile(QT);                       // elements per tile
  constexpr int NPASS = QT >= kTcThreads ? QT / kTcThreads : 1;  // 128-row passes per tile
  static_assert(EPT == 1 || !kRescale, "the rescaling form works one element at a time");
  extern __shared__ __align__(128) unsigned char smem[];  // operands need 16-byte alignment
  const Layout o = layout(QT, int(sizeof(S)), VROWS);
  uint64_t* bar_tile = reinterpret_cast<uint64_t*>(smem + o.bar);
  uint64_t* bar_mma = bar_tile + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + o.bar + 16);
  float* sA = reinterpret_cast<float*>(smem + o.A);
  float* sF = reinterpret_cast<float*>(smem + o.F);
  float* sB = reinterpret_cast<float*>(smem + o.B);
  float* sL = reinterpret_cast<float*>(smem + o.L);
  StageSmem<float, S> sm;
  sm.bar = bar_tile;
  sm.f = reinterpret_cast<S*>(smem + o.f);
  sm.res = nullptr;
  sm.tr = nullptr;
  sm.geo = reinterpret_cast<float*>(smem + o.geo);
  sm.nbr = reinterpret_cast<int*>(smem + o.nbr);
  sm.scale = reinterpret_cast<float*>(smem + o.sc);       // element scale (deviation forms)
  sm.nscale = sm.scale + EPT;                              // the new scale (one element)
  sm.dmax = reinterpret_cast<unsigned*>(sm.scale + EPT + 1);  // max |f_new/w - 1| as float bits
  sm.mom = reinterpret_cast<float*>(smem + o.mom);
  sm.wn = reinterpret_cast<float*>(smem + o.wn);
  sm.vel = reinterpret_cast<float*>(smem + o.vel);

  const int tid = threadIdx.x, warp = tid >> 5;
  const float rkA = a.rkA, rkB = a.rkB, ab = a.ab;
  const bool read_res = rkA != 0.f;
  const bool third = a.eq_order == 3;
  const int64_t ntiles = (a.K + EPT - 1) / EPT;
  // this thread's row of a tile: element te of the tile, velocity lane ti
  const int te = QT >= kTcThreads ? 0 : int(threadIdx.x) / QT;
  const int ti = QT >= kTcThreads ? int(threadIdx.x) : int(threadIdx.x) % QT;
  auto tile_ne = [&](int64_t t) { return int(min(int64_t(EPT), a.K - t * EPT)); };
  const S* fin = static_cast<const S*>(a.f_in);
  S* fout = static_cast<S*>(a.f_out);

  if (tid == 0) {
    mbar_init(bar_tile, 32);
    mbar_init(bar_mma, 2);  // one commit from each of the two issuing threads
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "n"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  for (int v = tid; v < VROWS * QT; v += kTcThreads) sm.vel[v] = a.vel[v];
  // B operands from the FP64 operators: [Dr; Ds] (rows n, then ND + n) and LIFT
  for (int v = tid; v < 2 * ND * KD; v += kTcThreads) {
    const int n = v / KD, m = v % KD;
    const int nn = n < ND ? n : n - ND;
    double x = 0.0;
    if (nn < NP && m < NP) x = c_ops64[(n < ND ? OFF_DR : OFF_DS) + nn * NP + m];
    const float h = __uint_as_float(tf32_round_bits(float(x)));
    sB[kidx(n, m, KCD)] = h;
    sB[2 * ND * KD + kidx(n, m, KCD)] = float(x - double(h));
  }
  for (int v = tid; v < NL * KL; v += kTcThreads) {
    const int n = v / KL, j = v % KL;
    const double x = (n < NP && j < NF) ? c_ops64[OFF_LIFT + n * NF + j] : 0.0;
    const float h = __uint_as_float(tf32_round_bits(float(x)));
    sL[kidx(n, j, KCL)] = h;
    sL[NL * KL + kidx(n, j, KCL)] = float(x - double(h));
  }
  fence_proxy_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;

  int64_t tile = blockIdx.x;
  if (tid < 32 && tile < ntiles) tc_issue_tile<ST>(a, sm, QT, tile * EPT, tile_ne(tile));

  // matrix descriptors of the operand starts; a byte offset d inside an operand
  // adds d >> 4 to the start-address field (all operands lie below 256 KB)
  const uint64_t dA = sdesc(smem_u32(sA), 128, KCD * 128), dF = sdesc(smem_u32(sF), 128, KCL * 128);
  const uint64_t dB = sdesc(smem_u32(sB), 128, KCD * 128), dL = sdesc(smem_u32(sL), 128, KCL * 128);
  constexpr uint32_t idD = idesc_tf32(128, 2 * ND), idL = idesc_tf32(128, NL);
  constexpr uint32_t aHalfD = kTcThreads * KD * 4, aHalfL = kTcThreads * KL * 4;  // hi -> lo bytes
  constexpr uint32_t bHalfD = 2 * ND * KD * 4, bHalfL = NL * KL * 4;
  const uint32_t ta = tmem + (uint32_t(32 * warp) << 16);  // this warp's accumulator lanes

  // residual and neighbour-trace columns of (element k, velocity i), loaded
  // one pass ahead of their use
  // (the traces stay as stored, with each face's neighbour scale, and are
  // decoded where they are used, so that nothing waits on the loads here)
  constexpr int NSX = ST::dev ? 3 : 1;  // neighbour scales, deviation forms only
  auto fetch = [&](int64_t k, int i, float (&rx)[NP], S (&tx)[NF], float (&sx)[NSX]) {
#pragma unroll
    for (int n = 0; n < NP; ++n) rx[n] = read_res ? __ldg(a.res + (k * NP + n) * QT + i) : 0.f;
#pragma unroll
    for (int fcx = 0; fcx < 3; ++fcx) {
      const int code = __ldg(a.nbr + k * 3 + fcx);
      const int64_t kn = code >= 0 ? int64_t(code >> 3) : k;  // walls: an in-bounds address, not used
      const int fn = (code >> 1) & 3;
      if constexpr (ST::dev) sx[fcx] = __ldg(a.scale_in + kn);
#pragma unroll
      for (int aa = 0; aa < NFP; ++aa) {
        const int a2 = (code & 1) ? NFP - 1 - aa : aa;
        const int node = fn == 0 ? face_node(0, a2) : (fn == 1 ? face_node(1, a2) : face_node(2, a2));
        tx[fcx * NFP + aa] = fin[(kn * NP + node) * QT + i];  // walls: not used
      }
    }
  };
  // element of this thread's row in tile t (the last element for a ragged tail)
  auto row_elem = [&](int64_t t) { return min(t * EPT + te, a.K - 1); };
  float rcur[NP], scur[NSX];
  S tcur[NF];
  if (tile < ntiles) fetch(row_elem(tile), ti, rcur, tcur, scur);

  bool failed = false;
  int pending = -1;   // parity of a tile copy issued but not yet waited for
  int mma_pending = -1;  // phase of committed MMAs whose barrier wait gave up
  uint32_t mph = 0;   // phase of the MMA barrier
  for (int j = 0; tile < ntiles; ++j, tile += gridDim.x) {
    const int ne = tile_ne(tile);
    const bool valid = te < ne;                  // a ragged tail leaves rows empty
    const int64_t k0 = tile * EPT + te;          // this row's element
    // warp 0 waits for the tile (suspended in try_wait), the others at the
    // block barrier; then one try_wait gives each thread its acquire
    bool ok = true;
    if (tid < 32) ok = mbar_wait_bounded(bar_tile, uint32_t(j & 1), 2000000000ull);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (tid >= 32) mbar_try_wait(bar_tile, uint32_t(j & 1));
    pending = -1;

    // ---- node moments and wall numerators (as in the FMA kernel) -----------------
    if (!a.collision) {
      for (int v = tid; v < EPT * NP * 8; v += kTcThreads) sm.mom[v] = 0.f;
    } else if (a.red == kRedFP64) {
      tile_moments<ST, AccD, QT, kTcThreads, EPT>(a, sm.f, sm.scale, sm.geo, sm.mom, ne, sm.vel);
    } else if (a.red == kRedCompFP32) {
      tile_moments<ST, AccN, QT, kTcThreads, EPT>(a, sm.f, sm.scale, sm.geo, sm.mom, ne, sm.vel);
    } else {
      tile_moments<ST, AccF, QT, kTcThreads, EPT>(a, sm.f, sm.scale, sm.geo, sm.mom, ne, sm.vel);
    }
    if (a.wall_any) tile_wall_numerators<ST, QT>(a, sm.f, sm.geo, sm.nbr, sm.scale, sm.wn, ne, sm.vel);
    __syncthreads();
    const float* geo = sm.geo + te * kGeoStrideDev;  // this row's element
    const float dt = geo[kGeoDt], inv_tau = geo[kGeoInvTau];
    const float s_el = ST::dev ? sm.scale[te] : 0.f;
    const float inv_s_el = ST::dev ? 1.0f / s_el : 0.f;
    if (kKeepScale && valid && ti == 0) a.scale_out[k0] = s_el;
    float dloc = 0.f;  // FP16 form: this thread's max |f_new/w - 1|

#pragma unroll 1
    for (int pass = 0; pass < NPASS; ++pass) {
      const int i = pass * kTcThreads + ti;
      const float ex = sm.vel[kVelEx * QT + i], ey = sm.vel[kVelEy * QT + i];
      const float w = ST::dev ? sm.vel[kVelW * QT + i] : __ldg(a.vel + kVelW * QT + i);  // the FP32 copy has no w row
      const float invw = ST::dev ? __ldg(a.vel + kVelInvW * QT + i) : 0.f;
      const float ar = ex * geo[0] + ey * geo[2], as = ex * geo[1] + ey * geo[3];
      const S* frow = sm.f + te * NP * QT + i;
      float fc[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) fc[m] = valid ? decode<ST>(frow[m * QT], w, w * s_el) : 0.f;
      {
        float flux[NF];
#pragma unroll
        for (int fcx = 0; fcx < 3; ++fcx) {
          const float en = ex * geo[4 + 3 * fcx] + ey * geo[5 + 3 * fcx];
          const float c = valid ? 0.5f * (en - ab * fabsf(en)) * geo[6 + 3 * fcx] : 0.f;  // empty rows: no flux
          const int code = valid ? sm.nbr[te * 3 + fcx] : 0;
          if (code >= 0) {
#pragma unroll
            for (int aa = 0; aa < NFP; ++aa)
              flux[fcx * NFP + aa] =
                  c * (fc[face_node(fcx, aa)] - decode<ST>(tcur[fcx * NFP + aa], w, ST::dev ? w * scur[fcx % NSX] : 0.f));
          } else {
            const int slot = -code - 1;  // wall slot: 4 * case + side
            const float fb = __ldg(a.wall_feq + slot * QT + i);
            const float den_inv = __ldg(a.wall_den_inv + slot);
            const bool diffuse = den_inv > 0.f;
            const float scale = diffuse ? den_inv * fb : 0.f;
            // incoming velocities take the wall state; outgoing ones have no jump
#pragma unroll
            for (int aa = 0; aa < NFP; ++aa) {
              const float fp = diffuse ? sm.wn[te * NF + fcx * NFP + aa] * scale : fb;
              flux[fcx * NFP + aa] = en < 0.f ? c * (fc[face_node(fcx, aa)] - fp) : 0.f;
            }
          }
        }
        put_row<KCD, NP>(sA, sA + kTcThreads * KD, tid, fc, fc[0]);
        put_row<KCL, NF>(sF, sF + kTcThreads * KL, tid, flux, 0.f);
      }
      fence_proxy_async_smem();
      fence_before_sync();
      __syncthreads();  // operand rows written (and, in the last pass, the tile read)

      const bool last = pass == NPASS - 1;
      if (!kRescale && last && tile + gridDim.x < ntiles) {
        if (tid < 32) tc_issue_tile<ST>(a, sm, QT, (tile + gridDim.x) * EPT, tile_ne(tile + gridDim.x));
        pending = (j + 1) & 1;
      }
      // two threads in different warps issue the two products side by side
      if (tid == 0) {
        fence_after_sync();
#pragma unroll
        for (int ks = 0; ks < KD / 8; ++ks) {
          const uint64_t ko = uint64_t(ks * 256) >> 4;
          const uint64_t ah = dA + ko, al = dA + ((aHalfD >> 4) + ko);
          const uint64_t bh = dB + ko, bl = dB + ((bHalfD >> 4) + ko);
          mma_tf32(tmem, ah, bh, idD, ks > 0);
          mma_tf32(tmem, al, bh, idD, 1);
          mma_tf32(tmem, ah, bl, idD, 1);
        }
        mma_commit(bar_mma);
      } else if (tid == 32) {
        fence_after_sync();
#pragma unroll
        for (int ks = 0; ks < KL / 8; ++ks) {
          const uint64_t ko = uint64_t(ks * 256) >> 4;
          const uint64_t ah = dF + ko, al = dF + ((aHalfL >> 4) + ko);
          const uint64_t bh = dL + ko, bl = dL + ((bHalfL >> 4) + ko);
          mma_tf32(tmem + 2 * ND, ah, bh, idL, ks > 0);
          mma_tf32(tmem + 2 * ND, al, bh, idL, 1);
          mma_tf32(tmem + 2 * ND, ah, bl, idL, 1);
        }
        mma_commit(bar_mma);
      }
      // the next pass's (or next element's first pass's) loads fly during the MMAs
      float rnext[NP], snext[NSX];
      S tnext[NF];
      if (!last) fetch(k0, i + kTcThreads, rnext, tnext, snext);
      else if (tile + gridDim.x < ntiles) fetch(row_elem(tile + gridDim.x), ti, rnext, tnext, snext);

      bool mok = true;
      if (tid < 32) mok = mbar_wait_bounded(bar_mma, mph, 2000000000ull);
      if (__syncthreads_or(!mok)) {
        failed = true;
        mma_pending = int(mph);  // the MMAs may still write tensor memory
        break;
      }
      if (tid >= 32) mbar_try_wait(bar_mma, mph);
      mph ^= 1u;
      fence_after_sync();

      // ---- epilogue: rhs, collision, update; outputs straight from registers -------
#pragma unroll
      for (int c = 0; c < (NP + 7) / 8; ++c) {
        float V[8], W[8], Lf[8];
        tmem_ld8(ta + 8 * c, V);
        tmem_ld8(ta + ND + 8 * c, W);
        tmem_ld8(ta + 2 * ND + 8 * c, Lf);
        tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int n = 8 * c + q;
          if (n < NP && valid) {
            float rhs = fmaf(-ar, V[q], fmaf(-as, W[q], Lf[q]));
            rhs += collision<float>(sm.mom + (te * NP + n) * 8, ex, ey, w, fc[n], inv_tau, third);
            float r = dt * rhs;
            if (read_res) r = fmaf(rkA, rcur[n], r);
            a.res[(k0 * NP + n) * QT + i] = r;
            const float fnew = new_f<ST>(fc[n], rkB, r);
            if constexpr (kRescale) {
              dloc = fmaxf(dloc, fabsf((fnew - w) * invw));
            } else if constexpr (kKeepScale) {
              const float qv = (fnew - w) * invw * inv_s_el;
              const size_t gi = (k0 * NP + n) * QT + i;
              if (a.sr_step) fout[gi] = bf16_round_stochastic(qv, sr_hash(gi, __ldg(a.sr_step), uint32_t(a.sr_stage)));
              else fout[gi] = ST::from_r(qv);
            } else {
              fout[(k0 * NP + n) * QT + i] = fnew;
            }
          }
        }
      }
#pragma unroll
      for (int n = 0; n < NP; ++n) rcur[n] = rnext[n];
#pragma unroll
      for (int q = 0; q < NF; ++q) tcur[q] = tnext[q];
      if constexpr (ST::dev) {
#pragma unroll
        for (int q = 0; q < NSX; ++q) scur[q] = snext[q];
      }
      fence_before_sync();
      __syncthreads();  // accumulators and operand rows are free for the next pass
    }
    if (failed) break;

    // ---- FP16 form: new element scale, then encode from the old tile -----------
    if constexpr (kRescale) {
      atomicMax(sm.dmax, __float_as_uint(dloc));
      __syncthreads();
      if (tid == 0) {
        const float md = __uint_as_float(sm.dmax[0]);
        float sc = 1.0f;
        if (md > 0.f) {
          int ex2;
          frexpf(md, &ex2);
          sc = ldexpf(1.0f, ex2 - ST::qmax_log2);
        }
        sm.nscale[0] = sc;
        a.scale_out[k0] = sc;
      }
      __syncthreads();
      const float inv_s = 1.0f / sm.nscale[0];
#pragma unroll 1
      for (int pass = 0; pass < NPASS; ++pass) {
        const int i = pass * kTcThreads + tid;
        const float w = sm.vel[kVelW * QT + i], invw = __ldg(a.vel + kVelInvW * QT + i);
#pragma unroll
        for (int n = 0; n < NP; ++n) {
          // the residual this thread stored above, and the same f_new as there
          const float fold = decode<ST>(sm.f[n * QT + i], w, w * s_el);
          const float fnew = new_f<ST>(fold, rkB, a.res[(k0 * NP + n) * QT + i]);
          fout[(k0 * NP + n) * QT + i] = ST::from_r((fnew - w) * invw * inv_s);
        }
      }
      __syncthreads();  // the state tile, scale and maximum are free for the next element
      if (tile + gridDim.x < ntiles) {
        if (tid < 32) tc_issue_tile<ST>(a, sm, QT, (tile + gridDim.x) * EPT, tile_ne(tile + gridDim.x));
        pending = (j + 1) & 1;
      }
    }
  }
  if (failed) {
    if (tid == 0 && a.err) atomicExch(a.err, 1);
    // a copy of the next tile may still be in flight: let it land (bounded)
    if (pending >= 0) mbar_wait_bounded(bar_tile, uint32_t(pending), 1000000000ull);
    // committed MMAs must finish with tensor memory before it is released (bounded)
    if (mma_pending >= 0) mbar_wait_bounded(bar_mma, uint32_t(mma_pending), 1000000000ull);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTcCols));
  }
}

// Largest degree with a tensor-core form.
constexpr int kTcMaxP = 5;

// Dynamic shared memory of the tensor-core kernel (0 = no tensor-core form).
size_t tc_smem(int store_kind, int Qp) {
  if (P > kTcMaxP || store_kind == kStoreF64 || (Qp != 16 && Qp != 128 && Qp != 256 && Qp != 1024)) return 0;
  if (Qp == 16 && store_kind == kStoreF16) return 0;  // stacked tiles: not the rescaling form
  const bool dev = store_kind != kStoreF32;
  return tc::layout(Qp, dev ? 2 : 4, dev ? 3 : 2).end;
}

// Tensor-memory columns one CTA of the tensor-core kernel allocates.
int tc_tmem_cols(int) { return tc::kTcCols; }

// Calls fn with the tensor-core kernel of a store kind and velocity count.
template <class Fn>
cudaError_t with_tc_kernel(int store_kind, int Qp, Fn fn) {
  if constexpr (P <= kTcMaxP) {
    auto by_q = [&](auto st) -> cudaError_t {
      using ST = decltype(st);
      if constexpr (!ST::dev || keeps_scale<ST>())
        if (Qp == 16) return fn(stage_kernel_tc<ST, 16>);
      if (Qp == 256) return fn(stage_kernel_tc<ST, 256>);
      if (Qp == 128) return fn(stage_kernel_tc<ST, 128>);
      if (Qp == 1024) return fn(stage_kernel_tc<ST, 1024>);
      return cudaErrorInvalidValue;
    };
    if (store_kind == kStoreF32) return by_q(StoreF32{});
    if (store_kind == kStoreBF16) return by_q(StoreBF16{});
    if (store_kind == kStoreF16) return by_q(StoreF16{});
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_tc(int store_kind, const void* args, int grid, size_t smem, cudaStream_t st) {
  const auto& a = *static_cast<const StageArgs<float>*>(args);
  cudaError_t e = with_tc_kernel(store_kind, a.Qp, [&](auto kernel) {
    kernel<<<grid, tc::kTcThreads, smem, st>>>(a);
    return cudaSuccess;
  });
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t set_smem_tc(int store_kind, int Qp, size_t smem) {
  return with_tc_kernel(store_kind, Qp, [smem](auto kernel) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    // all of the SM's unified L1/shared storage as shared memory, so that
    // several of these tiles are resident at once
    return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  });
}

// Resident CTAs per SM from the kernel's registers, its shared memory (with
// the per-block reservation) and the thread limit.
int occupancy_tc(int store_kind, int Qp, size_t smem) {
  cudaFuncAttributes fa;
  if (with_tc_kernel(store_kind, Qp, [&fa](auto kernel) { return cudaFuncGetAttributes(&fa, kernel); }) !=
      cudaSuccess)
    return 0;
  int dev = 0, regs_sm = 0, smem_sm = 0, thr_sm = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;  // allocated per warp in units of 256
  const int by_regs = regs_sm / (regs_warp * (tc::kTcThreads / 32));
  const int by_smem = int(size_t(smem_sm) / (smem + fa.sharedSizeBytes + size_t(reserved)));
  const int by_thr = thr_sm / tc::kTcThreads;
  return std::min(by_regs, std::min(by_smem, by_thr));
}
