// Velocity-split form of the stage kernel: one thread-block cluster of NCL
// CTAs (2, 4 or 8) shares each element tile, CTA r of the cluster owning the
// velocities [r Qc, (r+1) Qc), Qc = Qp / NCL.  Included by stage_impl.cuh
// inside its namespace; it serves the velocity sets whose whole element tile
// does not fit one CTA's shared memory (NC 33 x 33 = D2Q1089 at degree 5 and
// 6, Sec. III.B), for FP64, FP32 and BF16 deviation state.
//
// Everything in a stage is local to one velocity except two reductions over
// all velocities of a node: the moments rho, rho u that feed f^eq (Sec.
// II.A.2) and the numerators of eq. FullBC at wall nodes.  Each CTA reduces its
// own slice, writes the partial sums to its shared memory, and after a cluster
// barrier every CTA adds the NCL partial sums of every node, rank by rank in
// the same order, from the peers' shared memory (distributed shared memory,
// ld.shared::cluster), so all CTAs of the cluster hold the same node records.
// The partial-sum buffers alternate between tiles, so one cluster barrier per
// tile suffices: a CTA overwrites a buffer only after every peer has passed the
// barrier that follows the peers' last read of it.
//
// A CTA whose bounded tile wait gives up records the timeout and keeps taking
// part in the cluster barriers without loading, computing or storing until
// the loop ends, so that no peer waits at a cluster barrier for a CTA that has
// left; results are then invalid and the host reports FEDBM_ETIMEOUT.

namespace cl {

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_index() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster; release/acquire order the shared
// memory writes before the barrier with the peers' reads after it
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared-memory address of the same variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ double ld_peer(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}

constexpr int kThreads = 256;

// Shared-memory layout of one CTA (byte offsets): the slice of the element
// tile, residual and neighbour traces, per-element data, double-buffered
// partial sums, node records, wall numerators, velocity rows of the slice.
struct Layout {
  size_t bar, f, res, tr, geo, nbr, scale, nscale, part, wpart, mom, wn, vel, end;
};
__host__ __device__ inline Layout layout(int epc, int Qc, int s_bytes, int r_bytes) {
  Layout o;
  size_t b = 0;
  o.bar = b;    b += 16;
  o.f = b;      b += align16(size_t(epc) * NP * Qc * s_bytes);
  o.res = b;    b += align16(size_t(epc) * NP * Qc * r_bytes);
  o.tr = b;     b += align16(size_t(epc) * NF * Qc * s_bytes);
  o.geo = b;    b += align16(size_t(epc) * kGeoStrideDev * r_bytes);
  o.nbr = b;    b += align16(size_t(epc) * 3 * 4);
  o.scale = b;  b += align16(size_t(epc) * 4);
  o.nscale = b; b += align16(size_t(epc) * 3 * 4);
  o.part = b;   b += size_t(2) * epc * NP * 3 * 8;   // [2][epc*NP][3] FP64 partial moments
  o.wpart = b;  b += size_t(2) * epc * NF * 8;       // [2][epc*NF] FP64 partial wall numerators
  o.mom = b;    b += align16(size_t(epc) * NP * 8 * r_bytes);
  o.wn = b;     b += align16(size_t(epc) * NF * r_bytes);
  o.vel = b;    b += align16(size_t(3) * Qc * r_bytes);
  o.end = b;
  return o;
}

// Two resident CTAs of 256 threads per SM (at most 128 registers) for the
// FP32-arithmetic forms: one CTA per SM leaves too few warps to hide latency;
// the FP64 form keeps the whole register file (it would spill heavily).
template <class ST>
__host__ __device__ constexpr int cl_min_blocks() {
  return sizeof(typename ST::R) == 8 ? 1 : 2;
}

template <class ST>
__global__ void __launch_bounds__(kThreads, cl_min_blocks<ST>()) stage_kernel_cl(const StageArgs<typename ST::R> a) {
  using R = typename ST::R;
  using S = typename ST::S;
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const uint32_t rank = cluster_rank(), ncl = cluster_size();
  const int Qp = a.Qp, Qc = Qp / int(ncl), v0 = int(rank) * Qc;
  const int epc = a.epc;
  const Layout o = layout(epc, Qc, int(sizeof(S)), int(sizeof(R)));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + o.bar);
  S* s_f = reinterpret_cast<S*>(smem + o.f);
  R* s_res = reinterpret_cast<R*>(smem + o.res);
  S* s_tr = reinterpret_cast<S*>(smem + o.tr);
  R* s_geo = reinterpret_cast<R*>(smem + o.geo);
  int* s_nbr = reinterpret_cast<int*>(smem + o.nbr);
  float* s_scale = reinterpret_cast<float*>(smem + o.scale);
  float* s_nscale = reinterpret_cast<float*>(smem + o.nscale);
  double* s_part = reinterpret_cast<double*>(smem + o.part);
  double* s_wpart = reinterpret_cast<double*>(smem + o.wpart);
  R* s_mom = reinterpret_cast<R*>(smem + o.mom);
  R* s_wn = reinterpret_cast<R*>(smem + o.wn);
  R* s_vel = reinterpret_cast<R*>(smem + o.vel);  // e_x, e_y, w of the slice
  const R rkA = a.rkA, rkB = a.rkB, ab = a.ab;
  const bool read_res = rkA != R(0);
  const bool third = a.eq_order == 3;
  const S* fin = static_cast<const S*>(a.f_in);
  S* fout = static_cast<S*>(a.f_out);
  const size_t row_bytes = size_t(Qc) * sizeof(S);
  const size_t rrow_bytes = size_t(Qc) * sizeof(R);
  const int64_t ntiles = (a.K + epc - 1) / epc;
  constexpr bool kImm = kHaveOpsTable && sizeof(R) == 4 && P <= 5;

  for (int v = tid; v < 3 * Qc; v += nth) s_vel[v] = a.vel[(v / Qc) * Qp + v0 + v % Qc];
  if (tid == 0) {
    mbar_init(bar, 32);
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  __syncthreads();

  // warp 0: bulk copies of this CTA's slice of tile t (element rows, residual
  // rows, neighbour face rows) and the tile's geometry, on the tile barrier
  auto issue = [&](int64_t k0, int ne) {
    const int lane = tid & 31;
    for (int v = lane; v < ne * 3; v += 32) {
      const int code = __ldg(a.nbr + k0 * 3 + v);
      s_nbr[v] = code;
      if constexpr (ST::dev) s_nscale[v] = code >= 0 ? __ldg(a.scale_in + (code >> 3)) : 0.f;
    }
    if constexpr (ST::dev)
      for (int v = lane; v < ne; v += 32) s_scale[v] = __ldg(a.scale_in + k0 + v);
    uint32_t bytes = lane == 0 ? uint32_t(size_t(ne) * kGeoStrideDev * sizeof(R)) + a.extra_tx : 0u;
    for (int row = lane; row < ne * NP; row += 32) bytes += uint32_t(row_bytes + (read_res ? rrow_bytes : 0));
    for (int row = lane; row < ne * NF; row += 32) {
      const int code = __ldg(a.nbr + (k0 + row / NF) * 3 + (row % NF) / NFP);
      if (code >= 0) bytes += uint32_t(row_bytes);
    }
    mbar_arrive_expect_tx(bar, bytes);
    if (lane == 0) bulk_load(s_geo, a.geo + k0 * kGeoStrideDev, uint32_t(size_t(ne) * kGeoStrideDev * sizeof(R)), bar);
    for (int row = lane; row < ne * NP; row += 32) {
      const size_t g = (size_t(k0) * NP + row) * Qp + v0;
      bulk_load(s_f + size_t(row) * Qc, fin + g, uint32_t(row_bytes), bar);
      if (read_res) bulk_load(s_res + size_t(row) * Qc, a.res + g, uint32_t(rrow_bytes), bar);
    }
    for (int row = lane; row < ne * NF; row += 32) {
      const int e = row / NF, fc = (row % NF) / NFP, aa = row % NFP;
      const int code = __ldg(a.nbr + (k0 + e) * 3 + fc);
      if (code >= 0) {
        const int64_t kn = code >> 3;
        const int fn = (code >> 1) & 3;
        const int a2 = (code & 1) ? NFP - 1 - aa : aa;
        const int node = face_node(fn, a2);
        bulk_load(s_tr + size_t(row) * Qc, fin + (size_t(kn) * NP + node) * Qp + v0, uint32_t(row_bytes), bar);
      }
    }
  };

  bool dead = false;     // a tile wait of this CTA gave up
  uint32_t dead_parity = 0;  // phase of the copies it gave up on
  int64_t tile = cluster_index();
  const int64_t tstride = cluster_count();
  if (tid < 32 && tile < ntiles) issue(tile * epc, int(min(int64_t(epc), a.K - tile * epc)));
  for (int j = 0; tile < ntiles; ++j, tile += tstride) {
    const int64_t k0 = tile * epc;
    const int ne = int(min(int64_t(epc), a.K - k0));
    const uint32_t parity = uint32_t(j & 1);
    if (!dead) {
      bool ok = true;
      if (tid < 32) ok = mbar_wait_bounded(bar, parity, 2000000000ull);
      if (__syncthreads_or(!ok)) {
        dead = true;
        dead_parity = parity;
        if (tid == 0 && a.err) atomicExch(a.err, 1);
      } else if (tid >= 32) {
        mbar_try_wait(bar, parity);  // this thread's acquire of the copied slice
      }
    }
    double* part = s_part + size_t(j & 1) * epc * NP * 3;
    double* wpart = s_wpart + size_t(j & 1) * epc * NF;

    // ---- partial moments and wall numerators of this slice ----------------------
    if (!dead) {
      const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
      for (int node = warp; node < ne * NP; node += nwarp) {
        const S* row = s_f + size_t(node) * Qc;
        double m0 = 0, m1 = 0, m2 = 0;
        if (a.collision) {
          R c0 = 0, c1 = 0, c2 = 0;
          for (int i = lane; i < Qc; i += 32) {
            R f;
            if constexpr (ST::dev) f = s_vel[2 * Qc + i] * ST::to_r(row[i]);
            else f = row[i];
            c0 += f;
            c1 = fma(s_vel[i], f, c1);
            c2 = fma(s_vel[Qc + i], f, c2);
          }
          m0 = double(c0);
          m1 = double(c1);
          m2 = double(c2);
          for (int off = 16; off > 0; off >>= 1) {
            m0 += __shfl_xor_sync(kFull, m0, off);
            m1 += __shfl_xor_sync(kFull, m1, off);
            m2 += __shfl_xor_sync(kFull, m2, off);
          }
        }
        if (lane == 0) {
          part[node * 3 + 0] = m0;
          part[node * 3 + 1] = m1;
          part[node * 3 + 2] = m2;
        }
      }
      for (int trip = warp; trip < ne * NF; trip += nwarp) {
        const int e = trip / NF, fc = (trip % NF) / NFP, aa = trip % NFP;
        const int code = s_nbr[e * 3 + fc];
        double acc = 0;
        if (code < 0 && __ldg(a.wall_den_inv + (-code - 1)) > R(0)) {
          const R nxf = s_geo[e * kGeoStrideDev + 4 + 3 * fc];
          const R nyf = s_geo[e * kGeoStrideDev + 5 + 3 * fc];
          const S* row = s_f + (size_t(e) * NP + face_node(fc, aa)) * Qc;
          const R sc = ST::dev ? s_scale[e] : R(0);
          R c = 0;
          for (int i = lane; i < Qc; i += 32) {
            const R en = s_vel[i] * nxf + s_vel[Qc + i] * nyf;
            const R w = ST::dev ? s_vel[2 * Qc + i] : R(0);
            if (en > 0) c += en * decode<ST>(row[i], w, w * sc);
          }
          acc = double(c);
          for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
        }
        if (lane == 0) wpart[trip] = acc;
      }
    }
    cluster_sync();

    // ---- totals over the cluster (same rank order in every CTA), node records ----
    if (!dead) {
      for (int node = tid; node < ne * NP; node += nth) {
        double t0 = 0, t1 = 0, t2 = 0;
        for (uint32_t r = 0; r < ncl; ++r) {
          t0 += ld_peer(peer_addr(part + node * 3 + 0, r));
          t1 += ld_peer(peer_addr(part + node * 3 + 1, r));
          t2 += ld_peer(peer_addr(part + node * 3 + 2, r));
        }
        R* mm = s_mom + size_t(node) * 8;
        if (!a.collision) {
          for (int q = 0; q < 8; ++q) mm[q] = R(0);
          continue;
        }
        R rho, jx, jy;
        if constexpr (ST::dev) {
          const R sc = s_scale[node / NP];
          rho = a.W0 + sc * R(t0);
          jx = a.W1x + sc * R(t1);
          jy = a.W1y + sc * R(t2);
        } else {
          rho = R(t0);
          jx = R(t1);
          jy = R(t2);
        }
        const R irho = R(1) / rho;
        const R it = s_geo[(node / NP) * kGeoStrideDev + kGeoInvTau];
        const R ux = jx * irho, uy = jy * irho, uu = ux * ux + uy * uy;
        mm[0] = rho * (R(1) - R(0.5) * uu) * it;
        mm[1] = jx * it;
        mm[2] = jy * it;
        mm[3] = R(0.5) * rho * it;
        mm[4] = ux;
        mm[5] = uy;
        mm[6] = third ? rho * it * R(1.0 / 6.0) : R(0);
        mm[7] = third ? R(0.5) * rho * uu * it : R(0);
      }
      for (int trip = tid; trip < ne * NF; trip += nth) {
        double t = 0;
        for (uint32_t r = 0; r < ncl; ++r) t += ld_peer(peer_addr(wpart + trip, r));
        s_wn[trip] = R(t);
      }
    }
    __syncthreads();

    // ---- residual and update of every (element, velocity) of the slice --------
    if (!dead) {
      for (int item = tid; item < ne * Qc; item += nth) {
        const int e = item / Qc, i = item - e * Qc, ig = v0 + i;
        const R ex = s_vel[i], ey = s_vel[Qc + i];
        const R w = s_vel[2 * Qc + i];
        const R* g = s_geo + e * kGeoStrideDev;
        const R dt = g[kGeoDt], inv_tau = g[kGeoInvTau];
        const R ar = ex * g[0] + ey * g[2], as = ex * g[1] + ey * g[3];
        const R ws = ST::dev ? w * R(s_scale[e]) : R(0);
        S* frow = s_f + size_t(e) * NP * Qc + i;
        R* rrow = s_res + size_t(e) * NP * Qc + i;
        R fr[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) fr[m] = decode<ST>(frow[m * Qc], w, ws);
        R flux[NF];
#pragma unroll
        for (int fc = 0; fc < 3; ++fc) {
          const R en = ex * g[4 + 3 * fc] + ey * g[5 + 3 * fc];
          const R c = R(0.5) * (en - ab * fabs(en)) * g[6 + 3 * fc];
          const int code = s_nbr[e * 3 + fc];
          if (code >= 0) {
            const R wsn = ST::dev ? w * R(s_nscale[e * 3 + fc]) : R(0);
            const S* trow = s_tr + size_t(e * NF + fc * NFP) * Qc + i;
#pragma unroll
            for (int aa = 0; aa < NFP; ++aa)
              flux[fc * NFP + aa] = c * (fr[face_node(fc, aa)] - decode<ST>(trow[aa * Qc], w, wsn));
          } else {
            const int slot = -code - 1;
            const R fb = a.wall_feq[slot * Qp + ig];
            const R den_inv = __ldg(a.wall_den_inv + slot);
            const bool diffuse = den_inv > R(0);
#pragma unroll
            for (int aa = 0; aa < NFP; ++aa) {
              const R fp = diffuse ? s_wn[e * NF + fc * NFP + aa] * den_inv * fb : fb;
              flux[fc * NFP + aa] = en < R(0) ? c * (fr[face_node(fc, aa)] - fp) : R(0);
            }
          }
        }
        R invw = R(0);
        if constexpr (ST::dev) invw = a.vel[kVelInvW * Qp + ig] / R(s_scale[e]);
#pragma unroll
        for (int n = 0; n < NP; ++n) {
          R dr = 0, ds = 0, lf = 0;
#pragma unroll
          for (int m = 0; m < NP; ++m) {
            dr = fma(opv<R, kImm>(OFF_DR + n * NP + m), fr[m], dr);
            ds = fma(opv<R, kImm>(OFF_DS + n * NP + m), fr[m], ds);
          }
#pragma unroll
          for (int q = 0; q < NF; ++q) lf = fma(opv<R, kImm>(OFF_LIFT + n * NF + q), flux[q], lf);
          R rhs = fma(-ar, dr, fma(-as, ds, lf));
          rhs += collision<R>(s_mom + (size_t(e) * NP + n) * 8, ex, ey, w, fr[n], inv_tau, third);
          R r = dt * rhs;
          if (read_res) r = fma(rkA, rrow[n * Qc], r);
          rrow[n * Qc] = r;
          const R fnew = new_f<ST>(fr[n], rkB, r);
          if constexpr (ST::dev) {
            const R qv = (fnew - w) * invw;
            if (a.sr_step) {
              const uint64_t gi = (uint64_t(k0 + e) * NP + n) * uint64_t(Qp) + uint64_t(ig);
              frow[n * Qc] = bf16_round_stochastic(qv, sr_hash(gi, __ldg(a.sr_step), uint32_t(a.sr_stage)));
            } else {
              frow[n * Qc] = ST::from_r(qv);
            }
          } else {
            frow[n * Qc] = S(fnew);
          }
        }
      }
      if constexpr (ST::dev)
        for (int e = tid; e < ne; e += nth)
          if (rank == 0) a.scale_out[k0 + e] = s_scale[e];  // BF16 keeps the element scale
    }

    // ---- bulk stores of the slice, then the next tile's copies ------------------
    fence_proxy_async_smem();
    __syncthreads();
    if (!dead && tid < 32) {
      const int lane = tid;
      for (int row = lane; row < ne * NP; row += 32) {
        const size_t g = (size_t(k0) * NP + row) * Qp + v0;
        bulk_store(fout + g, s_f + size_t(row) * Qc, uint32_t(row_bytes));
        bulk_store(a.res + g, s_res + size_t(row) * Qc, uint32_t(rrow_bytes));
      }
      bulk_commit();
      const int64_t next = tile + tstride;
      if (next < ntiles) {
        bulk_wait_read();  // this lane's stores have read the tile buffers
        __syncwarp();
        issue(next * epc, int(min(int64_t(epc), a.K - next * epc)));
      }
    }
  }
  if (tid < 32) bulk_wait_read();
  if (dead && tid < 32) mbar_wait_bounded(bar, dead_parity, 1000000000ull);  // copies still in flight land (bounded)
  cluster_sync();  // no CTA leaves while a peer may still read its partial sums
}

}  // namespace cl

// ---- host side of the velocity-split form ------------------------------------
// Dynamic shared memory of one CTA (elements per tile epc, Qp/ncl velocities).
size_t cl_smem(int store_kind, int Qp, int ncl, int epc) {
  if (store_kind == kStoreF16 || ncl < 2 || Qp % (8 * ncl) != 0) return 0;
  const int s_bytes = store_kind == kStoreF64 ? 8 : store_kind == kStoreF32 ? 4 : 2;
  const int r_bytes = store_kind == kStoreF64 ? 8 : 4;
  return cl::layout(epc, Qp / ncl, s_bytes, r_bytes).end;
}

template <class Fn>
cudaError_t with_cl_kernel(int store_kind, Fn fn) {
  if (store_kind == kStoreF64) return fn(cl::stage_kernel_cl<StoreF64>);
  if (store_kind == kStoreF32) return fn(cl::stage_kernel_cl<StoreF32>);
  if (store_kind == kStoreBF16) return fn(cl::stage_kernel_cl<StoreBF16>);
  return cudaErrorInvalidValue;
}

template <class ST>
cudaError_t launch_cl_as(const void* args, int nclusters, int ncl, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(nclusters * ncl), 1, 1);
  cfg.blockDim = dim3(cl::kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = unsigned(ncl);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cl::stage_kernel_cl<ST>, *static_cast<const StageArgs<typename ST::R>*>(args));
}

cudaError_t launch_cl(int store_kind, const void* args, int nclusters, int ncl, size_t smem, cudaStream_t st) {
  if (store_kind == kStoreF64) return launch_cl_as<StoreF64>(args, nclusters, ncl, smem, st);
  if (store_kind == kStoreF32) return launch_cl_as<StoreF32>(args, nclusters, ncl, smem, st);
  if (store_kind == kStoreBF16) return launch_cl_as<StoreBF16>(args, nclusters, ncl, smem, st);
  return cudaErrorInvalidValue;
}

cudaError_t set_smem_cl(int store_kind, size_t smem) {
  return with_cl_kernel(store_kind, [smem](auto kernel) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  });
}

// Clusters of ncl CTAs that can be resident at once on the device.
int occupancy_cl(int store_kind, int ncl, size_t smem) {
  int n = 0;
  cudaError_t e = with_cl_kernel(store_kind, [&](auto kernel) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(ncl), 1, 1);
    cfg.blockDim = dim3(cl::kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(ncl);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(&n, kernel, &cfg);
  });
  return e == cudaSuccess ? n : 0;
}
