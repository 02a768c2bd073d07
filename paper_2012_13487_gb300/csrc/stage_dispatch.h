// Per-degree entry points of the fused stage kernel (one translation unit per
// polynomial degree, so the degrees compile in parallel).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace fedbm {

struct StageEntry {
  cudaError_t (*launch)(int store_kind, const void* args, int grid, int block, size_t smem, cudaStream_t st);
  cudaError_t (*set_smem)(int store_kind, int Qp, size_t smem);
  cudaError_t (*upload)(const double* Dr, const double* Ds, const double* LIFT);
  int (*occupancy)(int store_kind, int Qp, int block, size_t smem);  // resident CTAs per SM
  // tensor-core form (FP32, BF16 or FP16 state; 128, 256 or 1024 velocities;
  // one element per CTA)
  size_t (*tc_smem)(int store_kind, int Qp);  // dynamic shared memory; 0 = no such form
  int (*tc_tmem_cols)(int Qp);                 // tensor-memory columns per CTA
  cudaError_t (*launch_tc)(int store_kind, const void* args, int grid, size_t smem, cudaStream_t st);
  cudaError_t (*set_smem_tc)(int store_kind, int Qp, size_t smem);
  int (*occupancy_tc)(int store_kind, int Qp, size_t smem);
  // velocity-split form (a cluster of ncl CTAs per element tile; FP64, FP32,
  // BF16 state; Qp a multiple of 8 ncl)
  size_t (*cl_smem)(int store_kind, int Qp, int ncl, int epc);  // 0 = no such form
  cudaError_t (*launch_cl)(int store_kind, const void* args, int nclusters, int ncl, size_t smem, cudaStream_t st);
  cudaError_t (*set_smem_cl)(int store_kind, size_t smem);
  int (*occupancy_cl)(int store_kind, int ncl, size_t smem);  // resident clusters on the device
  // warp-specialised form (a producer warp filling a three-stage ring of
  // element tiles for eight consumer warps; FP32 or BF16 state, 256 padded
  // velocities, degree <= 5)
  size_t (*ws_smem)(int store_kind, int Qp);  // 0 = no such form
  cudaError_t (*launch_ws)(int store_kind, const void* args, int grid, size_t smem, cudaStream_t st);
  cudaError_t (*set_smem_ws)(int store_kind, size_t smem);
  int (*occupancy_ws)(int store_kind, size_t smem);  // resident CTAs per SM
};

StageEntry stage_entry_p0();
StageEntry stage_entry_p1();
StageEntry stage_entry_p2();
StageEntry stage_entry_p3();
StageEntry stage_entry_p4();
StageEntry stage_entry_p5();
StageEntry stage_entry_p6();

}  // namespace fedbm
