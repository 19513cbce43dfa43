// voxel.cuh -- launch interface of the voxelizer kernels (voxel.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gp_common.cuh"

namespace gp {

constexpr int VOX_TILE = 8;  // 8^3 voxel tiles (Sec. 4.3, "Differentiable Voxelization")

struct VoxArgs {
  const float* mu;
  const float* scale;
  const float* quat;
  const float* alpha;
  int n;
  float mod;
  float k2;          // 2 ln(1/eps)
  int X, Y, Z;
  int TX, TY, TZ;    // tile grid
};

void launch_vox_pre(const VoxArgs& a, VoxRec* rec, unsigned long long* counts, cudaStream_t st);
void launch_vox_emit(const VoxArgs& a, const VoxRec* rec, const unsigned long long* offsets,
                     const unsigned long long* counts, uint32_t* keys, uint32_t* vals, uint32_t* emit_gid,
                     cudaStream_t st);
cudaError_t launch_vox_fwd(const VoxArgs& a, const VoxRec* rec, const uint32_t* vals, const uint32_t* emit_gid,
                           const uint2* ranges, float* vol, cudaStream_t st);
cudaError_t launch_vox_bwd(const VoxArgs& a, bool deterministic, const VoxRec* rec, const uint32_t* vals,
                           const uint32_t* emit_gid, const uint2* ranges, const float* dL_dV, float* accum,
                           float4* partial, cudaStream_t st);
void launch_vox_det_reduce(int n, const unsigned long long* offsets, const unsigned long long* counts,
                           const float4* partial, float* accum, cudaStream_t st);
void launch_vox_count(const VoxArgs& a, const VoxRec* rec, unsigned long long* out, cudaStream_t st);
void launch_vox_bwd_pre(const VoxArgs& a, const float* accum, float* d_mu, float* d_scale, float* d_quat,
                        float* d_alpha, cudaStream_t st);

}  // namespace gp
