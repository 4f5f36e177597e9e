// Host-side launchers of the libdisc kernels (all enqueue on the given stream).
#pragma once

#include <cuda_runtime.h>

#include "disc_common.cuh"

namespace disc {

// Eq. 1, coverage, weights + image quality terms, exact pooling
void launch_features(const FrameParams& fp, const Scratch& sc, cudaStream_t st, int cov_smem_limit);
cudaError_t set_feature_kernel_attrs(int max_dyn_smem);

// tensor-core pooling GEMM (fast embedding used by the association gate)
void launch_pool_gemm(const FrameParams& fp, const Scratch& sc, cudaStream_t st);
cudaError_t set_gemm_kernel_attrs();
size_t gemm_smem_bytes(int NT);

// map side
void launch_frame_begin(const Scratch& sc, FrameCounters* prev, const int* next_id, int D, int sticky,
                        cudaStream_t st);
void launch_geometry(const FrameParams& fp, const Scratch& sc, const VoxelTable& vt, const Instances& inst,
                     cudaStream_t st);
void launch_associate(const FrameParams& fp, const Scratch& sc, const Instances& inst, int* next_id, float eta,
                      float dot_err, cudaStream_t st);
void launch_insert(const Scratch& sc, const VoxelTable& vt, const Instances& inst, cudaStream_t st);
void launch_rehash(const VoxelTable& from, const VoxelTable& to, int* err, cudaStream_t st);
void launch_query_topk(const float* q, int nq, int D, const Instances& inst, int nid, float* scores, int k,
                       int* ids, float* out, cudaStream_t st);
void launch_query_points(const float* xyz, long long n, float voxel, const VoxelTable& vt, const Instances& inst,
                         int* ids, cudaStream_t st);
void launch_load_voxels(const unsigned long long* keys, const int* labels, long long n, const VoxelTable& vt,
                        int* err, cudaStream_t st);

}  // namespace disc
