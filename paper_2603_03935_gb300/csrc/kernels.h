// Host-side launchers of the libdisc kernels.  Each enqueues on the given
// stream and returns the number of kernels it launched.
#pragma once

#include <cuda_runtime.h>

#include "disc_common.cuh"

namespace disc {

// per-frame phases, in enqueue order
enum Phase {
    PH_BEGIN = 0,     // clear the previous frame's scratch
    PH_TOKENS,        // Eq. 1 (4 kernels)
    PH_COVERAGE,      // mask -> patch coverage
    PH_WEIGHTS,       // pooling weights, S_size / S_sem / S_dist
    PH_POOL_EXACT,    // exact D-weighted pooled embedding
    PH_POOL_GEMM,     // tcgen05 pooled embedding (fast score)
    PH_BACKPROJECT,   // depth -> voxel keys, normals, per-segment sets
    PH_ENTRIES,       // S_angle terms, map lookup, overlap histogram
    PH_ASSOCIATE,     // gates, union, new ids, merges, fusion
    PH_INSERT,        // new voxels
    PH_COUNT
};

int launch_frame_begin(const Scratch& sc, FrameCounters* prev, const int* next_id, int D, int sticky,
                       cudaStream_t st);
int launch_token_stats(const FrameParams& fp, const Scratch& sc, cudaStream_t st);
int launch_coverage(const FrameParams& fp, const Scratch& sc, cudaStream_t st, int cov_smem_limit);
int launch_weights(const FrameParams& fp, const Scratch& sc, cudaStream_t st);
int launch_pool_exact(const FrameParams& fp, const Scratch& sc, cudaStream_t st);
int launch_pool_gemm(const FrameParams& fp, const Scratch& sc, cudaStream_t st);
int launch_backproject(const FrameParams& fp, const Scratch& sc, cudaStream_t st);
int launch_entries(const FrameParams& fp, const Scratch& sc, const VoxelTable& vt, const Instances& inst,
                   cudaStream_t st);
int launch_associate(const FrameParams& fp, const Scratch& sc, const Instances& inst, int* next_id, float eta,
                     float dot_err, cudaStream_t st);
int launch_insert(const FrameParams& fp, const Scratch& sc, const VoxelTable& vt, const Instances& inst,
                  cudaStream_t st);

cudaError_t set_feature_kernel_attrs(int max_dyn_smem);
cudaError_t set_gemm_kernel_attrs();
cudaError_t set_map_kernel_attrs();
size_t gemm_smem_bytes(int NT);

// maintenance and queries
void launch_rehash(const VoxelTable& from, const VoxelTable& to, int* err, cudaStream_t st);
void launch_query_topk(const float* q, int nq, int D, const Instances& inst, int nid, float* scores, int k,
                       int* ids, float* out, cudaStream_t st);
void launch_query_points(const float* xyz, long long n, float voxel, const VoxelTable& vt, const Instances& inst,
                         int* ids, cudaStream_t st);
void launch_load_voxels(const unsigned long long* keys, const int* labels, long long n, const VoxelTable& vt,
                        int* err, cudaStream_t st);

}  // namespace disc
