// Host-side launchers of the libdisc kernels.  Each enqueues on the given
// stream and returns the number of kernels it launched.
//
// A batch of B frames runs in two parts:
//   batched (one launch covers every frame slot; nothing here writes the map):
//     slot_clear, token_stats (Eq. 1), coverage, weights, pool_exact,
//     pool_gemm (tcgen05), backproject, entries (+ Q)
//   serial (per frame of each map, in order; these read and write the maps,
//   all maps of the batch side by side in one launch):
//     overlap, score, union, apply
#pragma once

#include <cuda_runtime.h>

#include "disc_common.cuh"

namespace disc {

// phases timed by disc_map_phase_times, in enqueue order
enum Phase {
    PH_CLEAR = 0,     // clear the frame slots' scratch from their last use
    PH_TOKENS,        // Eq. 1
    PH_COVERAGE,      // mask -> patch coverage
    PH_WEIGHTS,       // pooling weights, S_size / S_sem / S_dist
    PH_POOL_EXACT,    // exact D-weighted pooled embedding
    PH_POOL_GEMM,     // tcgen05 pooled embedding (fast score)
    PH_DBSCAN,        // Sec. III-A noise filter of the segment points (chunks of frames)
    PH_BACKPROJECT,   // depth -> voxel keys, normals, per-segment sets (chunks of frames)
    PH_ENTRIES,       // S_angle terms, |V_m|, labels at batch start (chunks), then Q
    PH_OVERLAP,       // per frame: overlap histogram against the current map
    PH_SCORE,         // per frame: geometry and cosine gates
    PH_UNION,         // per frame: union, new ids, merges, fusion (one CTA)
    PH_APPLY,         // per frame: embeddings, new voxels, parent flattening
    PH_LOOKUP,        // every entry of the batch: label at the batch start, or first frame of the batch
    PH_ASSOCIATE,     // one CTA per map: its frames in order (pairs, gates, union, fusion, counts)
    PH_COMMIT,        // the batch's new voxels into the maps, parent tables flattened
    PH_COUNT
};

// batched
int launch_slot_clear(const BatchScratch& bs, int B, int D, int MM, cudaStream_t st);
int launch_view_clear(const BatchScratch& bs, int B, int D, int MM, cudaStream_t st);
int launch_token_stats(const FrameParams* fps, const BatchScratch& bs, int B, int P, int D, bool any_bf16,
                       bool any_f32, cudaStream_t st);
int launch_coverage(const FrameParams* fps, const BatchScratch& bs, int B, int Ph, int Pw, int Mmax, cudaStream_t st);
int launch_weights(const FrameParams* fps, const BatchScratch& bs, int B, int Mmax, cudaStream_t st);
int launch_pool_exact(const FrameParams* fps, const BatchScratch& bs, int B, int P, int D, int Mmax, bool any_bf16,
                      bool any_f32, cudaStream_t st);
// one launch per (token dtype, precision) present: any[tok_bf16][prec_bf16]
int launch_pool_gemm(const FrameParams* fps, const BatchScratch& bs, int B, int D, int Mmax, const bool any[2][3],
                     cudaStream_t st);
// back-projection and the per-entry pass (S_angle terms, |V_m|, labels at
// batch start) on frames [f0, f0 + nb); then Q of every segment
int launch_backproject(const FrameParams* fps, const BatchScratch& bs, int f0, int nb, int H, int W, cudaStream_t st);
// DBSCAN noise flags of frames [f0, f0 + nb) (frames without DBSCAN return at once)
int launch_dbscan(const FrameParams* fps, const BatchScratch& bs, int f0, int nb, int H, int W, cudaStream_t st);
int launch_entries(const FrameParams* fps, const BatchScratch& bs, const MapRefs* refs, int f0, int nb, int Mmax,
                   bool lookup, cudaStream_t st);
int launch_quality(const FrameParams* fps, const BatchScratch& bs, int B, cudaStream_t st);
// default frames per back-projection/entries/DBSCAN launch (their per-frame
// hashes stay in L2); the runner's tuning may pick another
constexpr int GEOMETRY_CHUNK = 8;

// start of a batch's serial part: every map's edge and copy counters to zero
int launch_e4m3_copies(const Instances& inst, int n, int D, cudaStream_t st);
int launch_room(const MapRefs* refs, int G, const int* slot_of, int J, const BatchScratch& bs, unsigned long long* out,
                cudaStream_t st);
int launch_serial_begin(const MapRefs* refs, int G, cudaStream_t st);
// serial part, step st.j over the G maps of a batch: phase 0 overlap,
// 1 score, 2 union, 3 apply
int launch_serial_step(const FrameParams* fps, const BatchScratch& bs, const SerialStep& st, int G, int phase,
                       cudaStream_t stream);

// The frame chain as one pass per batch (k_serial.cu): lookup of every entry
// of the batch's S slots in the maps as they stand (k_lookup, then k_absent);
// each of the G maps' frames in order in one CTA (k_associate); the batch's
// new voxels into the maps (k_commit).  The absent-voxel hash is empty
// before k_lookup and after k_commit.
// probe_width: lanes per key in the voxel-table lookup (1, 2, 4, 8);
// cluster: CTAs per map of the association kernel (0: as many as the maps
// leave room for, up to 8; else 1, 2, 4 or 8, capped by the device)
int launch_lookup(const FrameParams* fps, const BatchScratch& bs, const MapRefs* refs, const AbsentHash& ah, int S,
                  int probe_width, cudaStream_t st);
int launch_associate(const FrameParams* fps, const BatchScratch& bs, const SerialStep& st, int G, int cluster,
                     cudaStream_t s);
int launch_commit(const BatchScratch& bs, const SerialStep& st, const AbsentHash& ah, int G, cudaStream_t s);
// bytes of the union region a map keeps in global memory (SerialScratch::ureg)
size_t union_region_bytes_full();

size_t coverage_smem_bytes(int max_masks, int Pw);
size_t gemm_smem_bytes(int NT);
cudaError_t set_feature_kernel_attrs(int max_dyn_smem);
cudaError_t set_gemm_kernel_attrs();
cudaError_t set_gemm_stall(bool on);
cudaError_t set_serial_kernel_attrs();

// end-of-trajectory finalisation, phases 0..2 (k_final.cu)
int launch_finalize(int phase, const VoxelTable& vt, const Instances& inst, int nid, int D, const FinalizeScratch& fs,
                    int min_voxels, int num, int den, float tau, cudaStream_t st);

// maintenance and queries
void launch_rehash(const VoxelTable& from, const VoxelTable& to, int* err, cudaStream_t st);
void launch_query_topk(const float* q, int nq, int D, const Instances& inst, int nid, float* scores, int k,
                       int* ids, float* out, cudaStream_t st);
void launch_query_points(const float* xyz, long long n, float voxel, const VoxelTable& vt, const Instances& inst,
                         int* ids, cudaStream_t st);
void launch_load_voxels(const unsigned long long* keys, const int* labels, long long n, const VoxelTable& vt,
                        int* err, cudaStream_t st);

}  // namespace disc
