// Map maintenance and query kernels: table growth, checkpoint loading,
// open-vocabulary top-k over the instance embeddings, point -> instance lookup.
#include <climits>

#include "disc_common.cuh"
#include "kernels.h"

namespace disc {

// ---- growth: re-insert every entry of the old table into a larger one ----------
__global__ void k_rehash(VoxelTable from, VoxelTable to, int* err)
{
    const unsigned long long cap = from.mask + 1;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long key = from.keys[i];
        if (key == EMPTY_KEY) continue;
        unsigned long long h = mix64(key) & to.mask;
        unsigned long long probes = 0;
        while (true) {
            unsigned long long prev = atomicCAS(&to.keys[h], EMPTY_KEY, key);
            if (prev == EMPTY_KEY) { to.labels[h] = from.labels[i]; break; }
            h = (h + 1) & to.mask;
            if (++probes > to.mask) { atomicExch(err, DISC_ERR_TABLE_FULL); return; }
        }
    }
}

// ---- queries -----------------------------------------------------------------------
// cosine of each query against every live instance; scores [nq][nid]
__global__ void k_query_scores(const float* q, int nq, int D, Instances inst, int nid, float* scores)
{
    const int lane = threadIdx.x & 31;
    const int qi = blockIdx.y;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= nid || qi >= nq) return;
    float s = -INFINITY;
    if (inst.parent[i] == i && inst.n_obs[i] > 0) {  // live (a dropped instance has no observations)
        const float* a = q + (size_t)qi * D;
        const float* b = inst.E + (size_t)i * D;
        float dt = 0.0f, na = 0.0f, nb = 0.0f;
        for (int d = lane; d < D; d += 32) {
            dt += a[d] * b[d];
            na += a[d] * a[d];
            nb += b[d] * b[d];
        }
        dt = warp_sum(dt);
        na = warp_sum(na);
        nb = warp_sum(nb);
        s = (na > 0.0f && nb > 0.0f) ? dt / (sqrtf(na) * sqrtf(nb)) : 0.0f;
    }
    if (lane == 0) scores[(size_t)qi * nid + i] = s;
}

// k best per query: repeated block arg-max (score descending, id ascending)
__global__ void k_query_topk(float* scores, int nid, int k, int* ids, float* out)
{
    __shared__ float bs[32];
    __shared__ int bi[32];
    const int qi = blockIdx.x;
    float* sc = scores + (size_t)qi * nid;
    for (int j = 0; j < k; j++) {
        float best = -INFINITY;
        int bid = INT_MAX;
        for (int i = threadIdx.x; i < nid; i += blockDim.x) {
            float s = sc[i];
            if (s > best || (s == best && i < bid)) { best = s; bid = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            float s2 = __shfl_xor_sync(0xffffffffu, best, o);
            int i2 = __shfl_xor_sync(0xffffffffu, bid, o);
            if (s2 > best || (s2 == best && i2 < bid)) { best = s2; bid = i2; }
        }
        if ((threadIdx.x & 31) == 0) { bs[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = bid; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); w++)
                if (bs[w] > bs[0] || (bs[w] == bs[0] && bi[w] < bi[0])) { bs[0] = bs[w]; bi[0] = bi[w]; }
            const bool found = bi[0] != INT_MAX && bs[0] > -INFINITY;
            ids[(size_t)qi * k + j] = found ? bi[0] : -1;
            out[(size_t)qi * k + j] = found ? bs[0] : -INFINITY;
            if (found) sc[bi[0]] = -INFINITY;
            else bi[0] = INT_MAX;
        }
        __syncthreads();
    }
}

__global__ void k_query_points(const float* xyz, long long n, float voxel, VoxelTable vt, Instances inst, int* ids)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long key;
        int out = -1;
        if (voxel_key(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], __fdiv_rn(1.0f, voxel), &key)) {
            unsigned long long h = mix64(key) & vt.mask;
            for (unsigned long long pr = 0; pr <= vt.mask; pr++) {
                unsigned long long kk = vt.keys[h];
                if (kk == key) {
                    const int lab = vt.labels[h];
                    out = lab >= 0 ? inst.parent[lab] : -1;  // -1: the voxel's instance was dropped
                    break;
                }
                if (kk == EMPTY_KEY) break;
                h = (h + 1) & vt.mask;
            }
        }
        ids[i] = out;
    }
}

// insert checkpointed voxels (keys unique, table sized beforehand)
__global__ void k_load_voxels(const unsigned long long* keys, const int* labels, long long n, VoxelTable vt, int* err)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[i];
        unsigned long long h = mix64(key) & vt.mask;
        unsigned long long probes = 0;
        while (true) {
            unsigned long long prev = atomicCAS(&vt.keys[h], EMPTY_KEY, key);
            if (prev == EMPTY_KEY || prev == key) { vt.labels[h] = labels[i]; break; }
            h = (h + 1) & vt.mask;
            if (++probes > vt.mask) { atomicExch(err, DISC_ERR_TABLE_FULL); return; }
        }
    }
}

// ---- host launchers ------------------------------------------------------------------
void launch_rehash(const VoxelTable& from, const VoxelTable& to, int* err, cudaStream_t st)
{
    k_rehash<<<152 * 8, 256, 0, st>>>(from, to, err);
}

void launch_query_topk(const float* q, int nq, int D, const Instances& inst, int nid, float* scores, int k,
                       int* ids, float* out, cudaStream_t st)
{
    dim3 g((nid + 7) / 8, nq);
    k_query_scores<<<g, 256, 0, st>>>(q, nq, D, inst, nid, scores);
    k_query_topk<<<nq, 256, 0, st>>>(scores, nid, k, ids, out);
}

void launch_query_points(const float* xyz, long long n, float voxel, const VoxelTable& vt, const Instances& inst,
                         int* ids, cudaStream_t st)
{
    k_query_points<<<152 * 4, 256, 0, st>>>(xyz, n, voxel, vt, inst, ids);
}

void launch_load_voxels(const unsigned long long* keys, const int* labels, long long n, const VoxelTable& vt,
                        int* err, cudaStream_t st)
{
    k_load_voxels<<<152 * 4, 256, 0, st>>>(keys, labels, n, vt, err);
}

}  // namespace disc
