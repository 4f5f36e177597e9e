// End of the trajectory (Sec. III-B, last paragraph): merge the remaining
// orphaned candidates, then drop instances with too few voxels.
//
//   contact(a, b) = voxels of a or b with a face neighbour in the other
//   merge a, b   when contact * den >= num * min(|a|, |b|) and the exact
//                cosine of their embeddings >= tau (state at the start)
//   components   transitive, represented by the smallest id; Q and
//                embedding of the member with the highest Q (ties: smallest
//                id); voxel and observation counts summed
//   filter       live instances with 0 < count < min_voxels are dropped: their
//                voxels carry no instance (label -1), count/observations/Q = 0
//
// Kernels in order: contacts (six face-neighbour lookups per voxel, distinct
// neighbouring instances per voxel, a (pair -> count) hash), gates (one warp
// per pair, exact fixed-point cosine), union by smallest id (lock-free
// hooking, bounded retries), winner per component, merge, fusion, parent
// flattening, filter.
#include <climits>

#include "disc_common.cuh"
#include "kernels.h"

namespace disc {

namespace {

__device__ __forceinline__ void fin_err(FinalizeScratch fs, int code) { atomicCAS(&fs.ctr[FIN_ERR], 0, code); }

// label of a key in the table, or -2 when absent
__device__ __forceinline__ int table_label(const VoxelTable& vt, unsigned long long key)
{
    unsigned long long h = mix64(key) & vt.mask;
    for (unsigned long long pr = 0; pr <= vt.mask; pr++) {
        const unsigned long long kk = vt.keys[h];
        if (kk == key) return vt.labels[h];
        if (kk == EMPTY_KEY) return -2;
        h = (h + 1) & vt.mask;
    }
    return -2;
}

__device__ __forceinline__ int find_comp(const int* comp, int x)
{
    for (int it = 0; it < (1 << 26); it++) {
        const int p = ((volatile const int*)comp)[x];
        if (p == x) return x;
        x = p;
    }
    return x;
}

}  // namespace

__global__ void k_fin_contacts(VoxelTable vt, const int32_t* parent, FinalizeScratch fs)
{
    const unsigned long long cap = vt.mask + 1;
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap;
         s += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long key = vt.keys[s];
        if (key == EMPTY_KEY) continue;
        const int lab = vt.labels[s];
        if (lab < 0) continue;
        const int a = parent[lab];
        int k[3];
        unpack_key(key, k);
        int seen[6];
        int ns = 0;
        for (int ax = 0; ax < 3; ax++) {
            for (int sg = -1; sg <= 1; sg += 2) {
                int q[3] = {k[0], k[1], k[2]};
                q[ax] += sg;
                if (q[ax] < -KEY_BIAS || q[ax] > KEY_BIAS - 1) continue;
                const unsigned long long nk = ((unsigned long long)(q[0] + KEY_BIAS) << (2 * KEY_BITS)) |
                                              ((unsigned long long)(q[1] + KEY_BIAS) << KEY_BITS) |
                                              (unsigned long long)(q[2] + KEY_BIAS);
                const int nl = table_label(vt, nk);
                if (nl < 0) continue;
                const int b = parent[nl];
                if (b == a) continue;
                bool dup = false;
                for (int j = 0; j < ns; j++) dup |= seen[j] == b;
                if (!dup) seen[ns++] = b;
            }
        }
        for (int j = 0; j < ns; j++) {
            const int b = seen[j];
            const unsigned long long pk = ((unsigned long long)min(a, b) << 32) | (unsigned)max(a, b);
            unsigned long long h = mix64(pk) & fs.pmask;
            for (unsigned long long pr = 0;; pr++) {
                const unsigned long long prev = atomicCAS(&fs.pkeys[h], EMPTY_KEY, pk);
                if (prev == EMPTY_KEY) {
                    const int at = atomicAdd(&fs.ctr[FIN_PAIRS], 1);
                    fs.plist[at] = (int)h;
                    break;
                }
                if (prev == pk) break;
                h = (h + 1) & fs.pmask;
                if (pr > fs.pmask) {
                    fin_err(fs, DISC_ERR_TABLE_FULL);
                    return;
                }
            }
            atomicAdd(&fs.pcnt[h], 1);
        }
    }
}

// one warp per contact pair: the contact gate, then the exact cosine
__global__ void k_fin_gates(Instances inst, int D, FinalizeScratch fs, int num, int den, float tau)
{
    const int lane = threadIdx.x & 31;
    const int np = fs.ctr[FIN_PAIRS];
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < np; i += (gridDim.x * blockDim.x) >> 5) {
        const int h = fs.plist[i];
        const unsigned long long pk = fs.pkeys[h];
        const int a = (int)(pk >> 32), b = (int)(pk & 0xffffffffu);
        const long long mn = min(inst.count[a], inst.count[b]);
        if ((long long)fs.pcnt[h] * den < (long long)num * mn) continue;
        // the association features with a second grid, else the embeddings
        const float* Sm = scoring_master(inst);
        const int Ds = scoring_dim(inst, D);
        const float* ea = Sm + (size_t)a * Ds;
        const float* eb = Sm + (size_t)b * Ds;
        long long xd = 0, xa = 0, xb = 0;
        for (int d = lane; d < Ds; d += 32) {
            const float x = ea[d], y = eb[d];
            xd += fix32f(__fmul_rn(x, y), S_SQ);
            xa += fix32f(__fmul_rn(x, x), S_SQ);
            xb += fix32f(__fmul_rn(y, y), S_SQ);
        }
        xd = warp_sum(xd);
        xa = warp_sum(xa);
        xb = warp_sum(xb);
        float c = 0.0f;
        if (xa != 0 && xb != 0)
            c = __double2float_rn(__ddiv_rn(unfix(xd, S_SQ), __dmul_rn(__dsqrt_rn(unfix(xa, S_SQ)), __dsqrt_rn(unfix(xb, S_SQ)))));
        if (lane == 0 && c >= tau) {
            const int e = atomicAdd(&fs.ctr[FIN_EDGES], 1);
            fs.ea[e] = a;
            fs.eb[e] = b;
        }
    }
}

// union of every accepted pair: the root with the larger id hooks under the
// smaller one, so each component's root is its smallest id
__global__ void k_fin_union(FinalizeScratch fs)
{
    const int ne = fs.ctr[FIN_EDGES];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        int x = fs.ea[e], y = fs.eb[e];
        bool done = false;
        for (int it = 0; it < (1 << 20) && !done; it++) {
            x = find_comp(fs.comp, x);
            y = find_comp(fs.comp, y);
            if (x == y) {
                done = true;
                break;
            }
            const int lo = min(x, y), hi = max(x, y);
            if (atomicCAS(&fs.comp[hi], hi, lo) == hi) done = true;
        }
        if (!done) fin_err(fs, DISC_ERR_TIMEOUT);
    }
}

// component of every id; the winner key (Q bits, inverted id) of each
// component over its live instances
__global__ void k_fin_winner(Instances inst, int nid, FinalizeScratch fs)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nid; i += gridDim.x * blockDim.x) {
        const int c = find_comp(fs.comp, i);
        fs.comp[i] = c;
        if (inst.parent[i] != i || inst.count[i] <= 0) continue;
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(inst.Q[i]) << 32) | (0xffffffffu - (unsigned)i);  // Q >= 0
        atomicMax(&fs.win[c], key);
    }
}

// live instances join their component's smallest id
__global__ void k_fin_merge(Instances inst, int nid, FinalizeScratch fs)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nid; i += gridDim.x * blockDim.x) {
        const int c = fs.comp[i];
        if (c == i || inst.parent[i] != i || inst.count[i] <= 0) continue;
        atomicAdd((unsigned long long*)&inst.count[c], (unsigned long long)inst.count[i]);
        atomicAdd(&inst.n_obs[c], inst.n_obs[i]);
        inst.count[i] = 0;
        inst.parent[i] = c;
        atomicAdd(&fs.ctr[FIN_MERGED], 1);
    }
}

// the component's Q and embedding from its winner (one warp per id)
__global__ void k_fin_fuse(Instances inst, int nid, int D, FinalizeScratch fs)
{
    const int lane = threadIdx.x & 31;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nid; c += (gridDim.x * blockDim.x) >> 5) {
        const unsigned long long key = fs.win[c];
        if (key == 0ull || fs.comp[c] != c) continue;
        const int w = (int)(0xffffffffu - (unsigned)(key & 0xffffffffu));
        if (w == c) continue;
        for (int d = lane; d < D; d += 32) inst.E[(size_t)c * D + d] = inst.E[(size_t)w * D + d];
        // the scoring copies are rows of the scoring master's length
        const int Ds = scoring_dim(inst, D);
        for (int d = lane; d < Ds; d += 32) {
            if (inst.A) inst.A[(size_t)c * Ds + d] = inst.A[(size_t)w * Ds + d];
            if (inst.Eb) inst.Eb[(size_t)c * Ds + d] = inst.Eb[(size_t)w * Ds + d];
            if (inst.E8) inst.E8[(size_t)c * Ds + d] = inst.E8[(size_t)w * Ds + d];
        }
        if (lane == 0) {
            inst.Q[c] = inst.Q[w];
            if (inst.Er) inst.Er[c] = inst.Er[w];
        }
    }
}

// parents two levels deep at most after the merge: one jump makes them flat
__global__ void k_fin_flatten(Instances inst, int nid)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nid; i += gridDim.x * blockDim.x)
        inst.parent[i] = inst.parent[inst.parent[i]];
}

__global__ void k_fin_filter_inst(Instances inst, int nid, int min_voxels, FinalizeScratch fs)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nid; i += gridDim.x * blockDim.x) {
        fs.drop[i] = 0;
        if (inst.parent[i] == i && inst.count[i] > 0 && inst.count[i] < min_voxels) {
            fs.drop[i] = 1;
            inst.count[i] = 0;
            inst.n_obs[i] = 0;
            inst.Q[i] = 0.0f;
            atomicAdd(&fs.ctr[FIN_REMOVED], 1);
        }
    }
}

__global__ void k_fin_filter_vox(VoxelTable vt, const int32_t* parent, FinalizeScratch fs)
{
    const unsigned long long cap = vt.mask + 1;
    int removed = 0;
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap;
         s += (unsigned long long)gridDim.x * blockDim.x) {
        if (vt.keys[s] == EMPTY_KEY) continue;
        const int lab = vt.labels[s];
        if (lab >= 0 && fs.drop[parent[lab]]) {
            vt.labels[s] = -1;
            removed++;
        }
    }
    removed = warp_sum(removed);
    if ((threadIdx.x & 31) == 0 && removed) atomicAdd((unsigned long long*)fs.removed_voxels, (unsigned long long)removed);
}

__global__ void k_fin_init(int nid, FinalizeScratch fs)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nid; i += gridDim.x * blockDim.x) {
        fs.comp[i] = i;
        fs.win[i] = 0ull;
    }
}

// phase 0: init + contacts; 1: gates, union, winners; 2: merge, fuse,
// flatten, filter (no error paths)
int launch_finalize(int phase, const VoxelTable& vt, const Instances& inst, int nid, int D, const FinalizeScratch& fs,
                    int min_voxels, int num, int den, float tau, cudaStream_t st)
{
    const int g = 152 * 4;
    switch (phase) {
        case 0:
            k_fin_init<<<g, 256, 0, st>>>(nid, fs);
            k_fin_contacts<<<g, 256, 0, st>>>(vt, inst.parent, fs);
            return 2;
        case 1:
            k_fin_gates<<<g, 256, 0, st>>>(inst, D, fs, num, den, tau);
            k_fin_union<<<g, 256, 0, st>>>(fs);
            k_fin_winner<<<g, 256, 0, st>>>(inst, nid, fs);
            return 3;
        default:
            k_fin_merge<<<g, 256, 0, st>>>(inst, nid, fs);
            k_fin_fuse<<<g, 256, 0, st>>>(inst, nid, D, fs);
            k_fin_flatten<<<g, 256, 0, st>>>(inst, nid);
            k_fin_filter_inst<<<g, 256, 0, st>>>(inst, nid, min_voxels, fs);
            k_fin_filter_vox<<<g, 256, 0, st>>>(vt, inst.parent, fs);
            return 5;
    }
}

}  // namespace disc
