// Geometry and map-side kernels of the integration step:
//   Sec. III-A  masked depth -> world points -> voxel keys, pixel normals;
//               per-segment voxel sets V_m in a per-frame hash
//   Eq. 3       S_angle from the voxel normals and view rays
//   Sec. III-B  exact overlap of each V_m with the map (state before the
//               frame), cosine gate, union of segments and instances,
//               new instance ids, merging through the parent table
//   Sec. III-C  Q-replacement fusion of the stored embeddings
//   insertion of the frame's new voxels
#include <climits>

#include "disc_common.cuh"
#include "kernels.h"

namespace disc {

__device__ __forceinline__ void set_err(FrameCounters* c, int code) { atomicCAS(&c->err, 0, code); }

// ---- frame start: clear what the previous frame used --------------------------
// The per-frame hashes are cleared slot by slot from the previous frame's used
// lists; prev/cur are the two alternating counter blocks.
__global__ void k_frame_begin(Scratch sc, FrameCounters* prev, const int* next_id, int D, int max_masks, int sticky)
{
    const int ne = prev->n_entries, np = prev->n_pairs, nn = prev->n_new;
    const long long scap = (long long)sc.smask + 1;
    const int n = max(max(ne, np), max(nn, max(D, max_masks)));
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < ne) {
            int s = sc.slist[i];
            sc.skeys[s] = 0ull;
            sc.snpx[s] = 0;
            sc.snrm[s] = 0;
            sc.snrm[scap + s] = 0;
            sc.snrm[2 * scap + s] = 0;
        }
        if (i < np) {
            int s = sc.olist[i];
            sc.okeys[s] = EMPTY_KEY;
            sc.ocnt[s] = 0;
        }
        if (i < nn) {
            int s = sc.nlist[i];
            sc.nkeys[s] = EMPTY_KEY;
            sc.nown[s] = INT_MAX;
        }
        if (i < D) sc.sumF[i] = 0;
        if (i < max_masks) {
            sc.npix[i] = 0;
            sc.ang[i] = 0;
            sc.nvox[i] = 0;
            sc.segrep[i] = -1;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *sc.gg = 0;
        *sc.nsum = 0;
        FrameCounters z = {};
        // within one batch of frames an error stops the frames after it
        if (sticky && prev->err) z.err = prev->err;
        z.next_id = *next_id;
        *sc.ctr = z;
    }
}

// ---- Sec. III-A: world point of pixel (u, v) at depth z -------------------------
__device__ __forceinline__ void world_point(const FrameParams& fp, int u, int v, float z, float p[3])
{
    float xc = __fdiv_rn(__fmul_rn(__fsub_rn(__fadd_rn((float)u, 0.5f), fp.cx), z), fp.fx);
    float yc = __fdiv_rn(__fmul_rn(__fsub_rn(__fadd_rn((float)v, 0.5f), fp.cy), z), fp.fy);
#pragma unroll
    for (int r = 0; r < 3; r++)
        p[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(fp.R[3 * r], xc), __fmul_rn(fp.R[3 * r + 1], yc)),
                                   __fmul_rn(fp.R[3 * r + 2], z)),
                         fp.t[r]);
}

__device__ __forceinline__ bool pix_valid(const FrameParams& fp, int u, int v, int lab)
{
    if (u < 0 || v < 0 || u >= fp.W || v >= fp.H) return false;
    size_t i = (size_t)v * fp.W + u;
    if (fp.labels[i] != lab) return false;
    float z = fp.depth[i];
    return z >= fp.z_min && z <= fp.z_max;
}

// ---- back-projection + per-segment voxel dedupe (one thread per pixel) ----------
// Block (32, 8): a warp is 32 consecutive pixels of one row; its counters are
// aggregated with ballots before one atomic per warp.
__global__ void k_backproject(FrameParams fp, Scratch sc)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    const bool inside = u < fp.W && v < fp.H;
    int lab = 0;
    float z = 0.0f;
    bool active = inside && !sc.ctr->err;
    if (active) {
        const size_t idx = (size_t)v * fp.W + u;
        lab = fp.labels[idx];
        active = lab >= 1 && lab <= fp.M && sc.npix[lab - 1] >= fp.min_px;
        if (active) {
            z = fp.depth[idx];
            active = z >= fp.z_min && z <= fp.z_max;
        }
    }
    float p0[3] = {0.0f, 0.0f, 0.0f};
    unsigned long long key = 0;
    bool keyed = false;
    if (active) {
        world_point(fp, u, v, z, p0);
        keyed = voxel_key(p0[0], p0[1], p0[2], fp.voxel, &key);
    }
    const unsigned wmask = __activemask();
    const unsigned nvalid = __popc(__ballot_sync(wmask, keyed));
    const unsigned ndrop = __popc(__ballot_sync(wmask, active && !keyed));
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(wmask) - 1;
    if (lane == leader) {
        if (nvalid) atomicAdd(&sc.ctr->valid_pixels, (int)nvalid);
        if (ndrop) atomicAdd(&sc.ctr->dropped_pixels, (int)ndrop);
    }
    int probes = 0;
    if (keyed) {
        // image-space tangents: forward differences, backward at the mask's edge
        long long nfix[3] = {0, 0, 0};
        bool has_n = false;
        int ua = -1, ub = -1, va = -1, vb = -1;
        if (pix_valid(fp, u + 1, v, lab)) { ua = u + 1; ub = u; }
        else if (pix_valid(fp, u - 1, v, lab)) { ua = u; ub = u - 1; }
        if (pix_valid(fp, u, v + 1, lab)) { va = v + 1; vb = v; }
        else if (pix_valid(fp, u, v - 1, lab)) { va = v; vb = v - 1; }
        if (ua >= 0 && va >= 0) {
            float pa[3], pb[3], qa[3], qb[3];
            world_point(fp, ua, v, fp.depth[(size_t)v * fp.W + ua], pa);
            world_point(fp, ub, v, fp.depth[(size_t)v * fp.W + ub], pb);
            world_point(fp, u, va, fp.depth[(size_t)va * fp.W + u], qa);
            world_point(fp, u, vb, fp.depth[(size_t)vb * fp.W + u], qb);
            float e1[3], e2[3], n[3];
#pragma unroll
            for (int r = 0; r < 3; r++) {
                e1[r] = __fsub_rn(pa[r], pb[r]);
                e2[r] = __fsub_rn(qa[r], qb[r]);
            }
            n[0] = __fsub_rn(__fmul_rn(e2[1], e1[2]), __fmul_rn(e2[2], e1[1]));
            n[1] = __fsub_rn(__fmul_rn(e2[2], e1[0]), __fmul_rn(e2[0], e1[2]));
            n[2] = __fsub_rn(__fmul_rn(e2[0], e1[1]), __fmul_rn(e2[1], e1[0]));
            float l2 = __fadd_rn(__fadd_rn(__fmul_rn(n[0], n[0]), __fmul_rn(n[1], n[1])), __fmul_rn(n[2], n[2]));
            if (l2 > 0.0f) {
                float l = __fsqrt_rn(l2);
#pragma unroll
                for (int r = 0; r < 3; r++) n[r] = __fdiv_rn(n[r], l);
                // orient toward the camera
                float vd = __fadd_rn(__fadd_rn(__fmul_rn(__fsub_rn(p0[0], fp.t[0]), n[0]),
                                               __fmul_rn(__fsub_rn(p0[1], fp.t[1]), n[1])),
                                     __fmul_rn(__fsub_rn(p0[2], fp.t[2]), n[2]));
                if (vd > 0.0f) {
#pragma unroll
                    for (int r = 0; r < 3; r++) n[r] = -n[r];
                }
#pragma unroll
                for (int r = 0; r < 3; r++) nfix[r] = fix32f(n[r], S_VEC);
                has_n = true;
            }
        }

        // insert (mask, voxel) into the per-frame hash; the winner of an empty
        // slot appends it to the used list
        const unsigned long long hk = ((unsigned long long)lab << 54) | key;
        unsigned long long s = mix64(hk) & sc.smask;
        bool ok = true;
        while (true) {
            unsigned long long cur = sc.skeys[s];
            if (cur == hk) break;
            if (cur == 0ull) {
                unsigned long long prev = atomicCAS(&sc.skeys[s], 0ull, hk);
                if (prev == 0ull) {
                    int at = atomicAdd(&sc.ctr->n_entries, 1);
                    sc.slist[at] = (int)s;
                    break;
                }
                if (prev == hk) break;
            }
            s = (s + 1) & sc.smask;
            if (++probes > (int)sc.smask) {
                set_err(sc.ctr, DISC_ERR_TABLE_FULL);
                ok = false;
                break;
            }
        }
        if (ok) {
            atomicAdd(&sc.snpx[s], 1);
            if (has_n) {
                const long long scap = (long long)sc.smask + 1;
                atomicAdd((unsigned long long*)&sc.snrm[s], (unsigned long long)nfix[0]);
                atomicAdd((unsigned long long*)&sc.snrm[scap + s], (unsigned long long)nfix[1]);
                atomicAdd((unsigned long long*)&sc.snrm[2 * scap + s], (unsigned long long)nfix[2]);
            }
        }
    }
    const int pmax = __reduce_max_sync(wmask, probes);
    if (lane == leader && pmax > 0) atomicMax(&sc.ctr->max_probe, pmax);
}

// ---- per unique (segment, voxel): Eq. 3 term and the map lookup ------------------
__global__ void k_entries(FrameParams fp, Scratch sc, VoxelTable vt, Instances inst)
{
    const int ne = sc.ctr->n_entries;
    if (sc.ctr->err) return;
    const long long scap = (long long)sc.smask + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += gridDim.x * blockDim.x) {
        const int s = sc.slist[i];
        const unsigned long long hk = sc.skeys[s];
        const int m = (int)(hk >> 54);
        const unsigned long long key = hk & ((1ull << 54) - 1);
        // Eq. 3: max(0, -r_v . n_v) with n_v the normalised normal sum
        float N[3] = {__double2float_rn(unfix(sc.snrm[s], S_VEC)),
                      __double2float_rn(unfix(sc.snrm[scap + s], S_VEC)),
                      __double2float_rn(unfix(sc.snrm[2 * scap + s], S_VEC))};
        float l2 = __fadd_rn(__fadd_rn(__fmul_rn(N[0], N[0]), __fmul_rn(N[1], N[1])), __fmul_rn(N[2], N[2]));
        float term = 0.0f;
        if (l2 > 0.0f) {
            float l = __fsqrt_rn(l2);
            float nv[3] = {__fdiv_rn(N[0], l), __fdiv_rn(N[1], l), __fdiv_rn(N[2], l)};
            int k[3];
            unpack_key(key, k);
            float r[3];
#pragma unroll
            for (int a = 0; a < 3; a++) r[a] = __fsub_rn(__fmul_rn(__fadd_rn((float)k[a], 0.5f), fp.voxel), fp.t[a]);
            float rl2 = __fadd_rn(__fadd_rn(__fmul_rn(r[0], r[0]), __fmul_rn(r[1], r[1])), __fmul_rn(r[2], r[2]));
            if (rl2 > 0.0f) {
                float rl = __fsqrt_rn(rl2);
                float dot = __fadd_rn(__fadd_rn(__fmul_rn(r[0], nv[0]), __fmul_rn(r[1], nv[1])), __fmul_rn(r[2], nv[2]));
                term = __fdiv_rn(-dot, rl);
                if (!(term > 0.0f)) term = 0.0f;
            }
        }
        atomicAdd((unsigned long long*)&sc.ang[m - 1], (unsigned long long)fix32f(term, S_VEC));
        atomicAdd(&sc.nvox[m - 1], 1);

        // Sec. III-B: label of the voxel in the map before this frame
        unsigned long long h = mix64(key) & vt.mask;
        int lab = -1, probes = 0;
        while (true) {
            unsigned long long kk = vt.keys[h];
            if (kk == key) { lab = vt.labels[h]; break; }
            if (kk == EMPTY_KEY) break;
            h = (h + 1) & vt.mask;
            if (++probes > (int)vt.mask) { set_err(sc.ctr, DISC_ERR_TABLE_FULL); return; }
        }
        atomicMax(&sc.ctr->max_probe, probes);
        if (lab >= 0) {
            const int root = inst.parent[lab];
            const unsigned long long ok = ((unsigned long long)m << 32) | (unsigned)root;
            unsigned long long t = mix64(ok) & sc.omask;
            int pr = 0;
            while (true) {
                unsigned long long cur = sc.okeys[t];
                if (cur == ok) break;
                if (cur == EMPTY_KEY) {
                    unsigned long long prev = atomicCAS(&sc.okeys[t], EMPTY_KEY, ok);
                    if (prev == EMPTY_KEY) { sc.olist[atomicAdd(&sc.ctr->n_pairs, 1)] = (int)t; break; }
                    if (prev == ok) break;
                }
                t = (t + 1) & sc.omask;
                if (++pr > (int)sc.omask) { set_err(sc.ctr, DISC_ERR_TABLE_FULL); return; }
            }
            atomicAdd(&sc.ocnt[t], 1);
        } else {
            unsigned long long t = mix64(key) & sc.nmask;
            int pr = 0;
            while (true) {
                unsigned long long cur = sc.nkeys[t];
                if (cur == key) break;
                if (cur == EMPTY_KEY) {
                    unsigned long long prev = atomicCAS(&sc.nkeys[t], EMPTY_KEY, key);
                    if (prev == EMPTY_KEY) { sc.nlist[atomicAdd(&sc.ctr->n_new, 1)] = (int)t; break; }
                    if (prev == key) break;
                }
                t = (t + 1) & sc.nmask;
                if (++pr > (int)sc.nmask) { set_err(sc.ctr, DISC_ERR_TABLE_FULL); return; }
            }
            atomicMin(&sc.nown[t], m);
        }
    }
}

// ---- association, union, new ids, merging and fusion (one block) ---------------
constexpr int ASSOC_THREADS = 1024;
constexpr int PAIR_CAP = 8192;   // distinct (segment, instance) overlaps per frame
constexpr size_t ASSOC_SMEM = (size_t)PAIR_CAP * 16;  // roots, uf, best_src, best_q

struct AssocParams {
    float eta;      // relative error bound of the tensor-core pooled embedding
    float dot_err;  // error bound of an fp32 warp dot product (relative)
};

__device__ __forceinline__ int lower_bound_u32(const unsigned* a, int n, unsigned x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ int uf_find(int* uf, int x)
{
    while (uf[x] != x) x = uf[x];
    return x;
}

__global__ void __launch_bounds__(ASSOC_THREADS, 1)
k_associate(FrameParams fp, Scratch sc, Instances inst, int* next_id, AssocParams ap)
{
    extern __shared__ __align__(16) unsigned char assoc_smem[];
    unsigned* roots = (unsigned*)assoc_smem;            // sorted distinct roots (active set)
    int* uf = (int*)(roots + PAIR_CAP);                  // union-find over local indices
    int* best_src = uf + PAIR_CAP;                       // fusion winner per component
    float* best_q = (float*)(best_src + PAIR_CAP);
    __shared__ int first[MAX_MASKS];
    __shared__ int s_nroots, s_nedge, s_live, s_border, s_merges, s_new;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = ASSOC_THREADS / 32;
    FrameCounters* ctr = sc.ctr;
    if (ctr->err) return;
    const int M = fp.M, D = fp.D;
    const int npairs = ctr->n_pairs;
    if (npairs > PAIR_CAP) {
        if (tid == 0) set_err(ctr, DISC_ERR_CAPACITY);
        return;
    }
    if (tid == 0) { s_live = 0; s_border = 0; s_merges = 0; s_new = 0; s_nedge = 0; }
    // (1) Eq. 3 mean and Q = S_size * S_angle * S_sem * S_dist
    for (int m = tid; m < MAX_MASKS; m += ASSOC_THREADS) first[m] = -1;
    __syncthreads();
    for (int m = tid; m < M; m += ASSOC_THREADS) {
        float* S = sc.S + 5 * m;
        const int nv = sc.nvox[m];
        float sa = 0.0f;
        if (nv > 0) {
            sa = __double2float_rn(__ddiv_rn(unfix(sc.ang[m], S_VEC), (double)nv));
            atomicAdd(&s_live, 1);
        }
        S[1] = sa;
        S[4] = __fmul_rn(__fmul_rn(__fmul_rn(S[0], sa), S[2]), S[3]);
    }
    // (2) active set: sorted distinct roots of all overlaps
    int n2 = 1;
    while (n2 < npairs) n2 <<= 1;
    for (int i = tid; i < n2; i += ASSOC_THREADS)
        roots[i] = i < npairs ? (unsigned)(sc.okeys[sc.olist[i]] & 0xffffffffu) : 0xffffffffu;
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < n2; i += ASSOC_THREADS) {
                int ixj = i ^ j;
                if (ixj > i) {
                    unsigned a = roots[i], b = roots[ixj];
                    bool up = (i & k) == 0;
                    if ((a > b) == up) { roots[i] = b; roots[ixj] = a; }
                }
            }
            __syncthreads();
        }
    if (tid == 0) {
        int n = 0;
        for (int i = 0; i < npairs; i++)
            if (i == 0 || roots[i] != roots[i - 1]) roots[n++] = roots[i];
        s_nroots = n;
    }
    __syncthreads();
    const int nroots = s_nroots;
    for (int i = tid; i < nroots; i += ASSOC_THREADS) uf[i] = i;
    // (3) edges: overlap gate (exact) and cosine gate (fast score, exact re-score
    //     inside the error band), one warp per overlap pair
    for (int i = warp; i < npairs; i += nwarps) {
        const int slot = sc.olist[i];
        const unsigned long long okey = sc.okeys[slot];
        const int m = (int)(okey >> 32) - 1;
        const int k = (int)(okey & 0xffffffffu);
        const long long ov = sc.ocnt[slot];
        // overlap coefficient |V_m & V_k| / min(|V_m|, |V_k|) >= ov_num / ov_den
        const long long denom = min((long long)sc.nvox[m], inst.count[k]);
        if (ov * (long long)fp.ov_den < (long long)fp.ov_num * denom) continue;
        const float* a = sc.Efast + (size_t)m * D;
        const float* b = inst.E + (size_t)k * D;
        float dt = 0.0f, na = 0.0f, nb = 0.0f;
        for (int d = lane; d < D; d += 32) {
            float x = a[d], y = b[d];
            dt += x * y;
            na += x * x;
            nb += y * y;
        }
        dt = warp_sum(dt);
        na = warp_sum(na);
        nb = warp_sum(nb);
        bool edge;
        float cf = (na > 0.0f && nb > 0.0f) ? dt / (sqrtf(na) * sqrtf(nb)) : 0.0f;
        float band = (na > 0.0f) ? 2.2f * ap.eta * sc.Bm[m] / sqrtf(na) + ap.dot_err + 1e-6f : 2.0f;
        if (fabsf(cf - fp.tau) > band) {
            edge = cf >= fp.tau;
        } else {
            // exact re-score with the exact pooled embedding (Sec. III-B gate)
            const float* ae = sc.Ecan + (size_t)m * D;
            long long xd = 0, xa = 0, xb = 0;
            for (int d = lane; d < D; d += 32) {
                float x = ae[d], y = b[d];
                xd += fix32f(__fmul_rn(x, y), S_SQ);
                xa += fix32f(__fmul_rn(x, x), S_SQ);
                xb += fix32f(__fmul_rn(y, y), S_SQ);
            }
            xd = warp_sum(xd);
            xa = warp_sum(xa);
            xb = warp_sum(xb);
            float ce = 0.0f;
            if (xa != 0 && xb != 0)
                ce = __double2float_rn(__ddiv_rn(unfix(xd, S_SQ),
                                                 __dmul_rn(__dsqrt_rn(unfix(xa, S_SQ)), __dsqrt_rn(unfix(xb, S_SQ)))));
            edge = ce >= fp.tau;
            if (lane == 0) atomicAdd(&s_border, 1);
        }
        if (edge && lane == 0) {
            int e = atomicAdd(&s_nedge, 1);
            if (e < sc.edge_cap) {
                sc.edge_m[e] = m;
                sc.edge_k[e] = lower_bound_u32(roots, nroots, (unsigned)k);
            } else {
                set_err(ctr, DISC_ERR_CAPACITY);
            }
        }
    }
    __syncthreads();
    if (ctr->err) return;
    const int nedge = s_nedge;
    // (4) union of the instances joined by one segment; representative =
    //     smallest id (local order == id order)
    if (tid == 0) {
        for (int e = 0; e < nedge; e++) {
            const int m = sc.edge_m[e], x = sc.edge_k[e];
            if (first[m] < 0) { first[m] = x; continue; }
            int a = uf_find(uf, first[m]), b = uf_find(uf, x);
            if (a != b) { if (a < b) uf[b] = a; else uf[a] = b; }
        }
    }
    __syncthreads();
    for (int m = tid; m < M; m += ASSOC_THREADS)
        sc.segrep[m] = first[m] >= 0 ? (int)roots[uf_find(uf, first[m])] : -1;
    __syncthreads();
    // (5) new instances for live segments without an edge, in mask order
    if (tid == 0) {
        int id = *next_id;
        for (int m = 0; m < M; m++) {
            if (sc.nvox[m] > 0 && sc.segrep[m] < 0) {
                if (id >= inst.cap) { set_err(ctr, DISC_ERR_CAPACITY); break; }
                sc.segrep[m] = id;
                inst.parent[id] = id;
                inst.count[id] = 0;
                inst.Q[id] = sc.S[5 * m + 4];
                inst.n_obs[id] = 1;
                id++;
                s_new++;
            }
        }
        if (!ctr->err) *next_id = id;
    }
    __syncthreads();
    if (ctr->err) return;
    // (6) fusion per component: candidates in the order (members by ascending
    //     id, then segments by ascending mask); the first strictly larger Q wins
    //     (Sec. III-C).  best_src >= 0: an instance id; < 0: segment -(m+1).
    // compress every chain to its root (concurrent writes only store roots)
    for (int x = tid; x < nroots; x += ASSOC_THREADS) uf[x] = uf_find(uf, x);
    __syncthreads();
    int* comp_of = uf;
    for (int r = tid; r < nroots; r += ASSOC_THREADS) {
        best_src[r] = INT_MIN;
        if (comp_of[r] != r) continue;
        // only components that were touched by an edge change
        bool touched = false;
        for (int m = 0; m < M && !touched; m++) touched = sc.segrep[m] == (int)roots[r];
        if (!touched) continue;
        int src = (int)roots[r];
        float q = inst.Q[src];
        int obs = 0;
        for (int x = 0; x < nroots; x++) {
            if (comp_of[x] != r) continue;
            obs += inst.n_obs[roots[x]];
            if (x != r && inst.Q[roots[x]] > q) { q = inst.Q[roots[x]]; src = (int)roots[x]; }
        }
        for (int m = 0; m < M; m++) {
            if (sc.segrep[m] != (int)roots[r]) continue;
            obs++;
            const float qm = sc.S[5 * m + 4];
            if (qm > q) { q = qm; src = -(m + 1); }
        }
        best_src[r] = src;
        best_q[r] = q;
        inst.n_obs[roots[r]] = obs;
    }
    __syncthreads();
    // copy the winning embeddings (sources are never written in this frame)
    for (int r = warp; r < nroots; r += nwarps) {
        const int src = best_src[r];
        if (src == INT_MIN) continue;
        const int rep = (int)roots[r];
        if (src == rep) continue;
        const float* from = src >= 0 ? inst.E + (size_t)src * D : sc.Ecan + (size_t)(-src - 1) * D;
        float* to = inst.E + (size_t)rep * D;
        for (int d = lane; d < D; d += 32) to[d] = from[d];
        if (lane == 0) inst.Q[rep] = best_q[r];
    }
    // embeddings of the new instances
    for (int m = warp; m < M; m += nwarps) {
        if (sc.nvox[m] == 0) continue;
        const int id = sc.segrep[m];
        if (first[m] >= 0) continue;
        const float* from = sc.Ecan + (size_t)m * D;
        float* to = inst.E + (size_t)id * D;
        for (int d = lane; d < D; d += 32) to[d] = from[d];
    }
    __syncthreads();
    // (7) merge members into their representative
    for (int x = tid; x < nroots; x += ASSOC_THREADS) {
        const int r = comp_of[x];
        if (r == x) continue;
        const int k = (int)roots[x], rep = (int)roots[r];
        inst.parent[k] = rep;
        atomicAdd((unsigned long long*)&inst.count[rep], (unsigned long long)inst.count[k]);
        inst.count[k] = 0;
        atomicAdd(&s_merges, 1);
    }
    __syncthreads();
    // (8) keep the parent table flat (two levels at most after this frame)
    if (s_merges > 0) {
        const int nid = *next_id;
        for (int i = tid; i < nid; i += ASSOC_THREADS) inst.parent[i] = inst.parent[inst.parent[i]];
    }
    if (tid == 0) {
        ctr->active_instances = nroots;
        ctr->new_instances = s_new;
        ctr->merges = s_merges;
        ctr->live_segments = s_live;
        ctr->borderline = s_border;
        ctr->n_edges = nedge;
        ctr->next_id = *next_id;
    }
}

// ---- insertion of the new voxels (lowest segment index owns a voxel) -----------
__global__ void k_insert(Scratch sc, VoxelTable vt, Instances inst)
{
    if (sc.ctr->err) return;
    const int nn = sc.ctr->n_new;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(vt.used, (unsigned long long)nn);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
        const int t = sc.nlist[i];
        const unsigned long long key = sc.nkeys[t];
        const int lab = sc.segrep[sc.nown[t] - 1];
        unsigned long long h = mix64(key) & vt.mask;
        int probes = 0;
        while (true) {
            unsigned long long prev = atomicCAS(&vt.keys[h], EMPTY_KEY, key);
            if (prev == EMPTY_KEY) { vt.labels[h] = lab; break; }
            h = (h + 1) & vt.mask;
            if (++probes > (int)vt.mask) { set_err(sc.ctr, DISC_ERR_TABLE_FULL); return; }
        }
        atomicAdd((unsigned long long*)&inst.count[lab], 1ull);
    }
}

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
    if (inst.parent[i] == i) {
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
        if (voxel_key(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], voxel, &key)) {
            unsigned long long h = mix64(key) & vt.mask;
            for (unsigned long long pr = 0; pr <= vt.mask; pr++) {
                unsigned long long kk = vt.keys[h];
                if (kk == key) { out = inst.parent[vt.labels[h]]; break; }
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

// ---- host launchers (each returns the number of kernels it enqueued) ---------------
int launch_frame_begin(const Scratch& sc, FrameCounters* prev, const int* next_id, int D, int sticky,
                       cudaStream_t st)
{
    k_frame_begin<<<304, 256, 0, st>>>(sc, prev, next_id, D, MAX_MASKS, sticky);
    return 1;
}

int launch_backproject(const FrameParams& fp, const Scratch& sc, cudaStream_t st)
{
    if (fp.M <= 0) return 0;
    dim3 b(32, 8), g((fp.W + 31) / 32, (fp.H + 7) / 8);
    k_backproject<<<g, b, 0, st>>>(fp, sc);
    return 1;
}

int launch_entries(const FrameParams& fp, const Scratch& sc, const VoxelTable& vt, const Instances& inst,
                   cudaStream_t st)
{
    if (fp.M <= 0) return 0;
    k_entries<<<152 * 4, 256, 0, st>>>(fp, sc, vt, inst);
    return 1;
}

int launch_associate(const FrameParams& fp, const Scratch& sc, const Instances& inst, int* next_id,
                     float eta, float dot_err, cudaStream_t st)
{
    if (fp.M <= 0) return 0;
    AssocParams ap{eta, dot_err};
    k_associate<<<1, ASSOC_THREADS, ASSOC_SMEM, st>>>(fp, sc, inst, next_id, ap);
    return 1;
}

int launch_insert(const FrameParams& fp, const Scratch& sc, const VoxelTable& vt, const Instances& inst,
                  cudaStream_t st)
{
    if (fp.M <= 0) return 0;
    k_insert<<<152 * 2, 256, 0, st>>>(sc, vt, inst);
    return 1;
}

cudaError_t set_map_kernel_attrs()
{
    return cudaFuncSetAttribute(k_associate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ASSOC_SMEM);
}

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
