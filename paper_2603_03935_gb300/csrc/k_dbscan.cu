// Sec. III-A: the points of each segment are filtered by DBSCAN before they
// are voxelised.  A point (pixel of an active mask with valid depth and an
// in-range voxel) is core when at least min_pts points of its segment, itself
// included, lie within eps -- ((dx*dx + dy*dy) + dz*dz) <= eps*eps in fp32 --
// and kept when it is core or within eps of a core point; the other points
// are noise and count as invalid depth for the back-projection.
//
// Per frame (chunks of frames like the back-projection):
//   k_db_points      world point of every point pixel; its (mask, cell) in a
//                    hash of cells 1.001 eps wide, so every point within eps
//                    of a point lies in the 27 cells around it
//   k_db_ranges      a range of the cell-ordered point list for every cell
//   k_db_scatter     the points in cell order
//   k_db_core        core flags from the 5x5 pixels around each point: those
//                    are distinct points of the frame, so min_pts of them
//                    within eps already make the point core
//   k_db_core_full   the points the window left undecided, one warp each,
//                    over the 27 cells (counting stops at min_pts)
//   k_db_noise       a non-core point with a core point among its 5x5
//                    pixels within eps is kept
//   k_db_noise_full  the rest, one warp each: noise when no core point of
//                    the 27 cells lies within eps
// Counting and "any core" do not depend on the order of the points, so the
// order in which cells claim their ranges and points their places does not
// reach the result.
#include <algorithm>

#include "disc_common.cuh"
#include "kernels.h"

namespace disc {

namespace {

__device__ __forceinline__ void db_err(const Scratch& sc, int code) { atomicCAS(&sc.ctr->err, 0, code); }

__device__ __forceinline__ unsigned long long cell_key(int lab, int cx, int cy, int cz)
{
    return ((unsigned long long)lab << 54) | ((unsigned long long)(cx + KEY_BIAS) << (2 * KEY_BITS)) |
           ((unsigned long long)(cy + KEY_BIAS) << KEY_BITS) | (unsigned long long)(cz + KEY_BIAS);
}

__device__ __forceinline__ void cell_of(const FrameParams& fp, float4 p, int c[3])
{
    c[0] = (int)floorf(__fmul_rn(p.x, fp.db_inv_cell));
    c[1] = (int)floorf(__fmul_rn(p.y, fp.db_inv_cell));
    c[2] = (int)floorf(__fmul_rn(p.z, fp.db_inv_cell));
}

// hash slot of a cell, or -1
__device__ __forceinline__ long long find_cell(const Scratch& sc, unsigned long long key)
{
    unsigned long long h = mix64(key) & sc.smask;
    for (unsigned long long pr = 0; pr <= sc.smask; pr++) {
        const unsigned long long cur = sc.dkey[h];
        if (cur == key) return (long long)h;
        if (cur == 0ull) return -1;
        h = (h + 1) & sc.smask;
    }
    return -1;
}

__device__ __forceinline__ bool within(float4 a, float4 b, float eps2)
{
    const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)) <= eps2;
}

// Warp-wide walk over the points of the 27 cells around point p (same mask),
// 32 points at a time: f(hit, k) gets each lane's "within eps" and the
// point's position k in the cell-ordered list, and returns true (uniform over
// the warp) to stop.  Lane t < 27 looks up cell t at once (the point's own
// cell on lane 0); the walk then runs over the cells' ranges laid end to end.
// Every lane holds the same p, so the walk is uniform.
template <class F>
__device__ __forceinline__ void warp_neighbours(const FrameParams& fp, const Scratch& sc, float4 p, F&& f)
{
    int c[3];
    cell_of(fp, p, c);
    const int lab = __float_as_int(p.w);
    const int lane = threadIdx.x & 31;
    int s0 = 0, n = 0;
    if (lane < 27) {
        const int o27 = lane == 0 ? 13 : (lane <= 13 ? lane - 1 : lane);  // 13 = offset (0, 0, 0)
        const int q[3] = {c[0] + o27 / 9 - 1, c[1] + (o27 / 3) % 3 - 1, c[2] + o27 % 3 - 1};
        if (q[0] >= -KEY_BIAS && q[0] <= KEY_BIAS - 1 && q[1] >= -KEY_BIAS && q[1] <= KEY_BIAS - 1 &&
            q[2] >= -KEY_BIAS && q[2] <= KEY_BIAS - 1) {
            const long long h = find_cell(sc, cell_key(lab, q[0], q[1], q[2]));
            if (h >= 0) {
                s0 = sc.dstart[sc.dpos[h]];
                n = sc.dcnt[h];
            }
        }
    }
    int incl = n;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    const int excl = incl - n;  // non-decreasing over the lanes; lanes 27..31 hold the total
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int j0 = 0; j0 < total; j0 += 32) {
        const int j = j0 + lane;
        int cc = 0;  // the last lane whose range starts at or before j: the cell holding j
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int e = __shfl_sync(0xffffffffu, excl, cc + step);
            if (e <= j) cc += step;
        }
        const int k = __shfl_sync(0xffffffffu, s0, cc) + j - __shfl_sync(0xffffffffu, excl, cc);
        const bool hit = j < total && within(p, sc.dsp[k], fp.db_eps2);
        if (f(hit, k)) return;
    }
}

// Appends v to list (counter cnt) for the lanes with take; all 32 lanes call.
__device__ __forceinline__ void warp_append(int* list, int* cnt, bool take, int v)
{
    const unsigned m = __ballot_sync(0xffffffffu, take);
    if (!m) return;
    const int lane = threadIdx.x & 31, lead = __ffs(m) - 1;
    int base = 0;
    if (lane == lead) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, lead);
    if (take) list[base + __popc(m & ((1u << lane) - 1))] = v;
}

// Visit the points among the 5x5 pixels around pixel (u, v), itself
// included, of the same mask and within eps; f returns false to stop.
// Returns false when f stopped the walk.
template <class F>
__device__ __forceinline__ bool for_window(const FrameParams& fp, const Scratch& sc, int u, int v, float4 p, F&& f)
{
    const int lab = __float_as_int(p.w);
    for (int dv = -2; dv <= 2; dv++) {
        const int vv = v + dv;
        if (vv < 0 || vv >= fp.H) continue;
        for (int du = -2; du <= 2; du++) {
            const int uu = u + du;
            if (uu < 0 || uu >= fp.W) continue;
            const int o = vv * fp.W + uu;
            if (sc.dcell[o] < 0) continue;
            const float4 q = sc.dpt[o];
            if (__float_as_int(q.w) == lab && within(p, q, fp.db_eps2) && !f(o)) return false;
        }
    }
    return true;
}

}  // namespace

// one thread per pixel of frames [f0, f0 + gridDim.y)
__global__ void k_db_points(const FrameParams* fps, BatchScratch bs, int f0)
{
    const FrameParams& fp = fps[f0 + blockIdx.y];
    const Scratch sc = bs.frame(f0 + blockIdx.y);
    if (fp.db_min_pts <= 0 || fp.M <= 0 || sc.ctr->err) return;  // uniform per block
    const int npx = fp.W * fp.H;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool pt = false;
    float p[3] = {0.0f, 0.0f, 0.0f};
    int lab = 0;
    if (idx < npx) {
        const int u = idx % fp.W, v = idx / fp.W;
        lab = fp.labels[idx];
        const float z = fp.depth[idx];
        if (lab >= 1 && lab <= fp.M && sc.npix[lab - 1] >= fp.min_px && z >= fp.z_min && z <= fp.z_max) {
            world_point(fp, u, v, z, p);
            unsigned long long vk;
            pt = voxel_key(p[0], p[1], p[2], fp.inv_voxel, &vk);
        }
        sc.dflag[idx] = 0;
        sc.dpt[idx] = make_float4(p[0], p[1], p[2], __int_as_float(lab));
    }
    // the pixels of a warp that share a cell claim it once
    unsigned long long key = 0ull;
    if (pt) {
        int c[3];
        cell_of(fp, make_float4(p[0], p[1], p[2], 0.0f), c);
        key = cell_key(lab, c[0], c[1], c[2]);
    }
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    long long h = -1;
    if (pt && lane == __ffs(grp) - 1) {
        unsigned long long s = mix64(key) & sc.smask;
        for (unsigned long long pr = 0;; pr++) {
            const unsigned long long cur = sc.dkey[s];
            if (cur == key) break;
            if (cur == 0ull) {
                const unsigned long long prev = atomicCAS(&sc.dkey[s], 0ull, key);
                if (prev == 0ull) {
                    const int at = atomicAdd(&sc.ctr->n_cells, 1);
                    sc.dlist[at] = (int)s;
                    sc.dpos[s] = at;
                    break;
                }
                if (prev == key) break;
            }
            s = (s + 1) & sc.smask;
            if (pr > sc.smask) {
                db_err(sc, DISC_ERR_TABLE_FULL);
                s = ~0ull;
                break;
            }
        }
        if (s != ~0ull) {
            h = (long long)s;
            atomicAdd(&sc.dcnt[s], __popc(grp));
        }
    }
    if (pt) h = __shfl_sync(grp, h, __ffs(grp) - 1);
    if (idx < npx) sc.dcell[idx] = pt ? (int)h : -1;
}

// a range of the cell-ordered list per cell: each warp claims the sum of
// its cells' sizes at once and splits it by a scan
__global__ void k_db_ranges(const FrameParams* fps, BatchScratch bs, int f0)
{
    const FrameParams& fp = fps[f0 + blockIdx.y];
    const Scratch sc = bs.frame(f0 + blockIdx.y);
    if (fp.db_min_pts <= 0 || fp.M <= 0 || sc.ctr->err) return;
    const int n = sc.ctr->n_cells;
    const int lane = threadIdx.x & 31;
    for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {  // uniform per block
        const int i = i0 + threadIdx.x;
        const int x = i < n ? sc.dcnt[sc.dlist[i]] : 0;
        int incl = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        int base = 0;
        if (lane == 31) base = atomicAdd(&sc.ctr->db_cursor, incl);
        base = __shfl_sync(0xffffffffu, base, 31);
        if (i < n) {
            sc.dstart[i] = base + incl - x;
            sc.dfill[i] = 0;
        }
    }
}

__global__ void k_db_scatter(const FrameParams* fps, BatchScratch bs, int f0)
{
    const FrameParams& fp = fps[f0 + blockIdx.y];
    const Scratch sc = bs.frame(f0 + blockIdx.y);
    if (fp.db_min_pts <= 0 || fp.M <= 0 || sc.ctr->err) return;
    const int npx = fp.W * fp.H;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int h = idx < npx ? sc.dcell[idx] : -1;
    const unsigned grp = __match_any_sync(0xffffffffu, h);
    if (h < 0) return;
    const int lp = sc.dpos[h];
    int base = 0;
    const int lead = __ffs(grp) - 1;
    if (lane == lead) base = atomicAdd(&sc.dfill[lp], __popc(grp));
    base = __shfl_sync(grp, base, lead);
    const int k = sc.dstart[lp] + base + __popc(grp & ((1u << lane) - 1));
    sc.dorder[k] = idx;
    sc.dsp[k] = sc.dpt[idx];
}

__global__ void k_db_core(const FrameParams* fps, BatchScratch bs, int f0)
{
    const FrameParams& fp = fps[f0 + blockIdx.y];
    const Scratch sc = bs.frame(f0 + blockIdx.y);
    if (fp.db_min_pts <= 0 || fp.M <= 0 || sc.ctr->err) return;
    const int npx = fp.W * fp.H;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    bool left = false;
    if (idx < npx && sc.dcell[idx] >= 0) {
        int cnt = 0;
        const int need = fp.db_min_pts;
        for_window(fp, sc, idx % fp.W, idx / fp.W, sc.dpt[idx], [&](int) { return ++cnt < need; });
        if (cnt >= need)
            sc.dflag[idx] = 1;
        else
            left = true;
    }
    warp_append(sc.dund, &sc.ctr->db_left[0], left, idx);
}

// one warp per point the window left undecided
__global__ void k_db_core_full(const FrameParams* fps, BatchScratch bs, int f0)
{
    const FrameParams& fp = fps[f0 + blockIdx.y];
    const Scratch sc = bs.frame(f0 + blockIdx.y);
    if (fp.db_min_pts <= 0 || fp.M <= 0 || sc.ctr->err) return;
    const int n = sc.ctr->db_left[0], need = fp.db_min_pts;
    const int wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += gridDim.x * wpb) {  // uniform per warp
        const int idx = sc.dund[i];
        int cnt = 0;
        warp_neighbours(fp, sc, sc.dpt[idx], [&](bool hit, int) {
            cnt += __popc(__ballot_sync(0xffffffffu, hit));
            return cnt >= need;
        });
        if ((threadIdx.x & 31) == 0 && cnt >= need) sc.dflag[idx] = 1;
    }
}

__global__ void k_db_noise(const FrameParams* fps, BatchScratch bs, int f0)
{
    const FrameParams& fp = fps[f0 + blockIdx.y];
    const Scratch sc = bs.frame(f0 + blockIdx.y);
    if (fp.db_min_pts <= 0 || fp.M <= 0 || sc.ctr->err) return;
    const int npx = fp.W * fp.H;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    bool left = false;
    if (idx < npx && sc.dcell[idx] >= 0 && !(sc.dflag[idx] & 1)) {
        bool near_core = false;
        for_window(fp, sc, idx % fp.W, idx / fp.W, sc.dpt[idx], [&](int o) {
            near_core = (sc.dflag[o] & 1) != 0;
            return !near_core;
        });
        left = !near_core;
    }
    warp_append(sc.dund, &sc.ctr->db_left[1], left, idx);
}

// one warp per non-core point with no core point in its window
__global__ void k_db_noise_full(const FrameParams* fps, BatchScratch bs, int f0)
{
    const FrameParams& fp = fps[f0 + blockIdx.y];
    const Scratch sc = bs.frame(f0 + blockIdx.y);
    if (fp.db_min_pts <= 0 || fp.M <= 0 || sc.ctr->err) return;
    const int n = sc.ctr->db_left[1];
    const int wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += gridDim.x * wpb) {  // uniform per warp
        const int idx = sc.dund[i];
        bool kept = false;
        warp_neighbours(fp, sc, sc.dpt[idx], [&](bool hit, int k) {
            kept = __any_sync(0xffffffffu, hit && (sc.dflag[sc.dorder[k]] & 1));
            return kept;
        });
        if ((threadIdx.x & 31) == 0 && !kept) {
            sc.dflag[idx] = 2;
            atomicAdd(&sc.ctr->denoised, 1);
        }
    }
}

int launch_dbscan(const FrameParams* fps, const BatchScratch& bs, int f0, int nb, int H, int W, cudaStream_t st)
{
    const int npx = H * W;
    // the warp-wide searches: up to 64 resident warps on each of 152 SMs
    const dim3 g((npx + 255) / 256, nb), gl(std::max(8, 1216 / std::max(nb, 1)), nb);
    k_db_points<<<g, 256, 0, st>>>(fps, bs, f0);
    k_db_ranges<<<dim3(16, nb), 256, 0, st>>>(fps, bs, f0);
    k_db_scatter<<<g, 256, 0, st>>>(fps, bs, f0);
    k_db_core<<<g, 256, 0, st>>>(fps, bs, f0);
    k_db_core_full<<<gl, 256, 0, st>>>(fps, bs, f0);
    k_db_noise<<<g, 256, 0, st>>>(fps, bs, f0);
    k_db_noise_full<<<gl, 256, 0, st>>>(fps, bs, f0);
    return 7;
}

}  // namespace disc
