// Shared device-side definitions of libdisc: the exact fixed-point arithmetic,
// voxel keys, hash probing, and the per-map / per-frame device state.
//
// Numerical contract (identical on every GPU run, independent of thread order):
//   * element-wise arithmetic is IEEE fp32 in a fixed operation order; the
//     library is compiled with -fmad=false so no multiply-add is fused;
//   * sums that decide labels are exact: each term is scaled by 2^S, rounded
//     to the nearest integer (ties to even) and added in int64 with atomics or
//     shuffles -- integer addition is associative, so any order gives the
//     same bits;
//   * scalar quotients/square roots of those sums are taken in fp64 and
//     rounded once to fp32.
#pragma once

#include <cstdint>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "../../include/disc.h"

namespace disc {

// fixed-point scales (bits after the binary point) of the exact sums
constexpr int S_TOK = 32;   // token sums (mean token, Eq. 1)
constexpr int S_SQ = 28;    // sums over the embedding dimension
constexpr int S_NRM = 28;   // sum of residual norms (Eq. 1)
constexpr int S_A = 24;     // coverage x distinctiveness sums
constexpr int S_SEM = 32;   // coverage x ReLU(cosine) sums
constexpr int S_EMB = 40;   // pooled embedding sums
constexpr int S_VEC = 32;   // voxel normal and S_angle sums

constexpr float TOKEN_LIMIT = 1024.0f;
constexpr int KEY_BITS = 18;
constexpr int32_t KEY_BIAS = 1 << (KEY_BITS - 1);
constexpr unsigned long long EMPTY_KEY = ~0ull;
constexpr int MAX_MASKS = 256;
constexpr int GEMM_MT = 128;    // token-dimension rows per GEMM tile
constexpr int GEMM_KC = 32;     // patches per GEMM pipeline chunk

// llrint(x * 2^S), S <= 62.  The product is exact (a power-of-two scale).
// Kept off the fp64 pipe, which converts float -> int64 at a small fraction
// of the fp32 rate on this part: below 2^31 in magnitude a 32-bit
// conversion rounds it (to nearest, ties to even, as llrint); from 2^31 on
// the float is an integer and its significand and exponent give it exactly.
__device__ __forceinline__ long long fix32f(float x, int S)
{
    const float y = __fmul_rn(x, __int_as_float((127 + S) << 23));
    if (fabsf(y) < 2147483648.0f) return (long long)__float2int_rn(y);
    const unsigned b = __float_as_uint(y);
    const int e = min((int)((b >> 23) & 0xffu) - 150, 39);  // >= 8 here; |y| < 2^63 for finite inputs in range
    const long long v = (long long)((b & 0x7fffffu) | 0x800000u) << e;
    return (b >> 31) ? -v : v;
}
__device__ __forceinline__ double unfix(long long n, int S)
{
    return __dmul_rn(__ll2double_rn(n), __longlong_as_double((long long)(1023 - S) << 52));
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// floor(p * inv_s) per axis (inv_s = 1/s rounded once to fp32), packed as
// three biased 18-bit fields; false when a coordinate is out of range.
__device__ __forceinline__ bool voxel_key(float px, float py, float pz, float inv_s,
                                          unsigned long long* key)
{
    float k[3] = {floorf(__fmul_rn(px, inv_s)), floorf(__fmul_rn(py, inv_s)), floorf(__fmul_rn(pz, inv_s))};
    unsigned long long out = 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (!(k[a] >= -(float)KEY_BIAS && k[a] <= (float)(KEY_BIAS - 1))) return false;
        out = (out << KEY_BITS) | (unsigned long long)((int)k[a] + KEY_BIAS);
    }
    *key = out;
    return true;
}

__device__ __forceinline__ void unpack_key(unsigned long long key, int k[3])
{
    const unsigned long long mask = (1ull << KEY_BITS) - 1;
    k[0] = (int)((key >> (2 * KEY_BITS)) & mask) - KEY_BIAS;
    k[1] = (int)((key >> KEY_BITS) & mask) - KEY_BIAS;
    k[2] = (int)(key & mask) - KEY_BIAS;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Device state.  Plain structs of device pointers, passed to kernels by value.

struct VoxelTable {              // open addressing, linear probing
    unsigned long long* keys;    // EMPTY_KEY = free
    int32_t* labels;             // instance id at insertion (resolve via parent)
    unsigned long long mask;     // capacity - 1 (capacity is a power of two)
    unsigned long long* used;    // number of occupied slots
};

struct Instances {
    int32_t* parent;             // flat between batches: parent[i] is always a root (inside a batch
                                 // merges may leave chains, followed to the root)
    long long* count;            // voxels per root
    float* Q;
    float* E;                    // [cap][D] stored embedding
    uint16_t* Eb;                // [cap][D] bf16 scoring copy of E (BF16 precision), else NULL
    uint8_t* E8;                 // [cap][D] E4M3 scoring copy of E / 2^e (FP8 precision), else NULL
    float* Er;                   // [cap] bound of ||2^e E8 - E|| / ||E|| for the E4M3 copy
    float* A;                    // [cap][Da] association features (second token grid), else NULL;
                                 // with them, the scoring copies Eb/E8/Er are copies of A, not E
    int32_t Da;
    int32_t* n_obs;
    int32_t cap;
};

// counters of one frame, written on the device and copied back to the host
struct FrameCounters {
    int32_t n_entries;           // unique (segment, voxel) pairs
    int32_t n_pairs;             // distinct (segment, root) overlaps
    int32_t n_new;               // distinct absent voxels
    int32_t valid_pixels;
    int32_t dropped_pixels;
    int32_t active_instances;
    int32_t new_instances;
    int32_t merges;
    int32_t live_segments;
    int32_t borderline;
    int32_t max_probe;
    int32_t err;                 // disc_status of the frame (0 = ok)
    int32_t next_id;             // instance ids handed out so far
    int32_t num_masks;           // of the frame
    int32_t n_edges;
    int32_t n_cells;             // DBSCAN grid cells of the frame
    int32_t denoised;            // pixels DBSCAN marked as noise
    int32_t db_left[2];          // DBSCAN points left to the warp-wide core / noise search
    int32_t db_cursor;           // DBSCAN cell ranges handed out
    int32_t n_absent;            // entries whose voxel was absent from the map at the batch start
    int32_t n_pre;               // distinct (segment, label) and (segment, earlier frame's segment) items
    int32_t n_scored;            // (segment, instance) pairs that passed the overlap gate (cosine taken)
    int32_t n_copies;            // embeddings written (new instances and fusion winners)
};

// One slot of the per-frame (segment, voxel) hash: one 32-byte sector.
struct __align__(32) SegSlot {
    unsigned long long key;     // (mask << 54 | voxel key); 0 = empty
    long long n[3];             // exact sums of the pixel normals (2^-32 fixed point)
};

// Per-frame scratch of one frame slot (pointers already offset to the slot).
struct Scratch {
    // Eq. 1
    long long* sumF;    // [D]
    float* fbar;        // [D]
    float* gvec;        // [D]
    long long* gg;      // [1]
    long long* nsum;    // [1]
    long long* dotg;    // [P]
    long long* ffp;     // [P]
    float* nrm;         // [P]
    float* Dp;          // [P]
    float* cosg;        // [P]
    float* fnorm;       // [P]
    // E4M3 operands (FP8 precision): token p is quantised as f_p / 2^qexp[p]
    int32_t* qexp;      // [P]
    float* qmul;        // [Kpad] 2^-qexp[p] (0 past P): the GEMM's token scaling
    float* qerr;        // [P] bound of ||2^qexp q_p - f_p||
    float* qnrm;        // [P] bound of ||q_p|| (quantised units)
    int32_t* qexpm;     // [MM] mask m's weight row is quantised as 2^qexp[p] w / 2^qexpm[m]
    uint8_t* W8;        // [Npad_max][Kpad] E4M3 weight rows, zero padded
    // coverage / weights / pooling
    int32_t* cov;       // [MM][P]
    int32_t* npix;      // [MM]
    float* W;           // [Npad_max][Kpad] GEMM operand, zero padded
    float* S;           // [MM][5]
    float* Bm;          // [MM] sum_p w ||f_p|| (error-bound scale)
    float* Ecan;        // [MM][D]
    float* Efast;       // [MM][D]
    long long* ang;     // [MM]
    int32_t* nvox;      // [MM]
    int32_t* segrep;    // [MM]
    // per-frame (segment, voxel) hash, cleared slot by slot before reuse
    SegSlot* sslot;             // [scap] key (mask << 54 | voxel key; EMPTY = 0) + normal sums
    int32_t* slist;             // [scap] used slots, in claim order (entry i -> slot)
    unsigned long long* sent;   // [scap] key of entry i (dense copy of the slot key)
    int32_t* elab;              // [scap] per entry: label at batch start, -1 absent
    unsigned long long smask;
    // per-frame overlap items, counted over the whole batch before the frames
    // run in order (one hash per slot, capacity scap, cleared slot by slot):
    // key = mask << 33 | tag << 32 | x, tag 0: x = the voxel's label at the
    // batch start; tag 1: x = j0 << 9 | m0, the voxel was first seen in the
    // batch by frame j0 of the same map, its lowest segment there m0
    unsigned long long* pkey;   // [scap] EMPTY = ~0
    int32_t* pcnt;              // [scap] voxels of the item
    int32_t* plist;             // [scap] used slots, in claim order
    int32_t* aent;              // [scap] entries absent at the batch start
    int32_t* aslot;             // [scap] and their slot in the batch's absent-voxel hash (aent + scap)
    // the items again, dense (k_items, once k_absent is done with aent and
    // aslot): ikey over aent | aslot, icnt over plist
    unsigned long long* ikey;   // [n_pre] item keys
    int32_t* icnt;              // [n_pre] voxels of the item
    int32_t* newcnt;            // [MM] voxels this frame inserts, by their lowest segment
    FrameCounters* ctr;
    // DBSCAN (Sec. III-A), allocated once a frame asks for it
    unsigned long long* dkey;   // [scap] (mask << 54 | cell); EMPTY = 0
    int32_t* dcnt;              // [scap] points per cell
    int32_t* dpos;              // [scap] cell -> position in the cell list
    int32_t* dlist;             // [scap] cell list (hash slots, claim order)
    int32_t* dstart;            // [scap] first point of list position i in dorder
    int32_t* dfill;             // [scap] scatter cursor per list position
    float4* dpt;                // [px] world point and mask of each point
    int32_t* dcell;             // [px] hash slot of the pixel's cell, -1: not a point
    int32_t* dorder;            // [px] points in cell order
    unsigned char* dflag;       // [px] bit 0 core, bit 1 noise
    float4* dsp;                // [px] the points in cell order (copies of dpt)
    int32_t* dund;              // [px] points the pixel window left undecided
};

// The frame slots of one batch: base pointers plus the per-frame stride of
// every array (in elements).
struct BatchScratch {
    Scratch base;
    long long sD, sP, sMM, sMMP, sW, sMMD, sS, scap, spx, sK;
    __host__ __device__ Scratch frame(int f) const
    {
        Scratch s = base;
        s.sumF += f * sD;
        s.fbar += f * sD;
        s.gvec += f * sD;
        s.gg += f;
        s.nsum += f;
        s.dotg += f * sP;
        s.ffp += f * sP;
        s.nrm += f * sP;
        s.Dp += f * sP;
        s.cosg += f * sP;
        s.fnorm += f * sP;
        s.qexp += f * sP;
        s.qmul += f * sK;
        s.qerr += f * sP;
        s.qnrm += f * sP;
        s.qexpm += f * sMM;
        s.W8 += f * sW;
        s.cov += f * sMMP;
        s.npix += f * sMM;
        s.W += f * sW;
        s.S += f * sS;
        s.Bm += f * sMM;
        s.Ecan += f * sMMD;
        s.Efast += f * sMMD;
        s.ang += f * sMM;
        s.nvox += f * sMM;
        s.segrep += f * sMM;
        s.sslot += f * scap;
        s.slist += f * scap;
        s.sent += f * scap;
        s.elab += f * scap;
        if (s.pkey) {
            s.pkey += f * scap;
            s.pcnt += f * scap;
            s.plist += f * scap;
            s.aent += f * 2 * scap;
            s.aslot = s.aent + scap;
            s.ikey = (unsigned long long*)s.aent;
            s.icnt = s.plist;
            s.newcnt += f * sMM;
        }
        s.ctr += f;
        if (s.dkey) {
            s.dkey += f * scap;
            s.dcnt += f * scap;
            s.dpos += f * scap;
            s.dlist += f * scap;
            s.dstart += f * scap;
            s.dfill += f * scap;
            s.dpt += f * spx;
            s.dcell += f * spx;
            s.dorder += f * spx;
            s.dflag += f * spx;
            s.dsp += f * spx;
            s.dund += f * spx;
        }
        return s;
    }
};

// Map-level scratch of the serial (per-frame) phases.
struct SerialScratch {
    unsigned long long* okeys;  // (mask << 32 | root); EMPTY = ~0
    int32_t* ocnt;
    int32_t* olist;
    unsigned long long omask;
    unsigned long long* nkeys;  // absent voxel key; EMPTY = ~0
    int32_t* nown;              // lowest mask label containing it
    int32_t* nlist;
    unsigned long long nmask;
    int32_t* edge_m;            // [edge_cap] accepted (segment, local root) edges
    int32_t* edge_k;
    int32_t* edge_n;            // [1] number of edges
    int32_t edge_cap;
    int32_t* copy_dst;          // [copy_cap] instance id receiving an embedding
    int32_t* copy_src;          // >= 0 instance id, < 0: segment -(m+1)
    int32_t* copy_n;            // [1]
    int32_t copy_cap;
    unsigned char* ureg;        // a union region of the full capacities (frames past the shared ones)
};

// Everything the kernels need of one map's resident state.  A batch holds an
// array of these in device memory (one per map of the batch), so captured
// launch sequences stay valid when a map's tables grow.
struct MapRefs {
    VoxelTable vt;
    Instances inst;
    SerialScratch ss;
    int* next_id;               // [1] next unused instance id
};

// End-of-trajectory finalisation scratch (k_final.cu)
enum { FIN_PAIRS = 0, FIN_EDGES, FIN_MERGED, FIN_REMOVED, FIN_ERR, FIN_NCTR };
struct FinalizeScratch {
    unsigned long long* pkeys;  // (min id << 32 | max id) of instances in contact; EMPTY = ~0
    int32_t* pcnt;              // contact voxels per pair
    int32_t* plist;             // occupied pair slots
    unsigned long long pmask;
    int32_t* ea;                // accepted pairs
    int32_t* eb;
    int32_t* comp;              // [nid] union-find over ids
    unsigned long long* win;    // [nid] winner key per component
    unsigned char* drop;        // [nid] dropped by the voxel count
    int32_t* ctr;               // [FIN_NCTR]
    unsigned long long* removed_voxels;
};

// One step of the serial part over the maps of a batch: block row g runs the
// j-th frame of map g.
struct SerialStep {
    const MapRefs* refs;        // [G]
    const int* slot_of;         // [G * J] frame slot of frame j of map g, -1: none
    const int* prev_hist;       // [G] index in hist of the frame before this batch, -1: none
    const FrameCounters* hist;  // counters of the call's earlier batches
    int J;                      // frames per map in this batch
    int j;                      // this step
    BatchScratch view;          // the second grid's features per slot (zero when the runner has none)
    int cta_scale;              // serial kernels' CTAs, in quarters of the default count (4 = default)
    int* merged;                // [G] some frame of map g merged instances in this batch (k_associate)
};

// Voxels absent from their map when a batch starts, over all maps of the
// batch: key (map + 1) << 54 | voxel key (never 0 = EMPTY), value the least
// (frame position j << 9 | segment m) of the batch's segments that contain
// the voxel.  Filled by k_lookup, read by k_absent, emptied by k_commit,
// which inserts each voxel with its first frame's label.
struct AbsentHash {
    unsigned long long* key;    // [cap]
    int32_t* val;               // [cap] above every (j << 9 | m) when empty
    int32_t* list;              // [cap] used slots
    int32_t* n;                 // [1] used slots
    unsigned long long mask;    // cap - 1
};

// frame parameters passed by value
struct FrameParams {
    int32_t H, W, M, P, D, Ph, Pw, Kpad, Npad;
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float voxel, z_min, z_max, eps, tau, lambda_size;
    float inv_fx, inv_fy, inv_voxel;   // 1/fx, 1/fy, 1/voxel rounded once to fp32
    int32_t ov_num, ov_den, min_px;
    int32_t token_bf16;
    int32_t map;           // position of the frame's map in the batch (MapRefs index)
    int32_t jpos;          // position of the frame among its map's frames in the batch
    int32_t precision;     // disc_precision of the fast pooled embedding and scoring
    int32_t dilate;        // overlap_dilation: 26-neighbour overlap
    int32_t assoc;         // the map has a second grid: association on its features
    int32_t uniform_w;     // this is the second grid's view: pixel-mean weights c_p / |M|
    int32_t db_min_pts;    // DBSCAN core threshold; 0: no DBSCAN for this frame
    float db_eps2;         // eps * eps
    float db_inv_cell;     // 1 / (1.001 eps): grid cells a little wider than eps
    float eta;             // bound of |E_fast - E| relative to sum_p w_p ||f_p||
    float dot_err;         // bound of the fast cosine's own error
    const float* depth;
    const uint16_t* labels;
    const void* tokens;
    const float* gembed;   // nullable
};

// ---- Sec. III-A: world point of pixel (u, v) at depth z -------------------------
__device__ __forceinline__ void world_point(const FrameParams& fp, int u, int v, float z, float p[3])
{
    float xc = __fmul_rn(__fmul_rn(__fsub_rn(__fadd_rn((float)u, 0.5f), fp.cx), z), fp.inv_fx);
    float yc = __fmul_rn(__fmul_rn(__fsub_rn(__fadd_rn((float)v, 0.5f), fp.cy), z), fp.inv_fy);
#pragma unroll
    for (int r = 0; r < 3; r++)
        p[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(fp.R[3 * r], xc), __fmul_rn(fp.R[3 * r + 1], yc)),
                                   __fmul_rn(fp.R[3 * r + 2], z)),
                         fp.t[r]);
}

// ---- E4M3 (OCP FP8: 4 exponent bits, 3 mantissa bits, largest finite 448) ----
// Power-of-two scales keep the scaling itself exact: a vector with largest
// magnitude mx is stored as x / 2^e with e the least integer such that
// mx <= 448 * 2^e, so the conversion rounds once (to nearest even, finite).
__device__ __forceinline__ int e4m3_exp(float mx)
{
    if (!(mx > 0.0f) || !(mx <= 3.0e38f)) return 0;
    int e = ilogbf(mx) - 8;  // 448 = 1.75 * 2^8
    for (int i = 0; i < 4 && mx > ldexpf(448.0f, e); i++) e++;
    for (int i = 0; i < 4 && mx <= ldexpf(448.0f, e - 1); i++) e--;
    return e;
}

// x * 2^e, correctly rounded (exact unless the result is subnormal): one
// multiply by the power of two when that is a normal float, else ldexpf
__device__ __forceinline__ float scale_pow2(float x, int e)
{
    if (e >= -126 && e <= 127) return __fmul_rn(x, __int_as_float((127 + e) << 23));
    return ldexpf(x, e);
}

__device__ __forceinline__ uint8_t to_e4m3(float x)
{
    return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

__device__ __forceinline__ float from_e4m3(uint8_t q)
{
    __nv_fp8_e4m3 v;
    v.__x = (__nv_fp8_storage_t)q;
    return (float)v;
}

// One warp writes the E4M3 scoring copy q = rn(x / 2^e) of an embedding row
// and a bound of its relative error ||2^e q - x|| / ||x||, taken from the
// actual residue (fp32 sums widened by 1 + 2^-9).  All 32 lanes call.
__device__ __forceinline__ void e4m3_copy_row(const float* x, int D, uint8_t* q8, float* er)
{
    const int lane = threadIdx.x & 31;
    float mx = 0.0f;
    for (int d = lane; d < D; d += 32) mx = fmaxf(mx, fabsf(x[d]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = e4m3_exp(mx);
    float se = 0.0f, sn = 0.0f;
    for (int d = lane; d < D; d += 32) {
        const float v = x[d];
        const uint8_t q = to_e4m3(scale_pow2(v, -e));
        q8[d] = q;
        const float r = __fsub_rn(scale_pow2(from_e4m3(q), e), v);
        se = __fadd_rn(se, __fmul_rn(r, r));
        sn = __fadd_rn(sn, __fmul_rn(v, v));
    }
    for (int o = 16; o > 0; o >>= 1) {
        se = __fadd_rn(se, __shfl_xor_sync(0xffffffffu, se, o));
        sn = __fadd_rn(sn, __shfl_xor_sync(0xffffffffu, sn, o));
    }
    if (lane == 0) *er = sn > 0.0f ? __fmul_rn(__fdiv_rn(sqrtf(se), sqrtf(sn)), 1.0f + 0x1p-9f) : 0.0f;
}

// The embedding the association gate scores against: the association
// feature with a second grid, else the stored embedding; its length.
__host__ __device__ __forceinline__ const float* scoring_master(const Instances& in) { return in.A ? in.A : in.E; }
__host__ __device__ __forceinline__ int scoring_dim(const Instances& in, int D) { return in.A ? in.Da : D; }

}  // namespace disc
