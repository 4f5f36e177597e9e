/*
 * DISC integration-step ORACLE -- test infrastructure only.
 *
 * A plain, slow, single-threaded CPU restatement of the per-frame integration
 * step of DISC (arxiv 2603.03935, Sec. III-A to III-C, Eq. 1-3).  Only the
 * tests, the package smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code with the CUDA library.
 *
 * Arithmetic contract (the readings of the paper are listed in the design
 * notes of the repository):
 *   - element-wise work is IEEE fp32 in the written operation order, no FMA;
 *   - every sum that feeds a decision is taken exactly in int64 fixed point
 *     (value * 2^S rounded to nearest-even per term), so its result does not
 *     depend on summation order;
 *   - a handful of scalar quotients and square roots are taken in fp64 and
 *     rounded once to fp32.
 */
#ifndef DISC_ORACLE_H
#define DISC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    float voxel_size;      /* metres */
    float z_min, z_max;    /* valid depth range, metres */
    float eps;             /* epsilon of Eq. 1 */
    float tau_cos;         /* cosine threshold of the association gate */
    float lambda_size;     /* lambda of S_size (3.3) */
    int32_t ov_num, ov_den;/* overlap gate: ov / |V_m| >= ov_num / ov_den */
    int32_t embed_dim;     /* D */
    int32_t patch_h, patch_w;
    int32_t min_mask_pixels;
    float dbscan_eps;        /* > 0: per-segment DBSCAN denoise before voxelisation (radius, metres) */
    int32_t dbscan_min_pts;  /* core point: at least this many points of its segment within eps */
    int32_t overlap_dilation;/* 1: a segment voxel also overlaps the instances of its 26 neighbours */
    int32_t assoc_dim;       /* > 0: a second token grid [assoc_patch_h * assoc_patch_w][assoc_dim]
                                drives association (Sec. III-A/B: DINOv2 tokens for tracking, CLIP
                                tokens for the stored embedding); its pooled feature per mask is the
                                pixel-level mean over the mask (w_p = c_p / |M|) */
    int32_t assoc_patch_h, assoc_patch_w;
} oracle_config;

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;      /* finite, fx and fy non-zero */
    double T_world_cam[16];    /* row-major camera->world; top three rows finite as fp32 */
    const float* depth;        /* [H][W] */
    const uint16_t* labels;    /* [H][W], 0 = none, 1..num_masks */
    const float* tokens;       /* [Ph*Pw][D] */
    int32_t num_masks;
    const float* global_embed; /* [D] or NULL (then the mean token) */
    const float* assoc_tokens; /* [assoc_patch_h * assoc_patch_w][assoc_dim] when assoc_dim > 0 */
} oracle_frame;

/* Per-frame intermediates; every pointer is optional (NULL = not wanted).
 * Arrays over masks have num_masks rows, mask label m in row m - 1. */
typedef struct {
    float* fbar;        /* [D]   mean token */
    float* Dp;          /* [P]   distinctiveness (Eq. 1) */
    float* cosg;        /* [P]   cosine of each token with the global embedding */
    int32_t* cov;       /* [M][P] pixels of mask m inside patch p */
    int32_t* npix;      /* [M]   |M_m| */
    float* W;           /* [M][P] pooling weights */
    float* E;           /* [M][D] pooled embeddings */
    float* S;           /* [M][5] S_size, S_angle, S_sem, S_dist, Q */
    int32_t* nvox;      /* [M]   |V_m| */
    int32_t* rep;       /* [M]   instance the segment joined, -1 if none */
    uint64_t* seg_keys; /* [seg_cap] unique (segment, voxel) pairs ordered by (m, key) */
    int32_t* seg_m;     /* [seg_cap] their mask label */
    int64_t seg_cap;
    int64_t n_seg;      /* out: number of unique (segment, voxel) pairs */
    int32_t valid_pixels, dropped_pixels, new_voxels, active_instances;
    int32_t new_instances, merges, live_segments, overlap_pairs;
    int32_t denoised_pixels;   /* pixels DBSCAN marked as noise */
    float* A;           /* [M][assoc_dim] pooled association features (assoc_dim > 0) */
} oracle_report;

enum { ORACLE_OK = 0, ORACLE_ERR_INVALID_ARG = -1, ORACLE_ERR_RANGE = -7 };

typedef struct oracle_map oracle_map;

oracle_map* oracle_map_create(const oracle_config* cfg);
void oracle_map_destroy(oracle_map* map);
int oracle_integrate_frame(oracle_map* map, const oracle_frame* frame, oracle_report* rep);

int64_t oracle_num_voxels(const oracle_map* map);
/* Voxel keys ascending with their resolved instance ids. */
void oracle_export_voxels(const oracle_map* map, uint64_t* keys, int32_t* ids);
int32_t oracle_num_ids(const oracle_map* map);
/* Per id (0..num_ids-1): parent (== id for live instances), voxel count, Q,
 * embedding [D], observations. */
void oracle_export_instances(const oracle_map* map, int32_t* parent, int64_t* count, float* Q,
                             float* E, int32_t* n_obs);

/* Per id: the association feature [assoc_dim] (assoc_dim > 0). */
void oracle_export_assoc(const oracle_map* map, float* A);

/* Fig. 2: the distinctiveness-weighted cosine heatmap of a query vector q [D]
 * over a token grid [P][D]: heat_p = D_p * cos(f_p, q), D_p of Eq. 1 and the
 * exact cosine, their product rounded once to fp32. */
int oracle_query_heatmap(const float* F, int32_t P, int32_t D, const float* q, float eps, float* heat);

/* End of the trajectory (Sec. III-B, last paragraph): merge the remaining
 * orphaned candidates, then drop instances below a voxel count.  Reading:
 *   contact(a, b) = number of voxels of a or b with a face neighbour (one of
 *                   the 6 voxels sharing a face) in the other instance;
 *   a and b merge when contact * contact_den >= contact_num * min(|a|, |b|)
 *   and the exact cosine of their embeddings (the association features when
 *   the map has a second token grid) is >= tau_cos (counts and
 *   embeddings as they stand when finalisation starts); merges are
 *   transitive, the smallest id represents a component, whose Q and
 *   embedding are those of its member with the highest Q (ties: smallest id)
 *   and whose voxel and observation counts are the members' sums;
 *   then every live instance with 0 < count < min_voxels is dropped: its
 *   voxels carry no instance (id -1) and its count, observations and Q are 0.
 * The map is final afterwards (integration returns ORACLE_ERR_INVALID_ARG). */
typedef struct {
    int32_t min_voxels;
    int32_t contact_num, contact_den;
    float tau_cos;
} oracle_finalize_config;

typedef struct {
    int32_t contact_pairs;   /* instance pairs in contact */
    int32_t merged;          /* instances merged into another */
    int32_t removed;         /* instances dropped by the voxel count */
    int64_t removed_voxels;  /* their voxels */
} oracle_finalize_report;

int oracle_finalize(oracle_map* map, const oracle_finalize_config* cfg, oracle_finalize_report* rep);

/* Replace the map's state (test construction of exact situations): voxels
 * keys[n] with instance labels (>= 0), instance arrays over nid ids. */
void oracle_set_state(oracle_map* map, const uint64_t* keys, const int32_t* labels, int64_t n,
                      const int32_t* parent, const int64_t* count, const float* Q, const float* E,
                      const int32_t* n_obs, int32_t nid);
/* With a second token grid: the association features [nid][assoc_dim]. */
void oracle_set_assoc(oracle_map* map, const float* A, int32_t nid);

/* DBSCAN noise of Sec. III-A (the step between back-projection and
 * voxelisation), per segment.  Reading: a point is core when at least
 * min_pts points of its segment (itself included) lie within eps; a point is
 * kept when it is core or within eps of a core point of its segment; the
 * others are noise (noise[i] = 1).  Distances are compared squared in fp32:
 * ((dx*dx + dy*dy) + dz*dz) <= eps*eps, with dx = x_i - x_j, no FMA.
 * Requires eps > 0; pts [n][3], seg [n]. */
void oracle_dbscan_noise(const float* pts, const int32_t* seg, int64_t n, float eps, int32_t min_pts,
                         uint8_t* noise);

/* Stage functions (Eq. 1, mask coverage, pooling) for unit pins. */
int oracle_token_stats(const float* F, int32_t P, int32_t D, const float* g, float eps,
                       float* fbar, float* n, float* Dp, float* cosg);
void oracle_mask_coverage(const uint16_t* labels, int32_t H, int32_t W, int32_t Ph, int32_t Pw,
                          int32_t M, int32_t* cov, int32_t* npix);
/* Voxel key of a world point, the same quantisation as the integration step;
 * returns 0 when out of range. */
int oracle_point_key(float x, float y, float z, float voxel_size, uint64_t* key);
void oracle_unpack_key(uint64_t key, int32_t* kx, int32_t* ky, int32_t* kz);
float oracle_cosine(const float* a, const float* b, int32_t D);

/* FP64 twin of Eq. 1 and the D-weighted pooling, for error statements. */
void oracle_pool_f64(const float* F, int32_t P, int32_t D, const int32_t* cov, const int32_t* npix,
                     int32_t M, double eps, double* Dp, double* E);

#ifdef __cplusplus
}
#endif
#endif
