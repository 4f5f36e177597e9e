/*
 * libdisc -- the per-frame integration step of DISC (Dense Integrated Semantic
 * Context, arxiv 2603.03935) as a C ABI over hand-written sm_103a kernels.
 *
 * One map = one sparse voxel hash table (voxel key -> instance id) plus an
 * instance table (union-find parent, voxel count, view quality Q, embedding),
 * all resident on one GPU.  Each integrated frame runs the paper's per-frame
 * pipeline:
 *   - distinctiveness map D over the frame's patch tokens (Sec. III-C, Eq. 1),
 *   - D-weighted pooling of the tokens inside each mask (Sec. III-C),
 *   - view quality Q = S_size * S_angle * S_sem * S_dist (Sec. III-C, Eq. 2-3),
 *   - back-projection of the masked depth into per-segment voxel sets
 *     (Sec. III-A),
 *   - exact voxel overlap of each segment with the map, the cosine gate, and
 *     on-the-fly merging of instances (Sec. III-B),
 *   - Q-replacement fusion of the instance embeddings (Sec. III-C).
 *
 * Conventions shared by every entry point:
 *   - Status codes only; nothing throws across the ABI.  A frame is all or
 *     nothing: when integration fails the map keeps its pre-frame state.
 *   - The caller owns every buffer it passes; the map owns its device state.
 *     Inputs must stay valid until the call returns (for the asynchronous
 *     integration calls: until the call is finished, see
 *     disc_integrate_frames_async).
 *   - Work is ordered on the map's CUDA stream (config.cuda_stream, or a
 *     stream the map creates).  Every call returns after its results are on
 *     the host unless stated otherwise (the *_async calls).
 *   - One host thread per map at a time; different maps are independent.
 *   - Instance ids are resolved roots (the smallest id of a merged group);
 *     -1 means "none".
 *   - Camera: OpenCV pinhole (x right, y down, z forward), pixel centres at
 *     (u + 0.5, v + 0.5); pose camera->world, row-major 4x4 doubles, rounded
 *     once to fp32 on the host.
 */
#ifndef DISC_H
#define DISC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DISC_OK = 0,
    DISC_ERR_INVALID_ARG = -1, /* bad pointer, size or configuration */
    DISC_ERR_OOM = -2,         /* a device or host allocation failed */
    DISC_ERR_TABLE_FULL = -3,  /* hash probe limit reached */
    DISC_ERR_CUDA = -4,        /* a CUDA runtime call failed */
    DISC_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    DISC_ERR_BUDGET = -6,      /* reserved for admission under a memory budget */
    DISC_ERR_RANGE = -7,       /* a token is non-finite or |value| > 1024 */
    DISC_ERR_CAPACITY = -8     /* more association edges/pairs than a frame may hold */
} disc_status;

typedef struct disc_map disc_map; /* opaque; owns all device state of one map */

typedef enum { DISC_FP32 = 0, DISC_BF16 = 1, DISC_FP8_E4M3 = 2 } disc_precision;
typedef enum { DISC_TOKENS_F32 = 0, DISC_TOKENS_BF16 = 1 } disc_token_dtype;

typedef struct {
    float voxel_size;        /* metres per voxel edge (> 0) */
    float z_min, z_max;      /* depth range that counts as valid, metres */
    float eps;               /* epsilon of Eq. 1 */
    float tau_cos;           /* association gate: cosine >= tau_cos (Sec. III-B) */
    float lambda_size;       /* lambda of S_size, 3.3 in the paper */
    int32_t ov_num, ov_den;  /* geometry gate: overlap * ov_den >= ov_num * |V_m| */
    int32_t embed_dim;       /* D, <= 4096 */
    int32_t patch_h, patch_w;/* token grid; Ph * Pw <= 16384 */
    int32_t max_width, max_height; /* largest frame this map accepts (H*W <= 2^24) */
    int32_t max_masks;       /* largest num_masks per frame, <= 256 */
    int32_t min_mask_pixels; /* masks with fewer pixels are ignored (Sec. III-A filter) */
    int64_t voxel_capacity;  /* initial hash slots (rounded up to a power of two) */
    float max_load;          /* the table doubles before its load would pass this */
    int32_t instance_capacity; /* initial instance slots (grows on demand) */
    int32_t precision;       /* disc_precision of the fast pooling/scoring path (Sec. III-B gate):
                                FP32 = TF32x3 tensor-core pooling, fp32 scoring copies;
                                BF16 = bf16 operands and scoring copies, fp32 accumulation;
                                FP8_E4M3 = E4M3 operands with power-of-two per-vector scales
                                (per token, per weight row, per stored embedding), fp32
                                accumulation.  Every precision re-scores the pairs whose fast
                                cosine lies within its error bound of tau_cos exactly, so
                                labels, counts and stored embeddings are the same for all */
    void* cuda_stream;       /* cudaStream_t, or NULL: the map creates one */
    int32_t device;          /* CUDA device ordinal */
    int32_t batch_frames;    /* frames whose stateless phases share one launch (1..256) */
    float dbscan_eps;        /* > 0: per-segment DBSCAN noise filter before voxelisation (Sec. III-A):
                                a point is core with >= dbscan_min_pts points of its segment within
                                this radius (metres, >= voxel_size), kept when core or within the
                                radius of a core point; noise pixels count as invalid depth */
    int32_t dbscan_min_pts;  /* >= 1 when dbscan_eps > 0 */
    int32_t serial_sms;      /* > 0: calls of several batches overlap the next batch's stateless steps
                                with this batch's serial steps, which run on their own set of this many
                                SMs (a green context; without one, a high-priority stream); <= 0: no
                                overlap (the default: the overlap measured slower on GB300) */
    int32_t overlap_dilation;/* 1: a segment voxel also overlaps the instances labelling any of its 26
                                neighbours (the neighbourhood reading of Sec. III-B), once per
                                instance; 0 (default): the voxel itself only */
    int32_t assoc_dim;       /* > 0: frames carry a second token grid [assoc_patch_h * assoc_patch_w]
                                [assoc_dim] (the association encoder's, e.g. DINOv2, Sec. III-A)
                                that drives association: each mask's association feature is the
                                pixel-level mean of that grid's tokens over the mask, the cosine
                                gate (and disc_map_finalize) compares those features, and each
                                instance keeps one, replaced with its embedding when a better view
                                wins the fusion; Eq. 1, the quality terms, the stored embedding
                                and the queries stay on the first grid (CLIP).  0: one grid */
    int32_t assoc_patch_h, assoc_patch_w; /* the second grid; product <= 16384; assoc_dim <= 4096 */
} disc_map_config;

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;    /* pinhole intrinsics, pixels; finite, fx and fy non-zero */
    double T_world_cam[16];  /* row-major camera -> world; its top three rows finite as fp32 (a frame
                                with a non-finite intrinsic or pose is refused: DISC_ERR_INVALID_ARG) */
    const float* depth;      /* [H][W] metres; invalid = outside [z_min, z_max] or NaN */
    const uint16_t* labels;  /* [H][W] mask label, 0 = none, 1..num_masks */
    const void* tokens;      /* [Ph*Pw][D] row-major patch tokens (token_dtype) */
    int32_t token_dtype;     /* disc_token_dtype */
    int32_t num_masks;       /* labels above num_masks count as background */
    const float* global_embed; /* [D] global image embedding, or NULL -> mean token */
    int32_t inputs_on_device;  /* 1: pointers are device memory; 0: host memory */
    const void* assoc_tokens;  /* [assoc_patch_h*assoc_patch_w][assoc_dim] (token_dtype) when the
                                  map has a second grid; else ignored */
} disc_frame;

typedef struct {
    int32_t valid_pixels;       /* masked pixels with valid depth and in-range keys */
    int32_t dropped_pixels;     /* valid depth but voxel key out of range */
    int32_t unique_seg_voxels;  /* unique (segment, voxel) pairs = voxel updates */
    int32_t new_voxels;         /* voxels inserted into the map */
    int32_t active_instances;   /* distinct instances the segments overlap */
    int32_t overlap_pairs;      /* distinct (segment, instance) overlaps */
    int32_t new_instances;
    int32_t merges;             /* instances merged into another */
    int32_t live_segments;      /* masks that produced at least one voxel */
    int32_t borderline_rescored;/* fast cosines re-scored exactly near tau_cos */
    int32_t max_probe;          /* longest hash probe of the frame */
    int32_t status;             /* disc_status of the frame */
    int32_t denoised_pixels;    /* pixels the DBSCAN filter removed */
    int32_t scored_pairs;       /* (segment, instance) pairs past the overlap gate, cosine taken */
    int32_t embedding_copies;   /* instance embeddings written (new instances, fusion winners) */
} disc_frame_stats;

/* Intermediates of the most recent frame, copied to caller host buffers (any
 * pointer may be NULL).  Rows over masks: label m in row m - 1. */
typedef struct {
    float* fbar;      /* [D] mean token (Eq. 1) */
    float* Dp;        /* [P] distinctiveness (Eq. 1) */
    float* cosg;      /* [P] cosine of each token with the global embedding */
    int32_t* cov;     /* [M][P] pixels of mask m inside patch p */
    int32_t* npix;    /* [M] |M_m| */
    float* W;         /* [M][P] pooling weights (sum to 1 per valid mask) */
    float* E;         /* [M][D] pooled embeddings, exact path */
    float* E_fast;    /* [M][D] pooled embeddings, tensor-core path */
    float* S;         /* [M][5] S_size, S_angle, S_sem, S_dist, Q */
    int32_t* nvox;    /* [M] |V_m| */
    int32_t* rep;     /* [M] instance each segment joined, -1 if none */
    uint64_t* seg_keys; /* [seg_cap] unique (segment, voxel) pairs, unordered */
    int32_t* seg_m;     /* [seg_cap] their mask label */
    int64_t seg_cap;
    int64_t n_seg;      /* out: number of pairs */
    int32_t num_masks;  /* out */
    float* E_bound;     /* [M] the bound of ||E_fast - E|| the association gate's re-score band uses
                           (of ||A_fast - A|| with a second grid) */
    float* A;           /* [M][assoc_dim] association features, exact path (second grid) */
    float* A_fast;      /* [M][assoc_dim] association features, tensor-core path (second grid) */
} disc_frame_report;

/* Fills a config with the defaults used throughout (eps 1e-6, tau_cos 0.75,
 * lambda 3.3, overlap 1/5, depth 0.1..10 m, 640x480, 24x24x768, 40 masks). */
void disc_config_default(disc_map_config* cfg);

/* Creates a map on cfg->device.  Returns DISC_ERR_INVALID_ARG for an invalid
 * config and DISC_ERR_OOM when the resident state does not fit. */
disc_status disc_map_create(const disc_map_config* cfg, disc_map_config* resolved, disc_map** out_map);

/* Integrates one frame (all steps above).  stats may be NULL. */
disc_status disc_integrate_frame(disc_map* map, const disc_frame* frame, disc_frame_stats* stats);

/* Integrates n frames in order.  Frames are processed in batches of
 * config.batch_frames: the steps that do not touch the map (Eq. 1, coverage,
 * pooling, back-projection, S_angle, Q, the lookup of every voxel in the map
 * as it stood when the batch started) run for the whole batch in one launch
 * each; overlap, association, merging, fusion and insertion then run frame
 * after frame on the device with no host round trip.  The result is the same
 * as n calls of disc_integrate_frame.  stats (nullable) receives one entry per
 * frame.  On an error the frames before the failing one stay integrated;
 * *n_done (nullable) says how many. */
disc_status disc_integrate_frames(disc_map* map, const disc_frame* frames, int32_t n,
                                  disc_frame_stats* stats, int32_t* n_done);

/* Asynchronous form of disc_integrate_frames (the paper integrates a stream
 * of frames; this lets the next call's frames start while the last frames of
 * the previous call still associate, Sec. III-B, so the map's frame chain and
 * the next frames' per-frame kernels share the GPU).  The call enqueues the
 * frames and returns DISC_OK without waiting for them; it is finished later
 * by disc_map_wait, by a third asynchronous call on the map (at most two stay
 * unfinished; the oldest is finished first), or by any other call on the map,
 * which sees the map after every earlier call.  When a call is finished its
 * results are written: stats (nullable, n entries), *n_done (nullable) and
 * *result (nullable, the status disc_integrate_frames would have returned).
 * Until then the caller keeps stats, n_done and result valid, and the
 * frames' input buffers (host or device) unchanged; the disc_frame array
 * itself is read before the call returns.  Frames run in call order: a frame
 * that fails on the device stops every later frame of the map, in this call
 * and in calls enqueued while it was unfinished (their *result is that
 * error).  A frame that fails the host checks, and a map whose calls cannot
 * overlap (phase timing on, or the neighbourhood overlap without serial_sms),
 * make the call run synchronously: earlier calls finish first and the results
 * are written before it returns, with the status also returned.  Work on the
 * map's stream is not made to wait for an unfinished call.  Errors returned
 * directly: DISC_ERR_INVALID_ARG (bad arguments, a finalised map), and the
 * synchronous cases' statuses. */
disc_status disc_integrate_frames_async(disc_map* map, const disc_frame* frames, int32_t n,
                                        disc_frame_stats* stats, int32_t* n_done, disc_status* result);

/* Finishes the unfinished asynchronous calls that hold the map (its own, or a
 * group's: then every call of that group), oldest first, writing their
 * results.  Returns the first of their statuses that is not DISC_OK. */
disc_status disc_map_wait(disc_map* map);

/* ---- Groups: many maps integrated side by side --------------------------
 * A group owns the scratch of one batch over up to max_maps maps with up to
 * frames_per_map frames each (the paper has no counterpart: it processes one
 * map; this serves many independent maps on one GPU).  Every launch of a
 * batch covers the frames of all its maps; the stateful steps (overlap,
 * association, merging, fusion, insertion) run frame j of every map in one
 * launch, so maps hide each other's per-frame latency.  Each map's result is
 * bit for bit the result of integrating its frames alone.  Maps keep their
 * tables (resident on the device) between calls and may join any group call
 * whose embed_dim, patch grid and device match theirs. */
typedef struct disc_group disc_group; /* opaque */

typedef struct {
    int32_t max_maps;        /* maps per call (1..1024) */
    int32_t frames_per_map;  /* frames of one map per batch (1..256); max_maps * frames_per_map <= 4096 */
    int32_t embed_dim;       /* D of every map of the group */
    int32_t patch_h, patch_w;/* token grid of every map of the group */
    int32_t max_width, max_height; /* largest frame of any map */
    int32_t max_masks;       /* largest num_masks of any frame (<= 256) */
    void* cuda_stream;       /* cudaStream_t, or NULL: the group creates one */
    int32_t device;
    int32_t serial_sms;      /* as in disc_map_config */
    int32_t assoc_dim, assoc_patch_h, assoc_patch_w; /* the second grid of maps that have one (0: none);
                                                        such maps need a group with the same grid */
} disc_group_config;

/* Defaults: 16 maps x 4 frames, 640x480, 24x24x768, 40 masks. */
void disc_group_config_default(disc_group_config* cfg);

/* Allocates the batch scratch (about 26 MB per frame slot at 640x480).
 * DISC_ERR_INVALID_ARG for an invalid config, DISC_ERR_OOM when it does not
 * fit. */
disc_status disc_group_create(const disc_group_config* cfg, disc_group** out_group);

/* Integrates counts[i] frames (frames[i], in order) into maps[i] for every i,
 * each map's frames in order and the maps independently: a frame that fails
 * stops the later frames of its own map only.  stats (nullable; stats[i]
 * nullable) receives one entry per frame of each map; n_done (nullable)
 * [n_maps] how many frames of each map were integrated.  A map may appear
 * once per call.  Returns DISC_OK when every frame was integrated, else the
 * first failure in map order.  Returns after all results are complete. */
disc_status disc_group_integrate(disc_group* group, disc_map* const* maps, int32_t n_maps,
                                 const disc_frame* const* frames, const int32_t* counts,
                                 disc_frame_stats* const* stats, int32_t* n_done);

/* Asynchronous form of disc_group_integrate, with the semantics of
 * disc_integrate_frames_async: the batch's frame chains overlap the next
 * call's per-frame kernels.  stats[i] (the arrays, not the outer array),
 * n_done [n_maps] and result stay valid until the call is finished, by
 * disc_group_wait, a third asynchronous call on the group, another call on
 * the group, or any call on one of its maps (disc_map_wait finishes every
 * call of the group).  A map whose earlier asynchronous calls are held by
 * another runner (its own, or another group) has them finished first. */
disc_status disc_group_integrate_async(disc_group* group, disc_map* const* maps, int32_t n_maps,
                                       const disc_frame* const* frames, const int32_t* counts,
                                       disc_frame_stats* const* stats, int32_t* n_done, disc_status* result);

/* Finishes the group's unfinished asynchronous calls, oldest first, writing
 * their results; returns the first of their statuses that is not DISC_OK. */
disc_status disc_group_wait(disc_group* group);

/* Per-phase timing of the group's batches (as disc_map_set_phase_timing). */
disc_status disc_group_set_phase_timing(disc_group* group, int32_t enable);
disc_status disc_group_phase_times(disc_group* group, double* ms, int64_t* launches, int64_t* calls,
                                   int32_t n);
/* Kernels the group has launched since creation (graph nodes counted per
 * replay), and the device bytes its scratch holds; 0 for a NULL group. */
int64_t disc_group_kernel_launches(disc_group* group);
int64_t disc_group_device_bytes(disc_group* group);
/* Frees the group's streams, graphs and scratch; the maps it integrated stay
 * valid (its unfinished asynchronous calls are finished first).  Must not
 * overlap a disc_group_integrate on the same group. */
void disc_group_destroy(disc_group* group); /* NULL-safe */

/* ---- Serving: a request loop over many resident maps ----------------------
 * Clients (any host threads) submit integrate and query requests for maps the
 * server holds resident on the device.  Worker threads batch continuously,
 * each with a group of its own: a worker's batch takes, for up to
 * group.max_maps maps with work that no other batch holds (oldest request
 * first), the leading frames of each map's queue (up to
 * group.frames_per_map, stopping at the map's first query) and runs them as
 * one group call; requests arriving meanwhile join a later batch.  While
 * other workers wait for work, a worker takes only its share of the free
 * maps (their number over the waiting workers plus one), so under a full
 * load batches stay in flight side by side: one batch's input copies and
 * stateless kernels run while another's frame chain computes.  A map is in one batch at a time and a query
 * runs after the frames submitted before it on the same map and before those
 * after it, so every result equals the one of the same requests served alone.
 * Maps are admitted while the device memory of the workers' group scratch and
 * all open maps stays within hbm_budget_bytes (the paper has no counterpart
 * of this layer). */
typedef struct disc_server disc_server; /* opaque */

typedef struct {
    disc_group_config group;  /* batch shape and limits of every map */
    int64_t hbm_budget_bytes; /* admission limit for the group scratch plus the open maps */
    int32_t max_queue;        /* requests queued or running at most; more: DISC_ERR_BUDGET */
    int32_t workers;          /* batches in flight at once, 1..4 (0: 2) */
} disc_server_config;

typedef struct {
    int64_t frames, queries, batches; /* completed since creation or the last reset */
    int64_t pending;                  /* requests queued or running */
    int64_t resident_bytes;           /* the workers' group scratch + open maps at admission */
    double busy_ms;                   /* host time inside batches, summed over the workers */
    double wall_ms;                   /* since creation or the last reset */
    double p50_ms, p99_ms;            /* frame latency, submission to completion */
} disc_server_report;

/* Creates the server, its worker threads and their groups.  DISC_ERR_BUDGET
 * when the groups' scratch alone passes the budget; DISC_ERR_INVALID_ARG for
 * workers outside 0..4. */
disc_status disc_server_create(const disc_server_config* cfg, disc_server** out_server);

/* Opens a map (cfg's embed_dim, patch grid and device equal to the group's;
 * frame size and masks within the group's).  DISC_ERR_BUDGET when admitting
 * it would pass the budget. */
disc_status disc_server_open_map(disc_server* server, const disc_map_config* cfg, int32_t* map_id);

/* Waits for the map's requests, then frees it. */
disc_status disc_server_close_map(disc_server* server, int32_t map_id);

/* The map behind map_id, for export and checkpoints between requests (NULL
 * when not open).  Do not use it while the map has requests pending. */
disc_map* disc_server_map(disc_server* server, int32_t map_id);

/* Queues one frame of map_id.  Its inputs (host or device, inputs_on_device)
 * are copied before the call returns.  *ticket identifies the request. */
disc_status disc_server_submit_frame(disc_server* server, int32_t map_id, const disc_frame* frame,
                                     int64_t* ticket);

/* As disc_server_submit_frame, but the inputs are not copied: the batch that
 * takes the frame reads the caller's buffers in place (device memory, or host
 * memory: pinned memory lets the copies run asynchronously).  They must stay
 * allocated and unchanged until disc_server_wait has returned for the
 * ticket. */
disc_status disc_server_submit_frame_borrowed(disc_server* server, int32_t map_id, const disc_frame* frame,
                                              int64_t* ticket);

/* Queues a top-k query: queries [nq][D] host memory, copied before return. */
disc_status disc_server_submit_query(disc_server* server, int32_t map_id, const float* queries, int32_t nq,
                                     int32_t k, int64_t* ticket);

/* Waits for a request and returns its status.  A frame fills stats
 * (nullable); a query fills ids and scores [nq][k] (nullable).  latency_ms
 * (nullable): submission to completion.  A ticket has one waiter: it can be
 * waited for once, and a second wait on it, concurrent or later, returns
 * DISC_ERR_INVALID_ARG. */
disc_status disc_server_wait(disc_server* server, int64_t ticket, disc_frame_stats* stats, int32_t* ids,
                             float* scores, double* latency_ms);

/* The counters and latency percentiles of disc_server_report (out: caller
 * memory); callable from any thread.  reset_stats zeroes the completed
 * counts, busy and wall time and the latency samples (pending and resident
 * bytes are states, not counts, and stay).  DISC_ERR_INVALID_ARG for NULL. */
disc_status disc_server_stats(disc_server* server, disc_server_report* out);
disc_status disc_server_reset_stats(disc_server* server);

/* Drains every queued request, then frees the maps, the group and the worker. */
void disc_server_destroy(disc_server* server); /* NULL-safe */

/* Copies the intermediates of the most recent frame that the map integrated
 * through disc_integrate_frame(s) (see disc_frame_report). */
disc_status disc_map_last_frame(disc_map* map, disc_frame_report* report);

/* Open-vocabulary query (Sec. IV retrieval): cosine of each query vector
 * [nq][D] (host) against every live instance embedding; per query the k best
 * ids and scores (descending score, ascending id on ties; -1 / -inf pad). */
disc_status disc_query_topk(disc_map* map, const float* queries, int32_t nq, int32_t k, int32_t* ids,
                            float* scores);

/* Instance id of the voxel containing each world point [n][3] (host), -1 if
 * the voxel is not mapped. */
disc_status disc_query_points(disc_map* map, const float* xyz, int64_t n, int32_t* ids);

/* Map export.  Voxels come sorted by key with resolved instance ids; instance
 * arrays cover ids 0..num_ids-1 (parent[i] == i marks a live instance). */
disc_status disc_map_counts(disc_map* map, int64_t* num_voxels, int32_t* num_ids);
disc_status disc_map_export_voxels(disc_map* map, uint64_t* keys, int32_t* ids, int64_t cap);
/* The association feature [assoc_dim] of every id 0..num_ids-1 (maps with a
 * second grid), into a host buffer of cap rows. */
disc_status disc_map_export_assoc(disc_map* map, float* A, int32_t cap);

disc_status disc_map_export_instances(disc_map* map, int32_t* parent, int64_t* count, float* Q,
                                      float* E, int32_t* n_obs, int32_t cap);

/* Checkpoint: a host file holding the config, the voxel table and the
 * instance table.  disc_map_load creates a new map (stream and device taken
 * from cfg_override when it is not NULL). */
disc_status disc_map_save(disc_map* map, const char* path);
disc_status disc_map_load(const char* path, const disc_map_config* cfg_override, disc_map** out_map);

/* Token statistics without device allocation.  The paper has no counterpart
 * of this entry point: it serves callers that cannot call cudaMalloc (code
 * whose device memory footprint must stay fixed after start-up, or hosts that
 * hand the library only buffers they registered themselves).  It computes the
 * same distinctiveness D_p (Eq. 1) and token/global-embedding cosine as one
 * frame of disc_integrate_frame, bit for bit, for one token grid:
 *   tokens       [P][D] device memory, disc_token_dtype;
 *   global_embed [D] device memory or NULL (then the mean token);
 *   Dp, cosg     [P] device memory, written;
 *   cuda_stream  cudaStream_t of the current device (NULL = default stream).
 * Limits: P <= 16384, D <= 4096; larger sizes return DISC_ERR_INVALID_ARG.
 * Its working set (~450 KB) is a file-scope __device__ array that every GPU
 * loading the library holds until the process exits; every call on a GPU
 * shares it, so calls whose GPU work overlaps race.  The first call on each
 * device looks up that array's device address (the current device must be
 * the one the stream and pointers belong to); make that first call before any
 * stream capture.  Returns after the results are complete; DISC_ERR_RANGE for
 * a non-finite token or |token| > 1024. */
disc_status disc_token_stats_static(const void* tokens, int32_t token_dtype, int32_t P, int32_t D,
                                    const float* global_embed, float eps, float* Dp, float* cosg,
                                    void* cuda_stream);

/* ---- Test hooks (failure paths, made without a GPU fault) -------------------
 * disc_debug_fail_alloc_after: after n more device allocations of the library
 * the next ones fail as out of memory, until called again with n < 0 (also
 * read once from the environment variable DISC_FAULT_ALLOC_AFTER).  Calls that
 * hit it return DISC_ERR_OOM and leave maps as they were.
 * disc_debug_gemm_stall: while on, the pooling GEMM on `device` issues no
 * MMA, so its bounded waits (about 1 s) run out and each frame it serves fails
 * with DISC_ERR_TIMEOUT, the map unchanged and the context usable. */
void disc_debug_fail_alloc_after(int64_t n);
disc_status disc_debug_gemm_stall(int32_t device, int32_t on);

/* ---- Launch schedule and autotuner -----------------------------------------
 * How a map's (or a group's) batches are cut into launches: the frames per
 * launch of the geometry kernels (back-projection, entries, DBSCAN), whose
 * per-frame hashes should stay in L2; the CTA counts of the four serial
 * kernels per frame of maps with the neighbourhood overlap; how many lanes
 * look one voxel up in the table together (warp-cooperative probing: each
 * round a group of probe_width lanes reads that many consecutive slots of the
 * probe sequence); how many CTAs (a thread-block cluster) carry one map's
 * frames in the association kernel; and into how many smaller batches a call
 * whose frames fit one batch is cut, so that each smaller batch's stateless
 * kernels run beside the frame chain of the one before it.  None changes any
 * result. */
typedef struct {
    int32_t geometry_chunk;  /* frames per geometry launch, 1..32 (default 8) */
    int32_t serial_ctas;     /* serial kernels' CTAs in quarters of the default count, 1..32 (default 4) */
    int32_t probe_width;     /* lanes per key of the voxel-table lookup: 1, 2, 4 or 8 (0 or 1: one lane) */
    int32_t assoc_cluster;   /* CTAs per map in the association kernel: 0 (as many as the batch's maps leave
                                SMs for, up to 8), or 1, 2, 4, 8 (capped by what the device co-schedules) */
    int32_t batch_split;     /* smaller batches per call that fits one batch: 0 (2 for one map's synchronous
                                calls of 16 frames or more, else 1: an asynchronous call's frame chain
                                already overlaps the next call), or 1, 2, 4, 8; each keeps at least 4 frames */
} disc_schedule;

typedef struct {
    disc_schedule best;      /* the schedule kept */
    double best_ms;          /* its time for the sample (minimum over the timed repetitions) */
    double default_ms;       /* the default schedule's time */
    int32_t candidates;      /* schedules timed */
} disc_tune_report;

disc_status disc_map_set_schedule(disc_map* map, const disc_schedule* schedule);
disc_status disc_group_set_schedule(disc_group* group, const disc_schedule* schedule);

/* Autotuner: times each candidate schedule (geometry_chunk in {2, 4, 8} x
 * probe_width in {1, 2, 4} x assoc_cluster automatic or half of it, then the
 * fastest of these with batch_split at each of {1, 2, 4} other than the
 * automatic one) on the sample frames, integrated into fresh maps
 * with the given maps' configurations (created and destroyed here; the given
 * maps are not changed), two untimed passes then `reps` timed ones, and keeps
 * the fastest for the map or group.  report may be NULL. */
disc_status disc_map_autotune(disc_map* map, const disc_frame* frames, int32_t n, int32_t reps,
                              disc_tune_report* report);
disc_status disc_group_autotune(disc_group* group, disc_map* const* maps, int32_t n_maps,
                                const disc_frame* const* frames, const int32_t* counts, int32_t reps,
                                disc_tune_report* report);

/* Fig. 2: the distinctiveness-weighted cosine heatmap of a query vector over a
 * frame's token grid, heat_p = D_p * cos(f_p, q): D_p of Eq. 1 and the exact
 * cosine, their product rounded once to fp32 (the heatmap the paper shows for
 * a text query).  Arguments and the shared allocation-free working set as in
 * disc_token_stats_static, with q [D] (device memory) in the place of the
 * global embedding and heat [P] (device memory) written. */
disc_status disc_query_heatmap(const void* tokens, int32_t token_dtype, int32_t P, int32_t D, const float* query,
                               float eps, float* heat, void* cuda_stream);

/* End of the trajectory (Sec. III-B, last paragraph): merge the remaining
 * orphaned candidates, then drop noisy instances below a voxel count.  The
 * paper fixes no criteria; this call takes:
 *   contact(a, b) = voxels of instance a or b with a face neighbour (one of
 *                   the 6 voxels sharing a face) in the other instance;
 *   a and b merge when contact * contact_den >= contact_num * min(|a|, |b|)
 *   and the cosine of their stored embeddings (exact sums, as in the
 *   association gate) >= tau_cos, on the state as it stands at the call;
 *   merges are transitive; a component keeps its smallest id, the Q and
 *   embedding of its member with the highest Q (ties: smallest id), and the
 *   sums of its voxel and observation counts;
 *   then live instances with 0 < voxel count < min_voxels are dropped: their
 *   voxels report instance -1, their count, observations and Q become 0, and
 *   queries skip them.
 * The map is final afterwards: integration calls (and group calls naming it)
 * return DISC_ERR_INVALID_ARG; exports, queries and checkpoints still work
 * (a checkpoint of a final map reloads final).  Same result bit for bit as
 * the plain CPU statement of these steps. */
typedef struct {
    int32_t min_voxels;
    int32_t contact_num, contact_den;
    float tau_cos;
} disc_finalize_config;

typedef struct {
    int32_t contact_pairs;  /* instance pairs in contact */
    int32_t merged;         /* instances merged into another */
    int32_t removed;        /* instances dropped by the voxel count */
    int64_t removed_voxels; /* their voxels */
} disc_finalize_report;

disc_status disc_map_finalize(disc_map* map, const disc_finalize_config* cfg, disc_finalize_report* report);

/* Voxel key packing: three signed 18-bit voxel coordinates (x, y, z), each
 * biased by 2^17, in bits 36..53, 18..35 and 0..17. */
uint64_t disc_pack_key(int32_t kx, int32_t ky, int32_t kz);

/* The map's resolved configuration (capacities after rounding/growth). */
disc_status disc_map_get_config(disc_map* map, disc_map_config* out);

/* Kernels this map has enqueued since creation (every kernel of every phase). */
int64_t disc_map_kernel_launches(disc_map* map);

/* Per-phase timing with CUDA events recorded on the map's stream around each
 * phase of every frame (off by default; enabling resets the totals).  Phases:
 * 0 clear, 1 token_stats (Eq. 1), 2 coverage, 3 weights, 4 pool_exact,
 * 5 pool_gemm -- one interval per batch each --, 6 dbscan, 7 backproject and
 * 8 entries (S_angle, |V_m|; then Q) -- one interval per chunk of frames --,
 * 13 lookup (every entry of the batch in the map as the batch starts),
 * 14 associate (each map's frames in order: overlap pairs, gates, union,
 * fusion, voxel counts), 15 commit (the batch's new voxels) -- one interval
 * per batch each --, and, for maps with the neighbourhood overlap, 9 overlap,
 * 10 score, 11 union, 12 apply -- one interval per frame step each (the
 * entries phase then also looks the voxels up).  disc_phase_name(i) names
 * phase i.  With timing on, each batch is captured with event-record nodes and
 * launched once as a graph.  ms/launches/calls: [n] accumulated device time,
 * kernels launched and timed intervals per phase (any may be NULL).  Kernel
 * launches count only the map's own calls (not group calls). */
disc_status disc_map_set_phase_timing(disc_map* map, int32_t enable);
disc_status disc_map_phase_times(disc_map* map, double* ms, int64_t* launches, int64_t* calls, int32_t n);
const char* disc_phase_name(int32_t phase);

/* Device memory held by the map, bytes. */
int64_t disc_map_device_bytes(disc_map* map);

/* Frees the map; its unfinished asynchronous calls (and those of a group
 * call that holds it) are finished first, writing their results. */
void disc_map_destroy(disc_map* map); /* NULL-safe */
const char* disc_status_str(int32_t status);

#ifdef __cplusplus
}
#endif
#endif
