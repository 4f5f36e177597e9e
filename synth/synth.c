/*
 * Seeded synthetic RGB-D-like frames for the DISC integration step.
 *
 * This module is INPUT PLUMBING shared by the CUDA path, the oracle, the tests
 * and the benchmark.  It holds none of the integration method's arithmetic: it
 * ray-casts axis-aligned boxes and ellipsoids inside a box-shaped room, picks
 * the largest visible objects as instance masks, and draws patch tokens as a
 * per-object mean plus noise.  Everything is a pure function of (seed, frame,
 * pixel/patch, dimension) through a counter-based generator, so frames can be
 * produced in any order and in parallel.
 *
 * Conventions (OpenCV pinhole): camera x right, y down, z forward; the pose is
 * camera->world, row-major 4x4 doubles.  Depth is the camera-frame z of the
 * first hit.  Pixel (u, v) is sampled at its centre (u + 0.5, v + 0.5).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t kind;   /* 0 = axis-aligned box (h = half extents), 1 = ellipsoid (h = radii) */
    int32_t id;     /* object id, >= 1 */
    double c[3];
    double h[3];
} synth_prim;

typedef struct {
    double room_lo[3], room_hi[3];   /* room interior; the six faces carry ids */
    int32_t face_id[6];              /* -x, +x, -y, +y, -z (floor), +z (ceiling) */
    double tile;                     /* > 0: faces are cut into tile x tile m panels, each its own id */
    int32_t n_prims;
    const synth_prim* prims;
    int32_t width, height;
    double fx, fy, cx, cy;
    double depth_noise;              /* relative sigma of multiplicative depth noise */
    int32_t patch_h, patch_w, dim;   /* token grid and embedding dimension */
    double token_noise;              /* sigma of the per-patch token noise */
    int32_t max_masks;
    int32_t max_id;                  /* ids are in [0, max_id] */
    uint64_t seed;
    /* optional 2D uniform grid over (x, y) for scenes with many primitives:
     * cell (i, j) lists the primitives whose (x, y) extent overlaps it,
     * cell_items[cell_start[c] .. cell_start[c + 1]) with c = j * grid_nx + i */
    int32_t grid_nx, grid_ny;        /* 0: test every primitive */
    double grid_x0, grid_y0, grid_cell;
    const int32_t* cell_start;
    const int32_t* cell_items;
} synth_scene;

/* ---- counter-based generator (splitmix64 finaliser as a hash) ---------- */
static uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t hash4(uint64_t seed, uint64_t a, uint64_t b, uint64_t c)
{
    return mix64(mix64(mix64(mix64(seed) ^ a) ^ b) ^ c);
}

/* Approximately standard normal: centred sum of four uniforms, unit variance.
 * Only additions and multiplications, so it is identical on every host. */
static double normal4(uint64_t seed, uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t h = hash4(seed, a, b, c);
    double s = 0.0;
    for (int i = 0; i < 4; i++) {
        h = mix64(h + (uint64_t)i);
        s += (double)(h >> 11) * 0x1p-53;
    }
    return (s - 2.0) * 1.7320508075688772; /* sqrt(12/4) */
}

enum { STREAM_MEAN = 1, STREAM_TOKEN = 2, STREAM_DEPTH = 3, STREAM_AMEAN = 4, STREAM_ATOKEN = 5 };

/* ---- ray casting --------------------------------------------------------- */
static int hit_box(const synth_prim* p, const double o[3], const double d[3], double* t_out)
{
    double t0 = -INFINITY, t1 = INFINITY;
    for (int a = 0; a < 3; a++) {
        double lo = p->c[a] - p->h[a], hi = p->c[a] + p->h[a];
        if (d[a] == 0.0) {
            if (o[a] < lo || o[a] > hi) return 0;
            continue;
        }
        double inv = 1.0 / d[a];
        double ta = (lo - o[a]) * inv, tb = (hi - o[a]) * inv;
        if (ta > tb) { double s = ta; ta = tb; tb = s; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return 0;
    }
    if (t0 <= 1e-9) return 0; /* camera inside or behind: not visible */
    *t_out = t0;
    return 1;
}

static int hit_ellipsoid(const synth_prim* p, const double o[3], const double d[3], double* t_out)
{
    double oo[3], dd[3];
    for (int a = 0; a < 3; a++) {
        oo[a] = (o[a] - p->c[a]) / p->h[a];
        dd[a] = d[a] / p->h[a];
    }
    double A = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
    double B = oo[0] * dd[0] + oo[1] * dd[1] + oo[2] * dd[2];
    double C = oo[0] * oo[0] + oo[1] * oo[1] + oo[2] * oo[2] - 1.0;
    double disc = B * B - A * C;
    if (disc < 0.0 || C <= 0.0) return 0;
    double t = (-B - sqrt(disc)) / A;
    if (t <= 1e-9) return 0;
    *t_out = t;
    return 1;
}

/* Exit of the room box from inside: returns t and the face index. */
static double room_exit(const synth_scene* s, const double o[3], const double d[3], int* face)
{
    double best = INFINITY;
    int bf = -1;
    for (int a = 0; a < 3; a++) {
        if (d[a] < 0.0) {
            double t = (s->room_lo[a] - o[a]) / d[a];
            if (t < best) { best = t; bf = 2 * a; }
        } else if (d[a] > 0.0) {
            double t = (s->room_hi[a] - o[a]) / d[a];
            if (t < best) { best = t; bf = 2 * a + 1; }
        }
    }
    *face = bf;
    return best;
}

/* Id of the room panel hit at o + t d on face `face`: the face's base id plus
 * the panel index along the face's two in-plane axes (lower axis first). */
static int32_t face_tile_id(const synth_scene* s, const double o[3], const double d[3], double t, int face)
{
    if (s->tile <= 0.0) return s->face_id[face];
    int a = face / 2, b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
    int n1 = (int)ceil((s->room_hi[b1] - s->room_lo[b1]) / s->tile);
    int i = (int)floor((o[b0] + t * d[b0] - s->room_lo[b0]) / s->tile);
    int j = (int)floor((o[b1] + t * d[b1] - s->room_lo[b1]) / s->tile);
    int n0 = (int)ceil((s->room_hi[b0] - s->room_lo[b0]) / s->tile);
    if (i < 0) i = 0;
    if (i >= n0) i = n0 - 1;
    if (j < 0) j = 0;
    if (j >= n1) j = n1 - 1;
    return s->face_id[face] + i * n1 + j;
}

/* Render one frame: depth (camera z, metres; 0 where nothing is hit) and the
 * object id seen at each pixel. */
static void render_ids(const synth_scene* s, const double* T, uint64_t frame,
                       float* depth, int32_t* ids)
{
    const int W = s->width, H = s->height;
    double o[3] = {T[3], T[7], T[11]};
    for (int v = 0; v < H; v++) {
        for (int u = 0; u < W; u++) {
            double dc[3] = {((double)u + 0.5 - s->cx) / s->fx, ((double)v + 0.5 - s->cy) / s->fy, 1.0};
            double d[3];
            for (int r = 0; r < 3; r++) d[r] = T[4 * r + 0] * dc[0] + T[4 * r + 1] * dc[1] + T[4 * r + 2] * dc[2];
            int face;
            double tbest = room_exit(s, o, d, &face);
            int32_t id = face >= 0 ? face_tile_id(s, o, d, tbest, face) : 0;
            if (s->grid_nx > 0) {
                /* walk the (x, y) cells the ray crosses, nearest first; stop
                 * once the nearest hit so far lies within the current cell */
                const double cs = s->grid_cell;
                int ix = (int)floor((o[0] - s->grid_x0) / cs), iy = (int)floor((o[1] - s->grid_y0) / cs);
                if (ix < 0) ix = 0;
                if (ix >= s->grid_nx) ix = s->grid_nx - 1;
                if (iy < 0) iy = 0;
                if (iy >= s->grid_ny) iy = s->grid_ny - 1;
                const int sx = d[0] > 0.0 ? 1 : -1, sy = d[1] > 0.0 ? 1 : -1;
                double tmx = d[0] != 0.0 ? (s->grid_x0 + (ix + (d[0] > 0.0)) * cs - o[0]) / d[0] : INFINITY;
                double tmy = d[1] != 0.0 ? (s->grid_y0 + (iy + (d[1] > 0.0)) * cs - o[1]) / d[1] : INFINITY;
                const double tdx = d[0] != 0.0 ? cs / fabs(d[0]) : INFINITY;
                const double tdy = d[1] != 0.0 ? cs / fabs(d[1]) : INFINITY;
                while (1) {
                    const int c = iy * s->grid_nx + ix;
                    for (int k = s->cell_start[c]; k < s->cell_start[c + 1]; k++) {
                        double t;
                        const synth_prim* p = &s->prims[s->cell_items[k]];
                        int hit = p->kind == 0 ? hit_box(p, o, d, &t) : hit_ellipsoid(p, o, d, &t);
                        if (hit && (t < tbest || (t == tbest && p->id < id))) { tbest = t; id = p->id; }
                    }
                    const double texit = tmx < tmy ? tmx : tmy;
                    if (tbest <= texit || !isfinite(texit)) break;
                    if (tmx < tmy) { ix += sx; tmx += tdx; } else { iy += sy; tmy += tdy; }
                    if (ix < 0 || ix >= s->grid_nx || iy < 0 || iy >= s->grid_ny) break;
                }
            } else {
                for (int i = 0; i < s->n_prims; i++) {
                    double t;
                    const synth_prim* p = &s->prims[i];
                    int hit = p->kind == 0 ? hit_box(p, o, d, &t) : hit_ellipsoid(p, o, d, &t);
                    if (hit && t < tbest) { tbest = t; id = p->id; }
                }
            }
            size_t idx = (size_t)v * W + u;
            if (!isfinite(tbest) || id == 0) {
                depth[idx] = 0.0f;
                ids[idx] = 0;
            } else {
                /* dc has z = 1, so the ray parameter is the camera-frame depth. */
                double z = tbest;
                if (s->depth_noise > 0.0)
                    z *= 1.0 + s->depth_noise * normal4(s->seed, STREAM_DEPTH, frame, idx);
                depth[idx] = (float)z;
                ids[idx] = id;
            }
        }
    }
}

/* Choose the <= max_masks largest visible ids (pixel count descending, id
 * ascending on ties) and write the label image (1-based mask index, 0 = none).
 * Returns the number of masks; mask_ids[k] is the object id of mask k + 1. */
static int32_t make_masks(const synth_scene* s, const int32_t* ids, uint16_t* labels,
                          int32_t* mask_ids, int64_t* counts /* scratch [max_id+1] */)
{
    const size_t n = (size_t)s->width * s->height;
    memset(counts, 0, sizeof(int64_t) * (size_t)(s->max_id + 1));
    for (size_t i = 0; i < n; i++)
        if (ids[i] > 0 && ids[i] <= s->max_id) counts[ids[i]]++;
    int32_t nm = 0;
    for (int32_t k = 0; k < s->max_masks; k++) {
        int32_t best = -1;
        for (int32_t id = 1; id <= s->max_id; id++) {
            if (counts[id] <= 0) continue;
            if (best < 0 || counts[id] > counts[best]) best = id;
        }
        if (best < 0) break;
        mask_ids[nm++] = best;
        counts[best] = -(int64_t)nm; /* taken; remembers its mask index */
    }
    for (int32_t k = nm; k < s->max_masks; k++) mask_ids[k] = 0;
    for (size_t i = 0; i < n; i++) {
        int32_t id = ids[i];
        uint16_t lab = 0;
        if (id > 0 && id <= s->max_id && counts[id] < 0) lab = (uint16_t)(-counts[id]);
        labels[i] = lab;
    }
    return nm;
}

/* Patch tokens of a Ph x Pw x Dd grid: the object at the patch-centre pixel
 * picks the mean vector (id 0 = background mean) of stream sm, plus
 * independent noise per (frame, patch, dim) of stream st. */
static void grid_tokens(const synth_scene* s, int Ph, int Pw, int Dd, int sm, int st, uint64_t frame,
                        const int32_t* ids, float* tokens)
{
    for (int i = 0; i < Ph; i++) {
        for (int j = 0; j < Pw; j++) {
            int vc = ((2 * i + 1) * s->height) / (2 * Ph);
            int uc = ((2 * j + 1) * s->width) / (2 * Pw);
            int32_t id = ids[(size_t)vc * s->width + uc];
            size_t p = (size_t)i * Pw + j;
            float* out = tokens + p * Dd;
            for (int d = 0; d < Dd; d++) {
                double mu = normal4(s->seed, sm, (uint64_t)id, (uint64_t)d);
                double nz = normal4(s->seed, st, frame * 1000003ull + p, (uint64_t)d);
                out[d] = (float)(mu + s->token_noise * nz);
            }
        }
    }
}

static void make_tokens(const synth_scene* s, uint64_t frame, const int32_t* ids, float* tokens)
{
    grid_tokens(s, s->patch_h, s->patch_w, s->dim, STREAM_MEAN, STREAM_TOKEN, frame, ids, tokens);
}

/*
 * Render n frames.  poses: [n][16] camera->world row-major; frame_ids: [n]
 * (the counter used for the noise streams).  Outputs (caller-owned):
 *   depth  [n][H][W] float,  labels [n][H][W] uint16,  tokens [n][Ph*Pw][dim] float,
 *   mask_ids [n][max_masks] int32,  num_masks [n] int32,  id_image [n][H][W] int32 (nullable).
 */
int synth_render(const synth_scene* s, int32_t n, const double* poses, const int64_t* frame_ids,
                 float* depth, uint16_t* labels, float* tokens, int32_t* mask_ids,
                 int32_t* num_masks, int32_t* id_image)
{
    if (!s || n < 0 || s->width <= 0 || s->height <= 0 || s->max_id < 1) return -1;
    const size_t npx = (size_t)s->width * s->height;
    const size_t ntok = (size_t)s->patch_h * s->patch_w * s->dim;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t f = 0; f < n; f++) {
        int32_t* ids = (int32_t*)malloc(sizeof(int32_t) * npx);
        int64_t* counts = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s->max_id + 1));
        if (!ids || !counts) {
            err = -2;
        } else {
            uint64_t fid = (uint64_t)frame_ids[f];
            render_ids(s, poses + 16 * (size_t)f, fid, depth + npx * f, ids);
            num_masks[f] = make_masks(s, ids, labels + npx * f, mask_ids + (size_t)s->max_masks * f, counts);
            make_tokens(s, fid, ids, tokens + ntok * f);
            if (id_image) memcpy(id_image + npx * f, ids, sizeof(int32_t) * npx);
        }
        free(ids);
        free(counts);
    }
    return err;
}

/* A second token grid (the association encoder's) of n rendered frames from
 * their id images [n][H][W]: per-object means and noise from streams of
 * their own.  out: [n][Ph*Pw][Dd]. */
int synth_assoc_tokens(const synth_scene* s, int32_t n, const int64_t* frame_ids, const int32_t* id_image,
                       int32_t Ph, int32_t Pw, int32_t Dd, float* out)
{
    if (!s || n < 0 || Ph <= 0 || Pw <= 0 || Dd <= 0) return -1;
    const size_t npx = (size_t)s->width * s->height;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t f = 0; f < n; f++)
        grid_tokens(s, Ph, Pw, Dd, STREAM_AMEAN, STREAM_ATOKEN, (uint64_t)frame_ids[f], id_image + npx * f,
                    out + (size_t)Ph * Pw * Dd * f);
    return 0;
}

/* Object mean vector (the noiseless token of an object), for query tests. */
void synth_object_mean(const synth_scene* s, int32_t id, float* out)
{
    for (int d = 0; d < s->dim; d++)
        out[d] = (float)normal4(s->seed, STREAM_MEAN, (uint64_t)id, (uint64_t)d);
}
