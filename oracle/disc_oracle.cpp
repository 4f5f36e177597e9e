// DISC integration-step ORACLE -- test infrastructure only (see disc_oracle.h).
//
// One frame is integrated by walking the paper's steps in order:
//   Sec. III-C, Eq. 1   distinctiveness map D over the frame's patch tokens
//   Sec. III-C          D-weighted pooling of the tokens inside each mask
//   Sec. III-C, Eq. 2-3 view quality Q = S_size * S_angle * S_sem * S_dist
//   Sec. III-A          masked depth -> 3D points -> voxels (per segment)
//   Sec. III-B          exact voxel overlap with the map, cosine gate, merges
//   Sec. III-C          fusion: keep the observation with the higher Q
// Built with -O2 -ffp-contract=off so no multiply-add is contracted.
#include "disc_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <array>
#include <functional>
#include <map>
#include <tuple>
#include <set>
#include <unordered_map>
#include <vector>

namespace {

// Exact fixed-point accumulation: every term is scaled by 2^S (exact for a
// float) and rounded to the nearest integer (ties to even), then summed in
// int64.  Integer sums are associative, so the value is order-independent.
int64_t fix(float x, int S) { return (int64_t)llrintf(ldexpf(x, S)); }
double unfix(int64_t n, int S) { return ldexp((double)n, -S); }

constexpr int S_TOK = 32;   // sums of tokens (mean token)
constexpr int S_SQ = 28;    // sums over the embedding dimension (norms, dots)
constexpr int S_NRM = 28;   // sum of residual norms
constexpr int S_A = 24;     // sums of coverage x distinctiveness
constexpr int S_SEM = 32;   // sums of coverage x ReLU(cosine)
constexpr int S_EMB = 40;   // pooled embedding sums
constexpr int S_VEC = 32;   // voxel normal sums and S_angle sums

constexpr float TOKEN_LIMIT = 1024.0f;
constexpr int KEY_BITS = 18;
constexpr int32_t KEY_BIAS = 1 << (KEY_BITS - 1);

// Cosine of two vectors with exact dot/norm sums (Sec. III-B association gate,
// Sec. III-C S_sem).  Zero when either vector is zero.
float cosine_exact(const float* a, const float* b, int D)
{
    int64_t dot = 0, na = 0, nb = 0;
    for (int d = 0; d < D; d++) {
        dot += fix(a[d] * b[d], S_SQ);
        na += fix(a[d] * a[d], S_SQ);
        nb += fix(b[d] * b[d], S_SQ);
    }
    if (na == 0 || nb == 0) return 0.0f;
    return (float)(unfix(dot, S_SQ) / (std::sqrt(unfix(na, S_SQ)) * std::sqrt(unfix(nb, S_SQ))));
}

// Voxel of a world point: floor(p * (1/s)) per axis, the reciprocal rounded
// once to fp32.
bool key_of(float px, float py, float pz, float s, uint64_t* key)
{
    const float is = 1.0f / s;
    float k[3] = {std::floor(px * is), std::floor(py * is), std::floor(pz * is)};
    uint64_t out = 0;
    for (int a = 0; a < 3; a++) {
        if (!(k[a] >= -(float)KEY_BIAS && k[a] <= (float)(KEY_BIAS - 1))) return false;
        out = (out << KEY_BITS) | (uint64_t)((int32_t)k[a] + KEY_BIAS);
    }
    *key = out;
    return true;
}

void unpack(uint64_t key, int32_t* k)
{
    const uint64_t mask = (1ull << KEY_BITS) - 1;
    k[0] = (int32_t)((key >> (2 * KEY_BITS)) & mask) - KEY_BIAS;
    k[1] = (int32_t)((key >> KEY_BITS) & mask) - KEY_BIAS;
    k[2] = (int32_t)(key & mask) - KEY_BIAS;
}

struct Pose {
    float R[3][3];
    float t[3];
};

// Pinhole back-projection of pixel (u, v) at depth z, then camera -> world
// (Sec. III-A: the masked depth becomes a world point cloud).  Pixel centres at +0.5;
// the focal lengths enter as reciprocals rounded once to fp32.
void world_point(const Pose& T, float fx, float fy, float cx, float cy, int u, int v, float z,
                 float p[3])
{
    const float ifx = 1.0f / fx, ify = 1.0f / fy;
    float xc = ((((float)u + 0.5f) - cx) * z) * ifx;
    float yc = ((((float)v + 0.5f) - cy) * z) * ify;
    float zc = z;
    for (int r = 0; r < 3; r++) p[r] = ((T.R[r][0] * xc + T.R[r][1] * yc) + T.R[r][2] * zc) + T.t[r];
}

}  // namespace

extern "C" {

struct oracle_map {
    oracle_config cfg;
    std::unordered_map<uint64_t, int32_t> vox;  // voxel key -> label at insertion
    std::vector<int32_t> parent;                // flat: parent[i] is always a root
    std::vector<int64_t> count;                 // voxels per root
    std::vector<float> Q;
    std::vector<std::vector<float>> E;
    std::vector<std::vector<float>> A;          // association features (second token grid)
    std::vector<int32_t> n_obs;
    bool final_ = false;  // finalised: no more frames
};

oracle_map* oracle_map_create(const oracle_config* cfg)
{
    if (!cfg || cfg->embed_dim <= 0 || cfg->patch_h <= 0 || cfg->patch_w <= 0 || !(cfg->voxel_size > 0.0f))
        return nullptr;
    if (cfg->assoc_dim < 0 || cfg->assoc_dim > 4096 ||
        (cfg->assoc_dim > 0 && (cfg->assoc_patch_h <= 0 || cfg->assoc_patch_w <= 0 ||
                                cfg->assoc_patch_h * cfg->assoc_patch_w > 16384)))
        return nullptr;
    oracle_map* m = new oracle_map();
    m->cfg = *cfg;
    return m;
}

void oracle_map_destroy(oracle_map* map) { delete map; }

// ---- Eq. 1: distinctiveness map ---------------------------------------------
// fbar = (1/P) sum_p f_p;  n_p = ||f_p - fbar||;  D_p = n_p / ((1/P) sum n + eps).
// cosg_p = cos(f_p, g) with g the global embedding (or fbar when g is NULL).
int oracle_token_stats(const float* F, int32_t P, int32_t D, const float* g, float eps,
                       float* fbar, float* n, float* Dp, float* cosg)
{
    for (int64_t i = 0; i < (int64_t)P * D; i++)
        if (!(std::fabs(F[i]) <= TOKEN_LIMIT)) return ORACLE_ERR_RANGE;
    if (g)
        for (int d = 0; d < D; d++)
            if (!(std::fabs(g[d]) <= TOKEN_LIMIT)) return ORACLE_ERR_RANGE;
    std::vector<float> mean(D);
    for (int d = 0; d < D; d++) {
        int64_t s = 0;
        for (int p = 0; p < P; p++) s += fix(F[(int64_t)p * D + d], S_TOK);
        mean[d] = (float)(unfix(s, S_TOK) / (double)P);
    }
    std::vector<float> norm(P);
    int64_t nsum = 0;
    for (int p = 0; p < P; p++) {
        int64_t ss = 0;
        for (int d = 0; d < D; d++) {
            float r = F[(int64_t)p * D + d] - mean[d];
            ss += fix(r * r, S_SQ);
        }
        norm[p] = (float)std::sqrt(unfix(ss, S_SQ));
        nsum += fix(norm[p], S_NRM);
    }
    double nbar = unfix(nsum, S_NRM) / (double)P;
    const float* gv = g ? g : mean.data();
    for (int p = 0; p < P; p++) {
        if (Dp) Dp[p] = (float)((double)norm[p] / (nbar + (double)eps));
        if (n) n[p] = norm[p];
        if (cosg) cosg[p] = cosine_exact(F + (int64_t)p * D, gv, D);
    }
    if (fbar) std::memcpy(fbar, mean.data(), sizeof(float) * D);
    return ORACLE_OK;
}

// ---- mask -> patch coverage ---------------------------------------------------
// cov[m][p] = #pixels of mask m whose patch is p, patch(u, v) = (v*Ph/H, u*Pw/W).
void oracle_mask_coverage(const uint16_t* labels, int32_t H, int32_t W, int32_t Ph, int32_t Pw,
                          int32_t M, int32_t* cov, int32_t* npix)
{
    const int P = Ph * Pw;
    std::memset(cov, 0, sizeof(int32_t) * (size_t)M * P);
    std::memset(npix, 0, sizeof(int32_t) * (size_t)M);
    for (int v = 0; v < H; v++)
        for (int u = 0; u < W; u++) {
            int m = labels[(size_t)v * W + u];
            if (m < 1 || m > M) continue;
            int p = (v * Ph / H) * Pw + (u * Pw / W);
            cov[(size_t)(m - 1) * P + p] += 1;
            npix[m - 1] += 1;
        }
}

int oracle_point_key(float x, float y, float z, float voxel_size, uint64_t* key)
{
    return key_of(x, y, z, voxel_size, key) ? 1 : 0;
}

void oracle_unpack_key(uint64_t key, int32_t* kx, int32_t* ky, int32_t* kz)
{
    int32_t k[3];
    unpack(key, k);
    *kx = k[0];
    *ky = k[1];
    *kz = k[2];
}

float oracle_cosine(const float* a, const float* b, int32_t D) { return cosine_exact(a, b, D); }

// ---- Sec. III-A: DBSCAN noise per segment ----------------------------------------
// Neighbours are looked for in the 27 grid cells around a point; the cells are
// 1.001 eps wide, so every point within eps lies in one of them (the grid only
// narrows the search, the decision is the exact squared-distance test).
void oracle_dbscan_noise(const float* pts, const int32_t* seg, int64_t n, float eps, int32_t min_pts,
                         uint8_t* noise)
{
    const float eps2 = eps * eps;
    const float inv_c = 1.0f / (eps * 1.001f);
    std::map<std::tuple<int32_t, int32_t, int32_t, int32_t>, std::vector<int64_t>> cells;
    std::vector<std::array<int32_t, 3>> cell_of(n);
    for (int64_t i = 0; i < n; i++) {
        for (int a = 0; a < 3; a++) cell_of[i][a] = (int32_t)std::floor(pts[3 * i + a] * inv_c);
        cells[{seg[i], cell_of[i][0], cell_of[i][1], cell_of[i][2]}].push_back(i);
    }
    auto within = [&](int64_t i, int64_t j) {
        const float dx = pts[3 * i] - pts[3 * j], dy = pts[3 * i + 1] - pts[3 * j + 1], dz = pts[3 * i + 2] - pts[3 * j + 2];
        return (dx * dx + dy * dy) + dz * dz <= eps2;
    };
    auto for_neighbours = [&](int64_t i, const std::function<bool(int64_t)>& f) {
        for (int dx = -1; dx <= 1; dx++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dz = -1; dz <= 1; dz++) {
                    auto it = cells.find({seg[i], cell_of[i][0] + dx, cell_of[i][1] + dy, cell_of[i][2] + dz});
                    if (it == cells.end()) continue;
                    for (int64_t j : it->second)
                        if (within(i, j) && !f(j)) return;
                }
    };
    std::vector<char> core(n, 0);
    for (int64_t i = 0; i < n; i++) {
        int64_t cnt = 0;
        for_neighbours(i, [&](int64_t) { return ++cnt < min_pts; });
        core[i] = cnt >= min_pts;
    }
    for (int64_t i = 0; i < n; i++) {
        bool keep = core[i];
        if (!keep)
            for_neighbours(i, [&](int64_t j) {
                keep = core[j] != 0;
                return !keep;
            });
        noise[i] = keep ? 0 : 1;
    }
}

// ---- one frame ----------------------------------------------------------------
int oracle_integrate_frame(oracle_map* map, const oracle_frame* fr, oracle_report* rep)
{
    if (!map || !fr || map->final_) return ORACLE_ERR_INVALID_ARG;
    const oracle_config& cfg = map->cfg;
    const int H = fr->height, Wd = fr->width, D = cfg.embed_dim;
    const int Ph = cfg.patch_h, Pw = cfg.patch_w, P = Ph * Pw;
    const int M = fr->num_masks;
    if (H <= 0 || Wd <= 0 || (int64_t)H * Wd > (1 << 24) || M < 0 || M > 1023 || P > 16384 ||
        D > 4096 || !fr->depth || !fr->labels || !fr->tokens)
        return ORACLE_ERR_INVALID_ARG;
    // a camera model and pose of finite numbers (the pose as it is rounded to fp32)
    if (!std::isfinite(fr->fx) || !std::isfinite(fr->fy) || !std::isfinite(fr->cx) || !std::isfinite(fr->cy) ||
        fr->fx == 0.0f || fr->fy == 0.0f)
        return ORACLE_ERR_INVALID_ARG;
    for (int i = 0; i < 12; i++)
        if (!std::isfinite((float)fr->T_world_cam[i])) return ORACLE_ERR_INVALID_ARG;
    const float s = cfg.voxel_size;
    const int Da = cfg.assoc_dim, Pa = cfg.assoc_patch_h * cfg.assoc_patch_w;
    if (Da > 0) {
        if (!fr->assoc_tokens) return ORACLE_ERR_INVALID_ARG;
        for (int64_t i = 0; i < (int64_t)Pa * Da; i++)
            if (!(std::fabs(fr->assoc_tokens[i]) <= TOKEN_LIMIT)) return ORACLE_ERR_RANGE;
    }

    // Pose rounded once to fp32.
    Pose T;
    for (int r = 0; r < 3; r++) {
        for (int c = 0; c < 3; c++) T.R[r][c] = (float)fr->T_world_cam[4 * r + c];
        T.t[r] = (float)fr->T_world_cam[4 * r + 3];
    }

    // (a1) Eq. 1.
    std::vector<float> fbar(D), Dp(P), cosg(P), nrm(P);
    int st = oracle_token_stats(fr->tokens, P, D, fr->global_embed, cfg.eps, fbar.data(), nrm.data(),
                                Dp.data(), cosg.data());
    if (st != ORACLE_OK) return st;

    // (a2) coverage.
    std::vector<int32_t> cov((size_t)std::max(M, 1) * P), npix(std::max(M, 1));
    oracle_mask_coverage(fr->labels, H, Wd, Ph, Pw, M, cov.data(), npix.data());
    const int min_px = std::max(1, cfg.min_mask_pixels);
    std::vector<char> mask_ok(M);
    for (int m = 0; m < M; m++) mask_ok[m] = npix[m] >= min_px;

    // (a3, a4) weights, pooled embeddings and the image-based quality terms.
    std::vector<float> Wt((size_t)M * P, 0.0f), Em((size_t)M * D, 0.0f);
    std::vector<float> S_size(M, 0.0f), S_sem(M, 0.0f), S_dist(M, 0.0f), S_ang(M, 0.0f), Qm(M, 0.0f);
    for (int m = 0; m < M; m++) {
        if (!mask_ok[m]) continue;
        const int32_t* c = &cov[(size_t)m * P];
        std::vector<float> a(P);
        int64_t A = 0, sem = 0;
        for (int p = 0; p < P; p++) {
            a[p] = (float)c[p] * Dp[p];
            A += fix(a[p], S_A);
            float rc = cosg[p] > 0.0f ? cosg[p] : 0.0f;  // ReLU
            sem += fix((float)c[p] * rc, S_SEM);
        }
        float* w = &Wt[(size_t)m * P];
        if (A > 0) {
            float Af = (float)unfix(A, S_A);
            for (int p = 0; p < P; p++) w[p] = a[p] / Af;
        } else {  // all distinctiveness zero: plain coverage mean
            for (int p = 0; p < P; p++) w[p] = (float)c[p] / (float)npix[m];
        }
        for (int d = 0; d < D; d++) {
            int64_t acc = 0;
            for (int p = 0; p < P; p++) acc += fix(w[p] * fr->tokens[(int64_t)p * D + d], S_EMB);
            Em[(size_t)m * D + d] = (float)unfix(acc, S_EMB);
        }
        float Dbar = (float)(unfix(A, S_A) / (double)npix[m]);
        S_dist[m] = 0.5f + 0.5f * Dbar;
        float sm = (float)(unfix(sem, S_SEM) / (double)npix[m]);
        S_sem[m] = std::min(std::max(sm, 0.0f), 1.0f);
        S_size[m] = std::min((cfg.lambda_size * (float)npix[m]) / (float)(H * Wd), 1.0f);
    }

    // (a3') with a second token grid: each mask's association feature, the
    // pixel-level mean of that grid's tokens over the mask
    std::vector<float> Am((size_t)M * std::max(Da, 1), 0.0f);
    if (Da > 0) {
        const int Pha = cfg.assoc_patch_h, Pwa = cfg.assoc_patch_w;
        std::vector<int32_t> cova((size_t)std::max(M, 1) * Pa), npa(std::max(M, 1));
        oracle_mask_coverage(fr->labels, H, Wd, Pha, Pwa, M, cova.data(), npa.data());
        for (int m = 0; m < M; m++) {
            if (!mask_ok[m]) continue;
            for (int d = 0; d < Da; d++) {
                int64_t acc = 0;
                for (int p = 0; p < Pa; p++) {
                    const float w = (float)cova[(size_t)m * Pa + p] / (float)npix[m];
                    acc += fix(w * fr->assoc_tokens[(int64_t)p * Da + d], S_EMB);
                }
                Am[(size_t)m * Da + d] = (float)unfix(acc, S_EMB);
            }
        }
    }

    // (a5') Sec. III-A: each segment's points (pixels of an active mask with
    // valid depth and an in-range voxel) filtered by DBSCAN; noise pixels
    // count as invalid depth from here on.
    std::vector<uint8_t> noise((size_t)H * Wd, 0);
    int denoised = 0;
    if (cfg.dbscan_eps > 0.0f) {
        std::vector<float> pts;
        std::vector<int32_t> sg;
        std::vector<size_t> at;
        for (int v = 0; v < H; v++)
            for (int u = 0; u < Wd; u++) {
                const size_t i = (size_t)v * Wd + u;
                const int lab = fr->labels[i];
                if (lab < 1 || lab > M || !mask_ok[lab - 1]) continue;
                const float z = fr->depth[i];
                if (!(z >= cfg.z_min && z <= cfg.z_max)) continue;
                float p0[3];
                world_point(T, fr->fx, fr->fy, fr->cx, fr->cy, u, v, z, p0);
                uint64_t key;
                if (!key_of(p0[0], p0[1], p0[2], s, &key)) continue;
                pts.insert(pts.end(), p0, p0 + 3);
                sg.push_back(lab);
                at.push_back(i);
            }
        std::vector<uint8_t> nz(at.size());
        if (!at.empty()) oracle_dbscan_noise(pts.data(), sg.data(), (int64_t)at.size(), cfg.dbscan_eps,
                                             cfg.dbscan_min_pts, nz.data());
        for (size_t k = 0; k < at.size(); k++)
            if (nz[k]) {
                noise[at[k]] = 1;
                denoised++;
            }
    }

    // (a5) back-projection, keys and pixel normals.
    auto valid_px = [&](int u, int v, int lab) -> bool {
        if (u < 0 || v < 0 || u >= Wd || v >= H) return false;
        size_t i = (size_t)v * Wd + u;
        if (fr->labels[i] != lab || noise[i]) return false;
        float z = fr->depth[i];
        return z >= cfg.z_min && z <= cfg.z_max;
    };
    struct Acc {
        int64_t n[3] = {0, 0, 0};
        int32_t npx = 0;
    };
    std::map<std::pair<int, uint64_t>, Acc> segvox;  // ordered by (m, key)
    int valid = 0, dropped = 0;
    for (int v = 0; v < H; v++)
        for (int u = 0; u < Wd; u++) {
            int lab = fr->labels[(size_t)v * Wd + u];
            if (lab < 1 || lab > M || !mask_ok[lab - 1]) continue;
            if (!valid_px(u, v, lab)) continue;
            float p0[3];
            world_point(T, fr->fx, fr->fy, fr->cx, fr->cy, u, v, fr->depth[(size_t)v * Wd + u], p0);
            uint64_t key;
            if (!key_of(p0[0], p0[1], p0[2], s, &key)) {
                dropped++;
                continue;
            }
            valid++;
            Acc& acc = segvox[{lab, key}];
            acc.npx += 1;
            // Image-space tangents: forward differences, backward ones at the
            // right/bottom edge of a mask (both point along +u / +v).
            int ua = -1, ub = -1, va = -1, vb = -1;
            if (valid_px(u + 1, v, lab)) { ua = u + 1; ub = u; }
            else if (valid_px(u - 1, v, lab)) { ua = u; ub = u - 1; }
            if (valid_px(u, v + 1, lab)) { va = v + 1; vb = v; }
            else if (valid_px(u, v - 1, lab)) { va = v; vb = v - 1; }
            if (ua >= 0 && va >= 0) {
                float pa[3], pb[3], qa[3], qb[3];
                world_point(T, fr->fx, fr->fy, fr->cx, fr->cy, ua, v, fr->depth[(size_t)v * Wd + ua], pa);
                world_point(T, fr->fx, fr->fy, fr->cx, fr->cy, ub, v, fr->depth[(size_t)v * Wd + ub], pb);
                world_point(T, fr->fx, fr->fy, fr->cx, fr->cy, u, va, fr->depth[(size_t)va * Wd + u], qa);
                world_point(T, fr->fx, fr->fy, fr->cx, fr->cy, u, vb, fr->depth[(size_t)vb * Wd + u], qb);
                float e1[3], e2[3], n[3];
                for (int r = 0; r < 3; r++) {
                    e1[r] = pa[r] - pb[r];
                    e2[r] = qa[r] - qb[r];
                }
                n[0] = e2[1] * e1[2] - e2[2] * e1[1];
                n[1] = e2[2] * e1[0] - e2[0] * e1[2];
                n[2] = e2[0] * e1[1] - e2[1] * e1[0];
                float l2 = (n[0] * n[0] + n[1] * n[1]) + n[2] * n[2];
                if (l2 > 0.0f) {
                    float l = std::sqrt(l2);
                    const float il = 1.0f / l;
                    for (int r = 0; r < 3; r++) n[r] = n[r] * il;
                    // orient toward the camera
                    float vd = ((p0[0] - T.t[0]) * n[0] + (p0[1] - T.t[1]) * n[1]) + (p0[2] - T.t[2]) * n[2];
                    if (vd > 0.0f)
                        for (int r = 0; r < 3; r++) n[r] = -n[r];
                    for (int r = 0; r < 3; r++) acc.n[r] += fix(n[r], S_VEC);
                }
            }
        }

    // (a6) segment voxel sets and Eq. 3.
    std::vector<int32_t> nvox(M, 0);
    std::vector<int64_t> ang(M, 0);
    for (auto& kv : segvox) {
        int m = kv.first.first - 1;
        nvox[m] += 1;
        const Acc& acc = kv.second;
        float N[3] = {(float)unfix(acc.n[0], S_VEC), (float)unfix(acc.n[1], S_VEC), (float)unfix(acc.n[2], S_VEC)};
        float l2 = (N[0] * N[0] + N[1] * N[1]) + N[2] * N[2];
        float term = 0.0f;
        if (l2 > 0.0f) {
            float l = std::sqrt(l2);
            float nv[3] = {N[0] / l, N[1] / l, N[2] / l};
            int32_t k[3];
            unpack(kv.first.second, k);
            float r[3];
            for (int a = 0; a < 3; a++) r[a] = (((float)k[a] + 0.5f) * s) - T.t[a];
            float rl2 = (r[0] * r[0] + r[1] * r[1]) + r[2] * r[2];
            if (rl2 > 0.0f) {
                float rl = std::sqrt(rl2);
                float dot = (r[0] * nv[0] + r[1] * nv[1]) + r[2] * nv[2];
                term = -dot / rl;
                if (!(term > 0.0f)) term = 0.0f;
            }
        }
        ang[m] += fix(term, S_VEC);
    }
    int live = 0;
    for (int m = 0; m < M; m++) {
        if (nvox[m] > 0) {
            S_ang[m] = (float)(unfix(ang[m], S_VEC) / (double)nvox[m]);
            live++;
        }
        Qm[m] = ((S_size[m] * S_ang[m]) * S_sem[m]) * S_dist[m];
    }

    // (a7) overlap with the map as it stood before this frame.  With
    // overlap_dilation (the neighbourhood reading of Sec. III-B) a segment
    // voxel overlaps every instance that labels it or one of its 26
    // neighbours, once per instance.
    std::vector<std::map<int32_t, int64_t>> ov(M);  // per segment: root -> voxels
    std::set<int32_t> active;
    for (auto& kv : segvox) {
        std::set<int32_t> roots;
        int32_t k[3];
        unpack(kv.first.second, k);
        const int reach = cfg.overlap_dilation ? 1 : 0;
        for (int dx = -reach; dx <= reach; dx++)
            for (int dy = -reach; dy <= reach; dy++)
                for (int dz = -reach; dz <= reach; dz++) {
                    const int32_t q[3] = {k[0] + dx, k[1] + dy, k[2] + dz};
                    bool in = true;
                    for (int a = 0; a < 3; a++) in = in && q[a] >= -KEY_BIAS && q[a] <= KEY_BIAS - 1;
                    if (!in) continue;
                    const uint64_t nk = ((uint64_t)(q[0] + KEY_BIAS) << (2 * KEY_BITS)) |
                                        ((uint64_t)(q[1] + KEY_BIAS) << KEY_BITS) | (uint64_t)(q[2] + KEY_BIAS);
                    auto it = map->vox.find(nk);
                    if (it != map->vox.end()) roots.insert(map->parent[it->second]);
                }
        for (int32_t root : roots) {
            ov[kv.first.first - 1][root] += 1;
            active.insert(root);
        }
    }
    int pairs = 0;
    for (int m = 0; m < M; m++) pairs += (int)ov[m].size();

    // (a8) association: an edge needs enough shared voxels AND similar embeddings.
    std::vector<std::vector<int32_t>> edges(M);
    for (int m = 0; m < M; m++) {
        if (nvox[m] == 0) continue;
        for (auto& kv : ov[m]) {
            // overlap coefficient |V_m & V_k| / min(|V_m|, |V_k|) against ov_num/ov_den
            int64_t vk = map->count[kv.first];
            int64_t denom = std::min<int64_t>(nvox[m], vk);
            bool geo = kv.second * (int64_t)cfg.ov_den >= (int64_t)cfg.ov_num * denom;
            if (!geo) continue;
            // the association feature: the second grid's when there is one
            float c = Da > 0 ? cosine_exact(&Am[(size_t)m * Da], map->A[kv.first].data(), Da)
                             : cosine_exact(&Em[(size_t)m * D], map->E[kv.first].data(), D);
            if (c >= cfg.tau_cos) edges[m].push_back(kv.first);
        }
    }
    // Components of the bipartite segment/instance graph.  Union-find over the
    // touched roots; representative = smallest instance id.
    std::map<int32_t, int32_t> uf;
    std::function<int32_t(int32_t)> find = [&](int32_t x) -> int32_t {
        while (uf[x] != x) x = uf[x];
        return x;
    };
    for (int m = 0; m < M; m++)
        for (int32_t k : edges[m])
            if (!uf.count(k)) uf[k] = k;
    for (int m = 0; m < M; m++)
        for (size_t i = 1; i < edges[m].size(); i++) {
            int32_t a = find(edges[m][0]), b = find(edges[m][i]);
            if (a != b) {
                if (a < b) uf[b] = a; else uf[a] = b;
            }
        }
    std::vector<int32_t> segrep(M, -1);
    int new_inst = 0, merges = 0;
    for (int m = 0; m < M; m++)
        if (!edges[m].empty()) segrep[m] = find(edges[m][0]);
    // Merge the instances of each component into its representative.
    std::map<int32_t, std::vector<int32_t>> comp;  // rep -> member roots (ascending)
    for (auto& kv : uf) comp[find(kv.first)].push_back(kv.first);
    // (a10) fusion candidates gathered before any state changes.
    // The winning observation brings both its embedding and (with a second
    // grid) its association feature.
    struct Cand {
        float q;
        const float* e;
        const float* a;
    };
    std::map<int32_t, std::vector<float>> fusedE, fusedA;
    std::map<int32_t, float> fusedQ;
    auto inst_a = [&](int32_t k) { return Da > 0 ? map->A[k].data() : nullptr; };
    for (auto& kv : comp) {
        int32_t r = kv.first;
        Cand best{map->Q[kv.second[0]], map->E[kv.second[0]].data(), inst_a(kv.second[0])};
        for (size_t i = 1; i < kv.second.size(); i++) {
            int32_t k = kv.second[i];
            if (map->Q[k] > best.q) best = {map->Q[k], map->E[k].data(), inst_a(k)};
        }
        for (int m = 0; m < M; m++)
            if (segrep[m] == r && Qm[m] > best.q) best = {Qm[m], &Em[(size_t)m * D], &Am[(size_t)m * std::max(Da, 1)]};
        fusedE[r] = std::vector<float>(best.e, best.e + D);
        if (Da > 0) fusedA[r] = std::vector<float>(best.a, best.a + Da);
        fusedQ[r] = best.q;
    }
    for (auto& kv : comp) {
        int32_t r = kv.first;
        int32_t obs = 0;
        for (int32_t k : kv.second) {
            obs += map->n_obs[k];
            if (k != r) {
                map->parent[k] = r;
                map->count[r] += map->count[k];
                map->count[k] = 0;
                merges++;
            }
        }
        for (int m = 0; m < M; m++)
            if (segrep[m] == r) obs++;
        map->E[r] = fusedE[r];
        if (Da > 0) map->A[r] = fusedA[r];
        map->Q[r] = fusedQ[r];
        map->n_obs[r] = obs;
    }
    // keep the parent table flat: every id points at its root
    if (merges)
        for (size_t i = 0; i < map->parent.size(); i++) map->parent[i] = map->parent[map->parent[i]];
    // Segments without an edge open new instances, in increasing mask order.
    for (int m = 0; m < M; m++) {
        if (nvox[m] == 0 || segrep[m] >= 0) continue;
        int32_t id = (int32_t)map->parent.size();
        map->parent.push_back(id);
        map->count.push_back(0);
        map->Q.push_back(Qm[m]);
        map->E.emplace_back(&Em[(size_t)m * D], &Em[(size_t)m * D] + D);
        if (Da > 0) map->A.emplace_back(&Am[(size_t)m * Da], &Am[(size_t)m * Da] + Da);
        map->n_obs.push_back(1);
        segrep[m] = id;
        new_inst++;
    }

    // (a9) new voxels: the lowest-index segment containing a voxel labels it.
    int new_vox = 0;
    {
        std::map<uint64_t, int> owner;  // voxel -> lowest mask label
        for (auto& kv : segvox) {
            uint64_t key = kv.first.second;
            if (map->vox.count(key)) continue;
            auto it = owner.find(key);
            if (it == owner.end() || kv.first.first < it->second) owner[key] = kv.first.first;
        }
        for (auto& kv : owner) {
            int32_t lab = segrep[kv.second - 1];
            map->vox[kv.first] = lab;
            map->count[lab] += 1;
            new_vox++;
        }
    }

    if (rep) {
        if (rep->fbar) std::memcpy(rep->fbar, fbar.data(), sizeof(float) * D);
        if (rep->Dp) std::memcpy(rep->Dp, Dp.data(), sizeof(float) * P);
        if (rep->cosg) std::memcpy(rep->cosg, cosg.data(), sizeof(float) * P);
        if (rep->cov && M) std::memcpy(rep->cov, cov.data(), sizeof(int32_t) * (size_t)M * P);
        if (rep->npix && M) std::memcpy(rep->npix, npix.data(), sizeof(int32_t) * M);
        if (rep->W && M) std::memcpy(rep->W, Wt.data(), sizeof(float) * (size_t)M * P);
        if (rep->E && M) std::memcpy(rep->E, Em.data(), sizeof(float) * (size_t)M * D);
        if (rep->A && M && Da > 0) std::memcpy(rep->A, Am.data(), sizeof(float) * (size_t)M * Da);
        if (rep->S)
            for (int m = 0; m < M; m++) {
                rep->S[5 * m + 0] = S_size[m];
                rep->S[5 * m + 1] = S_ang[m];
                rep->S[5 * m + 2] = S_sem[m];
                rep->S[5 * m + 3] = S_dist[m];
                rep->S[5 * m + 4] = Qm[m];
            }
        if (rep->nvox && M) std::memcpy(rep->nvox, nvox.data(), sizeof(int32_t) * M);
        if (rep->rep && M) std::memcpy(rep->rep, segrep.data(), sizeof(int32_t) * M);
        rep->n_seg = (int64_t)segvox.size();
        if (rep->seg_keys && rep->seg_m) {
            int64_t i = 0;
            for (auto& kv : segvox) {
                if (i >= rep->seg_cap) break;
                rep->seg_m[i] = kv.first.first;
                rep->seg_keys[i] = kv.first.second;
                i++;
            }
        }
        rep->valid_pixels = valid;
        rep->dropped_pixels = dropped;
        rep->new_voxels = new_vox;
        rep->active_instances = (int32_t)active.size();
        rep->new_instances = new_inst;
        rep->merges = merges;
        rep->live_segments = live;
        rep->overlap_pairs = pairs;
        rep->denoised_pixels = denoised;
    }
    return ORACLE_OK;
}

int64_t oracle_num_voxels(const oracle_map* map) { return (int64_t)map->vox.size(); }

void oracle_export_voxels(const oracle_map* map, uint64_t* keys, int32_t* ids)
{
    std::vector<std::pair<uint64_t, int32_t>> v(map->vox.begin(), map->vox.end());
    std::sort(v.begin(), v.end());
    for (size_t i = 0; i < v.size(); i++) {
        keys[i] = v[i].first;
        ids[i] = v[i].second >= 0 ? map->parent[v[i].second] : -1;
    }
}

int32_t oracle_num_ids(const oracle_map* map) { return (int32_t)map->parent.size(); }

void oracle_export_instances(const oracle_map* map, int32_t* parent, int64_t* count, float* Q,
                             float* E, int32_t* n_obs)
{
    const int D = map->cfg.embed_dim;
    for (size_t i = 0; i < map->parent.size(); i++) {
        if (parent) parent[i] = map->parent[i];
        if (count) count[i] = map->count[i];
        if (Q) Q[i] = map->Q[i];
        if (E) std::memcpy(E + i * D, map->E[i].data(), sizeof(float) * D);
        if (n_obs) n_obs[i] = map->n_obs[i];
    }
}

// ---- End of the trajectory: orphan merge and noise filter (Sec. III-B) --------
namespace {

int32_t find_root(std::vector<int32_t>& uf, int32_t x)
{
    while (uf[x] != x) x = uf[x];
    return x;
}

// face neighbours of a voxel key (in range)
int neighbours6(uint64_t key, uint64_t out[6])
{
    int32_t k[3];
    unpack(key, k);
    int n = 0;
    for (int a = 0; a < 3; a++)
        for (int s = -1; s <= 1; s += 2) {
            int32_t q[3] = {k[0], k[1], k[2]};
            q[a] += s;
            if (q[a] < -KEY_BIAS || q[a] > KEY_BIAS - 1) continue;
            out[n++] = ((uint64_t)(q[0] + KEY_BIAS) << (2 * KEY_BITS)) | ((uint64_t)(q[1] + KEY_BIAS) << KEY_BITS) |
                       (uint64_t)(q[2] + KEY_BIAS);
        }
    return n;
}

}  // namespace

int oracle_finalize(oracle_map* map, const oracle_finalize_config* cfg, oracle_finalize_report* rep)
{
    if (!map || !cfg || cfg->contact_den <= 0 || cfg->contact_num < 0 || map->final_) return ORACLE_ERR_INVALID_ARG;
    const int D = map->cfg.embed_dim;
    const int32_t nid = (int32_t)map->parent.size();
    oracle_finalize_report r{};
    // (1) contacts between the instances (roots) of face-adjacent voxels
    std::map<std::pair<int32_t, int32_t>, int64_t> contact;
    for (const auto& kv : map->vox) {
        if (kv.second < 0) continue;
        const int32_t a = map->parent[kv.second];
        uint64_t nb[6];
        const int n = neighbours6(kv.first, nb);
        std::set<int32_t> seen;
        for (int i = 0; i < n; i++) {
            auto it = map->vox.find(nb[i]);
            if (it == map->vox.end() || it->second < 0) continue;
            const int32_t b = map->parent[it->second];
            if (b != a) seen.insert(b);
        }
        for (int32_t b : seen) contact[{std::min(a, b), std::max(a, b)}] += 1;
    }
    r.contact_pairs = (int32_t)contact.size();
    // (2) gates on the state at the start; union by smallest id
    std::vector<int32_t> uf(nid);
    for (int32_t i = 0; i < nid; i++) uf[i] = i;
    for (const auto& c : contact) {
        const int32_t a = c.first.first, b = c.first.second;
        const int64_t mn = std::min(map->count[a], map->count[b]);
        if (c.second * (int64_t)cfg->contact_den < (int64_t)cfg->contact_num * mn) continue;
        const bool similar = map->cfg.assoc_dim > 0
                                 ? cosine_exact(map->A[a].data(), map->A[b].data(), map->cfg.assoc_dim) >= cfg->tau_cos
                                 : cosine_exact(map->E[a].data(), map->E[b].data(), D) >= cfg->tau_cos;
        if (!similar) continue;
        const int32_t ra = find_root(uf, a), rb = find_root(uf, b);
        if (ra != rb) uf[std::max(ra, rb)] = std::min(ra, rb);
    }
    // (3) per component: summed counts, the highest-Q member's Q and embedding
    std::vector<int32_t> comp(nid), winner(nid, -1);
    for (int32_t i = 0; i < nid; i++) comp[i] = find_root(uf, i);
    for (int32_t i = 0; i < nid; i++) {
        if (map->parent[i] != i || map->count[i] <= 0) continue;  // live instances only
        int32_t& w = winner[comp[i]];
        if (w < 0 || map->Q[i] > map->Q[w]) w = i;  // ascending ids: ties keep the smaller
    }
    const std::vector<int64_t> count0 = map->count;
    const std::vector<int32_t> obs0 = map->n_obs;
    for (int32_t i = 0; i < nid; i++) {
        if (map->parent[i] != i || count0[i] <= 0 || comp[i] == i) continue;
        const int32_t c = comp[i];
        map->count[c] += count0[i];
        map->n_obs[c] += obs0[i];
        map->count[i] = 0;
        map->parent[i] = c;
        r.merged++;
    }
    for (int32_t c = 0; c < nid; c++) {
        const int32_t w = winner[c];
        if (w >= 0 && w != c) {
            map->Q[c] = map->Q[w];
            map->E[c] = map->E[w];
            if (map->cfg.assoc_dim > 0) map->A[c] = map->A[w];
        }
    }
    for (int32_t i = 0; i < nid; i++) map->parent[i] = map->parent[map->parent[i]];  // flat again
    // (4) drop instances below the voxel count
    std::vector<char> drop(nid, 0);
    for (int32_t i = 0; i < nid; i++) {
        if (map->parent[i] == i && map->count[i] > 0 && map->count[i] < cfg->min_voxels) {
            drop[i] = 1;
            r.removed++;
            map->count[i] = 0;
            map->n_obs[i] = 0;
            map->Q[i] = 0.0f;
        }
    }
    for (auto& kv : map->vox) {
        if (kv.second >= 0 && drop[map->parent[kv.second]]) {
            kv.second = -1;
            r.removed_voxels++;
        }
    }
    map->final_ = true;
    if (rep) *rep = r;
    return ORACLE_OK;
}

void oracle_set_state(oracle_map* map, const uint64_t* keys, const int32_t* labels, int64_t n,
                      const int32_t* parent, const int64_t* count, const float* Q, const float* E,
                      const int32_t* n_obs, int32_t nid)
{
    const int D = map->cfg.embed_dim;
    map->vox.clear();
    for (int64_t i = 0; i < n; i++) map->vox[keys[i]] = labels[i];
    map->parent.assign(parent, parent + nid);
    map->count.assign(count, count + nid);
    map->Q.assign(Q, Q + nid);
    map->n_obs.assign(n_obs, n_obs + nid);
    map->E.assign(nid, std::vector<float>(D));
    for (int32_t i = 0; i < nid; i++) std::memcpy(map->E[i].data(), E + (size_t)i * D, sizeof(float) * D);
    map->A.assign(map->cfg.assoc_dim > 0 ? nid : 0, std::vector<float>(std::max(map->cfg.assoc_dim, 0)));
    map->final_ = false;
}

void oracle_set_assoc(oracle_map* map, const float* A, int32_t nid)
{
    const int Da = map->cfg.assoc_dim;
    if (Da <= 0) return;
    map->A.assign(nid, std::vector<float>(Da));
    for (int32_t i = 0; i < nid; i++) std::memcpy(map->A[i].data(), A + (size_t)i * Da, sizeof(float) * Da);
}

void oracle_export_assoc(const oracle_map* map, float* A)
{
    const int Da = map->cfg.assoc_dim;
    for (size_t i = 0; i < map->A.size() && Da > 0; i++) std::memcpy(A + i * Da, map->A[i].data(), sizeof(float) * Da);
}

// Fig. 2: Eq. 1 on the grid with the query in the place of the global
// embedding gives D_p and cos(f_p, q); the heatmap is their product.
int oracle_query_heatmap(const float* F, int32_t P, int32_t D, const float* q, float eps, float* heat)
{
    if (!F || !q || !heat || P <= 0 || D <= 0) return ORACLE_ERR_INVALID_ARG;
    std::vector<float> Dp(P), c(P);
    const int st = oracle_token_stats(F, P, D, q, eps, nullptr, nullptr, Dp.data(), c.data());
    if (st != ORACLE_OK) return st;
    for (int p = 0; p < P; p++) heat[p] = Dp[p] * c[p];
    return ORACLE_OK;
}

// ---- FP64 twin of Eq. 1 and the pooling (error statements only) ---------------
void oracle_pool_f64(const float* F, int32_t P, int32_t D, const int32_t* cov, const int32_t* npix,
                     int32_t M, double eps, double* Dp, double* E)
{
    std::vector<double> mean(D, 0.0), n(P, 0.0);
    for (int p = 0; p < P; p++)
        for (int d = 0; d < D; d++) mean[d] += (double)F[(int64_t)p * D + d];
    for (int d = 0; d < D; d++) mean[d] /= P;
    double nbar = 0.0;
    for (int p = 0; p < P; p++) {
        double ss = 0.0;
        for (int d = 0; d < D; d++) {
            double r = (double)F[(int64_t)p * D + d] - mean[d];
            ss += r * r;
        }
        n[p] = std::sqrt(ss);
        nbar += n[p];
    }
    nbar /= P;
    for (int p = 0; p < P; p++) Dp[p] = n[p] / (nbar + eps);
    for (int m = 0; m < M; m++) {
        double A = 0.0;
        for (int p = 0; p < P; p++) A += (double)cov[(size_t)m * P + p] * Dp[p];
        for (int d = 0; d < D; d++) {
            double acc = 0.0;
            for (int p = 0; p < P; p++) {
                double w = A > 0.0 ? (double)cov[(size_t)m * P + p] * Dp[p] / A
                                   : (npix[m] > 0 ? (double)cov[(size_t)m * P + p] / npix[m] : 0.0);
                acc += w * (double)F[(int64_t)p * D + d];
            }
            E[(size_t)m * D + d] = acc;
        }
    }
}

}  // extern "C"
