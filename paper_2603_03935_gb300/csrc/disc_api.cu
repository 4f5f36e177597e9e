// C ABI of libdisc (declared in include/disc.h): map lifetime, frame
// integration, queries, export and checkpoints.  Host code only orchestrates:
// every step of a frame runs in the kernels of k_features.cu, k_gemm.cu,
// k_geometry.cu and k_serial.cu, enqueued on the map's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

#include "disc_common.cuh"
#include "kernels.h"

using namespace disc;

namespace {

constexpr int PAIR_CAP = 8192;   // distinct (segment, instance) overlaps per frame (k_serial.cu)

struct DevAlloc {
    std::vector<void*> ptrs;
    int64_t bytes = 0;
    bool failed = false;
    template <typename T>
    T* get(size_t n)
    {
        void* p = nullptr;
        if (n == 0) n = 1;
        if (cudaMalloc(&p, sizeof(T) * n) != cudaSuccess) {
            cudaGetLastError();
            failed = true;
            return nullptr;
        }
        ptrs.push_back(p);
        bytes += (int64_t)(sizeof(T) * n);
        return (T*)p;
    }
    void release(void* p, size_t n)
    {
        auto it = std::find(ptrs.begin(), ptrs.end(), p);
        if (it != ptrs.end()) {
            cudaFree(p);
            ptrs.erase(it);
            bytes -= (int64_t)n;
        }
    }
    void free_all()
    {
        for (void* p : ptrs) cudaFree(p);
        ptrs.clear();
        bytes = 0;
    }
};

uint64_t next_pow2(uint64_t x)
{
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace

struct BatchGraph {
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
};

struct disc_map {
    disc_map_config cfg;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevAlloc mem;
    VoxelTable vt{};
    Instances inst{};
    int* d_next_id = nullptr;
    int* d_flag = nullptr;
    int* d_prev_err = nullptr;            // status of the frame before the running batch
    bool graphs_off = false;              // capture failed once: launch directly
    std::map<int, BatchGraph> graphs;     // captured batch sequences
    const void* graph_vt_keys = nullptr;
    const void* graph_inst_parent = nullptr;
    BatchScratch bs{};
    SerialScratch ss{};
    FrameParams* d_fps = nullptr;         // [Bmax] parameters of the batch's frames
    FrameCounters* d_hist = nullptr;      // [hist_cap] per-frame counters of one call
    int hist_cap = 0;
    int Bmax = 1;
    int MM = 1;                           // mask rows per frame slot
    int P = 0, Kpad = 0, D = 0, Npad_max = 16;
    // host-side bounds that avoid a synchronisation per frame
    uint64_t used_upper = 0;
    int64_t next_id_upper = 0;
    int last_slot = 0, last_M = 0;
    bool have_frame = false;
    // staging of host inputs, one slot per frame of a batch
    float* d_depth = nullptr;
    uint16_t* d_labels = nullptr;
    unsigned char* d_tokens = nullptr;
    float* d_gembed = nullptr;
    size_t px_cap = 0;
    // kernel accounting and optional per-phase CUDA-event timing
    int64_t launches = 0;
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Mark {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Mark> marks;
    double phase_ms[PH_COUNT] = {};
    int64_t phase_launches[PH_COUNT] = {};
    int64_t phase_calls[PH_COUNT] = {};
};

namespace {

disc_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return DISC_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DISC_ERR_OOM : DISC_ERR_CUDA;
}

#define CK(x)                                      \
    do {                                           \
        disc_status _s = cuda_status((x));         \
        if (_s != DISC_OK) return _s;              \
    } while (0)

bool config_ok(const disc_map_config& c)
{
    if (!(c.voxel_size > 0.0f) || !(c.z_max >= c.z_min) || !(c.eps >= 0.0f)) return false;
    if (c.ov_den <= 0 || c.ov_num < 0) return false;
    if (c.embed_dim <= 0 || c.embed_dim > 4096) return false;
    if (c.patch_h <= 0 || c.patch_w <= 0 || (int64_t)c.patch_h * c.patch_w > 16384) return false;
    if (c.max_width <= 0 || c.max_height <= 0 || (int64_t)c.max_width * c.max_height > (1 << 24)) return false;
    if (c.max_masks < 0 || c.max_masks > MAX_MASKS) return false;
    if (coverage_smem_bytes(c.max_masks, c.patch_w) > 200 * 1024) return false;
    if (c.voxel_capacity <= 0 || !(c.max_load > 0.0f && c.max_load < 1.0f)) return false;
    if (c.instance_capacity <= 0) return false;
    if (c.batch_frames < 0 || c.batch_frames > 256) return false;
    if (c.precision != DISC_FP32) return false;  // only the fp32 fast path is built
    return true;
}

disc_status alloc_voxel_table(disc_map* m, uint64_t cap, VoxelTable* out)
{
    VoxelTable t{};
    t.keys = m->mem.get<unsigned long long>(cap);
    t.labels = m->mem.get<int32_t>(cap);
    if (m->mem.failed) {
        m->mem.failed = false;
        if (t.keys) m->mem.release(t.keys, sizeof(unsigned long long) * cap);
        if (t.labels) m->mem.release(t.labels, sizeof(int32_t) * cap);
        return DISC_ERR_OOM;
    }
    CK(cudaMemsetAsync(t.keys, 0xFF, sizeof(unsigned long long) * cap, m->stream));
    t.mask = cap - 1;
    t.used = m->vt.used;
    *out = t;
    return DISC_OK;
}

disc_status alloc_instances(disc_map* m, int cap, Instances* out)
{
    Instances in{};
    in.cap = cap;
    in.parent = m->mem.get<int32_t>(cap);
    in.count = m->mem.get<long long>(cap);
    in.Q = m->mem.get<float>(cap);
    in.E = m->mem.get<float>((size_t)cap * m->D);
    in.n_obs = m->mem.get<int32_t>(cap);
    if (m->mem.failed) {
        m->mem.failed = false;
        if (in.parent) m->mem.release(in.parent, sizeof(int32_t) * cap);
        if (in.count) m->mem.release(in.count, sizeof(long long) * cap);
        if (in.Q) m->mem.release(in.Q, sizeof(float) * cap);
        if (in.E) m->mem.release(in.E, sizeof(float) * (size_t)cap * m->D);
        if (in.n_obs) m->mem.release(in.n_obs, sizeof(int32_t) * cap);
        return DISC_ERR_OOM;
    }
    *out = in;
    return DISC_OK;
}

int read_next_id(disc_map* m)
{
    int v = 0;
    cudaMemcpyAsync(&v, m->d_next_id, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
    cudaStreamSynchronize(m->stream);
    return v;
}

uint64_t read_used(disc_map* m)
{
    unsigned long long v = 0;
    cudaMemcpyAsync(&v, m->vt.used, sizeof(v), cudaMemcpyDeviceToHost, m->stream);
    cudaStreamSynchronize(m->stream);
    return v;
}

// Grow the voxel table so that `incoming` more voxels keep the load below
// max_load.  Uses a host bound first; synchronises only when the bound is hit.
disc_status ensure_voxel_room(disc_map* m, uint64_t incoming)
{
    const double lim = (double)m->cfg.max_load * (double)(m->vt.mask + 1);
    if ((double)(m->used_upper + incoming) <= lim) return DISC_OK;
    CK(cudaStreamSynchronize(m->stream));
    m->used_upper = read_used(m);
    uint64_t cap = m->vt.mask + 1;
    while ((double)(m->used_upper + incoming) > (double)m->cfg.max_load * (double)cap) cap <<= 1;
    if (cap == m->vt.mask + 1) return DISC_OK;
    VoxelTable nt{};
    disc_status s = alloc_voxel_table(m, cap, &nt);
    if (s != DISC_OK) return s;
    CK(cudaMemsetAsync(m->d_flag, 0, sizeof(int), m->stream));
    launch_rehash(m->vt, nt, m->d_flag, m->stream);
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    if (flag != 0) {
        m->mem.release(nt.keys, sizeof(unsigned long long) * cap);
        m->mem.release(nt.labels, sizeof(int32_t) * cap);
        return DISC_ERR_TABLE_FULL;
    }
    const uint64_t old = m->vt.mask + 1;
    m->mem.release(m->vt.keys, sizeof(unsigned long long) * old);
    m->mem.release(m->vt.labels, sizeof(int32_t) * old);
    m->vt = nt;
    return DISC_OK;
}

disc_status ensure_instance_room(disc_map* m, int64_t incoming)
{
    if (m->next_id_upper + incoming <= m->inst.cap) return DISC_OK;
    CK(cudaStreamSynchronize(m->stream));
    m->next_id_upper = read_next_id(m);
    if (m->next_id_upper + incoming <= m->inst.cap) return DISC_OK;
    int cap = m->inst.cap;
    while ((int64_t)cap < m->next_id_upper + incoming) {
        if (cap > (1 << 29)) return DISC_ERR_CAPACITY;
        cap *= 2;
    }
    Instances ni{};
    disc_status s = alloc_instances(m, cap, &ni);
    if (s != DISC_OK) return s;
    const int n = (int)m->next_id_upper;
    CK(cudaMemcpyAsync(ni.parent, m->inst.parent, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(ni.count, m->inst.count, sizeof(long long) * n, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(ni.Q, m->inst.Q, sizeof(float) * n, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(ni.E, m->inst.E, sizeof(float) * (size_t)n * m->D, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaMemcpyAsync(ni.n_obs, m->inst.n_obs, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    const int oc = m->inst.cap;
    m->mem.release(m->inst.parent, sizeof(int32_t) * oc);
    m->mem.release(m->inst.count, sizeof(long long) * oc);
    m->mem.release(m->inst.Q, sizeof(float) * oc);
    m->mem.release(m->inst.E, sizeof(float) * (size_t)oc * m->D);
    m->mem.release(m->inst.n_obs, sizeof(int32_t) * oc);
    m->inst = ni;
    return DISC_OK;
}

cudaEvent_t take_event(disc_map* m)
{
    if (m->ev_used == m->ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        m->ev_pool.push_back(e);
    }
    return m->ev_pool[m->ev_used++];
}

// Enqueue one phase; with timing on, bracket it with events on the map's
// stream (event-record nodes when the stream is being captured).
template <class F>
void run_phase(disc_map* m, int ph, F&& launch)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (m->timing && (a = take_event(m))) cudaEventRecordWithFlags(a, m->stream, cudaEventRecordExternal);
    const int n = launch();
    m->launches += n;
    m->phase_launches[ph] += n;
    if (a && (b = take_event(m))) {
        cudaEventRecordWithFlags(b, m->stream, cudaEventRecordExternal);
        if (n > 0) m->marks.push_back({ph, a, b});
    }
}

int enqueue_batch_kernels(disc_map* m, int B, bool any_bf16, bool any_f32);

// Timing run of one batch: the sequence with its phase events is captured and
// launched as one graph, so the device never waits on the host inside a
// timed interval.  false: capture is not possible here (plain launches).
bool launch_timed_graph(disc_map* m, int B, bool any_bf16, bool any_f32)
{
    const size_t marks0 = m->marks.size(), ev0 = m->ev_used;
    const int64_t l0 = m->launches;
    int64_t pl0[PH_COUNT];
    for (int i = 0; i < PH_COUNT; i++) pl0[i] = m->phase_launches[i];
    auto undo = [&] {
        m->marks.resize(marks0);
        m->ev_used = ev0;
        m->launches = l0;
        for (int i = 0; i < PH_COUNT; i++) m->phase_launches[i] = pl0[i];
        cudaGetLastError();
    };
    if (cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        undo();
        return false;
    }
    enqueue_batch_kernels(m, B, any_bf16, any_f32);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamEndCapture(m->stream, &graph) != cudaSuccess || !graph ||
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        undo();
        return false;
    }
    cudaGraphDestroy(graph);
    const bool ok = cudaGraphLaunch(exec, m->stream) == cudaSuccess;
    cudaGraphExecDestroy(exec);  // freed once the launch completes
    if (!ok) {
        undo();
        return false;
    }
    return true;
}

// After a synchronisation: fold the recorded phase intervals into the totals.
void collect_timing(disc_map* m)
{
    for (auto& mk : m->marks) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, mk.a, mk.b) == cudaSuccess) {
            m->phase_ms[mk.phase] += ms;
            m->phase_calls[mk.phase] += 1;
        } else {
            cudaGetLastError();
        }
    }
    m->marks.clear();
    m->ev_used = 0;
}

disc_status check_frame(const disc_map* m, const disc_frame* f)
{
    if (!f || !f->depth || !f->labels || !f->tokens) return DISC_ERR_INVALID_ARG;
    if (f->width <= 0 || f->height <= 0 || f->width > m->cfg.max_width || f->height > m->cfg.max_height)
        return DISC_ERR_INVALID_ARG;
    if (f->num_masks < 0 || f->num_masks > m->cfg.max_masks) return DISC_ERR_INVALID_ARG;
    if (f->token_dtype != DISC_TOKENS_F32 && f->token_dtype != DISC_TOKENS_BF16) return DISC_ERR_INVALID_ARG;
    if (!(f->fx != 0.0f) || !(f->fy != 0.0f)) return DISC_ERR_INVALID_ARG;
    return DISC_OK;
}

// Every kernel of one batch of B frame slots, in order.  Grids follow the
// map's maxima (frames smaller than that return early in their blocks), and
// per-frame values are read on the device, so the sequence is the same for
// every batch of B frames and can be replayed as a CUDA graph.
int enqueue_batch_kernels(disc_map* m, int B, bool any_bf16, bool any_f32)
{
    const int D = m->D, P = m->P, Mmax = m->cfg.max_masks;
    const int Hmax = m->cfg.max_height, Wmax = m->cfg.max_width;
    cudaStream_t st = m->stream;
    const BatchScratch& bs = m->bs;
    const FrameParams* dfp = m->d_fps;
    const int64_t before = m->launches;
    run_phase(m, PH_CLEAR, [&] { return launch_slot_clear(bs, B, D, m->MM, st); });
    run_phase(m, PH_TOKENS, [&] { return launch_token_stats(dfp, bs, B, P, D, any_bf16, any_f32, st); });
    run_phase(m, PH_COVERAGE, [&] { return launch_coverage(dfp, bs, B, m->cfg.patch_h, m->cfg.patch_w, Mmax, st); });
    run_phase(m, PH_WEIGHTS, [&] { return launch_weights(dfp, bs, B, Mmax, st); });
    run_phase(m, PH_POOL_EXACT, [&] { return launch_pool_exact(dfp, bs, B, P, D, Mmax, any_bf16, any_f32, st); });
    run_phase(m, PH_POOL_GEMM, [&] { return launch_pool_gemm(dfp, bs, B, D, Mmax, any_bf16, any_f32, st); });
    if (Mmax > 0) {
        for (int f0 = 0; f0 < B; f0 += GEOMETRY_CHUNK) {
            const int nb = std::min(GEOMETRY_CHUNK, B - f0);
            run_phase(m, PH_BACKPROJECT, [&] { return launch_backproject(dfp, bs, f0, nb, Hmax, Wmax, st); });
            run_phase(m, PH_ENTRIES, [&] { return launch_entries(dfp, bs, m->vt, f0, nb, Mmax, st); });
        }
        run_phase(m, PH_ENTRIES, [&] { return launch_quality(dfp, bs, B, st); });
    }
    // error bound of the tensor-core pooled embedding relative to
    // sum_p w_p ||f_p||: split residue 3 * 2^-22 plus fp32 accumulation of
    // 3 K products; and of a warp-level fp32 cosine
    const float eta = (float)(3.0 * std::ldexp(1.0, -22) + 3.0 * m->Kpad * std::ldexp(1.0, -24));
    const float dot_err = (float)(3.0 * D * std::ldexp(1.0, -24));
    SerialScratch ss = m->ss;
    ss.prev_err = m->d_prev_err;
    for (int j = 0; j < B; j++)
        for (int ph = 0; ph < 4; ph++)
            run_phase(m, PH_OVERLAP + ph, [&] {
                return launch_serial_frame(dfp, bs, j, ss, m->vt, m->inst, m->d_next_id, eta, dot_err, ph, st);
            });
    return (int)(m->launches - before);
}

// The batch's kernel sequence captured once per (B, token dtypes) and
// replayed; tables that move (growth) invalidate the cache.
disc_status batch_graph(disc_map* m, int B, bool any_bf16, bool any_f32, BatchGraph** out)
{
    const int key = B * 4 + (any_bf16 ? 2 : 0) + (any_f32 ? 1 : 0);
    if (m->graph_vt_keys != m->vt.keys || m->graph_inst_parent != m->inst.parent) {
        for (auto& kv : m->graphs) cudaGraphExecDestroy(kv.second.exec);
        m->graphs.clear();
        m->graph_vt_keys = m->vt.keys;
        m->graph_inst_parent = m->inst.parent;
    }
    auto it = m->graphs.find(key);
    if (it != m->graphs.end()) {
        *out = &it->second;
        return DISC_OK;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    const int64_t before = m->launches;
    const int n = enqueue_batch_kernels(m, B, any_bf16, any_f32);
    m->launches = before;  // counted when the graph is launched
    cudaError_t e = cudaStreamEndCapture(m->stream, &graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        return DISC_ERR_CUDA;
    }
    BatchGraph g;
    g.kernels = n;
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DISC_ERR_CUDA;
    }
    *out = &(m->graphs[key] = g);
    return DISC_OK;
}

// Enqueue frames[0..B) (B <= Bmax, all valid) as one batch; counters of frame
// j are copied to hist[j].  prev: counters of the frame before this batch in
// the same call (an error there stops this batch), or NULL.
disc_status enqueue_batch(disc_map* m, const disc_frame* frames, int B, FrameCounters* hist,
                          const FrameCounters* prev)
{
    const int D = m->D, P = m->P;
    uint64_t px = 0;
    int64_t masks = 0;
    bool any_bf16 = false, any_f32 = false;
    for (int j = 0; j < B; j++) {
        px += (uint64_t)frames[j].width * frames[j].height;
        masks += frames[j].num_masks;
        any_bf16 |= frames[j].token_dtype == DISC_TOKENS_BF16;
        any_f32 |= frames[j].token_dtype == DISC_TOKENS_F32;
    }
    disc_status s = ensure_voxel_room(m, px);
    if (s != DISC_OK) return s;
    s = ensure_instance_room(m, masks);
    if (s != DISC_OK) return s;

    std::vector<FrameParams> fps(B);
    for (int j = 0; j < B; j++) {
        const disc_frame* f = frames + j;
        FrameParams& fp = fps[j];
        fp.H = f->height;
        fp.W = f->width;
        fp.M = f->num_masks;
        fp.P = P;
        fp.D = D;
        fp.Ph = m->cfg.patch_h;
        fp.Pw = m->cfg.patch_w;
        fp.Kpad = m->Kpad;
        fp.Npad = std::max(16, (fp.M + 15) / 16 * 16);
        fp.fx = f->fx;
        fp.fy = f->fy;
        fp.cx = f->cx;
        fp.cy = f->cy;
        for (int r = 0; r < 3; r++) {
            for (int c = 0; c < 3; c++) fp.R[3 * r + c] = (float)f->T_world_cam[4 * r + c];
            fp.t[r] = (float)f->T_world_cam[4 * r + 3];
        }
        fp.voxel = m->cfg.voxel_size;
        // reciprocals rounded once to fp32 (host fp32 division is IEEE)
        fp.inv_fx = 1.0f / f->fx;
        fp.inv_fy = 1.0f / f->fy;
        fp.inv_voxel = 1.0f / m->cfg.voxel_size;
        fp.z_min = m->cfg.z_min;
        fp.z_max = m->cfg.z_max;
        fp.eps = m->cfg.eps;
        fp.tau = m->cfg.tau_cos;
        fp.lambda_size = m->cfg.lambda_size;
        fp.ov_num = m->cfg.ov_num;
        fp.ov_den = m->cfg.ov_den;
        fp.min_px = std::max(1, m->cfg.min_mask_pixels);
        fp.token_bf16 = f->token_dtype == DISC_TOKENS_BF16;
        const size_t npx = (size_t)fp.H * fp.W;
        const size_t tok_bytes = (size_t)P * D * (fp.token_bf16 ? 2 : 4);
        if (f->inputs_on_device) {
            fp.depth = f->depth;
            fp.labels = f->labels;
            fp.tokens = f->tokens;
            fp.gembed = f->global_embed;
        } else {
            float* dd = m->d_depth + (size_t)j * m->px_cap;
            uint16_t* dl = m->d_labels + (size_t)j * m->px_cap;
            unsigned char* dt = m->d_tokens + (size_t)j * P * D * 4;
            CK(cudaMemcpyAsync(dd, f->depth, sizeof(float) * npx, cudaMemcpyHostToDevice, m->stream));
            CK(cudaMemcpyAsync(dl, f->labels, sizeof(uint16_t) * npx, cudaMemcpyHostToDevice, m->stream));
            CK(cudaMemcpyAsync(dt, f->tokens, tok_bytes, cudaMemcpyHostToDevice, m->stream));
            fp.depth = dd;
            fp.labels = dl;
            fp.tokens = dt;
            fp.gembed = nullptr;
            if (f->global_embed) {
                float* dg = m->d_gembed + (size_t)j * D;
                CK(cudaMemcpyAsync(dg, f->global_embed, sizeof(float) * D, cudaMemcpyHostToDevice, m->stream));
                fp.gembed = dg;
            }
        }
    }
    // pageable source: the call returns once the parameters are staged
    CK(cudaMemcpyAsync(m->d_fps, fps.data(), sizeof(FrameParams) * B, cudaMemcpyHostToDevice, m->stream));
    // status of the frame before this batch (0 when it is the first of the call)
    if (prev) CK(cudaMemcpyAsync(m->d_prev_err, &prev->err, sizeof(int), cudaMemcpyDeviceToDevice, m->stream));
    else CK(cudaMemsetAsync(m->d_prev_err, 0, sizeof(int), m->stream));

    BatchGraph* g = nullptr;
    if (!m->timing && !m->graphs_off && batch_graph(m, B, any_bf16, any_f32, &g) != DISC_OK) {
        m->graphs_off = true;  // this stream or driver cannot capture the sequence
        g = nullptr;
    }
    if (g) {
        CK(cudaGraphLaunch(g->exec, m->stream));
        m->launches += g->kernels;
    } else if (!(m->timing && !m->graphs_off && launch_timed_graph(m, B, any_bf16, any_f32))) {
        enqueue_batch_kernels(m, B, any_bf16, any_f32);
    }
    // the batch's counters, in slot order, to the call's history
    CK(cudaMemcpyAsync(hist, m->bs.base.ctr, sizeof(FrameCounters) * B, cudaMemcpyDeviceToDevice, m->stream));
    CK(cudaGetLastError());
    m->used_upper += px;
    m->next_id_upper += masks;
    m->last_slot = B - 1;
    m->last_M = frames[B - 1].num_masks;
    m->have_frame = true;
    return DISC_OK;
}

void to_stats(const FrameCounters& c, disc_frame_stats* s)
{
    s->valid_pixels = c.valid_pixels;
    s->dropped_pixels = c.dropped_pixels;
    s->unique_seg_voxels = c.n_entries;
    s->new_voxels = c.n_new;
    s->active_instances = c.active_instances;
    s->overlap_pairs = c.n_pairs;
    s->new_instances = c.new_instances;
    s->merges = c.merges;
    s->live_segments = c.live_segments;
    s->borderline_rescored = c.borderline;
    s->max_probe = c.max_probe;
    s->status = c.err;
}

disc_status ensure_hist(disc_map* m, int n)
{
    if (n <= m->hist_cap) return DISC_OK;
    if (m->d_hist) m->mem.release(m->d_hist, sizeof(FrameCounters) * m->hist_cap);
    m->d_hist = m->mem.get<FrameCounters>(n);
    if (m->mem.failed) {
        m->mem.failed = false;
        m->hist_cap = 0;
        m->d_hist = nullptr;
        return DISC_ERR_OOM;
    }
    m->hist_cap = n;
    return DISC_OK;
}

// Integrate frames[0..n): batches of Bmax; stops at the first invalid frame
// (host check) or the first frame that fails on the device.
disc_status integrate(disc_map* m, const disc_frame* frames, int n, disc_frame_stats* stats, int* n_done)
{
    if (n_done) *n_done = 0;
    disc_status s = ensure_hist(m, std::max(n, 1));
    if (s != DISC_OK) return s;
    int valid = 0;
    while (valid < n && check_frame(m, frames + valid) == DISC_OK) valid++;
    int enq = 0;
    for (int lo = 0; lo < valid; lo += m->Bmax) {
        const int B = std::min(m->Bmax, valid - lo);
        s = enqueue_batch(m, frames + lo, B, m->d_hist + lo, lo > 0 ? m->d_hist + lo - 1 : nullptr);
        if (s != DISC_OK) break;
        enq += B;
    }
    std::vector<FrameCounters> c(std::max(enq, 1));
    if (enq > 0) CK(cudaMemcpyAsync(c.data(), m->d_hist, sizeof(FrameCounters) * enq, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    collect_timing(m);
    int done = 0;
    disc_status fs = DISC_OK;
    int exact_next_id = -1;  // frames without masks skip the kernel that records it
    for (int i = 0; i < enq; i++) {
        if (stats) to_stats(c[i], stats + i);
        if (c[i].err != 0) {
            fs = (disc_status)c[i].err;
            break;
        }
        exact_next_id = std::max(exact_next_id, c[i].next_id);
        done++;
    }
    if (exact_next_id > 0) m->next_id_upper = std::max<int64_t>(exact_next_id, 0);
    if (n_done) *n_done = done;
    if (fs != DISC_OK) return fs;
    if (s != DISC_OK) return s;
    if (valid < n) return DISC_ERR_INVALID_ARG;
    return DISC_OK;
}

}  // namespace

extern "C" {

void disc_config_default(disc_map_config* c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->voxel_size = 0.025f;
    c->z_min = 0.1f;
    c->z_max = 10.0f;
    c->eps = 1e-6f;
    c->tau_cos = 0.75f;
    c->lambda_size = 3.3f;
    c->ov_num = 1;
    c->ov_den = 5;
    c->embed_dim = 768;
    c->patch_h = 24;
    c->patch_w = 24;
    c->max_width = 640;
    c->max_height = 480;
    c->max_masks = 40;
    c->min_mask_pixels = 307;
    c->voxel_capacity = 1 << 22;
    c->max_load = 0.5f;
    c->instance_capacity = 1 << 14;
    c->precision = DISC_FP32;
    c->cuda_stream = nullptr;
    c->device = 0;
    c->batch_frames = 32;
}

disc_status disc_map_create(const disc_map_config* cfg, disc_map_config* resolved, disc_map** out_map)
{
    if (!cfg || !out_map) return DISC_ERR_INVALID_ARG;
    *out_map = nullptr;
    if (!config_ok(*cfg)) return DISC_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return DISC_ERR_CUDA;
    }
    CK(cudaSetDevice(cfg->device));
    disc_map* m = new disc_map();
    m->cfg = *cfg;
    m->cfg.voxel_capacity = (int64_t)next_pow2((uint64_t)cfg->voxel_capacity);
    if (m->cfg.batch_frames == 0) m->cfg.batch_frames = 32;
    m->Bmax = m->cfg.batch_frames;
    m->D = cfg->embed_dim;
    m->P = cfg->patch_h * cfg->patch_w;
    m->Kpad = (m->P + GEMM_KC - 1) / GEMM_KC * GEMM_KC;
    m->MM = std::max(1, cfg->max_masks);
    m->Npad_max = std::max(16, (m->MM + 15) / 16 * 16);
    if (cfg->cuda_stream) {
        m->stream = (cudaStream_t)cfg->cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete m;
            return DISC_ERR_CUDA;
        }
        m->own_stream = true;
    }
    static bool attrs_set = false;
    if (!attrs_set) {
        cudaError_t e = set_feature_kernel_attrs(200 * 1024);
        if (e == cudaSuccess) e = set_gemm_kernel_attrs();
        if (e == cudaSuccess) e = set_serial_kernel_attrs();
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (m->own_stream) cudaStreamDestroy(m->stream);
            delete m;
            return DISC_ERR_CUDA;
        }
        attrs_set = true;
    }
    const int D = m->D, P = m->P, MM = m->MM, B = m->Bmax;
    const uint64_t npx = (uint64_t)cfg->max_width * cfg->max_height;
    const uint64_t scap = next_pow2(npx + npx / 2);  // per-frame hashes: load <= 2/3
    m->px_cap = npx;
    DevAlloc& a = m->mem;
    m->vt.used = a.get<unsigned long long>(1);
    m->d_next_id = a.get<int>(1);
    m->d_flag = a.get<int>(1);
    m->d_prev_err = a.get<int>(1);
    m->d_fps = a.get<FrameParams>(B);
    BatchScratch& bs = m->bs;
    bs.sD = D;
    bs.sP = P;
    bs.sMM = MM;
    bs.sMMP = (long long)MM * P;
    bs.sW = (long long)m->Npad_max * m->Kpad;
    bs.sMMD = (long long)MM * D;
    bs.sS = 5LL * MM;
    bs.scap = (long long)scap;
    Scratch& sc = bs.base;
    sc.sumF = a.get<long long>((size_t)B * D);
    sc.fbar = a.get<float>((size_t)B * D);
    sc.gvec = a.get<float>((size_t)B * D);
    sc.gg = a.get<long long>(B);
    sc.nsum = a.get<long long>(B);
    sc.dotg = a.get<long long>((size_t)B * P);
    sc.ffp = a.get<long long>((size_t)B * P);
    sc.nrm = a.get<float>((size_t)B * P);
    sc.Dp = a.get<float>((size_t)B * P);
    sc.cosg = a.get<float>((size_t)B * P);
    sc.fnorm = a.get<float>((size_t)B * P);
    sc.cov = a.get<int32_t>((size_t)B * MM * P);
    sc.npix = a.get<int32_t>((size_t)B * MM);
    sc.W = a.get<float>((size_t)B * bs.sW);
    sc.S = a.get<float>((size_t)B * 5 * MM);
    sc.Bm = a.get<float>((size_t)B * MM);
    sc.Ecan = a.get<float>((size_t)B * MM * D);
    sc.Efast = a.get<float>((size_t)B * MM * D);
    sc.ang = a.get<long long>((size_t)B * MM);
    sc.nvox = a.get<int32_t>((size_t)B * MM);
    sc.segrep = a.get<int32_t>((size_t)B * MM);
    sc.sslot = a.get<SegSlot>((size_t)B * scap);
    sc.sent = a.get<unsigned long long>((size_t)B * scap);
    sc.slist = a.get<int32_t>((size_t)B * scap);
    sc.elab = a.get<int32_t>((size_t)B * scap);
    sc.smask = scap - 1;
    sc.ctr = a.get<FrameCounters>(B);
    SerialScratch& ss = m->ss;
    ss.okeys = a.get<unsigned long long>(scap);
    ss.ocnt = a.get<int32_t>(scap);
    ss.olist = a.get<int32_t>(scap);
    ss.omask = scap - 1;
    ss.nkeys = a.get<unsigned long long>(scap);
    ss.nown = a.get<int32_t>(scap);
    ss.nlist = a.get<int32_t>(scap);
    ss.nmask = scap - 1;
    ss.edge_cap = PAIR_CAP;
    ss.edge_m = a.get<int32_t>(PAIR_CAP);
    ss.edge_k = a.get<int32_t>(PAIR_CAP);
    ss.edge_n = a.get<int32_t>(1);
    ss.copy_cap = PAIR_CAP + MAX_MASKS;
    ss.copy_dst = a.get<int32_t>(ss.copy_cap);
    ss.copy_src = a.get<int32_t>(ss.copy_cap);
    ss.copy_n = a.get<int32_t>(1);
    ss.prev_err = nullptr;
    m->d_depth = a.get<float>((size_t)B * npx);
    m->d_labels = a.get<uint16_t>((size_t)B * npx);
    m->d_tokens = a.get<unsigned char>((size_t)B * P * D * 4);
    m->d_gembed = a.get<float>((size_t)B * D);
    disc_status st = DISC_OK;
    if (a.failed) st = DISC_ERR_OOM;
    if (st == DISC_OK) {
        VoxelTable vt{};
        st = alloc_voxel_table(m, (uint64_t)m->cfg.voxel_capacity, &vt);
        if (st == DISC_OK) m->vt = vt;
    }
    if (st == DISC_OK) st = alloc_instances(m, cfg->instance_capacity, &m->inst);
    if (st == DISC_OK) {
        cudaStream_t s = m->stream;
        cudaMemsetAsync(m->vt.used, 0, sizeof(unsigned long long), s);
        cudaMemsetAsync(m->d_next_id, 0, sizeof(int), s);
        cudaMemsetAsync(sc.ctr, 0, sizeof(FrameCounters) * B, s);
        cudaMemsetAsync(sc.W, 0, sizeof(float) * (size_t)B * bs.sW, s);
        cudaMemsetAsync(sc.cov, 0, sizeof(int32_t) * (size_t)B * MM * P, s);
        cudaMemsetAsync(sc.sslot, 0, sizeof(SegSlot) * B * scap, s);
        cudaMemsetAsync(ss.okeys, 0xFF, sizeof(unsigned long long) * scap, s);
        cudaMemsetAsync(ss.ocnt, 0, sizeof(int32_t) * scap, s);
        cudaMemsetAsync(ss.nkeys, 0xFF, sizeof(unsigned long long) * scap, s);
        cudaMemsetAsync(ss.nown, 0x7F, sizeof(int32_t) * scap, s);  // large positive sentinel
        cudaMemsetAsync(ss.edge_n, 0, sizeof(int32_t), s);
        cudaMemsetAsync(ss.copy_n, 0, sizeof(int32_t), s);
        cudaMemsetAsync(sc.Efast, 0, sizeof(float) * (size_t)B * MM * D, s);
        cudaMemsetAsync(sc.Ecan, 0, sizeof(float) * (size_t)B * MM * D, s);
        st = cuda_status(cudaStreamSynchronize(s));
    }
    if (st != DISC_OK) {
        m->mem.free_all();
        if (m->own_stream) cudaStreamDestroy(m->stream);
        delete m;
        return st;
    }
    if (resolved) *resolved = m->cfg;
    *out_map = m;
    return DISC_OK;
}

void disc_map_destroy(disc_map* m)
{
    if (!m) return;
    cudaSetDevice(m->cfg.device);
    cudaStreamSynchronize(m->stream);
    for (cudaEvent_t e : m->ev_pool) cudaEventDestroy(e);
    for (auto& kv : m->graphs) cudaGraphExecDestroy(kv.second.exec);
    m->mem.free_all();
    if (m->own_stream) cudaStreamDestroy(m->stream);
    delete m;
}

disc_status disc_integrate_frame(disc_map* m, const disc_frame* f, disc_frame_stats* stats)
{
    if (!m || !f) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    disc_status s = check_frame(m, f);
    if (s != DISC_OK) return s;
    return integrate(m, f, 1, stats, nullptr);
}

disc_status disc_integrate_frames(disc_map* m, const disc_frame* frames, int32_t n, disc_frame_stats* stats,
                                  int32_t* n_done)
{
    if (n_done) *n_done = 0;
    if (!m || (n > 0 && !frames) || n < 0) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    if (n == 0) return DISC_OK;
    return integrate(m, frames, n, stats, n_done);
}

disc_status disc_map_last_frame(disc_map* m, disc_frame_report* r)
{
    if (!m || !r) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    CK(cudaStreamSynchronize(m->stream));
    const int M = m->have_frame ? m->last_M : 0, P = m->P, D = m->D;
    const Scratch sc = m->bs.frame(m->last_slot);
    FrameCounters c{};
    CK(cudaMemcpy(&c, sc.ctr, sizeof(c), cudaMemcpyDeviceToHost));
    r->num_masks = M;
    if (r->fbar) CK(cudaMemcpy(r->fbar, sc.fbar, sizeof(float) * D, cudaMemcpyDeviceToHost));
    if (r->Dp) CK(cudaMemcpy(r->Dp, sc.Dp, sizeof(float) * P, cudaMemcpyDeviceToHost));
    if (r->cosg) CK(cudaMemcpy(r->cosg, sc.cosg, sizeof(float) * P, cudaMemcpyDeviceToHost));
    if (M > 0) {
        if (r->cov) CK(cudaMemcpy(r->cov, sc.cov, sizeof(int32_t) * (size_t)M * P, cudaMemcpyDeviceToHost));
        if (r->npix) CK(cudaMemcpy(r->npix, sc.npix, sizeof(int32_t) * M, cudaMemcpyDeviceToHost));
        if (r->W)
            CK(cudaMemcpy2D(r->W, sizeof(float) * P, sc.W, sizeof(float) * m->Kpad, sizeof(float) * P, M,
                            cudaMemcpyDeviceToHost));
        if (r->E) CK(cudaMemcpy(r->E, sc.Ecan, sizeof(float) * (size_t)M * D, cudaMemcpyDeviceToHost));
        if (r->E_fast) CK(cudaMemcpy(r->E_fast, sc.Efast, sizeof(float) * (size_t)M * D, cudaMemcpyDeviceToHost));
        if (r->S) CK(cudaMemcpy(r->S, sc.S, sizeof(float) * 5 * M, cudaMemcpyDeviceToHost));
        if (r->nvox) CK(cudaMemcpy(r->nvox, sc.nvox, sizeof(int32_t) * M, cudaMemcpyDeviceToHost));
        if (r->rep) CK(cudaMemcpy(r->rep, sc.segrep, sizeof(int32_t) * M, cudaMemcpyDeviceToHost));
    }
    r->n_seg = c.n_entries;
    if (r->seg_keys && r->seg_m && c.n_entries > 0) {
        const int n = c.n_entries;
        std::vector<unsigned long long> keys(n);
        CK(cudaMemcpy(keys.data(), sc.sent, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost));
        const int lim = (int)std::min<int64_t>(n, r->seg_cap);
        for (int i = 0; i < lim; i++) {
            const unsigned long long hk = keys[i];
            r->seg_m[i] = (int32_t)(hk >> 54);
            r->seg_keys[i] = hk & ((1ull << 54) - 1);
        }
    }
    return DISC_OK;
}

disc_status disc_map_counts(disc_map* m, int64_t* nv, int32_t* nid)
{
    if (!m) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    CK(cudaStreamSynchronize(m->stream));
    if (nv) *nv = (int64_t)read_used(m);
    if (nid) *nid = read_next_id(m);
    return DISC_OK;
}

disc_status disc_map_export_voxels(disc_map* m, uint64_t* keys, int32_t* ids, int64_t cap)
{
    if (!m || (cap > 0 && (!keys || !ids))) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    CK(cudaStreamSynchronize(m->stream));
    const uint64_t tc = m->vt.mask + 1;
    std::vector<unsigned long long> k(tc);
    std::vector<int32_t> l(tc);
    const int nid = read_next_id(m);
    std::vector<int32_t> parent(std::max(nid, 1));
    CK(cudaMemcpy(k.data(), m->vt.keys, sizeof(unsigned long long) * tc, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(l.data(), m->vt.labels, sizeof(int32_t) * tc, cudaMemcpyDeviceToHost));
    if (nid) CK(cudaMemcpy(parent.data(), m->inst.parent, sizeof(int32_t) * nid, cudaMemcpyDeviceToHost));
    std::vector<std::pair<uint64_t, int32_t>> v;
    for (uint64_t i = 0; i < tc; i++)
        if (k[i] != EMPTY_KEY) v.push_back({k[i], (l[i] >= 0 && l[i] < nid) ? parent[l[i]] : -1});
    std::sort(v.begin(), v.end());
    if ((int64_t)v.size() > cap) return DISC_ERR_INVALID_ARG;
    for (size_t i = 0; i < v.size(); i++) {
        keys[i] = v[i].first;
        ids[i] = v[i].second;
    }
    return DISC_OK;
}

disc_status disc_map_export_instances(disc_map* m, int32_t* parent, int64_t* count, float* Q, float* E,
                                      int32_t* n_obs, int32_t cap)
{
    if (!m) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    CK(cudaStreamSynchronize(m->stream));
    const int n = read_next_id(m);
    if (n > cap) return DISC_ERR_INVALID_ARG;
    if (n == 0) return DISC_OK;
    if (parent) CK(cudaMemcpy(parent, m->inst.parent, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    if (count) CK(cudaMemcpy(count, m->inst.count, sizeof(int64_t) * n, cudaMemcpyDeviceToHost));
    if (Q) CK(cudaMemcpy(Q, m->inst.Q, sizeof(float) * n, cudaMemcpyDeviceToHost));
    if (E) CK(cudaMemcpy(E, m->inst.E, sizeof(float) * (size_t)n * m->D, cudaMemcpyDeviceToHost));
    if (n_obs) CK(cudaMemcpy(n_obs, m->inst.n_obs, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    return DISC_OK;
}

disc_status disc_query_topk(disc_map* m, const float* q, int32_t nq, int32_t k, int32_t* ids, float* scores)
{
    if (!m || nq < 0 || k <= 0 || (nq > 0 && (!q || !ids || !scores))) return DISC_ERR_INVALID_ARG;
    if (nq == 0) return DISC_OK;
    CK(cudaSetDevice(m->cfg.device));
    CK(cudaStreamSynchronize(m->stream));
    const int nid = read_next_id(m);
    const int D = m->D;
    if (nid == 0) {
        for (int64_t i = 0; i < (int64_t)nq * k; i++) {
            ids[i] = -1;
            scores[i] = -INFINITY;
        }
        return DISC_OK;
    }
    float *dq = nullptr, *dsc = nullptr, *dout = nullptr;
    int* dids = nullptr;
    disc_status s = DISC_OK;
    if (cudaMalloc(&dq, sizeof(float) * (size_t)nq * D) != cudaSuccess ||
        cudaMalloc(&dsc, sizeof(float) * (size_t)nq * nid) != cudaSuccess ||
        cudaMalloc(&dout, sizeof(float) * (size_t)nq * k) != cudaSuccess ||
        cudaMalloc(&dids, sizeof(int) * (size_t)nq * k) != cudaSuccess) {
        cudaGetLastError();
        s = DISC_ERR_OOM;
    }
    if (s == DISC_OK) {
        cudaMemcpyAsync(dq, q, sizeof(float) * (size_t)nq * D, cudaMemcpyHostToDevice, m->stream);
        launch_query_topk(dq, nq, D, m->inst, nid, dsc, k, dids, dout, m->stream);
        cudaMemcpyAsync(ids, dids, sizeof(int) * (size_t)nq * k, cudaMemcpyDeviceToHost, m->stream);
        cudaMemcpyAsync(scores, dout, sizeof(float) * (size_t)nq * k, cudaMemcpyDeviceToHost, m->stream);
        s = cuda_status(cudaStreamSynchronize(m->stream));
    }
    cudaFree(dq);
    cudaFree(dsc);
    cudaFree(dout);
    cudaFree(dids);
    return s;
}

disc_status disc_query_points(disc_map* m, const float* xyz, int64_t n, int32_t* ids)
{
    if (!m || n < 0 || (n > 0 && (!xyz || !ids))) return DISC_ERR_INVALID_ARG;
    if (n == 0) return DISC_OK;
    CK(cudaSetDevice(m->cfg.device));
    float* dx = nullptr;
    int* di = nullptr;
    disc_status s = DISC_OK;
    if (cudaMalloc(&dx, sizeof(float) * 3 * n) != cudaSuccess || cudaMalloc(&di, sizeof(int) * n) != cudaSuccess) {
        cudaGetLastError();
        s = DISC_ERR_OOM;
    }
    if (s == DISC_OK) {
        cudaMemcpyAsync(dx, xyz, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, m->stream);
        launch_query_points(dx, n, m->cfg.voxel_size, m->vt, m->inst, di, m->stream);
        cudaMemcpyAsync(ids, di, sizeof(int) * n, cudaMemcpyDeviceToHost, m->stream);
        s = cuda_status(cudaStreamSynchronize(m->stream));
    }
    cudaFree(dx);
    cudaFree(di);
    return s;
}

// checkpoint file: magic, config, counts, voxels (key, label), instance table
static const char kMagic[8] = {'D', 'I', 'S', 'C', 'M', 'A', 'P', '1'};

disc_status disc_map_save(disc_map* m, const char* path)
{
    if (!m || !path) return DISC_ERR_INVALID_ARG;
    int64_t nv = 0;
    int32_t nid = 0;
    disc_status s = disc_map_counts(m, &nv, &nid);
    if (s != DISC_OK) return s;
    std::vector<uint64_t> keys(std::max<int64_t>(nv, 1));
    std::vector<int32_t> ids(std::max<int64_t>(nv, 1));
    s = disc_map_export_voxels(m, keys.data(), ids.data(), nv);
    if (s != DISC_OK) return s;
    const int D = m->D;
    std::vector<int32_t> parent(std::max(nid, 1)), obs(std::max(nid, 1));
    std::vector<int64_t> count(std::max(nid, 1));
    std::vector<float> Q(std::max(nid, 1)), E((size_t)std::max(nid, 1) * D);
    s = disc_map_export_instances(m, parent.data(), count.data(), Q.data(), E.data(), obs.data(), nid);
    if (s != DISC_OK) return s;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return DISC_ERR_INVALID_ARG;
    disc_map_config c = m->cfg;
    c.cuda_stream = nullptr;
    bool ok = std::fwrite(kMagic, 1, 8, fp) == 8 && std::fwrite(&c, sizeof(c), 1, fp) == 1 &&
              std::fwrite(&nv, sizeof(nv), 1, fp) == 1 && std::fwrite(&nid, sizeof(nid), 1, fp) == 1;
    if (ok && nv) ok = std::fwrite(keys.data(), 8, nv, fp) == (size_t)nv && std::fwrite(ids.data(), 4, nv, fp) == (size_t)nv;
    if (ok && nid)
        ok = std::fwrite(parent.data(), 4, nid, fp) == (size_t)nid && std::fwrite(count.data(), 8, nid, fp) == (size_t)nid &&
             std::fwrite(Q.data(), 4, nid, fp) == (size_t)nid &&
             std::fwrite(E.data(), 4, (size_t)nid * D, fp) == (size_t)nid * D && std::fwrite(obs.data(), 4, nid, fp) == (size_t)nid;
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? DISC_OK : DISC_ERR_INVALID_ARG;
}

disc_status disc_map_load(const char* path, const disc_map_config* over, disc_map** out)
{
    if (!path || !out) return DISC_ERR_INVALID_ARG;
    *out = nullptr;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return DISC_ERR_INVALID_ARG;
    char magic[8];
    disc_map_config c;
    int64_t nv = 0;
    int32_t nid = 0;
    bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(&c, sizeof(c), 1, fp) == 1 && std::fread(&nv, sizeof(nv), 1, fp) == 1 &&
              std::fread(&nid, sizeof(nid), 1, fp) == 1 && nv >= 0 && nid >= 0 && c.embed_dim > 0 &&
              c.embed_dim <= 4096;
    const int D = ok ? c.embed_dim : 1;
    std::vector<uint64_t> keys(std::max<int64_t>(nv, 1));
    std::vector<int32_t> ids(std::max<int64_t>(nv, 1));
    std::vector<int32_t> parent(std::max(nid, 1)), obs(std::max(nid, 1));
    std::vector<int64_t> count(std::max(nid, 1));
    std::vector<float> Q(std::max(nid, 1)), E((size_t)std::max(nid, 1) * D);
    if (ok && nv) ok = std::fread(keys.data(), 8, nv, fp) == (size_t)nv && std::fread(ids.data(), 4, nv, fp) == (size_t)nv;
    if (ok && nid)
        ok = std::fread(parent.data(), 4, nid, fp) == (size_t)nid && std::fread(count.data(), 8, nid, fp) == (size_t)nid &&
             std::fread(Q.data(), 4, nid, fp) == (size_t)nid &&
             std::fread(E.data(), 4, (size_t)nid * D, fp) == (size_t)nid * D && std::fread(obs.data(), 4, nid, fp) == (size_t)nid;
    std::fclose(fp);
    if (!ok) return DISC_ERR_INVALID_ARG;
    if (over) {
        c.cuda_stream = over->cuda_stream;
        c.device = over->device;
    } else {
        c.cuda_stream = nullptr;
    }
    while ((double)nv > (double)c.max_load * (double)c.voxel_capacity) c.voxel_capacity *= 2;
    c.instance_capacity = std::max(c.instance_capacity, nid);
    disc_map* m = nullptr;
    disc_status s = disc_map_create(&c, nullptr, &m);
    if (s != DISC_OK) return s;
    unsigned long long* dk = nullptr;
    int* dl = nullptr;
    if (nv) {
        if (cudaMalloc(&dk, 8 * nv) != cudaSuccess || cudaMalloc(&dl, 4 * nv) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(dk);
            disc_map_destroy(m);
            return DISC_ERR_OOM;
        }
        cudaMemcpyAsync(dk, keys.data(), 8 * nv, cudaMemcpyHostToDevice, m->stream);
        cudaMemcpyAsync(dl, ids.data(), 4 * nv, cudaMemcpyHostToDevice, m->stream);
        cudaMemsetAsync(m->d_flag, 0, sizeof(int), m->stream);
        launch_load_voxels(dk, dl, nv, m->vt, m->d_flag, m->stream);
        unsigned long long unv = (unsigned long long)nv;
        cudaMemcpyAsync(m->vt.used, &unv, sizeof(unv), cudaMemcpyHostToDevice, m->stream);
    }
    if (nid) {
        cudaMemcpyAsync(m->inst.parent, parent.data(), 4 * nid, cudaMemcpyHostToDevice, m->stream);
        cudaMemcpyAsync(m->inst.count, count.data(), 8 * nid, cudaMemcpyHostToDevice, m->stream);
        cudaMemcpyAsync(m->inst.Q, Q.data(), 4 * nid, cudaMemcpyHostToDevice, m->stream);
        cudaMemcpyAsync(m->inst.E, E.data(), 4 * (size_t)nid * D, cudaMemcpyHostToDevice, m->stream);
        cudaMemcpyAsync(m->inst.n_obs, obs.data(), 4 * nid, cudaMemcpyHostToDevice, m->stream);
        cudaMemcpyAsync(m->d_next_id, &nid, sizeof(int), cudaMemcpyHostToDevice, m->stream);
    }
    int flag = 0;
    cudaMemcpyAsync(&flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
    s = cuda_status(cudaStreamSynchronize(m->stream));
    cudaFree(dk);
    cudaFree(dl);
    if (s == DISC_OK && flag) s = DISC_ERR_TABLE_FULL;
    if (s != DISC_OK) {
        disc_map_destroy(m);
        return s;
    }
    m->used_upper = (uint64_t)nv;
    m->next_id_upper = nid;
    *out = m;
    return DISC_OK;
}

uint64_t disc_pack_key(int32_t kx, int32_t ky, int32_t kz)
{
    const uint64_t mask = (1ull << KEY_BITS) - 1;
    return (((uint64_t)(kx + KEY_BIAS) & mask) << (2 * KEY_BITS)) | (((uint64_t)(ky + KEY_BIAS) & mask) << KEY_BITS) |
           ((uint64_t)(kz + KEY_BIAS) & mask);
}

int64_t disc_map_device_bytes(disc_map* m) { return m ? m->mem.bytes : 0; }

int64_t disc_map_kernel_launches(disc_map* m) { return m ? m->launches : 0; }

disc_status disc_map_set_phase_timing(disc_map* m, int32_t enable)
{
    if (!m) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    CK(cudaStreamSynchronize(m->stream));
    collect_timing(m);
    m->timing = enable != 0;
    for (int i = 0; i < PH_COUNT; i++) {
        m->phase_ms[i] = 0.0;
        m->phase_launches[i] = 0;
        m->phase_calls[i] = 0;
    }
    return DISC_OK;
}

disc_status disc_map_phase_times(disc_map* m, double* ms, int64_t* launches, int64_t* calls, int32_t n)
{
    if (!m || n < 0) return DISC_ERR_INVALID_ARG;
    for (int i = 0; i < n && i < PH_COUNT; i++) {
        if (ms) ms[i] = m->phase_ms[i];
        if (launches) launches[i] = m->phase_launches[i];
        if (calls) calls[i] = m->phase_calls[i];
    }
    return DISC_OK;
}

const char* disc_phase_name(int32_t i)
{
    static const char* names[PH_COUNT] = {"clear",     "token_stats", "coverage", "weights", "pool_exact",
                                          "pool_gemm", "backproject", "entries",  "overlap", "score",
                                          "union",     "apply"};
    return (i >= 0 && i < PH_COUNT) ? names[i] : "";
}

disc_status disc_map_get_config(disc_map* m, disc_map_config* out)
{
    if (!m || !out) return DISC_ERR_INVALID_ARG;
    *out = m->cfg;
    out->voxel_capacity = (int64_t)(m->vt.mask + 1);
    out->instance_capacity = m->inst.cap;
    out->cuda_stream = m->stream;
    return DISC_OK;
}

const char* disc_status_str(int32_t s)
{
    switch (s) {
        case DISC_OK: return "ok";
        case DISC_ERR_INVALID_ARG: return "invalid argument";
        case DISC_ERR_OOM: return "out of memory";
        case DISC_ERR_TABLE_FULL: return "hash table full";
        case DISC_ERR_CUDA: return "CUDA error";
        case DISC_ERR_TIMEOUT: return "device wait timed out";
        case DISC_ERR_BUDGET: return "over budget";
        case DISC_ERR_RANGE: return "token out of range";
        case DISC_ERR_CAPACITY: return "per-frame capacity exceeded";
        default: return "unknown status";
    }
}

}  // extern "C"
