// Serving loop of libdisc (declared in include/disc.h): many resident maps,
// integrate and query requests from any host thread, continuous batching.
//
// Host orchestration only.  Every request is queued on its map in arrival
// order.  Worker threads, each with a group of its own, repeatedly form a
// batch from what is pending: for each map with work that no other batch
// holds (oldest first, up to the group's maps per batch) the leading frames
// of its queue up to the group's frames per map, stopping at the map's first
// query.  Queries at the head of a queue run first, so a query sees exactly
// the frames submitted before it.  The batch runs as one group call (every
// kernel spans all its maps); requests that arrive meanwhile join a later
// batch.  With two workers, one batch's host work, input copies and
// stateless kernels overlap the other's frame chain.  Maps are admitted
// against a device-memory budget.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/disc.h"

#include <cuda_runtime.h>

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    bool is_query = false;
    // frame: inputs copied at submission into pinned host memory
    disc_frame frame{};
    unsigned char* host = nullptr;  // pinned block holding depth | labels | tokens | global_embed
    size_t host_bytes = 0;
    // query
    std::vector<float> q;
    int nq = 0, k = 0;
    Clock::time_point t_submit;
};

struct Result {
    bool done = false;
    bool claimed = false;  // a waiter holds this ticket (a ticket has one waiter)
    disc_status status = DISC_OK;
    disc_frame_stats stats{};
    std::vector<int32_t> ids;
    std::vector<float> scores;
    double latency_ms = 0.0;
};

struct MapSlot {
    disc_map* m = nullptr;
    bool open = false;
    bool closing = false;
    int64_t bytes = 0;
    std::deque<Request> queue;
    int64_t busy = 0;  // requests of this map inside a running batch (of one worker at a time)
};

}  // namespace

struct disc_server {
    disc_server_config cfg;
    std::vector<disc_group*> groups;  // one per worker
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<MapSlot> maps;
    std::map<int64_t, Result> results;
    int64_t next_ticket = 1;
    int64_t pending = 0;
    int waiting = 0;  // workers waiting for work
    int64_t resident = 0;  // device bytes: group scratch + open maps
    bool stop = false;
    std::vector<std::thread> workers;
    // pinned staging blocks for frame inputs, reused
    std::vector<std::pair<unsigned char*, size_t>> free_blocks;
    // statistics
    std::vector<double> frame_latency;
    int64_t frames_done = 0, queries_done = 0, batches = 0;
    double busy_ms = 0.0;
    Clock::time_point t0;
};

namespace {

unsigned char* take_block(disc_server* s, size_t bytes)
{
    for (size_t i = 0; i < s->free_blocks.size(); i++) {
        if (s->free_blocks[i].second >= bytes) {
            unsigned char* p = s->free_blocks[i].first;
            s->free_blocks.erase(s->free_blocks.begin() + i);
            return p;
        }
    }
    void* p = nullptr;
    if (cudaHostAlloc(&p, bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (unsigned char*)p;
}

void give_block(disc_server* s, unsigned char* p, size_t bytes)
{
    if (p) s->free_blocks.push_back({p, bytes});
}

void finish(disc_server* s, const Request& r, disc_status st, const disc_frame_stats* fs, std::vector<int32_t>* ids,
            std::vector<float>* sc)
{
    Result& res = s->results[r.ticket];
    res.done = true;
    res.status = st;
    if (fs) res.stats = *fs;
    if (ids) res.ids.swap(*ids);
    if (sc) res.scores.swap(*sc);
    res.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r.t_submit).count();
    if (r.is_query) {
        s->queries_done++;
    } else {
        s->frames_done++;
        s->frame_latency.push_back(res.latency_ms);
    }
}

// a map whose queue has work and that no batch holds
bool takeable(const MapSlot& ms) { return ms.busy == 0 && !ms.queue.empty(); }

void worker_loop(disc_server* s, int wi)
{
    const int G = s->cfg.group.max_maps, J = s->cfg.group.frames_per_map;
    disc_group* group = s->groups[wi];
    cudaSetDevice(s->cfg.group.device);
    while (true) {
        std::vector<int> gl;                       // maps of the batch
        std::vector<disc_map*> mp;                 // and their handles, read under the lock: the slot
                                                   // vector may grow (open_map) while the batch runs
        std::vector<std::vector<Request>> frames;  // their frames
        std::vector<std::pair<int, Request>> queries;
        std::vector<disc_map*> qmaps;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // work on a map that another worker's batch holds waits for that
            // batch (its finish wakes the workers)
            s->waiting++;
            s->cv_work.wait(lk, [&] {
                if (s->stop && s->pending == 0) return true;
                for (const MapSlot& ms : s->maps)
                    if (takeable(ms)) return true;
                return false;
            });
            s->waiting--;
            if (s->stop && s->pending == 0) return;
            std::vector<char> free(s->maps.size());
            for (int i = 0; i < (int)s->maps.size(); i++) free[i] = s->maps[i].busy == 0;
            // queries at the head of a queue run before the batch
            for (int i = 0; i < (int)s->maps.size(); i++) {
                MapSlot& ms = s->maps[i];
                while (free[i] && !ms.queue.empty() && ms.queue.front().is_query) {
                    queries.push_back({i, std::move(ms.queue.front())});
                    qmaps.push_back(ms.m);
                    ms.queue.pop_front();
                    ms.busy++;
                }
            }
            // maps with frames waiting, oldest head first
            std::vector<std::pair<Clock::time_point, int>> order;
            for (int i = 0; i < (int)s->maps.size(); i++)
                if (free[i] && !s->maps[i].queue.empty() && !s->maps[i].queue.front().is_query)
                    order.push_back({s->maps[i].queue.front().t_submit, i});
            std::sort(order.begin(), order.end());
            // a fair share of the free maps when other workers wait, so that
            // batches stay in flight side by side under a full load
            const int share = std::min<int>(G, ((int)order.size() + s->waiting) / (s->waiting + 1));
            for (auto& o : order) {
                if ((int)gl.size() == std::max(share, 1)) break;
                MapSlot& ms = s->maps[o.second];
                std::vector<Request> fr;
                while ((int)fr.size() < J && !ms.queue.empty() && !ms.queue.front().is_query) {
                    fr.push_back(std::move(ms.queue.front()));
                    ms.queue.pop_front();
                }
                ms.busy += (int64_t)fr.size();
                gl.push_back(o.second);
                mp.push_back(ms.m);
                frames.push_back(std::move(fr));
            }
            if ((int)gl.size() < (int)order.size() && s->waiting > 0) s->cv_work.notify_one();  // the rest
        }
        // queries (the maps' earlier frames are complete: a map is in one
        // batch at a time and batches are synchronous)
        for (size_t qi = 0; qi < queries.size(); qi++) {
            auto& qr = queries[qi];
            const Request& r = qr.second;
            std::vector<int32_t> ids((size_t)r.nq * r.k);
            std::vector<float> sc((size_t)r.nq * r.k);
            const disc_status st = disc_query_topk(qmaps[qi], r.q.data(), r.nq, r.k, ids.data(), sc.data());
            std::lock_guard<std::mutex> lk(s->mu);
            finish(s, r, st, nullptr, &ids, &sc);
            s->maps[qr.first].busy--;
            s->pending--;
        }
        if (!queries.empty()) {
            s->cv_done.notify_all();
            s->cv_work.notify_all();  // their maps are free again
        }
        if (gl.empty()) continue;
        // the batch: one group call over all its maps
        const int n = (int)gl.size();
        std::vector<std::vector<disc_frame>> fv(n);
        std::vector<const disc_frame*> fptr(n);
        std::vector<int32_t> cnt(n), done(n);
        std::vector<std::vector<disc_frame_stats>> st(n);
        std::vector<disc_frame_stats*> sptr(n);
        for (int i = 0; i < n; i++) {
            for (const Request& r : frames[i]) fv[i].push_back(r.frame);
            fptr[i] = fv[i].data();
            cnt[i] = (int32_t)fv[i].size();
            st[i].resize(std::max<size_t>(fv[i].size(), 1));
            sptr[i] = st[i].data();
        }
        const auto tb = Clock::now();
        const disc_status gst =
            disc_group_integrate(group, mp.data(), n, fptr.data(), cnt.data(), sptr.data(), done.data());
        const double ms = std::chrono::duration<double, std::milli>(Clock::now() - tb).count();
        {
            // frames before a map's first failure are done, the failing frame
            // fails on its own, the map's later frames (stopped only because
            // they followed it in this batch) go back to the head of its queue
            std::lock_guard<std::mutex> lk(s->mu);
            s->batches++;
            s->busy_ms += ms;
            for (int i = 0; i < n; i++) {
                MapSlot& slot = s->maps[gl[i]];
                int settled = 0;
                for (int j = 0; j < cnt[i]; j++) {
                    const Request& r = frames[i][j];
                    if (j < done[i]) {
                        finish(s, r, DISC_OK, &st[i][j], nullptr, nullptr);
                    } else if (j == done[i]) {
                        disc_status fst = (disc_status)st[i][j].status;
                        // not run on the device: the call's own failure, else the host checks
                        if (fst == DISC_OK) fst = gst != DISC_OK ? gst : DISC_ERR_INVALID_ARG;
                        finish(s, r, fst, &st[i][j], nullptr, nullptr);
                    } else {
                        break;
                    }
                    give_block(s, r.host, r.host_bytes);
                    settled++;
                }
                for (int j = cnt[i] - 1; j >= settled; j--) slot.queue.push_front(std::move(frames[i][j]));
                slot.busy -= cnt[i];
                s->pending -= settled;
            }
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();  // the batch's maps are free for any worker
    }
}

}  // namespace

extern "C" {

disc_status disc_server_create(const disc_server_config* cfg, disc_server** out)
{
    if (!cfg || !out) return DISC_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->max_queue <= 0 || cfg->hbm_budget_bytes <= 0 || cfg->workers < 0 || cfg->workers > 4)
        return DISC_ERR_INVALID_ARG;
    disc_server* s = new disc_server();
    s->cfg = *cfg;
    if (s->cfg.workers == 0) s->cfg.workers = 2;
    disc_status st = DISC_OK;
    for (int i = 0; i < s->cfg.workers && st == DISC_OK; i++) {
        disc_group* g = nullptr;
        st = disc_group_create(&cfg->group, &g);
        if (st == DISC_OK) {
            s->groups.push_back(g);
            s->resident += disc_group_device_bytes(g);
        }
    }
    if (st == DISC_OK && s->resident > cfg->hbm_budget_bytes) st = DISC_ERR_BUDGET;
    if (st != DISC_OK) {
        for (disc_group* g : s->groups) disc_group_destroy(g);
        delete s;
        return st;
    }
    s->t0 = Clock::now();
    for (int i = 0; i < s->cfg.workers; i++) s->workers.emplace_back(worker_loop, s, i);
    *out = s;
    return DISC_OK;
}

disc_status disc_server_open_map(disc_server* s, const disc_map_config* cfg, int32_t* map_id)
{
    if (!s || !cfg || !map_id) return DISC_ERR_INVALID_ARG;
    const disc_group_config& g = s->cfg.group;
    if (cfg->device != g.device || cfg->embed_dim != g.embed_dim || cfg->patch_h != g.patch_h ||
        cfg->patch_w != g.patch_w || cfg->max_width > g.max_width || cfg->max_height > g.max_height ||
        cfg->max_masks > g.max_masks)
        return DISC_ERR_INVALID_ARG;
    // a second token grid needs the group's
    if (cfg->assoc_dim > 0 && (cfg->assoc_dim != g.assoc_dim || cfg->assoc_patch_h != g.assoc_patch_h ||
                               cfg->assoc_patch_w != g.assoc_patch_w))
        return DISC_ERR_INVALID_ARG;
    if (cudaSetDevice(g.device) != cudaSuccess) {
        cudaGetLastError();
        return DISC_ERR_CUDA;
    }
    disc_map_config c = *cfg;
    c.cuda_stream = nullptr;  // the map's own stream; batches run on the group's
    disc_map* m = nullptr;
    disc_status st = disc_map_create(&c, nullptr, &m);
    if (st != DISC_OK) return st;
    const int64_t bytes = disc_map_device_bytes(m);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->resident + bytes > s->cfg.hbm_budget_bytes) {
        disc_map_destroy(m);
        return DISC_ERR_BUDGET;
    }
    int id = -1;
    for (int i = 0; i < (int)s->maps.size(); i++)
        if (!s->maps[i].open && !s->maps[i].m) id = i;
    if (id < 0) {
        id = (int)s->maps.size();
        s->maps.emplace_back();
    }
    MapSlot& ms = s->maps[id];
    ms.m = m;
    ms.open = true;
    ms.closing = false;
    ms.bytes = bytes;
    s->resident += bytes;
    *map_id = id;
    return DISC_OK;
}

disc_map* disc_server_map(disc_server* s, int32_t map_id)
{
    if (!s) return nullptr;
    std::lock_guard<std::mutex> lk(s->mu);
    if (map_id < 0 || map_id >= (int)s->maps.size() || !s->maps[map_id].open) return nullptr;
    return s->maps[map_id].m;
}

disc_status disc_server_close_map(disc_server* s, int32_t map_id)
{
    if (!s) return DISC_ERR_INVALID_ARG;
    disc_map* m = nullptr;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (map_id < 0 || map_id >= (int)s->maps.size() || !s->maps[map_id].open) return DISC_ERR_INVALID_ARG;
        MapSlot& ms = s->maps[map_id];
        ms.closing = true;  // no new requests
        s->cv_done.wait(lk, [&] { return ms.queue.empty() && ms.busy == 0; });
        m = ms.m;
        s->resident -= ms.bytes;
        ms.m = nullptr;
        ms.open = false;
    }
    disc_map_destroy(m);
    return DISC_OK;
}

}  // extern "C"

namespace {

// Queue one frame.  borrow: the request keeps the caller's pointers (read
// when its batch runs); otherwise the inputs are copied into a pinned block
// of the server now.
disc_status submit_frame(disc_server* s, int32_t map_id, const disc_frame* f, int64_t* ticket, bool borrow)
{
    if (!s || !f || !ticket || !f->depth || !f->labels || !f->tokens || f->width <= 0 || f->height <= 0)
        return DISC_ERR_INVALID_ARG;
    if (borrow) {
        Request r;
        r.t_submit = Clock::now();
        r.frame = *f;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (map_id < 0 || map_id >= (int)s->maps.size() || !s->maps[map_id].open || s->maps[map_id].closing)
                return DISC_ERR_INVALID_ARG;
            if (s->pending >= s->cfg.max_queue) return DISC_ERR_BUDGET;
            r.ticket = s->next_ticket++;
            *ticket = r.ticket;
            s->results[r.ticket];
            s->maps[map_id].queue.push_back(std::move(r));
            s->pending++;
        }
        s->cv_work.notify_one();
        return DISC_OK;
    }
    const disc_group_config& g = s->cfg.group;
    if (cudaSetDevice(g.device) != cudaSuccess) {
        cudaGetLastError();
        return DISC_ERR_CUDA;
    }
    const size_t npx = (size_t)f->width * f->height;
    const size_t tok = (size_t)g.patch_h * g.patch_w * g.embed_dim * (f->token_dtype == DISC_TOKENS_BF16 ? 2 : 4);
    const size_t od = 0, ol = od + ((4 * npx + 15) & ~(size_t)15), ot = ol + ((2 * npx + 15) & ~(size_t)15);
    const size_t atok = f->assoc_tokens && g.assoc_dim > 0 ? (size_t)g.assoc_patch_h * g.assoc_patch_w * g.assoc_dim *
                                                                 (f->token_dtype == DISC_TOKENS_BF16 ? 2 : 4)
                                                           : 0;
    const size_t og = ot + ((tok + 15) & ~(size_t)15), oa = og + ((4 * (size_t)g.embed_dim + 15) & ~(size_t)15);
    const size_t total = oa + atok;
    auto copy = [&](void* dst, const void* src, size_t n) {
        if (!f->inputs_on_device) {
            std::memcpy(dst, src, n);
            return true;
        }
        return cudaMemcpy(dst, src, n, cudaMemcpyDeviceToHost) == cudaSuccess;
    };
    Request r;
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (map_id < 0 || map_id >= (int)s->maps.size() || !s->maps[map_id].open || s->maps[map_id].closing)
            return DISC_ERR_INVALID_ARG;
        if (s->pending >= s->cfg.max_queue) return DISC_ERR_BUDGET;
        r.host = take_block(s, total);
        if (!r.host) return DISC_ERR_OOM;
    }
    r.host_bytes = total;
    // the caller's inputs, copied now (host or device pointers)
    bool ok = copy(r.host + od, f->depth, 4 * npx) && copy(r.host + ol, f->labels, 2 * npx) &&
              copy(r.host + ot, f->tokens, tok);
    if (ok && f->global_embed) ok = copy(r.host + og, f->global_embed, 4 * (size_t)g.embed_dim);
    if (ok && atok) ok = copy(r.host + oa, f->assoc_tokens, atok);
    if (!ok) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(s->mu);
        give_block(s, r.host, total);
        return DISC_ERR_CUDA;
    }
    r.frame = *f;
    r.frame.depth = (const float*)(r.host + od);
    r.frame.labels = (const uint16_t*)(r.host + ol);
    r.frame.tokens = r.host + ot;
    r.frame.global_embed = f->global_embed ? (const float*)(r.host + og) : nullptr;
    r.frame.assoc_tokens = atok ? r.host + oa : nullptr;
    r.frame.inputs_on_device = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        // the map may have been closed while the inputs were copied
        if (!s->maps[map_id].open || s->maps[map_id].closing) {
            give_block(s, r.host, total);
            return DISC_ERR_INVALID_ARG;
        }
        r.ticket = s->next_ticket++;
        *ticket = r.ticket;
        s->results[r.ticket];
        s->maps[map_id].queue.push_back(std::move(r));
        s->pending++;
    }
    s->cv_work.notify_one();
    return DISC_OK;
}

}  // namespace

extern "C" {

disc_status disc_server_submit_frame(disc_server* s, int32_t map_id, const disc_frame* f, int64_t* ticket)
{
    return submit_frame(s, map_id, f, ticket, false);
}

disc_status disc_server_submit_frame_borrowed(disc_server* s, int32_t map_id, const disc_frame* f, int64_t* ticket)
{
    return submit_frame(s, map_id, f, ticket, true);
}

disc_status disc_server_submit_query(disc_server* s, int32_t map_id, const float* q, int32_t nq, int32_t k,
                                     int64_t* ticket)
{
    if (!s || !q || nq <= 0 || k <= 0 || !ticket) return DISC_ERR_INVALID_ARG;
    Request r;
    r.is_query = true;
    r.t_submit = Clock::now();
    r.nq = nq;
    r.k = k;
    r.q.assign(q, q + (size_t)nq * s->cfg.group.embed_dim);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (map_id < 0 || map_id >= (int)s->maps.size() || !s->maps[map_id].open || s->maps[map_id].closing)
            return DISC_ERR_INVALID_ARG;
        if (s->pending >= s->cfg.max_queue) return DISC_ERR_BUDGET;
        r.ticket = s->next_ticket++;
        *ticket = r.ticket;
        s->results[r.ticket];
        s->maps[map_id].queue.push_back(std::move(r));
        s->pending++;
    }
    s->cv_work.notify_one();
    return DISC_OK;
}

disc_status disc_server_wait(disc_server* s, int64_t ticket, disc_frame_stats* stats, int32_t* ids, float* scores,
                             double* latency_ms)
{
    if (!s) return DISC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    // a ticket has one waiter: a second thread waiting on it (or on one
    // already returned) is refused instead of sharing the entry
    if (it == s->results.end() || it->second.claimed) return DISC_ERR_INVALID_ARG;
    it->second.claimed = true;
    s->cv_done.wait(lk, [&] { return it->second.done; });
    Result& r = it->second;
    const disc_status st = r.status;
    if (stats) *stats = r.stats;
    if (ids && !r.ids.empty()) std::memcpy(ids, r.ids.data(), sizeof(int32_t) * r.ids.size());
    if (scores && !r.scores.empty()) std::memcpy(scores, r.scores.data(), sizeof(float) * r.scores.size());
    if (latency_ms) *latency_ms = r.latency_ms;
    s->results.erase(it);
    return st;
}

disc_status disc_server_stats(disc_server* s, disc_server_report* out)
{
    if (!s || !out) return DISC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->frames = s->frames_done;
    out->queries = s->queries_done;
    out->batches = s->batches;
    out->pending = s->pending;
    out->resident_bytes = s->resident;
    out->busy_ms = s->busy_ms;
    out->wall_ms = std::chrono::duration<double, std::milli>(Clock::now() - s->t0).count();
    if (!s->frame_latency.empty()) {
        std::vector<double> v = s->frame_latency;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const size_t i = std::min(v.size() - 1, (size_t)(p / 100.0 * (double)(v.size() - 1) + 0.5));
            return v[i];
        };
        out->p50_ms = pct(50.0);
        out->p99_ms = pct(99.0);
    }
    return DISC_OK;
}

disc_status disc_server_reset_stats(disc_server* s)
{
    if (!s) return DISC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    s->frame_latency.clear();
    s->frames_done = s->queries_done = s->batches = 0;
    s->busy_ms = 0.0;
    s->t0 = Clock::now();
    return DISC_OK;
}

void disc_server_destroy(disc_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (std::thread& t : s->workers)
        if (t.joinable()) t.join();
    for (MapSlot& ms : s->maps)
        if (ms.m) disc_map_destroy(ms.m);
    for (disc_group* g : s->groups) disc_group_destroy(g);
    for (auto& b : s->free_blocks) cudaFreeHost(b.first);
    delete s;
}

}  // extern "C"
