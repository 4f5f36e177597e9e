// C ABI of libdisc (declared in include/disc.h): map and group lifetime,
// frame integration, queries, export and checkpoints.  Host code only
// orchestrates: every step of a frame runs in the kernels of k_features.cu,
// k_gemm.cu, k_geometry.cu and k_serial.cu, enqueued on the stream of the
// map (its own calls) or of the group (batches over many maps).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include <cuda.h>

#include "disc_common.cuh"
#include "kernels.h"

using namespace disc;

namespace {

constexpr int PAIR_CAP = 8192;   // distinct (segment, instance) overlaps per frame (k_serial.cu)

// Host-side fault injection (tests): after this many more device
// allocations, the next one fails as if the device were out of memory
// (-1: off).  Set by disc_debug_fail_alloc_after or the environment variable
// DISC_FAULT_ALLOC_AFTER.
std::atomic<int64_t> g_fail_alloc_after{[] {
    const char* e = std::getenv("DISC_FAULT_ALLOC_AFTER");
    return e ? (int64_t)std::atoll(e) : (int64_t)-1;
}()};

bool injected_alloc_failure()
{
    int64_t n = g_fail_alloc_after.load();
    while (n >= 0) {
        if (n == 0) return true;  // stays at 0: every later allocation fails too, until reset
        if (g_fail_alloc_after.compare_exchange_weak(n, n - 1)) return false;
    }
    return false;
}

struct DevAlloc {
    std::vector<void*> ptrs;
    int64_t bytes = 0;
    bool failed = false;
    template <typename T>
    T* get(size_t n)
    {
        void* p = nullptr;
        if (n == 0) n = 1;
        if (injected_alloc_failure()) {
            failed = true;
            return nullptr;
        }
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

// The frames one call integrates into one map.
struct Work {
    disc_map* m = nullptr;
    const disc_frame* frames = nullptr;
    int n = 0;                        // frames asked for
    int valid = 0;                    // leading frames that pass the host checks
    disc_frame_stats* stats = nullptr;
    int done = 0;                     // frames integrated
    disc_status status = DISC_OK;     // first failure of this map
    std::vector<int> hist_idx;        // counters of each enqueued frame in the call's history
    int prev_idx = -1;                // history entry of the map's last frame in an unfinished
                                      // asynchronous call (its first frame waits on that one's status)
};

// An asynchronous call whose work may still be on the device.  A runner
// holds at most two; each writes its counters to its own half (region) of
// the history buffer, and its results reach the caller's pointers when it
// is finished (finish_oldest).
struct AsyncCall {
    std::vector<Work> w;
    int region = 0;
    std::vector<uint64_t> px_mark;    // per map: its px_total when the call was enqueued
    std::vector<int64_t> masks_mark;  // per map: its masks_total then
    int32_t* n_done = nullptr;        // the caller's outputs (one n_done per map)
    disc_status* result = nullptr;
};

// What one batch of frame slots needs besides the maps themselves: the
// slots' scratch, the per-batch parameter block, input staging, the per-frame
// counters of the running call, captured launch sequences and phase timing.
// A map owns one for its own calls (one map per batch); a group owns one for
// batches that span many maps.
struct Runner {
    int device = 0;
    cudaStream_t stream = nullptr;   // the caller's stream (everything when not pipelined)
    cudaStream_t stream2 = nullptr;  // stateless part of pipelined batches, lowest priority
    cudaStream_t stream3 = nullptr;  // serial part of pipelined batches, highest priority
    cudaEvent_t ev_join = nullptr;   // call start on the caller's stream, call end on stream3
    CUgreenCtx green[2] = {};        // SM partitions of stream3 / stream2 (when the driver offers them)
    int serial_sms = -1;             // SMs of the serial partition; < 0: no pipelining
    DevAlloc mem;
    int D = 0, P = 0, Ph = 0, Pw = 0, Kpad = 0, MM = 1, Npad_max = 16;
    int Hmax = 0, Wmax = 0, Mmax = 0;
    int Gmax = 1, Jmax = 1, S = 1;  // maps per batch, frames per map, slots = Gmax * Jmax
    size_t px_cap = 0;
    // Two sets of slot scratch and parameter blocks: batch b uses set b % 2,
    // so the stateless part of batch b + 1 runs while the serial part of
    // batch b still reads its own set.
    BatchScratch bs[2] = {};
    // parameter block: FrameParams[S] | MapRefs[Gmax] | slot_of[Gmax * Jmax] | prev_hist[Gmax]
    unsigned char* d_param[2] = {};
    size_t off_refs = 0, off_slot = 0, off_prev = 0, param_bytes = 0;
    cudaEvent_t ev_state[2] = {}, ev_serial[2] = {};  // stateless / serial part of the set's last batch done
    int cur = 0;                                        // set of the next batch
    FrameCounters* d_hist = nullptr;  // [2 hist_cap] per-frame counters: a synchronous call uses the
    int hist_cap = 0;                 // first half, asynchronous calls alternate between the halves
    FrameCounters* h_hist = nullptr;  // pinned [2 hist_cap]: asynchronous calls' counters
    unsigned long long* h_used = nullptr;  // pinned [2 Gmax]: their maps' voxel counts at the end
    cudaEvent_t ev_done[2] = {};      // an asynchronous call's work done, by history half
    std::deque<AsyncCall> pend;       // unfinished asynchronous calls, oldest first (at most two)
    cudaStream_t stream_in = nullptr; // host-to-device copies of host inputs
    unsigned long long* d_room = nullptr;  // [2 Gmax] per map of a batch: voxel count, pairs of its frames
    AbsentHash ah{};                  // voxels absent at a batch's start (k_lookup .. k_commit), grown on demand
    uint64_t ah_cap = 0;
    int* d_merged = nullptr;          // [Gmax] per map of a batch: some frame merged instances
    unsigned long long* h_room = nullptr;  // pinned copy of d_room
    cudaEvent_t ev_room = nullptr;
    cudaEvent_t ev_in_ready[2] = {}, ev_in_free[2] = {};  // staging set k filled / read by its last batch
    cudaEvent_t ev_in_half[2] = {};                        // the second half of set k filled
    float* d_depth = nullptr;         // staging of host inputs: two sets (one per scratch set) of one
                                      // slot per frame of a batch
    uint16_t* d_labels = nullptr;
    unsigned char* d_tokens = nullptr;
    float* d_gembed = nullptr;
    // The second token grid (association features), when the runner serves
    // maps that have one: a second view of the feature kernels, with its own
    // FrameParams per slot in the parameter block and its own slot scratch
    // (sharing the primary slots' counters).
    int Da = 0, Pha = 0, Pwa = 0, Pa = 0, Kpad_a = 0;
    BatchScratch bsa[2] = {};
    size_t off_fpa = 0;
    unsigned char* d_atok = nullptr;  // staging of host association tokens (two sets)
    // launch schedule (disc_*_set_schedule, disc_*_autotune)
    int geo_chunk = GEOMETRY_CHUNK;   // frames per back-projection / entries / DBSCAN launch
    int cta_scale = 4;                // serial kernels' CTAs in quarters of the default count
    int probe_width = 1;              // lanes per key of the batch's voxel-table lookup
    int assoc_cluster = 0;            // CTAs per map of the association kernel (0: automatic)
    int batch_split = 0;              // smaller batches per call that fits one (0: automatic)
    bool graphs_off = false;
    std::map<long long, BatchGraph> graphs;
    std::map<long long, int> shapes_seen;  // batch shapes launched directly so far
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
    int last_set = 0, last_slot = 0, last_M = 0;  // the most recent frame
    bool have_frame = false;

    const FrameParams* fps(int k) const { return (const FrameParams*)d_param[k]; }
    const MapRefs* refs(int k) const { return (const MapRefs*)(d_param[k] + off_refs); }
    const int* slot_of(int k) const { return (const int*)(d_param[k] + off_slot); }
    const FrameParams* fpa(int k) const { return (const FrameParams*)(d_param[k] + off_fpa); }
    const int* prev_hist(int k) const { return (const int*)(d_param[k] + off_prev); }
};

struct disc_map {
    disc_map_config cfg;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevAlloc mem;
    VoxelTable vt{};
    Instances inst{};
    SerialScratch ss{};
    int* d_next_id = nullptr;
    int* d_flag = nullptr;
    int D = 0, P = 0, Kpad = 0, MM = 1;
    // host-side bounds that avoid a synchronisation per frame
    uint64_t used_upper = 0;
    int64_t next_id_upper = 0;
    uint64_t px_total = 0;      // pixels of every frame enqueued on the map (bounds its new voxels)
    int64_t masks_total = 0;    // masks of every frame enqueued (bounds the ids handed out)
    Runner* pend_run = nullptr; // the runner holding the map's unfinished asynchronous calls
    int pend_calls = 0;         // how many of them
    int pend_last = -1;         // history entry of the map's last frame in them
    Runner* run = nullptr;  // created by the map's first own integration call
    bool timing_wanted = false;
    unsigned char* qscratch = nullptr;  // query buffers, grown on demand and kept
    size_t qcap = 0;
    bool finalized = false;  // after disc_map_finalize: no more frames
};

struct disc_group {
    disc_group_config cfg;
    bool own_stream = false;
    Runner run;
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
    if (c.precision != DISC_FP32 && c.precision != DISC_BF16 && c.precision != DISC_FP8_E4M3) return false;
    if (c.overlap_dilation != 0 && c.overlap_dilation != 1) return false;
    if (c.assoc_dim < 0 || c.assoc_dim > 4096) return false;
    if (c.assoc_dim > 0 && (c.assoc_patch_h <= 0 || c.assoc_patch_w <= 0 ||
                            (int64_t)c.assoc_patch_h * c.assoc_patch_w > 16384 ||
                            coverage_smem_bytes(c.max_masks, c.assoc_patch_w) > 200 * 1024))
        return false;
    // DBSCAN cells at least a voxel wide keep cell coordinates in key range
    if (!(c.dbscan_eps >= 0.0f) || (c.dbscan_eps > 0.0f && (c.dbscan_eps < c.voxel_size || c.dbscan_min_pts < 1)))
        return false;
    return true;
}

// kernel attributes (dynamic shared memory above 48 KB), once per process
// (maps and groups may be created from several host threads at once)
disc_status set_kernel_attrs()
{
    static std::mutex mu;
    static bool done = false;
    std::lock_guard<std::mutex> lk(mu);
    if (done) return DISC_OK;
    cudaError_t e = set_feature_kernel_attrs(200 * 1024);
    if (e == cudaSuccess) e = set_gemm_kernel_attrs();
    if (e == cudaSuccess) e = set_serial_kernel_attrs();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DISC_ERR_CUDA;
    }
    done = true;
    return DISC_OK;
}

// ---- runner ----------------------------------------------------------------------
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Driver entry points of the green-context API, looked up through the
// runtime (the library does not link the driver directly).
struct GreenApi {
    decltype(&::cuDeviceGet) deviceGet = nullptr;
    decltype(&::cuDeviceGetDevResource) getResource = nullptr;
    decltype(&::cuDevSmResourceSplitByCount) split = nullptr;
    decltype(&::cuDevResourceGenerateDesc) desc = nullptr;
    decltype(&::cuGreenCtxCreate) create = nullptr;
    decltype(&::cuGreenCtxStreamCreate) stream = nullptr;
    decltype(&::cuGreenCtxDestroy) destroy = nullptr;
    decltype(&::cuStreamDestroy) streamDestroy = nullptr;
    bool ok = false;
};

const GreenApi& green_api()
{
    static GreenApi g = [] {
        GreenApi a;
        auto get = [](const char* name, void** fn) {
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPoint(name, fn, cudaEnableDefault, &q) != cudaSuccess ||
                q != cudaDriverEntryPointSuccess) {
                cudaGetLastError();
                *fn = nullptr;
            }
            return *fn != nullptr;
        };
        a.ok = get("cuDeviceGet", (void**)&a.deviceGet) && get("cuDeviceGetDevResource", (void**)&a.getResource) &&
               get("cuDevSmResourceSplitByCount", (void**)&a.split) &&
               get("cuDevResourceGenerateDesc", (void**)&a.desc) && get("cuGreenCtxCreate", (void**)&a.create) &&
               get("cuGreenCtxStreamCreate", (void**)&a.stream) && get("cuGreenCtxDestroy", (void**)&a.destroy) &&
               get("cuStreamDestroy", (void**)&a.streamDestroy);
        return a;
    }();
    return g;
}

// Green contexts over disjoint SM sets: r.serial_sms SMs for stream3, the rest
// for stream2.  false when the driver does not offer them (nothing is kept).
bool make_green_streams(Runner& r)
{
    const GreenApi& g = green_api();
    if (!g.ok) return false;
    CUdevice dev;
    CUdevResource all, part[1], rest;
    unsigned n = 1;
    CUdevResourceDesc d0, d1;
    if (g.deviceGet(&dev, r.device) != CUDA_SUCCESS ||
        g.getResource(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS ||
        all.sm.smCount < (unsigned)r.serial_sms + 16u ||
        g.split(part, &n, &all, &rest, 0, (unsigned)r.serial_sms) != CUDA_SUCCESS || n != 1 ||
        g.desc(&d0, &part[0], 1) != CUDA_SUCCESS || g.desc(&d1, &rest, 1) != CUDA_SUCCESS)
        return false;
    if (g.create(&r.green[0], d0, dev, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS) return false;
    if (g.create(&r.green[1], d1, dev, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS) {
        g.destroy(r.green[0]);
        r.green[0] = nullptr;
        return false;
    }
    CUstream s3 = nullptr, s2 = nullptr;
    if (g.stream(&s3, r.green[0], CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS ||
        g.stream(&s2, r.green[1], CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS) {
        if (s3) g.streamDestroy(s3);
        g.destroy(r.green[0]);
        g.destroy(r.green[1]);
        r.green[0] = r.green[1] = nullptr;
        return false;
    }
    r.stream3 = (cudaStream_t)s3;
    r.stream2 = (cudaStream_t)s2;
    return true;
}

disc_status runner_init(Runner& r, int device, cudaStream_t stream, int D, int Ph, int Pw, int Hmax, int Wmax,
                        int Mmax, int Gmax, int Jmax, int serial_sms, int Da, int Pha, int Pwa)
{
    r.Da = Da > 0 ? Da : 0;
    r.Pha = r.Da ? Pha : 0;
    r.Pwa = r.Da ? Pwa : 0;
    r.Pa = r.Pha * r.Pwa;
    r.Kpad_a = (r.Pa + GEMM_KC - 1) / GEMM_KC * GEMM_KC;
    r.device = device;
    r.serial_sms = serial_sms == 0 ? -1 : serial_sms;  // overlap only on request: measured slower here
    r.stream = stream;
    r.D = D;
    r.Ph = Ph;
    r.Pw = Pw;
    r.P = Ph * Pw;
    r.Kpad = (r.P + GEMM_KC - 1) / GEMM_KC * GEMM_KC;
    r.Hmax = Hmax;
    r.Wmax = Wmax;
    r.Mmax = Mmax;
    r.MM = std::max(1, Mmax);
    r.Npad_max = std::max(16, (r.MM + 15) / 16 * 16);
    r.Gmax = Gmax;
    r.Jmax = Jmax;
    r.S = Gmax * Jmax;
    const int P = r.P, MM = r.MM, B = r.S;
    const uint64_t npx = (uint64_t)Wmax * Hmax;
    const uint64_t scap = next_pow2(npx + npx / 2);  // per-frame hashes: load <= 2/3
    r.px_cap = npx;
    DevAlloc& a = r.mem;
    r.off_refs = align256(sizeof(FrameParams) * B);
    r.off_slot = r.off_refs + align256(sizeof(MapRefs) * Gmax);
    r.off_prev = r.off_slot + align256(sizeof(int) * Gmax * Jmax);
    r.off_fpa = r.off_prev + align256(sizeof(int) * Gmax);
    r.param_bytes = r.off_fpa + (r.Da ? align256(sizeof(FrameParams) * B) : 0);
    for (int k = 0; k < 2; k++) {
        r.d_param[k] = a.get<unsigned char>(r.param_bytes);
        BatchScratch& bs = r.bs[k];
        bs.sD = D;
        bs.sP = P;
        bs.sMM = MM;
        bs.sMMP = (long long)MM * P;
        bs.sW = (long long)r.Npad_max * r.Kpad;
        bs.sMMD = (long long)MM * D;
        bs.sS = 5LL * MM;
        bs.scap = (long long)scap;
        bs.sK = r.Kpad;
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
        sc.qexp = a.get<int32_t>((size_t)B * P);
        sc.qmul = a.get<float>((size_t)B * r.Kpad);
        sc.qerr = a.get<float>((size_t)B * P);
        sc.qnrm = a.get<float>((size_t)B * P);
        sc.qexpm = a.get<int32_t>((size_t)B * MM);
        sc.W8 = a.get<uint8_t>((size_t)B * bs.sW);
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
        sc.pkey = a.get<unsigned long long>((size_t)B * scap);
        sc.pcnt = a.get<int32_t>((size_t)B * scap);
        sc.plist = a.get<int32_t>((size_t)B * scap);
        sc.aent = a.get<int32_t>((size_t)B * 2 * scap);  // per slot: aent [scap], aslot [scap]
        sc.newcnt = a.get<int32_t>((size_t)B * MM);
        sc.ctr = a.get<FrameCounters>(B);
    }
    r.d_depth = a.get<float>((size_t)2 * B * npx);
    r.d_labels = a.get<uint16_t>((size_t)2 * B * npx);
    r.d_tokens = a.get<unsigned char>((size_t)2 * B * P * D * 4);
    r.d_gembed = a.get<float>((size_t)2 * B * D);
    r.d_room = a.get<unsigned long long>((size_t)2 * Gmax);
    r.d_merged = a.get<int>((size_t)Gmax);
    if (r.Da) {
        // the second grid's view: the feature kernels' arrays at its sizes;
        // the counters are the primary slots' own
        const int Da_ = r.Da, Pa = r.Pa, Ka = r.Kpad_a;
        r.d_atok = a.get<unsigned char>((size_t)2 * B * Pa * Da_ * 4);
        for (int k = 0; k < 2; k++) {
            BatchScratch& v = r.bsa[k];
            v.sD = Da_;
            v.sP = Pa;
            v.sMM = MM;
            v.sMMP = (long long)MM * Pa;
            v.sW = (long long)r.Npad_max * Ka;
            v.sMMD = (long long)MM * Da_;
            v.sS = 5LL * MM;
            v.sK = Ka;
            Scratch& sc = v.base;
            sc.sumF = a.get<long long>((size_t)B * Da_);
            sc.fbar = a.get<float>((size_t)B * Da_);
            sc.gvec = a.get<float>((size_t)B * Da_);
            sc.gg = a.get<long long>(B);
            sc.nsum = a.get<long long>(B);
            sc.dotg = a.get<long long>((size_t)B * Pa);
            sc.ffp = a.get<long long>((size_t)B * Pa);
            sc.nrm = a.get<float>((size_t)B * Pa);
            sc.Dp = a.get<float>((size_t)B * Pa);
            sc.cosg = a.get<float>((size_t)B * Pa);
            sc.fnorm = a.get<float>((size_t)B * Pa);
            sc.qexp = a.get<int32_t>((size_t)B * Pa);
            sc.qmul = a.get<float>((size_t)B * Ka);
            sc.qerr = a.get<float>((size_t)B * Pa);
            sc.qnrm = a.get<float>((size_t)B * Pa);
            sc.qexpm = a.get<int32_t>((size_t)B * MM);
            sc.W8 = a.get<uint8_t>((size_t)B * v.sW);
            sc.cov = a.get<int32_t>((size_t)B * MM * Pa);
            sc.npix = a.get<int32_t>((size_t)B * MM);
            sc.W = a.get<float>((size_t)B * v.sW);
            sc.S = a.get<float>((size_t)B * 5 * MM);
            sc.Bm = a.get<float>((size_t)B * MM);
            sc.Ecan = a.get<float>((size_t)B * MM * Da_);
            sc.Efast = a.get<float>((size_t)B * MM * Da_);
            sc.ctr = r.bs[k].base.ctr;
        }
    }
    if (a.failed) return DISC_ERR_OOM;
    // Pipelined batches put the serial part (a latency-bound chain of small
    // launches) on its own partition of serial_sms SMs and the stateless part
    // of the next batch on the rest, so the chain never waits for SMs that
    // long stateless blocks hold.  Without green contexts: two streams of
    // highest / lowest priority.
    if (r.serial_sms < 0 || !make_green_streams(r)) {
        int prio_lo = 0, prio_hi = 0;
        CK(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        CK(cudaStreamCreateWithPriority(&r.stream2, cudaStreamNonBlocking, prio_lo));
        CK(cudaStreamCreateWithPriority(&r.stream3, cudaStreamNonBlocking, prio_hi));
    }
    CK(cudaEventCreateWithFlags(&r.ev_join, cudaEventDisableTiming));
    CK(cudaStreamCreateWithFlags(&r.stream_in, cudaStreamNonBlocking));
    CK(cudaHostAlloc(&r.h_room, sizeof(unsigned long long) * 2 * Gmax, cudaHostAllocDefault));
    CK(cudaHostAlloc(&r.h_used, sizeof(unsigned long long) * 2 * Gmax, cudaHostAllocDefault));
    CK(cudaEventCreateWithFlags(&r.ev_room, cudaEventDisableTiming));
    for (int k = 0; k < 2; k++) CK(cudaEventCreateWithFlags(&r.ev_done[k], cudaEventDisableTiming));
    for (int k = 0; k < 2; k++) {
        CK(cudaEventCreateWithFlags(&r.ev_in_ready[k], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&r.ev_in_half[k], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&r.ev_in_free[k], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&r.ev_state[k], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&r.ev_serial[k], cudaEventDisableTiming));
    }
    cudaStream_t s = r.stream;
    for (int k = 0; k < 2; k++) {
        const BatchScratch& bs = r.bs[k];
        const Scratch& sc = bs.base;
        CK(cudaMemsetAsync(r.d_param[k], 0, r.param_bytes, s));
        CK(cudaMemsetAsync(sc.ctr, 0, sizeof(FrameCounters) * B, s));
        CK(cudaMemsetAsync(sc.W, 0, sizeof(float) * (size_t)B * bs.sW, s));
        CK(cudaMemsetAsync(sc.W8, 0, (size_t)B * bs.sW, s));
        CK(cudaMemsetAsync(sc.qmul, 0, sizeof(float) * (size_t)B * r.Kpad, s));
        CK(cudaMemsetAsync(sc.qexpm, 0, sizeof(int32_t) * (size_t)B * MM, s));
        CK(cudaMemsetAsync(sc.cov, 0, sizeof(int32_t) * (size_t)B * MM * P, s));
        CK(cudaMemsetAsync(sc.sslot, 0, sizeof(SegSlot) * B * scap, s));
        CK(cudaMemsetAsync(sc.pkey, 0xff, sizeof(unsigned long long) * B * scap, s));
        CK(cudaMemsetAsync(sc.pcnt, 0, sizeof(int32_t) * B * scap, s));
        CK(cudaMemsetAsync(sc.newcnt, 0, sizeof(int32_t) * B * MM, s));
        CK(cudaMemsetAsync(sc.Efast, 0, sizeof(float) * (size_t)B * MM * D, s));
        CK(cudaMemsetAsync(sc.Ecan, 0, sizeof(float) * (size_t)B * MM * D, s));
        if (r.Da) {
            const BatchScratch& v = r.bsa[k];
            CK(cudaMemsetAsync(v.base.W, 0, sizeof(float) * (size_t)B * v.sW, s));
            CK(cudaMemsetAsync(v.base.W8, 0, (size_t)B * v.sW, s));
            CK(cudaMemsetAsync(v.base.qmul, 0, sizeof(float) * (size_t)B * r.Kpad_a, s));
            CK(cudaMemsetAsync(v.base.qexpm, 0, sizeof(int32_t) * (size_t)B * MM, s));
            CK(cudaMemsetAsync(v.base.Ecan, 0, sizeof(float) * (size_t)B * MM * r.Da, s));
            CK(cudaMemsetAsync(v.base.Efast, 0, sizeof(float) * (size_t)B * MM * r.Da, s));
        }
    }
    return cuda_status(cudaStreamSynchronize(s));
}

void runner_release(Runner& r)
{
    cudaStreamSynchronize(r.stream);
    for (cudaStream_t* sp : {&r.stream2, &r.stream3, &r.stream_in}) {
        if (*sp) {
            cudaStreamSynchronize(*sp);
            cudaStreamDestroy(*sp);
            *sp = nullptr;
        }
    }
    if (r.ev_join) cudaEventDestroy(r.ev_join);
    r.ev_join = nullptr;
    if (r.ev_room) cudaEventDestroy(r.ev_room);
    r.ev_room = nullptr;
    if (r.h_room) cudaFreeHost(r.h_room);
    r.h_room = nullptr;
    if (r.h_used) cudaFreeHost(r.h_used);
    r.h_used = nullptr;
    if (r.h_hist) cudaFreeHost(r.h_hist);
    r.h_hist = nullptr;
    for (int k = 0; k < 2; k++) {
        if (r.ev_done[k]) cudaEventDestroy(r.ev_done[k]);
        r.ev_done[k] = nullptr;
    }
    for (int i = 0; i < 2; i++) {
        if (r.green[i]) green_api().destroy(r.green[i]);
        r.green[i] = nullptr;
    }
    for (int k = 0; k < 2; k++) {
        if (r.ev_state[k]) cudaEventDestroy(r.ev_state[k]);
        if (r.ev_serial[k]) cudaEventDestroy(r.ev_serial[k]);
        if (r.ev_in_ready[k]) cudaEventDestroy(r.ev_in_ready[k]);
        if (r.ev_in_free[k]) cudaEventDestroy(r.ev_in_free[k]);
        if (r.ev_in_half[k]) cudaEventDestroy(r.ev_in_half[k]);
        r.ev_state[k] = r.ev_serial[k] = r.ev_in_ready[k] = r.ev_in_free[k] = r.ev_in_half[k] = nullptr;
    }
    for (cudaEvent_t e : r.ev_pool) cudaEventDestroy(e);
    r.ev_pool.clear();
    for (auto& kv : r.graphs) cudaGraphExecDestroy(kv.second.exec);
    r.graphs.clear();
    r.mem.free_all();
}

// The history buffer for calls of up to n frames (in each of its halves).
// Growing it replaces the buffer: no asynchronous call may be unfinished.
disc_status ensure_hist(Runner& r, int n)
{
    if (n <= r.hist_cap) return DISC_OK;
    if (r.d_hist) r.mem.release(r.d_hist, sizeof(FrameCounters) * 2 * r.hist_cap);
    if (r.h_hist) cudaFreeHost(r.h_hist);
    r.h_hist = nullptr;
    // captured sequences hold the old pointer
    for (auto& kv : r.graphs) cudaGraphExecDestroy(kv.second.exec);
    r.graphs.clear();
    r.shapes_seen.clear();
    const int cap = std::max(n, 2 * r.hist_cap);
    r.d_hist = r.mem.get<FrameCounters>((size_t)2 * cap);
    if (r.mem.failed || cudaHostAlloc(&r.h_hist, sizeof(FrameCounters) * 2 * cap, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        if (r.d_hist) r.mem.release(r.d_hist, sizeof(FrameCounters) * 2 * cap);
        r.mem.failed = false;
        r.hist_cap = 0;
        r.d_hist = nullptr;
        r.h_hist = nullptr;
        return DISC_ERR_OOM;
    }
    r.hist_cap = cap;
    return DISC_OK;
}

// The DBSCAN scratch of both slot sets, allocated when a frame first asks
// for the filter (captured graphs hold the old slot pointers).
disc_status ensure_dbscan(Runner& r)
{
    if (r.bs[0].base.dkey) return DISC_OK;
    const size_t B = r.S, scap = (size_t)r.bs[0].scap, px = r.px_cap;
    DevAlloc& a = r.mem;
    for (int k = 0; k < 2; k++) {
        Scratch& sc = r.bs[k].base;
        sc.dkey = a.get<unsigned long long>(B * scap);
        sc.dcnt = a.get<int32_t>(B * scap);
        sc.dpos = a.get<int32_t>(B * scap);
        sc.dlist = a.get<int32_t>(B * scap);
        sc.dstart = a.get<int32_t>(B * scap);
        sc.dfill = a.get<int32_t>(B * scap);
        sc.dpt = a.get<float4>(B * px);
        sc.dcell = a.get<int32_t>(B * px);
        sc.dorder = a.get<int32_t>(B * px);
        sc.dflag = a.get<unsigned char>(B * px);
        sc.dsp = a.get<float4>(B * px);
        sc.dund = a.get<int32_t>(B * px);
        r.bs[k].spx = (long long)px;
    }
    if (a.failed) {
        a.failed = false;
        for (int k = 0; k < 2; k++) r.bs[k].base.dkey = nullptr;
        return DISC_ERR_OOM;
    }
    for (int k = 0; k < 2; k++) {
        CK(cudaMemsetAsync(r.bs[k].base.dkey, 0, sizeof(unsigned long long) * B * scap, r.stream));
        CK(cudaMemsetAsync(r.bs[k].base.dcnt, 0, sizeof(int32_t) * B * scap, r.stream));
    }  // the slots' n_cells are 0 until a frame with the filter ran in them
    for (auto& kv : r.graphs) cudaGraphExecDestroy(kv.second.exec);
    r.graphs.clear();
    r.shapes_seen.clear();
    return cuda_status(cudaStreamSynchronize(r.stream));
}

// The batch-wide hash of voxels absent at a batch's start, sized for `keys`
// of them at load <= 1/2 (keys bounds the batch's unique (segment, voxel)
// pairs); it grows when a batch could exceed it.  Captured graphs hold its
// old pointers, so they are dropped on growth.
disc_status ensure_absent(Runner& r, uint64_t keys)
{
    const uint64_t cap = next_pow2(std::max<uint64_t>(2 * keys, 1 << 16));
    if (cap <= r.ah_cap) return DISC_OK;
    CK(cudaStreamSynchronize(r.stream3));  // no batch of the runner is using the old one
    CK(cudaStreamSynchronize(r.stream));
    DevAlloc& a = r.mem;
    if (r.ah.key) {
        a.release(r.ah.key, sizeof(unsigned long long) * r.ah_cap);
        a.release(r.ah.val, sizeof(int32_t) * r.ah_cap);
        a.release(r.ah.list, sizeof(int32_t) * r.ah_cap);
        a.release(r.ah.n, sizeof(int32_t));
    }
    r.ah = AbsentHash{};
    r.ah_cap = 0;
    for (auto& kv : r.graphs) cudaGraphExecDestroy(kv.second.exec);
    r.graphs.clear();
    r.shapes_seen.clear();
    AbsentHash h{};
    h.key = a.get<unsigned long long>(cap);
    h.val = a.get<int32_t>(cap);
    h.list = a.get<int32_t>(cap);
    h.n = a.get<int32_t>(1);
    h.mask = cap - 1;
    if (a.failed) {
        a.failed = false;
        if (h.key) a.release(h.key, sizeof(unsigned long long) * cap);
        if (h.val) a.release(h.val, sizeof(int32_t) * cap);
        if (h.list) a.release(h.list, sizeof(int32_t) * cap);
        if (h.n) a.release(h.n, sizeof(int32_t));
        return DISC_ERR_OOM;
    }
    CK(cudaMemsetAsync(h.key, 0, sizeof(unsigned long long) * cap, r.stream));
    CK(cudaMemsetAsync(h.val, 0x7f, sizeof(int32_t) * cap, r.stream));  // 0x7f7f7f7f: above every (j << 9 | m)
    CK(cudaMemsetAsync(h.n, 0, sizeof(int32_t), r.stream));
    disc_status st = cuda_status(cudaStreamSynchronize(r.stream));
    if (st != DISC_OK) return st;
    r.ah = h;
    r.ah_cap = cap;
    return DISC_OK;
}

// ---- map tables --------------------------------------------------------------------
disc_status alloc_voxel_table(disc_map* m, uint64_t cap, VoxelTable* out, cudaStream_t st)
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
    CK(cudaMemsetAsync(t.keys, 0xFF, sizeof(unsigned long long) * cap, st));
    // an empty slot's label reads -1: a lookup racing an insert sees a key
    // with no label yet as absent
    CK(cudaMemsetAsync(t.labels, 0xFF, sizeof(int32_t) * cap, st));
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
    // the scoring copies are copies of the association features when the map
    // has a second grid, else of E
    const int Da = m->cfg.assoc_dim, Ds = Da > 0 ? Da : m->D;
    in.Da = Da;
    in.A = Da > 0 ? m->mem.get<float>((size_t)cap * Da) : nullptr;
    in.Eb = m->cfg.precision == DISC_BF16 ? m->mem.get<uint16_t>((size_t)cap * Ds) : nullptr;
    in.E8 = m->cfg.precision == DISC_FP8_E4M3 ? m->mem.get<uint8_t>((size_t)cap * Ds) : nullptr;
    in.Er = m->cfg.precision == DISC_FP8_E4M3 ? m->mem.get<float>(cap) : nullptr;
    in.n_obs = m->mem.get<int32_t>(cap);
    if (m->mem.failed) {
        m->mem.failed = false;
        if (in.parent) m->mem.release(in.parent, sizeof(int32_t) * cap);
        if (in.count) m->mem.release(in.count, sizeof(long long) * cap);
        if (in.Q) m->mem.release(in.Q, sizeof(float) * cap);
        if (in.E) m->mem.release(in.E, sizeof(float) * (size_t)cap * m->D);
        if (in.A) m->mem.release(in.A, sizeof(float) * (size_t)cap * Da);
        if (in.Eb) m->mem.release(in.Eb, sizeof(uint16_t) * (size_t)cap * Ds);
        if (in.E8) m->mem.release(in.E8, (size_t)cap * Ds);
        if (in.Er) m->mem.release(in.Er, sizeof(float) * cap);
        if (in.n_obs) m->mem.release(in.n_obs, sizeof(int32_t) * cap);
        return DISC_ERR_OOM;
    }
    *out = in;
    return DISC_OK;
}

int read_next_id(disc_map* m, cudaStream_t st)
{
    int v = 0;
    cudaMemcpyAsync(&v, m->d_next_id, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return v;
}

uint64_t read_used(disc_map* m, cudaStream_t st)
{
    unsigned long long v = 0;
    cudaMemcpyAsync(&v, m->vt.used, sizeof(v), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return v;
}

// Grow the voxel table (doubling) until `need` voxels keep the load at or
// below max_load.  st is the stream the map's kernels run on; synchronises it
// when the table grows.
disc_status grow_voxel_table(disc_map* m, uint64_t need, cudaStream_t st)
{
    uint64_t cap = m->vt.mask + 1;
    while ((double)need > (double)m->cfg.max_load * (double)cap) cap <<= 1;
    if (cap == m->vt.mask + 1) return DISC_OK;
    VoxelTable nt{};
    disc_status s = alloc_voxel_table(m, cap, &nt, st);
    if (s != DISC_OK) return s;
    CK(cudaMemsetAsync(m->d_flag, 0, sizeof(int), st));
    launch_rehash(m->vt, nt, m->d_flag, st);
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
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

// Grow the voxel table so that `incoming` more voxels keep the load below
// max_load, from a host bound (H * W per frame); synchronises `st` only when
// the bound is hit.
disc_status ensure_voxel_room(disc_map* m, uint64_t incoming, cudaStream_t st)
{
    const double lim = (double)m->cfg.max_load * (double)(m->vt.mask + 1);
    if ((double)(m->used_upper + incoming) <= lim) return DISC_OK;
    CK(cudaStreamSynchronize(st));
    m->used_upper = read_used(m, st);
    return grow_voxel_table(m, m->used_upper + incoming, st);
}

disc_status ensure_instance_room(disc_map* m, int64_t incoming, cudaStream_t st)
{
    if (m->next_id_upper + incoming <= m->inst.cap) return DISC_OK;
    CK(cudaStreamSynchronize(st));
    m->next_id_upper = read_next_id(m, st);
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
    CK(cudaMemcpyAsync(ni.parent, m->inst.parent, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ni.count, m->inst.count, sizeof(long long) * n, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ni.Q, m->inst.Q, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ni.E, m->inst.E, sizeof(float) * (size_t)n * m->D, cudaMemcpyDeviceToDevice, st));
    const int Ds = scoring_dim(ni, m->D);
    if (ni.A) CK(cudaMemcpyAsync(ni.A, m->inst.A, sizeof(float) * (size_t)n * ni.Da, cudaMemcpyDeviceToDevice, st));
    if (ni.Eb)
        CK(cudaMemcpyAsync(ni.Eb, m->inst.Eb, sizeof(uint16_t) * (size_t)n * Ds, cudaMemcpyDeviceToDevice, st));
    if (ni.E8) {
        CK(cudaMemcpyAsync(ni.E8, m->inst.E8, (size_t)n * Ds, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(ni.Er, m->inst.Er, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
    }
    CK(cudaMemcpyAsync(ni.n_obs, m->inst.n_obs, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    const int oc = m->inst.cap;
    m->mem.release(m->inst.parent, sizeof(int32_t) * oc);
    m->mem.release(m->inst.count, sizeof(long long) * oc);
    m->mem.release(m->inst.Q, sizeof(float) * oc);
    m->mem.release(m->inst.E, sizeof(float) * (size_t)oc * m->D);
    if (m->inst.A) m->mem.release(m->inst.A, sizeof(float) * (size_t)oc * m->inst.Da);
    if (m->inst.Eb) m->mem.release(m->inst.Eb, sizeof(uint16_t) * (size_t)oc * Ds);
    if (m->inst.E8) m->mem.release(m->inst.E8, (size_t)oc * Ds);
    if (m->inst.Er) m->mem.release(m->inst.Er, sizeof(float) * oc);
    m->mem.release(m->inst.n_obs, sizeof(int32_t) * oc);
    m->inst = ni;
    return DISC_OK;
}

// device scratch of at least `bytes` for query calls (no allocation once it
// is large enough: a freed buffer would synchronise the device each call)
unsigned char* query_scratch(disc_map* m, size_t bytes)
{
    if (bytes <= m->qcap) return m->qscratch;
    if (m->qscratch) m->mem.release(m->qscratch, m->qcap);
    const size_t cap = std::max(bytes, 2 * m->qcap);
    m->qscratch = m->mem.get<unsigned char>(cap);
    if (m->mem.failed) {
        m->mem.failed = false;
        m->qscratch = nullptr;
        m->qcap = 0;
        return nullptr;
    }
    m->qcap = cap;
    return m->qscratch;
}

MapRefs map_refs(const disc_map* m)
{
    MapRefs r;
    r.vt = m->vt;
    r.inst = m->inst;
    r.ss = m->ss;
    r.next_id = m->d_next_id;
    return r;
}

// ---- phase timing ----------------------------------------------------------------
cudaEvent_t take_event(Runner& r)
{
    if (r.ev_used == r.ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        r.ev_pool.push_back(e);
    }
    return r.ev_pool[r.ev_used++];
}

// Enqueue one phase; with timing on, bracket it with events on the runner's
// stream (event-record nodes when the stream is being captured).
template <class F>
void run_phase(Runner& r, int ph, cudaStream_t st, F&& launch)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (r.timing && (a = take_event(r))) cudaEventRecordWithFlags(a, st, cudaEventRecordExternal);
    const int n = launch();
    r.launches += n;
    r.phase_launches[ph] += n;
    if (a && (b = take_event(r))) {
        cudaEventRecordWithFlags(b, st, cudaEventRecordExternal);
        if (n > 0) r.marks.push_back({ph, a, b});
    }
}

// After a synchronisation: fold the recorded phase intervals into the totals.
void collect_timing(Runner& r)
{
    for (auto& mk : r.marks) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, mk.a, mk.b) == cudaSuccess) {
            r.phase_ms[mk.phase] += ms;
            r.phase_calls[mk.phase] += 1;
        } else {
            cudaGetLastError();
        }
    }
    r.marks.clear();
    r.ev_used = 0;
}

void reset_timing(Runner& r, bool enable)
{
    collect_timing(r);
    r.timing = enable;
    for (int i = 0; i < PH_COUNT; i++) {
        r.phase_ms[i] = 0.0;
        r.phase_launches[i] = 0;
        r.phase_calls[i] = 0;
    }
}

// ---- one batch -------------------------------------------------------------------
// A batch of S frame slots over G maps (J frames per map at most) runs in two
// parts.  Grids follow the runner's maxima (smaller frames return early in
// their blocks) and per-frame values and map state are read on the device,
// so each part depends on its shape only and is replayed as a CUDA graph.
//   stateless: every kernel over all slots (reads no map state that frames
//              change except the voxel lookup of k_entries, see below)
//   serial:    overlap, score, union, apply for frame j of every map, j = 0..J-1
// k_entries may run while the serial part of the previous batch inserts
// voxels: a voxel's label never changes once written, an empty slot's label
// reads -1, so the lookup returns either the final label or "absent", and an
// absent voxel is looked up again by k_overlap after the earlier frames.

// combos: bit (3 * token_bf16 + precision) set for every kind of frame in
// the batch; bit COMBO_DBSCAN: some frame runs the DBSCAN filter; bit
// COMBO_ASSOC: the feature kernels also run on the second grid's view
constexpr int COMBO_DBSCAN = 1 << 6;
constexpr int COMBO_ASSOC = 1 << 7;   // some frame's map has a second token grid
constexpr int COMBO_DILATE = 1 << 8;  // some frame's map takes the neighbourhood overlap: the batch's
                                      // frames run as four kernels each (overlap, score, union, apply)

// slots [base, base + S) of set k (base > 0: the second half of a batch whose
// halves wait for their own input copies)
int enqueue_stateless(Runner& r, int k, int S, int combos, cudaStream_t st, int base = 0)
{
    const bool any_bf16 = (combos & 070) != 0, any_f32 = (combos & 07) != 0;  // bits 0-5
    bool any[2][3];
    for (int t = 0; t < 2; t++)
        for (int q = 0; q < 3; q++) any[t][q] = (combos >> (3 * t + q)) & 1;
    const int D = r.D, P = r.P, Mmax = r.Mmax;
    BatchScratch bs = r.bs[k];
    bs.base = r.bs[k].frame(base);
    const FrameParams* dfp = r.fps(k) + base;
    const MapRefs* refs = r.refs(k);
    const int64_t before = r.launches;
    run_phase(r, PH_CLEAR, st, [&] { return launch_slot_clear(bs, S, D, r.MM, st); });
    run_phase(r, PH_TOKENS, st, [&] { return launch_token_stats(dfp, bs, S, P, D, any_bf16, any_f32, st); });
    run_phase(r, PH_COVERAGE, st, [&] { return launch_coverage(dfp, bs, S, r.Ph, r.Pw, Mmax, st); });
    run_phase(r, PH_WEIGHTS, st, [&] { return launch_weights(dfp, bs, S, Mmax, st); });
    run_phase(r, PH_POOL_EXACT, st, [&] { return launch_pool_exact(dfp, bs, S, P, D, Mmax, any_bf16, any_f32, st); });
    run_phase(r, PH_POOL_GEMM, st, [&] { return launch_pool_gemm(dfp, bs, S, D, Mmax, any, st); });
    if ((combos & COMBO_ASSOC) && r.Da) {
        // the association features: the same kernels on the second grid's
        // view (pixel-mean weights; frames of maps without it are inert)
        BatchScratch va = r.bsa[k];
        va.base = r.bsa[k].frame(base);
        const FrameParams* dfa = r.fpa(k) + base;
        run_phase(r, PH_CLEAR, st, [&] { return launch_view_clear(va, S, r.Da, r.MM, st); });
        run_phase(r, PH_TOKENS, st, [&] { return launch_token_stats(dfa, va, S, r.Pa, r.Da, any_bf16, any_f32, st); });
        run_phase(r, PH_COVERAGE, st, [&] { return launch_coverage(dfa, va, S, r.Pha, r.Pwa, Mmax, st); });
        run_phase(r, PH_WEIGHTS, st, [&] { return launch_weights(dfa, va, S, Mmax, st); });
        run_phase(r, PH_POOL_EXACT, st,
                  [&] { return launch_pool_exact(dfa, va, S, r.Pa, r.Da, Mmax, any_bf16, any_f32, st); });
        run_phase(r, PH_POOL_GEMM, st, [&] { return launch_pool_gemm(dfa, va, S, r.Da, Mmax, any, st); });
    }
    if (Mmax > 0) {
        for (int f0 = 0; f0 < S; f0 += r.geo_chunk) {
            const int nb = std::min(r.geo_chunk, S - f0);
            if (combos & COMBO_DBSCAN)
                run_phase(r, PH_DBSCAN, st, [&] { return launch_dbscan(dfp, bs, f0, nb, r.Hmax, r.Wmax, st); });
            run_phase(r, PH_BACKPROJECT, st, [&] { return launch_backproject(dfp, bs, f0, nb, r.Hmax, r.Wmax, st); });
            run_phase(r, PH_ENTRIES, st,
                      [&] { return launch_entries(dfp, bs, refs, f0, nb, Mmax, (combos & COMBO_DILATE) != 0, st); });
        }
        run_phase(r, PH_ENTRIES, st, [&] { return launch_quality(dfp, bs, S, st); });
    }
    return (int)(r.launches - before);
}

// The serial part of a batch of S slots over G maps (J frames per map).
// Plain: every entry looked up at once, one CTA per map walks its frames
// (k_associate), the new voxels committed at the end.  With the
// neighbourhood overlap (COMBO_DILATE) each frame probes the map as its
// predecessors left it: four kernels per frame.
int enqueue_serial(Runner& r, int k, int S, int G, int J, int combos, cudaStream_t st)
{
    const BatchScratch& bs = r.bs[k];
    const FrameParams* dfp = r.fps(k);
    const int64_t before = r.launches;
    SerialStep step;
    step.refs = r.refs(k);
    step.slot_of = r.slot_of(k);
    step.prev_hist = r.prev_hist(k);
    step.hist = r.d_hist;
    step.J = J;
    step.view = r.bsa[k];  // zero when the runner has no second grid
    step.cta_scale = r.cta_scale;
    step.merged = r.d_merged;
    if (!(combos & COMBO_DILATE)) {
        step.j = 0;
        run_phase(r, PH_LOOKUP, st, [&] { return launch_lookup(dfp, bs, step.refs, r.ah, S, r.probe_width, st); });
        // on an SM partition (serial_sms) the chain runs one CTA per map: a
        // cluster's CTAs must fit the partition's SMs together
        const int cluster = r.green[0] ? 1 : r.assoc_cluster;
        run_phase(r, PH_ASSOCIATE, st, [&] { return launch_associate(dfp, bs, step, G, cluster, st); });
        run_phase(r, PH_COMMIT, st, [&] {
            const int n = launch_commit(bs, step, r.ah, G, st);
            cudaMemsetAsync(r.ah.n, 0, sizeof(int32_t), st);  // the hash is empty again
            return n;
        });
        return (int)(r.launches - before);
    }
    run_phase(r, PH_OVERLAP, st, [&] { return launch_serial_begin(step.refs, G, st); });
    for (int j = 0; j < J; j++) {
        step.j = j;
        for (int ph = 0; ph < 4; ph++)
            run_phase(r, PH_OVERLAP + ph, st, [&] { return launch_serial_step(dfp, bs, step, G, ph, st); });
    }
    return (int)(r.launches - before);
}

long long graph_key(int part, int k, int S, int G, int J, int combos)
{
    return (((((((long long)S << 11) | G) << 9) | J) << 9 | combos) << 3) | (part << 1) | k;
}

// A part's kernel sequence captured once per shape and replayed.  A shape
// seen for the first time runs as plain launches (*out = NULL): under a mixed
// load (groups, serving) most shapes are one-off and instantiating a graph
// costs more than launching the kernels.  At most kMaxGraphs are kept.
constexpr int kMaxGraphs = 96;

template <class F>
disc_status part_graph(Runner& r, long long key, cudaStream_t st, F&& enqueue, BatchGraph** out)
{
    *out = nullptr;
    auto it = r.graphs.find(key);
    if (it != r.graphs.end()) {
        *out = &it->second;
        return DISC_OK;
    }
    if (r.shapes_seen[key]++ == 0) return DISC_OK;
    if ((int)r.graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(r.graphs.begin()->second.exec);
        r.graphs.erase(r.graphs.begin());
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int64_t before = r.launches;
    int64_t pl0[PH_COUNT];
    for (int i = 0; i < PH_COUNT; i++) pl0[i] = r.phase_launches[i];
    const int n = enqueue();
    r.launches = before;  // counted when the graph is launched
    for (int i = 0; i < PH_COUNT; i++) r.phase_launches[i] = pl0[i];
    cudaError_t e = cudaStreamEndCapture(st, &graph);
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
    *out = &(r.graphs[key] = g);
    return DISC_OK;
}

// Run one part: its graph when there is one, else plain launches.
template <class F>
disc_status run_part(Runner& r, long long key, cudaStream_t st, F&& enqueue)
{
    BatchGraph* g = nullptr;
    if (!r.graphs_off && part_graph(r, key, st, enqueue, &g) != DISC_OK) {
        r.graphs_off = true;  // this stream or driver cannot capture the sequence
        g = nullptr;
    }
    if (g) {
        r.launches += g->kernels;
        return cuda_status(cudaGraphLaunch(g->exec, st));
    }
    enqueue();
    return DISC_OK;
}

// Timing run of one batch: both parts with their phase events, captured and
// launched as one graph on the runner's stream, so the device never waits on
// the host inside a timed interval.  false: capture is not possible here.
bool launch_timed_graph(Runner& r, int k, int S, int G, int J, int combos)
{
    const size_t marks0 = r.marks.size(), ev0 = r.ev_used;
    const int64_t l0 = r.launches;
    int64_t pl0[PH_COUNT];
    for (int i = 0; i < PH_COUNT; i++) pl0[i] = r.phase_launches[i];
    auto undo = [&] {
        r.marks.resize(marks0);
        r.ev_used = ev0;
        r.launches = l0;
        for (int i = 0; i < PH_COUNT; i++) r.phase_launches[i] = pl0[i];
        cudaGetLastError();
    };
    if (cudaStreamBeginCapture(r.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        undo();
        return false;
    }
    enqueue_stateless(r, k, S, combos, r.stream);
    enqueue_serial(r, k, S, G, J, combos, r.stream);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamEndCapture(r.stream, &graph) != cudaSuccess || !graph ||
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        undo();
        return false;
    }
    cudaGraphDestroy(graph);
    const bool ok = cudaGraphLaunch(exec, r.stream) == cudaSuccess;
    cudaGraphExecDestroy(exec);  // freed once the launch completes
    if (!ok) {
        undo();
        return false;
    }
    return true;
}

disc_status check_frame(const disc_map* m, const Runner& r, const disc_frame* f)
{
    if (!f || !f->depth || !f->labels || !f->tokens) return DISC_ERR_INVALID_ARG;
    if (f->width <= 0 || f->height <= 0 || f->width > m->cfg.max_width || f->height > m->cfg.max_height)
        return DISC_ERR_INVALID_ARG;
    if (f->width > r.Wmax || f->height > r.Hmax || (int64_t)f->width * f->height > (int64_t)r.px_cap)
        return DISC_ERR_INVALID_ARG;
    if (f->num_masks < 0 || f->num_masks > m->cfg.max_masks || f->num_masks > r.Mmax) return DISC_ERR_INVALID_ARG;
    if (f->token_dtype != DISC_TOKENS_F32 && f->token_dtype != DISC_TOKENS_BF16) return DISC_ERR_INVALID_ARG;
    // a camera model and pose of finite numbers (the pose as it is rounded to fp32)
    if (!std::isfinite(f->fx) || !std::isfinite(f->fy) || !std::isfinite(f->cx) || !std::isfinite(f->cy) ||
        f->fx == 0.0f || f->fy == 0.0f)
        return DISC_ERR_INVALID_ARG;
    for (int i = 0; i < 12; i++)
        if (!std::isfinite((float)f->T_world_cam[i])) return DISC_ERR_INVALID_ARG;
    if (m->cfg.assoc_dim > 0 && (!f->assoc_tokens || r.Da != m->cfg.assoc_dim || r.Pha != m->cfg.assoc_patch_h ||
                                 r.Pwa != m->cfg.assoc_patch_w))
        return DISC_ERR_INVALID_ARG;
    return DISC_OK;
}

// Frame parameters of frame f of map m in slot `slot` (map position g); host
// inputs are staged into the slot's buffers.

// Error bounds of the fast score: eta scales the per-mask Bm into the bound
// of |E_fast - E|, dot_err bounds the fast cosine's own error.
//   FP32: Bm = sum_p w_p ||f_p||; tf32 split residue 3 * 2^-22 plus fp32
//         accumulation of 3 K products; fp32 warp cosine 3 D 2^-24
//   BF16: both operands rounded to bf16, 2 * 2^-9, plus fp32 accumulation
//         of K products; the bf16 scoring copy of E_k adds 2^-9 relative,
//         at most 2 * 2^-9 on the cosine
//   FP8:  the weights kernel stores the whole bound of |E_fast - E| in Bm
//         (eta 1); each E4M3 scoring copy carries its own relative error
//         bound, added per instance in the gate
void fast_error_terms(int precision, int Kpad, int D, float* eta, float* dot_err)
{
    const double K = Kpad, u24 = std::ldexp(1.0, -24), u9 = std::ldexp(1.0, -9);
    if (precision == DISC_BF16) {
        *eta = (float)(2.0 * u9 + u9 * u9 + 3.0 * K * u24);
        *dot_err = (float)(3.0 * u9 + 3.0 * D * u24);
    } else if (precision == DISC_FP8_E4M3) {
        *eta = 1.0f;
        *dot_err = (float)(3.0 * D * u24);
    } else {
        *eta = (float)(3.0 * std::ldexp(1.0, -22) + 3.0 * K * u24);
        *dot_err = (float)(3.0 * D * u24);
    }
}

// Host-to-device copies of one batch's inputs, one list per input kind.
// Copies whose sources and destinations both continue the previous copy of
// the same kind (frames laid out back to back, as a trajectory in one host
// array) merge into one larger copy.
struct CopyList {
    struct Item { char* dst; const char* src; size_t bytes; };
    std::vector<Item> kind[5];  // depth, labels, tokens, global embedding, association tokens
    void add(int k, void* dst, const void* src, size_t bytes)
    {
        std::vector<Item>& v = kind[k];
        if (!v.empty() && v.back().dst + v.back().bytes == (char*)dst && v.back().src + v.back().bytes == (const char*)src)
            v.back().bytes += bytes;
        else
            v.push_back({(char*)dst, (const char*)src, bytes});
    }
    void append(CopyList& o)  // o's copies after this list's, merged where they continue
    {
        for (int k = 0; k < 5; k++) {
            for (const Item& it : o.kind[k]) add(k, it.dst, it.src, it.bytes);
            o.kind[k].clear();
        }
    }
    bool empty() const
    {
        for (const auto& v : kind)
            if (!v.empty()) return false;
        return true;
    }
    disc_status issue(cudaStream_t st)
    {
        for (auto& v : kind) {
            for (const Item& it : v) CK(cudaMemcpyAsync(it.dst, it.src, it.bytes, cudaMemcpyHostToDevice, st));
            v.clear();
        }
        return DISC_OK;
    }
};

// Host inputs are staged in staging set `set` (copies collected in cl).
// With a second grid, *outa receives the view of the frame on that grid (for
// maps without one, an inert view: no tokens, no masks).
disc_status frame_params(Runner& r, const disc_map* m, const disc_frame* f, int set, int slot, int g, int jpos,
                         FrameParams* out, FrameParams* outa, CopyList* cl)
{
    const int P = r.P, D = r.D;
    FrameParams fp{};
    fp.H = f->height;
    fp.W = f->width;
    fp.M = f->num_masks;
    fp.P = P;
    fp.D = D;
    fp.Ph = r.Ph;
    fp.Pw = r.Pw;
    fp.Kpad = r.Kpad;
    fp.Npad = std::max(16, (fp.M + 15) / 16 * 16);
    fp.fx = f->fx;
    fp.fy = f->fy;
    fp.cx = f->cx;
    fp.cy = f->cy;
    for (int i = 0; i < 3; i++) {
        for (int c = 0; c < 3; c++) fp.R[3 * i + c] = (float)f->T_world_cam[4 * i + c];
        fp.t[i] = (float)f->T_world_cam[4 * i + 3];
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
    fp.map = g;
    fp.jpos = jpos;
    fp.precision = m->cfg.precision;
    fp.dilate = m->cfg.overlap_dilation;
    fp.db_min_pts = m->cfg.dbscan_eps > 0.0f ? m->cfg.dbscan_min_pts : 0;
    fp.db_eps2 = m->cfg.dbscan_eps * m->cfg.dbscan_eps;
    fp.db_inv_cell = m->cfg.dbscan_eps > 0.0f ? 1.0f / (m->cfg.dbscan_eps * 1.001f) : 0.0f;
    const bool assoc = m->cfg.assoc_dim > 0;
    fp.assoc = assoc;
    // the fast score's bounds are those of the features the gate compares
    if (assoc)
        fast_error_terms(m->cfg.precision, r.Kpad_a, r.Da, &fp.eta, &fp.dot_err);
    else
        fast_error_terms(m->cfg.precision, r.Kpad, D, &fp.eta, &fp.dot_err);
    const size_t npx = (size_t)fp.H * fp.W;
    const size_t tok_bytes = (size_t)P * D * (fp.token_bf16 ? 2 : 4);
    if (f->inputs_on_device) {
        fp.depth = f->depth;
        fp.labels = f->labels;
        fp.tokens = f->tokens;
        fp.gembed = f->global_embed;
    } else {
        const size_t at = (size_t)set * r.S + slot;
        float* dd = r.d_depth + at * r.px_cap;
        uint16_t* dl = r.d_labels + at * r.px_cap;
        unsigned char* dt = r.d_tokens + at * P * D * 4;
        cl->add(0, dd, f->depth, sizeof(float) * npx);
        cl->add(1, dl, f->labels, sizeof(uint16_t) * npx);
        cl->add(2, dt, f->tokens, tok_bytes);
        fp.depth = dd;
        fp.labels = dl;
        fp.tokens = dt;
        fp.gembed = nullptr;
        if (f->global_embed) {
            float* dg = r.d_gembed + at * D;
            cl->add(3, dg, f->global_embed, sizeof(float) * D);
            fp.gembed = dg;
        }
    }
    *out = fp;
    if (r.Da) {
        FrameParams va = fp;
        va.uniform_w = 1;
        va.gembed = nullptr;
        va.D = va.P = va.M = 0;  // inert unless the map has a second grid
        va.tokens = nullptr;
        if (assoc) {
            va.D = r.Da;
            va.P = r.Pa;
            va.Ph = r.Pha;
            va.Pw = r.Pwa;
            va.Kpad = r.Kpad_a;
            va.M = fp.M;
            const size_t abytes = (size_t)r.Pa * r.Da * (fp.token_bf16 ? 2 : 4);
            if (f->inputs_on_device) {
                va.tokens = f->assoc_tokens;
            } else {
                unsigned char* da = r.d_atok + ((size_t)set * r.S + slot) * r.Pa * r.Da * 4;
                cl->add(4, da, f->assoc_tokens, abytes);
                va.tokens = da;
            }
        }
        *outa = va;
    }
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
    s->denoised_pixels = c.denoised;
    s->scored_pairs = c.n_scored;
    s->embedding_copies = c.n_copies;
}

// Between a batch's stateless and serial parts (on the serial stream, after
// the stateless part): each map's exact voxel count and the unique (segment,
// voxel) pairs of its frames, which bound the voxels the batch inserts, come
// back to the host; a table that could pass max_load grows (rehash) before
// the serial part, and the map's table pointers in the batch's parameter
// block are refreshed.  Only this small read is waited for, so the input
// copies of the next batch run while the serial part computes.
disc_status room_check(Runner& r, int k, int G, int J, std::vector<Work>& w, const std::vector<int>& gl,
                       MapRefs* hrefs, cudaStream_t sr)
{
    launch_room(r.refs(k), G, r.slot_of(k), J, r.bs[k], r.d_room, sr);
    r.launches++;
    CK(cudaMemcpyAsync(r.h_room, r.d_room, sizeof(unsigned long long) * 2 * G, cudaMemcpyDeviceToHost, sr));
    CK(cudaEventRecord(r.ev_room, sr));
    CK(cudaEventSynchronize(r.ev_room));
    uint64_t pairs = 0;  // bounds the voxels absent at the batch start
    for (int gi = 0; gi < G; gi++) pairs += r.h_room[2 * gi + 1];
    disc_status sa = ensure_absent(r, pairs);
    if (sa != DISC_OK) return sa;
    for (int gi = 0; gi < G; gi++) {
        disc_map* m = w[gl[gi]].m;
        const uint64_t need = r.h_room[2 * gi] + r.h_room[2 * gi + 1];
        m->used_upper = need;  // the count after this batch is at most this
        if ((double)need <= (double)m->cfg.max_load * (double)(m->vt.mask + 1)) continue;
        disc_status s = grow_voxel_table(m, need, sr);
        if (s != DISC_OK) return s;
        hrefs[gi] = map_refs(m);
        CK(cudaMemcpyAsync(r.d_param[k] + r.off_refs + sizeof(MapRefs) * gi, &hrefs[gi], sizeof(MapRefs),
                           cudaMemcpyHostToDevice, sr));
    }
    return DISC_OK;
}

// Integrate every map's frames: batch b holds frames [b*J, (b+1)*J) of each
// map; the maps of a batch run side by side, each map's frames in order.  A
// frame that fails stops the later frames of its map (on the device), not
// those of the other maps.  Returns the first status that is not DISC_OK.
// With `async` (an asynchronous call, its history half chosen by the
// caller) a call whose work can overlap later calls returns as soon as it is
// enqueued, with *queued set: its counters and voxel counts come back on the
// serial stream and ev_done[async->region] marks the end of its work, and
// finish_oldest hands out its results.  Otherwise (or when enqueueing
// fails) it completes before returning, as a synchronous call does.
disc_status run_call(Runner& r, std::vector<Work>& w, const AsyncCall* async = nullptr, bool* queued = nullptr)
{
    if (queued) *queued = false;
    int total = 0, most = 0;
    for (Work& wk : w) {
        wk.valid = 0;
        while (wk.valid < wk.n && check_frame(wk.m, r, wk.frames + wk.valid) == DISC_OK) wk.valid++;
        total += wk.valid;
        most = std::max(most, wk.valid);
    }
    // frames per map per batch: a call that fits in one batch runs as
    // batch_split smaller batches of at least 4 frames (automatic: two for one
    // map's synchronous call of 16 frames or more, else one), so that each
    // one's stateless kernels overlap the frame chain of the one before (an
    // asynchronous call's chain overlaps the next call's instead: measured on
    // 32-frame Room calls, 28.9k frames/s whole against 27.1k split in two)
    int pieces = r.batch_split > 0 ? r.batch_split : (w.size() == 1 && total >= 16 && !async ? 2 : 1);
    pieces = std::min(pieces, std::max(1, total / 4));
    const int Jb = (!r.timing && pieces > 1 && most <= r.Jmax) ? (most + pieces - 1) / pieces : r.Jmax;
    const int nbatch = (most + Jb - 1) / Jb;
    disc_status s = ensure_hist(r, std::max(total, 1));
    if (s != DISC_OK) return s;
    for (const Work& wk : w)
        if (wk.valid > 0 && wk.m->cfg.dbscan_eps > 0.0f) s = ensure_dbscan(r);
    if (s != DISC_OK) return s;
    // pipelined (calls of several batches): the runner's two streams start
    // after the caller's earlier work and the caller's stream waits for their
    // end; a single batch runs on the caller's stream
    bool dilate = false;
    for (const Work& wk : w) dilate |= wk.valid > 0 && wk.m->cfg.overlap_dilation != 0;
    // the serial part of a plain batch runs on one SM per map, so the next
    // batch's stateless part runs beside it on the other SMs (two streams,
    // the serial one of highest priority); the four-kernels-per-frame form
    // (neighbourhood overlap) overlaps only on SM partitions (serial_sms)
    const bool can_pipe = !r.timing && (r.serial_sms > 0 || !dilate);
    const bool pipe = can_pipe && (nbatch > 1 || async);
    const bool queue = async && can_pipe;  // returns once enqueued
    cudaStream_t sr = pipe ? r.stream3 : r.stream;  // serial part
    cudaStream_t ss = pipe ? r.stream2 : r.stream;  // stateless part
    // the input copies (and, pipelined, both parts) start after the caller's
    // earlier work on its stream
    s = cuda_status(cudaEventRecord(r.ev_join, r.stream));
    if (s == DISC_OK) s = cuda_status(cudaStreamWaitEvent(r.stream_in, r.ev_join, 0));
    if (pipe) {
        if (s == DISC_OK) s = cuda_status(cudaStreamWaitEvent(r.stream2, r.ev_join, 0));
        if (s == DISC_OK) s = cuda_status(cudaStreamWaitEvent(r.stream3, r.ev_join, 0));
    }
    if (s != DISC_OK) return s;
    const bool one_graph = r.timing && !r.graphs_off;
    // Batch b + 1's stateless part is enqueued after batch b's serial part:
    // the serial kernel (one cluster of large-shared-memory CTAs per map)
    // then takes its SMs first and the stateless part fills the rest.
    // (Enqueued before it, the stateless kernels hold every SM and the
    // serial kernel waits for them to drain: measured slower.)
    const int hbase = async ? async->region * r.hist_cap : 0;  // the call's half of the history
    int hoff = hbase;
    // One batch between its two halves of the loop below.
    struct Pending {
        int b = -1, k = 0, G = 0, J = 0, S = 0, combos = 0, hoff = 0;
        std::vector<int> gl;       // works with frames in this batch
        std::vector<size_t> mark;  // their history lengths before the batch
        std::vector<unsigned char> blk;
        bool copied = false, timed = false;
    };
    auto undo = [&](Pending& P) {
        for (int gi = 0; gi < (int)P.gl.size(); gi++) w[P.gl[gi]].hist_idx.resize(P.mark[gi]);
        P.b = -1;
    };
    // front: compose batch b, fill and upload its parameter block, copy its
    // host inputs and enqueue its stateless part (or, timed, the whole batch)
    auto front = [&](int b, Pending& P) -> disc_status {
        P.b = -1;
        const int lo = b * Jb;
        P.gl.clear();
        int J = 0, S = 0;
        for (int i = 0; i < (int)w.size(); i++) {
            const int cnt = std::min(Jb, w[i].valid - lo);
            if (cnt <= 0) continue;
            P.gl.push_back(i);
            J = std::max(J, cnt);
            S += cnt;
        }
        const int G = (int)P.gl.size();
        if (G == 0) return DISC_OK;
        int combos = 0;
        uint64_t batch_px = 0;
        disc_status st = DISC_OK;
        for (int gi = 0; gi < G && st == DISC_OK; gi++) {
            Work& wk = w[P.gl[gi]];
            const int cnt = std::min(Jb, wk.valid - lo);
            uint64_t px = 0;
            int64_t masks = 0;
            for (int j = 0; j < cnt; j++) {
                const disc_frame& f = wk.frames[lo + j];
                px += (uint64_t)f.width * f.height;
                masks += f.num_masks;
                combos |= 1 << (3 * (f.token_dtype == DISC_TOKENS_BF16) + wk.m->cfg.precision);
                if (wk.m->cfg.dbscan_eps > 0.0f) combos |= COMBO_DBSCAN;
                if (wk.m->cfg.assoc_dim > 0) combos |= COMBO_ASSOC;
                if (wk.m->cfg.overlap_dilation) combos |= COMBO_DILATE;
            }
            // one graph of both parts (phase timing): room from the host
            // bounds now; otherwise before the serial part (back)
            if (one_graph) {
                st = ensure_voxel_room(wk.m, px, sr);
                if (st == DISC_OK) st = ensure_instance_room(wk.m, masks, sr);
            }
            batch_px += px;
        }
        if (st == DISC_OK && one_graph) st = ensure_absent(r, batch_px);
        if (st != DISC_OK) return st;
        // set k: its previous batch's serial part must be done before the
        // stateless part of this batch overwrites the set
        const int k = r.cur;
        r.cur ^= 1;
        if (pipe) CK(cudaStreamWaitEvent(ss, r.ev_serial[k], 0));
        P.blk.assign(r.param_bytes, 0);
        FrameParams* hfp = (FrameParams*)P.blk.data();
        MapRefs* hrefs = (MapRefs*)(P.blk.data() + r.off_refs);
        int* hslot = (int*)(P.blk.data() + r.off_slot);
        int* hprev = (int*)(P.blk.data() + r.off_prev);
        FrameParams* hfpa = r.Da ? (FrameParams*)(P.blk.data() + r.off_fpa) : nullptr;
        int slot = 0;
        CopyList cl[2];  // host inputs of the batch's first and second half
        // a batch that fails before its counters reach the call's history
        // leaves no history entries behind: its frames count as not done
        P.mark.resize(G);
        for (int gi = 0; gi < G; gi++) P.mark[gi] = w[P.gl[gi]].hist_idx.size();
        P.b = b;
        P.k = k;
        P.G = G;
        P.J = J;
        P.S = S;
        P.combos = combos;
        P.hoff = hoff;
        // host inputs of this batch go to staging set k once the set's last
        // batch has read its inputs (its stateless part), on the input
        // stream, so they overlap the previous batch's kernels
        st = cuda_status(cudaStreamWaitEvent(r.stream_in, r.ev_in_free[k], 0));
        for (int gi = 0; gi < G && st == DISC_OK; gi++) {
            Work& wk = w[P.gl[gi]];
            const int cnt = std::min(Jb, wk.valid - lo);
            hrefs[gi] = map_refs(wk.m);
            hprev[gi] = wk.hist_idx.empty() ? wk.prev_idx : wk.hist_idx.back();
            for (int j = 0; j < J; j++) hslot[gi * J + j] = -1;
            for (int j = 0; j < cnt && st == DISC_OK; j++) {
                st = frame_params(r, wk.m, wk.frames + lo + j, k, slot, gi, j, hfp + slot, hfpa ? hfpa + slot : nullptr,
                                  &cl[2 * slot >= S ? 1 : 0]);
                hslot[gi * J + j] = slot;
                wk.hist_idx.push_back(hoff + slot);
                slot++;
            }
        }
        hoff += S;
        // With host inputs (and not one timed graph), the batch's stateless
        // part runs in two halves: the second half's copies run while the
        // first half computes.
        const bool copied = !cl[0].empty() || !cl[1].empty();
        P.copied = copied;
        const bool halves = copied && !one_graph && S >= 8;
        const int Sh = halves ? S / 2 : S;
        if (!halves) cl[0].append(cl[1]);
        if (st == DISC_OK && copied) {
            st = cl[0].issue(r.stream_in);
            if (st == DISC_OK) st = cuda_status(cudaEventRecord(r.ev_in_ready[k], r.stream_in));
            if (st == DISC_OK) st = cuda_status(cudaStreamWaitEvent(ss, r.ev_in_ready[k], 0));
            if (st == DISC_OK && halves) {
                st = cl[1].issue(r.stream_in);
                if (st == DISC_OK) st = cuda_status(cudaEventRecord(r.ev_in_half[k], r.stream_in));
            }
        }
        // pageable source: the call returns once the block is staged
        if (st == DISC_OK)
            st = cuda_status(cudaMemcpyAsync(r.d_param[k], P.blk.data(), r.param_bytes, cudaMemcpyHostToDevice, ss));
        if (st != DISC_OK) return st;
        P.timed = one_graph && launch_timed_graph(r, k, S, G, J, combos);
        if (P.timed) {
            // both parts with their phase events, one graph on the runner's stream
            if (copied) st = cuda_status(cudaEventRecord(r.ev_in_free[k], r.stream));
            return st;
        }
        if (halves) {
            st = run_part(r, graph_key(2, k, Sh, 0, 0, combos), ss,
                          [&] { return enqueue_stateless(r, k, Sh, combos, ss); });
            if (st == DISC_OK) st = cuda_status(cudaStreamWaitEvent(ss, r.ev_in_half[k], 0));
            if (st == DISC_OK)
                st = run_part(r, graph_key(3, k, S - Sh, Sh, 0, combos), ss,  // keyed by its first slot too
                              [&] { return enqueue_stateless(r, k, S - Sh, combos, ss, Sh); });
        } else {
            st = run_part(r, graph_key(0, k, S, 0, 0, combos), ss,
                          [&] { return enqueue_stateless(r, k, S, combos, ss); });
        }
        if (st == DISC_OK && copied) st = cuda_status(cudaEventRecord(r.ev_in_free[k], ss));
        if (st == DISC_OK && pipe) {
            st = cuda_status(cudaEventRecord(r.ev_state[k], ss));
            if (st == DISC_OK) st = cuda_status(cudaStreamWaitEvent(sr, r.ev_state[k], 0));
        }
        return st;
    };
    // back: room for the batch's new voxels and ids (the tables grow when
    // they could pass their limits, and the batch's map pointers follow),
    // its serial part, its counters to the call's history
    auto back = [&](Pending& P) -> disc_status {
        const int k = P.k, G = P.G, J = P.J, S = P.S, lo = P.b * Jb;
        disc_status st = DISC_OK;
        if (!P.timed) {
            MapRefs* hrefs = (MapRefs*)(P.blk.data() + r.off_refs);
            bool moved = false;
            for (int gi = 0; gi < G && st == DISC_OK; gi++) {
                Work& wk = w[P.gl[gi]];
                const int cnt = std::min(Jb, wk.valid - lo);
                int64_t masks = 0;
                for (int j = 0; j < cnt; j++) masks += wk.frames[lo + j].num_masks;
                st = ensure_instance_room(wk.m, masks, sr);
                const MapRefs now = map_refs(wk.m);
                if (std::memcmp(&now, &hrefs[gi], sizeof(MapRefs)) != 0) {
                    hrefs[gi] = now;
                    moved = true;
                }
            }
            if (st == DISC_OK && moved)
                st = cuda_status(cudaMemcpyAsync(r.d_param[k] + r.off_refs, hrefs, sizeof(MapRefs) * G,
                                                 cudaMemcpyHostToDevice, sr));
            // Room without a round trip when the host bound suffices: a batch
            // inserts at most one voxel per pixel of its frames, so each
            // map's count stays below its bound plus the batch's pixels, and
            // the absent-voxel hash below the batch's pixels (sized so at most
            // kAbsentPixelCap slots).  Otherwise the exact counts come back
            // (room_check) and set the bounds anew.
            constexpr uint64_t kAbsentPixelCap = 1ull << 25;
            bool fast = st == DISC_OK;
            uint64_t batch_px = 0;
            std::vector<uint64_t> px(G, 0);
            for (int gi = 0; gi < G; gi++) {
                Work& wk = w[P.gl[gi]];
                const int cnt = std::min(Jb, wk.valid - lo);
                for (int j = 0; j < cnt; j++) px[gi] += (uint64_t)wk.frames[lo + j].width * wk.frames[lo + j].height;
                batch_px += px[gi];
                const disc_map* m = wk.m;
                fast = fast && (double)(m->used_upper + px[gi]) <= (double)m->cfg.max_load * (double)(m->vt.mask + 1);
            }
            fast = fast && next_pow2(std::max<uint64_t>(2 * batch_px, 1 << 16)) <= kAbsentPixelCap;
            if (fast) {
                st = ensure_absent(r, batch_px);
                for (int gi = 0; gi < G && st == DISC_OK; gi++) w[P.gl[gi]].m->used_upper += px[gi];
            } else if (st == DISC_OK) {
                st = room_check(r, k, G, J, w, P.gl, hrefs, sr);
            }
            if (st == DISC_OK)
                st = run_part(r, graph_key(1, k, S, G, J, P.combos & COMBO_DILATE), sr,
                              [&] { return enqueue_serial(r, k, S, G, J, P.combos, sr); });
        }
        // the batch's counters, in slot order, to the call's history
        if (st == DISC_OK)
            st = cuda_status(cudaMemcpyAsync(r.d_hist + P.hoff, r.bs[k].base.ctr, sizeof(FrameCounters) * S,
                                             cudaMemcpyDeviceToDevice, sr));
        if (st == DISC_OK && pipe) st = cuda_status(cudaEventRecord(r.ev_serial[k], sr));
        if (st == DISC_OK) st = cuda_status(cudaGetLastError());
        if (st != DISC_OK) return st;
        for (int gi = 0; gi < G; gi++) {
            Work& wk = w[P.gl[gi]];
            const int cnt = std::min(Jb, wk.valid - lo);
            for (int j = 0; j < cnt; j++) {
                const disc_frame& f = wk.frames[lo + j];
                if (P.timed) wk.m->used_upper += (uint64_t)f.width * f.height;
                wk.m->next_id_upper += f.num_masks;
                wk.m->px_total += (uint64_t)f.width * f.height;
                wk.m->masks_total += f.num_masks;
            }
        }
        r.last_set = k;
        r.last_slot = S - 1;
        const Work& wl = w[P.gl[G - 1]];
        r.last_M = wl.frames[lo + std::min(Jb, wl.valid - lo) - 1].num_masks;
        r.have_frame = true;
        return DISC_OK;
    };
    Pending cur, nxt;
    if (nbatch > 0) {
        s = front(0, cur);
        if (s != DISC_OK && cur.b >= 0) undo(cur);
    }
    for (int b = 0; b < nbatch && s == DISC_OK && cur.b >= 0; b++) {
        s = back(cur);
        if (s != DISC_OK) {
            undo(cur);
            break;
        }
        const disc_status sn = b + 1 < nbatch ? front(b + 1, nxt) : DISC_OK;
        if (sn != DISC_OK) {
            if (nxt.b >= 0) undo(nxt);
            s = sn;
            break;
        }
        std::swap(cur, nxt);
        nxt.b = -1;
    }
    if (queue && s == DISC_OK) {
        // every map's exact voxel count and the call's counters come back
        // behind its last batch; the caller's stream is not made to wait
        const int nu = std::min<int>((int)w.size(), r.Gmax);
        unsigned long long* hu = r.h_used + (size_t)async->region * r.Gmax;
        for (int i = 0; i < nu && s == DISC_OK; i++)
            s = cuda_status(cudaMemcpyAsync(hu + i, w[i].m->vt.used, sizeof(unsigned long long),
                                            cudaMemcpyDeviceToHost, r.stream3));
        if (s == DISC_OK && hoff > hbase)
            s = cuda_status(cudaMemcpyAsync(r.h_hist + hbase, r.d_hist + hbase, sizeof(FrameCounters) * (hoff - hbase),
                                            cudaMemcpyDeviceToHost, r.stream3));
        if (s == DISC_OK) s = cuda_status(cudaEventRecord(r.ev_done[async->region], r.stream3));
        if (s == DISC_OK) {
            *queued = true;
            return DISC_OK;
        }
    }
    if (pipe) {
        // the caller's stream continues after the call's work
        cudaEventRecord(r.ev_join, r.stream3);
        cudaStreamWaitEvent(r.stream, r.ev_join, 0);
    }
    std::vector<FrameCounters> c(std::max(hoff, 1));
    // every map's exact voxel count once the call's work is done, into the
    // pinned room buffer: the next call's host bounds start from it
    const int nread = std::min<int>((int)w.size(), 2 * r.Gmax);
    for (int i = 0; i < nread; i++)
        if (cudaMemcpyAsync(r.h_room + i, w[i].m->vt.used, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                            r.stream) != cudaSuccess)
            cudaGetLastError();
    if (hoff > hbase) {
        disc_status s2 = cuda_status(cudaMemcpyAsync(c.data() + hbase, r.d_hist + hbase,
                                                     sizeof(FrameCounters) * (hoff - hbase), cudaMemcpyDeviceToHost,
                                                     r.stream));
        if (s == DISC_OK) s = s2;
    }
    disc_status s3 = cuda_status(cudaStreamSynchronize(r.stream));
    if (s == DISC_OK) s = s3;
    s3 = cuda_status(cudaStreamSynchronize(r.stream2));
    if (s == DISC_OK) s = s3;
    // no copy from the caller's host buffers outlives the call
    s3 = cuda_status(cudaStreamSynchronize(r.stream_in));
    if (s == DISC_OK) s = s3;
    collect_timing(r);
    if (s == DISC_OK)
        for (int i = 0; i < nread; i++) w[i].m->used_upper = (uint64_t)r.h_room[i];
    disc_status first = s;
    for (Work& wk : w) {
        int exact_next_id = -1;  // frames without masks skip the kernel that records it
        wk.done = 0;
        wk.status = DISC_OK;
        for (size_t i = 0; i < wk.hist_idx.size() && hoff > hbase; i++) {
            const FrameCounters& fc = c[wk.hist_idx[i]];
            if (wk.stats) to_stats(fc, wk.stats + i);
            if (wk.status != DISC_OK) continue;
            if (fc.err != 0) {
                wk.status = (disc_status)fc.err;
                continue;
            }
            exact_next_id = std::max(exact_next_id, fc.next_id);
            wk.done++;
        }
        if (exact_next_id > 0) wk.m->next_id_upper = std::max<int64_t>(exact_next_id, 0);
        if (wk.status == DISC_OK && wk.valid < wk.n && wk.done == wk.valid) wk.status = DISC_ERR_INVALID_ARG;
        if (wk.status == DISC_OK && s != DISC_OK && wk.done < wk.valid) wk.status = s;
        if (first == DISC_OK) first = wk.status;
    }
    return first;
}

// the map's own runner, created on first use
disc_status map_runner(disc_map* m)
{
    if (m->run) return DISC_OK;
    Runner* r = new Runner();
    disc_status s = runner_init(*r, m->cfg.device, m->stream, m->D, m->cfg.patch_h, m->cfg.patch_w,
                                m->cfg.max_height, m->cfg.max_width, m->cfg.max_masks, 1, m->cfg.batch_frames,
                                m->cfg.serial_sms, m->cfg.assoc_dim, m->cfg.assoc_patch_h, m->cfg.assoc_patch_w);
    if (s != DISC_OK) {
        runner_release(*r);
        delete r;
        return s;
    }
    r->timing = m->timing_wanted;
    m->run = r;
    return DISC_OK;
}

// Finish the runner's oldest asynchronous call: wait for its work, hand its
// per-frame counters, frames done and status to the caller's pointers, and
// tighten its maps' host bounds: the exact voxel count and next id at its end
// plus what the calls enqueued after it may add (a voxel per pixel, an id per
// mask).  Returns the call's status.
disc_status finish_oldest(Runner& r)
{
    AsyncCall a = std::move(r.pend.front());
    r.pend.pop_front();
    const disc_status s = cuda_status(cudaEventSynchronize(r.ev_done[a.region]));
    const unsigned long long* hu = r.h_used + (size_t)a.region * r.Gmax;
    disc_status first = s;
    for (size_t i = 0; i < a.w.size(); i++) {
        Work& wk = a.w[i];
        disc_map* m = wk.m;
        int exact_next_id = -1;
        wk.done = 0;
        wk.status = DISC_OK;
        for (size_t j = 0; j < wk.hist_idx.size() && s == DISC_OK; j++) {
            const FrameCounters& fc = r.h_hist[wk.hist_idx[j]];
            if (wk.stats) to_stats(fc, wk.stats + j);
            if (wk.status != DISC_OK) continue;
            if (fc.err != 0) {
                wk.status = (disc_status)fc.err;
                continue;
            }
            exact_next_id = std::max(exact_next_id, fc.next_id);
            wk.done++;
        }
        if (s == DISC_OK) {
            if ((int)i < r.Gmax)
                m->used_upper = std::min<uint64_t>(m->used_upper, (uint64_t)hu[i] + (m->px_total - a.px_mark[i]));
            if (exact_next_id > 0)
                m->next_id_upper =
                    std::min<int64_t>(m->next_id_upper, (int64_t)exact_next_id + (m->masks_total - a.masks_mark[i]));
        }
        if (wk.status == DISC_OK && s != DISC_OK && wk.done < wk.valid) wk.status = s;
        if (first == DISC_OK) first = wk.status;
        if (a.n_done) a.n_done[i] = wk.done;
        if (--m->pend_calls <= 0) {
            m->pend_calls = 0;
            m->pend_run = nullptr;
            m->pend_last = -1;
        }
    }
    if (a.result) *a.result = first;
    return first;
}

// Finish every asynchronous call of the runner, oldest first; returns the
// first status that is not DISC_OK.
disc_status finish_all(Runner& r)
{
    disc_status first = DISC_OK;
    while (!r.pend.empty()) {
        const disc_status s = finish_oldest(r);
        if (first == DISC_OK) first = s;
    }
    return first;
}

// Finish the unfinished asynchronous calls that hold the map (its own or a
// group's), so that what follows sees the map after them.
disc_status wait_pending(disc_map* m)
{
    return m->pend_run ? finish_all(*m->pend_run) : DISC_OK;
}

// Enqueue an asynchronous call of the works on runner r (at most two stay
// unfinished: a third finishes the oldest first).  A call with a frame that
// fails the host checks, or one that cannot overlap later calls, runs
// synchronously after the earlier calls have finished, and its results are
// written before returning.
disc_status enqueue_async(Runner& r, std::vector<Work>&& w, int32_t* n_done, disc_status* result)
{
    int64_t frames = 0;
    bool ok = true;
    for (Work& wk : w) {
        if (wk.m->pend_run && wk.m->pend_run != &r) finish_all(*wk.m->pend_run);
        frames += wk.n;
        for (int i = 0; i < wk.n && ok; i++) ok = check_frame(wk.m, r, wk.frames + i) == DISC_OK;
    }
    // calls that cannot overlap run on the caller's stream, after every
    // earlier call has finished
    bool dilate = false;
    for (const Work& wk : w) dilate |= wk.n > 0 && wk.m->cfg.overlap_dilation != 0;
    const bool overlap = !r.timing && (r.serial_sms > 0 || !dilate);
    if (!ok || !overlap || frames > r.hist_cap) finish_all(r);
    while (r.pend.size() >= 2) finish_oldest(r);
    AsyncCall a;
    a.region = r.pend.empty() ? 0 : (r.pend.back().region ^ 1);
    a.n_done = n_done;
    a.result = result;
    a.w = std::move(w);
    for (Work& wk : a.w) wk.prev_idx = wk.m->pend_run == &r ? wk.m->pend_last : -1;
    bool queued = false;
    const disc_status s = run_call(r, a.w, ok && overlap ? &a : nullptr, &queued);
    if (!queued) {
        for (size_t i = 0; i < a.w.size() && n_done; i++) n_done[i] = a.w[i].done;
        if (result) *result = s;
        return s;
    }
    for (Work& wk : a.w) {
        disc_map* m = wk.m;
        a.px_mark.push_back(m->px_total);
        a.masks_mark.push_back(m->masks_total);
        m->pend_run = &r;
        m->pend_calls++;
        if (!wk.hist_idx.empty()) m->pend_last = wk.hist_idx.back();
    }
    r.pend.push_back(std::move(a));
    return DISC_OK;
}

disc_status integrate(disc_map* m, const disc_frame* frames, int n, disc_frame_stats* stats, int* n_done)
{
    if (n_done) *n_done = 0;
    if (m->finalized) return DISC_ERR_INVALID_ARG;
    wait_pending(m);
    disc_status s = map_runner(m);
    if (s != DISC_OK) return s;
    std::vector<Work> w(1);
    w[0].m = m;
    w[0].frames = frames;
    w[0].n = n;
    w[0].stats = stats;
    s = run_call(*m->run, w);
    if (n_done) *n_done = w[0].done;
    return s;
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
    if (set_kernel_attrs() != DISC_OK) return DISC_ERR_CUDA;
    disc_map* m = new disc_map();
    m->cfg = *cfg;
    m->cfg.voxel_capacity = (int64_t)next_pow2((uint64_t)cfg->voxel_capacity);
    if (m->cfg.batch_frames == 0) m->cfg.batch_frames = 32;
    m->D = cfg->embed_dim;
    m->P = cfg->patch_h * cfg->patch_w;
    m->Kpad = (m->P + GEMM_KC - 1) / GEMM_KC * GEMM_KC;
    m->MM = std::max(1, cfg->max_masks);
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
    const uint64_t npx = (uint64_t)cfg->max_width * cfg->max_height;
    const uint64_t scap = next_pow2(npx + npx / 2);  // per-frame hashes: load <= 2/3
    DevAlloc& a = m->mem;
    m->vt.used = a.get<unsigned long long>(1);
    m->d_next_id = a.get<int>(1);
    m->d_flag = a.get<int>(1);
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
    ss.ureg = a.get<unsigned char>(union_region_bytes_full());
    disc_status st = DISC_OK;
    if (a.failed) st = DISC_ERR_OOM;
    if (st == DISC_OK) {
        VoxelTable vt{};
        st = alloc_voxel_table(m, (uint64_t)m->cfg.voxel_capacity, &vt, m->stream);
        if (st == DISC_OK) m->vt = vt;
    }
    if (st == DISC_OK) st = alloc_instances(m, cfg->instance_capacity, &m->inst);
    if (st == DISC_OK) {
        cudaStream_t s = m->stream;
        cudaMemsetAsync(m->vt.used, 0, sizeof(unsigned long long), s);
        cudaMemsetAsync(m->d_next_id, 0, sizeof(int), s);
        cudaMemsetAsync(ss.okeys, 0xFF, sizeof(unsigned long long) * scap, s);
        cudaMemsetAsync(ss.ocnt, 0, sizeof(int32_t) * scap, s);
        cudaMemsetAsync(ss.nkeys, 0xFF, sizeof(unsigned long long) * scap, s);
        cudaMemsetAsync(ss.nown, 0x7F, sizeof(int32_t) * scap, s);  // large positive sentinel
        cudaMemsetAsync(ss.edge_n, 0, sizeof(int32_t), s);
        cudaMemsetAsync(ss.copy_n, 0, sizeof(int32_t), s);
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
    wait_pending(m);
    cudaStreamSynchronize(m->stream);
    if (m->run) {
        runner_release(*m->run);
        delete m->run;
    }
    m->mem.free_all();
    if (m->own_stream) cudaStreamDestroy(m->stream);
    delete m;
}

disc_status disc_integrate_frame(disc_map* m, const disc_frame* f, disc_frame_stats* stats)
{
    if (!m || !f) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
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

disc_status disc_integrate_frames_async(disc_map* m, const disc_frame* frames, int32_t n, disc_frame_stats* stats,
                                        int32_t* n_done, disc_status* result)
{
    if (!m || (n > 0 && !frames) || n < 0 || m->finalized) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    if (n == 0) {
        if (n_done) *n_done = 0;
        if (result) *result = DISC_OK;
        return DISC_OK;
    }
    disc_status s = map_runner(m);
    if (s != DISC_OK) return s;
    std::vector<Work> w(1);
    w[0].m = m;
    w[0].frames = frames;
    w[0].n = n;
    w[0].stats = stats;
    return enqueue_async(*m->run, std::move(w), n_done, result);
}

disc_status disc_map_wait(disc_map* m)
{
    if (!m) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    return wait_pending(m);
}

disc_status disc_map_last_frame(disc_map* m, disc_frame_report* r)
{
    if (!m || !r) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    wait_pending(m);
    CK(cudaStreamSynchronize(m->stream));
    const Runner* run = m->run;
    const bool have = run && run->have_frame;
    const int M = have ? run->last_M : 0, P = m->P, D = m->D;
    r->num_masks = M;
    r->n_seg = 0;
    if (!have) return DISC_OK;
    const Scratch sc = run->bs[run->last_set].frame(run->last_slot);
    FrameCounters c{};
    CK(cudaMemcpy(&c, sc.ctr, sizeof(c), cudaMemcpyDeviceToHost));
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
        // with a second grid, the gate's features and their bound are the view's
        const bool assoc = m->cfg.assoc_dim > 0 && run->Da > 0;
        const Scratch va = assoc ? run->bsa[run->last_set].frame(run->last_slot) : Scratch{};
        if (r->E_bound) {
            float eta = 0.0f, dot_err = 0.0f;
            if (assoc)
                fast_error_terms(m->cfg.precision, run->Kpad_a, run->Da, &eta, &dot_err);
            else
                fast_error_terms(m->cfg.precision, m->Kpad, D, &eta, &dot_err);
            CK(cudaMemcpy(r->E_bound, assoc ? va.Bm : sc.Bm, sizeof(float) * M, cudaMemcpyDeviceToHost));
            for (int i = 0; i < M; i++) r->E_bound[i] *= eta;
        }
        if (assoc && r->A) CK(cudaMemcpy(r->A, va.Ecan, sizeof(float) * (size_t)M * run->Da, cudaMemcpyDeviceToHost));
        if (assoc && r->A_fast)
            CK(cudaMemcpy(r->A_fast, va.Efast, sizeof(float) * (size_t)M * run->Da, cudaMemcpyDeviceToHost));
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

// ---- groups of maps --------------------------------------------------------------------
void disc_group_config_default(disc_group_config* c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->max_maps = 16;
    c->frames_per_map = 4;
    c->embed_dim = 768;
    c->patch_h = 24;
    c->patch_w = 24;
    c->max_width = 640;
    c->max_height = 480;
    c->max_masks = 40;
    c->cuda_stream = nullptr;
    c->device = 0;
}

disc_status disc_group_create(const disc_group_config* cfg, disc_group** out)
{
    if (!cfg || !out) return DISC_ERR_INVALID_ARG;
    *out = nullptr;
    const disc_group_config& c = *cfg;
    if (c.max_maps <= 0 || c.max_maps > 1024 || c.frames_per_map <= 0 || c.frames_per_map > 256 ||
        (int64_t)c.max_maps * c.frames_per_map > 4096)
        return DISC_ERR_INVALID_ARG;
    if (c.embed_dim <= 0 || c.embed_dim > 4096 || c.patch_h <= 0 || c.patch_w <= 0 ||
        (int64_t)c.patch_h * c.patch_w > 16384)
        return DISC_ERR_INVALID_ARG;
    if (c.max_width <= 0 || c.max_height <= 0 || (int64_t)c.max_width * c.max_height > (1 << 24))
        return DISC_ERR_INVALID_ARG;
    if (c.max_masks < 0 || c.max_masks > MAX_MASKS || coverage_smem_bytes(c.max_masks, c.patch_w) > 200 * 1024)
        return DISC_ERR_INVALID_ARG;
    if (c.assoc_dim < 0 || c.assoc_dim > 4096 ||
        (c.assoc_dim > 0 && (c.assoc_patch_h <= 0 || c.assoc_patch_w <= 0 ||
                             (int64_t)c.assoc_patch_h * c.assoc_patch_w > 16384 ||
                             coverage_smem_bytes(c.max_masks, c.assoc_patch_w) > 200 * 1024)))
        return DISC_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
        cudaGetLastError();
        return DISC_ERR_CUDA;
    }
    CK(cudaSetDevice(c.device));
    if (set_kernel_attrs() != DISC_OK) return DISC_ERR_CUDA;
    disc_group* g = new disc_group();
    g->cfg = c;
    cudaStream_t st = (cudaStream_t)c.cuda_stream;
    if (!st) {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete g;
            return DISC_ERR_CUDA;
        }
        g->own_stream = true;
    }
    disc_status s = runner_init(g->run, c.device, st, c.embed_dim, c.patch_h, c.patch_w, c.max_height,
                                c.max_width, c.max_masks, c.max_maps, c.frames_per_map, c.serial_sms, c.assoc_dim,
                                c.assoc_patch_h, c.assoc_patch_w);
    if (s != DISC_OK) {
        runner_release(g->run);
        if (g->own_stream) cudaStreamDestroy(st);
        delete g;
        return s;
    }
    *out = g;
    return DISC_OK;
}

disc_status disc_group_integrate(disc_group* g, disc_map* const* maps, int32_t n_maps,
                                 const disc_frame* const* frames, const int32_t* counts,
                                 disc_frame_stats* const* stats, int32_t* n_done)
{
    if (!g || n_maps < 0 || n_maps > g->cfg.max_maps || (n_maps > 0 && (!maps || !frames || !counts)))
        return DISC_ERR_INVALID_ARG;
    if (n_done)
        for (int i = 0; i < n_maps; i++) n_done[i] = 0;
    std::vector<Work> w(n_maps);
    for (int i = 0; i < n_maps; i++) {
        disc_map* m = maps[i];
        if (!m || counts[i] < 0 || (counts[i] > 0 && !frames[i])) return DISC_ERR_INVALID_ARG;
        if (m->cfg.device != g->cfg.device || m->D != g->cfg.embed_dim || m->cfg.patch_h != g->cfg.patch_h ||
            m->cfg.patch_w != g->cfg.patch_w)
            return DISC_ERR_INVALID_ARG;
        for (int k = 0; k < i; k++)
            if (maps[k] == m) return DISC_ERR_INVALID_ARG;  // one entry per map
        if (m->finalized) return DISC_ERR_INVALID_ARG;
        w[i].m = m;
        w[i].frames = frames[i];
        w[i].n = counts[i];
        w[i].stats = stats ? stats[i] : nullptr;
    }
    if (n_maps == 0) return DISC_OK;
    CK(cudaSetDevice(g->cfg.device));
    // earlier asynchronous calls of the group or of its maps finish first
    finish_all(g->run);
    for (int i = 0; i < n_maps; i++) wait_pending(maps[i]);
    // the maps' own streams may still hold work of earlier calls
    for (int i = 0; i < n_maps; i++) CK(cudaStreamSynchronize(maps[i]->stream));
    disc_status s = run_call(g->run, w);
    if (n_done)
        for (int i = 0; i < n_maps; i++) n_done[i] = w[i].done;
    return s;
}

disc_status disc_group_integrate_async(disc_group* g, disc_map* const* maps, int32_t n_maps,
                                       const disc_frame* const* frames, const int32_t* counts,
                                       disc_frame_stats* const* stats, int32_t* n_done, disc_status* result)
{
    if (!g || n_maps < 0 || n_maps > g->cfg.max_maps || (n_maps > 0 && (!maps || !frames || !counts)))
        return DISC_ERR_INVALID_ARG;
    std::vector<Work> w(n_maps);
    for (int i = 0; i < n_maps; i++) {
        disc_map* m = maps[i];
        if (!m || counts[i] < 0 || (counts[i] > 0 && !frames[i])) return DISC_ERR_INVALID_ARG;
        if (m->cfg.device != g->cfg.device || m->D != g->cfg.embed_dim || m->cfg.patch_h != g->cfg.patch_h ||
            m->cfg.patch_w != g->cfg.patch_w)
            return DISC_ERR_INVALID_ARG;
        for (int k = 0; k < i; k++)
            if (maps[k] == m) return DISC_ERR_INVALID_ARG;  // one entry per map
        if (m->finalized) return DISC_ERR_INVALID_ARG;
        w[i].m = m;
        w[i].frames = frames[i];
        w[i].n = counts[i];
        w[i].stats = stats ? stats[i] : nullptr;
    }
    if (n_maps == 0) {
        if (result) *result = DISC_OK;
        return DISC_OK;
    }
    CK(cudaSetDevice(g->cfg.device));
    for (int i = 0; i < n_maps; i++) CK(cudaStreamSynchronize(maps[i]->stream));
    return enqueue_async(g->run, std::move(w), n_done, result);
}

disc_status disc_group_wait(disc_group* g)
{
    if (!g) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(g->cfg.device));
    return finish_all(g->run);
}

// ---- test hooks: failures made on the host, waits that run out ---------------

void disc_debug_fail_alloc_after(int64_t n) { g_fail_alloc_after.store(n < 0 ? -1 : n); }

disc_status disc_debug_gemm_stall(int32_t device, int32_t on)
{
    CK(cudaSetDevice(device));
    return cuda_status(set_gemm_stall(on != 0));
}

// ---- launch schedule and autotuner -------------------------------------------

namespace {

disc_status set_schedule(Runner& r, const disc_schedule* sch)
{
    if (!sch || sch->geometry_chunk < 1 || sch->geometry_chunk > 32 || sch->serial_ctas < 1 || sch->serial_ctas > 32)
        return DISC_ERR_INVALID_ARG;
    const int pw = sch->probe_width == 0 ? 1 : sch->probe_width;
    if (pw != 1 && pw != 2 && pw != 4 && pw != 8) return DISC_ERR_INVALID_ARG;
    const int ac = sch->assoc_cluster;
    if (ac != 0 && ac != 1 && ac != 2 && ac != 4 && ac != 8) return DISC_ERR_INVALID_ARG;
    const int bsp = sch->batch_split;
    if (bsp != 0 && bsp != 1 && bsp != 2 && bsp != 4 && bsp != 8) return DISC_ERR_INVALID_ARG;
    if (r.geo_chunk == sch->geometry_chunk && r.cta_scale == sch->serial_ctas && r.probe_width == pw &&
        r.assoc_cluster == ac && r.batch_split == bsp)
        return DISC_OK;
    CK(cudaStreamSynchronize(r.stream));
    r.geo_chunk = sch->geometry_chunk;
    r.cta_scale = sch->serial_ctas;
    r.probe_width = pw;
    r.assoc_cluster = ac;
    r.batch_split = bsp;
    for (auto& kv : r.graphs) cudaGraphExecDestroy(kv.second.exec);  // captured with the old schedule
    r.graphs.clear();
    r.shapes_seen.clear();
    return DISC_OK;
}

// Times every candidate schedule on the sample: fresh maps with the given
// configurations take the frames through run_call on runner r; two untimed
// passes (the second captures the graphs), then reps timed ones.
disc_status autotune(Runner& r, const std::vector<const disc_map_config*>& cfgs,
                     const std::vector<std::pair<const disc_frame*, int>>& frames, int reps, disc_tune_report* out)
{
    if (reps < 1 || reps > 100) return DISC_ERR_INVALID_ARG;
    const disc_schedule keep{r.geo_chunk, r.cta_scale, r.probe_width, r.assoc_cluster, r.batch_split};
    disc_tune_report rep{};
    rep.best_ms = 1e300;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    disc_status s = DISC_OK;
    // one candidate's best time over the timed passes
    auto time_schedule = [&](const disc_schedule& cand) -> double {
        if (s != DISC_OK) return 1e300;  // an earlier candidate failed
        s = set_schedule(r, &cand);
        double best = 1e300;
        for (int pass = 0; pass < reps + 2 && s == DISC_OK; pass++) {
            std::vector<disc_map*> maps(cfgs.size(), nullptr);
            std::vector<Work> w(cfgs.size());
            for (size_t i = 0; i < cfgs.size() && s == DISC_OK; i++) {
                disc_map_config c = *cfgs[i];
                c.cuda_stream = r.stream;
                s = disc_map_create(&c, nullptr, &maps[i]);
                w[i].m = maps[i];
                w[i].frames = frames[i].first;
                w[i].n = frames[i].second;
            }
            if (s == DISC_OK) {
                s = cuda_status(cudaEventRecord(e0, r.stream));
                if (s == DISC_OK) s = run_call(r, w);
                if (s == DISC_OK) s = cuda_status(cudaEventRecord(e1, r.stream));
                if (s == DISC_OK) s = cuda_status(cudaEventSynchronize(e1));
                float ms = 0.0f;
                if (s == DISC_OK) s = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
                if (s == DISC_OK && pass >= 2) best = std::min(best, (double)ms);
            }
            for (disc_map* m : maps) disc_map_destroy(m);
        }
        if (s == DISC_OK) {
            rep.candidates++;
            if (best < rep.best_ms) {
                rep.best_ms = best;
                rep.best = cand;
            }
        }
        return best;
    };
    // frames per geometry launch x lanes per key of the lookup x CTAs per
    // map of the association kernel (automatic, or the next smaller cluster),
    // the automatic batch split
    for (int geo : {4, 2, 8})  // the default first
        for (int pw : {1, 2, 4})
            for (int ac : {0, -1}) {
                disc_schedule cand{geo, r.cta_scale, pw, ac, 0};
                if (ac < 0) {  // half the automatic cluster of these maps
                    int c = 1;
                    while (c * 2 <= 8 && (c * 2) * (int)cfgs.size() <= 152) c *= 2;
                    if (c == 1) continue;
                    cand.assoc_cluster = c / 2;
                }
                const double ms = time_schedule(cand);
                if (geo == 4 && pw == 1 && ac == 0) rep.default_ms = ms;
            }
    // then the fastest of these with each other batch split
    const int auto_split = cfgs.size() == 1 ? 2 : 1;
    const disc_schedule base = rep.best;
    for (int bsp : {1, 2, 4}) {
        if (bsp == auto_split) continue;
        disc_schedule cand = base;
        cand.batch_split = bsp;
        time_schedule(cand);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != DISC_OK) {
        set_schedule(r, &keep);
        return s;
    }
    s = set_schedule(r, &rep.best);
    if (out) *out = rep;
    return s;
}

}  // namespace

disc_status disc_map_set_schedule(disc_map* m, const disc_schedule* sch)
{
    if (!m || !sch) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    wait_pending(m);
    disc_status s = map_runner(m);
    return s != DISC_OK ? s : set_schedule(*m->run, sch);
}

disc_status disc_group_set_schedule(disc_group* g, const disc_schedule* sch)
{
    if (!g || !sch) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(g->cfg.device));
    finish_all(g->run);
    return set_schedule(g->run, sch);
}

disc_status disc_map_autotune(disc_map* m, const disc_frame* frames, int32_t n, int32_t reps, disc_tune_report* report)
{
    if (!m || !frames || n <= 0) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    disc_status s = map_runner(m);
    if (s != DISC_OK) return s;
    wait_pending(m);
    CK(cudaStreamSynchronize(m->stream));
    return autotune(*m->run, {&m->cfg}, {{frames, n}}, reps, report);
}

disc_status disc_group_autotune(disc_group* g, disc_map* const* maps, int32_t n_maps, const disc_frame* const* frames,
                                const int32_t* counts, int32_t reps, disc_tune_report* report)
{
    if (!g || !maps || !frames || !counts || n_maps <= 0 || n_maps > g->cfg.max_maps) return DISC_ERR_INVALID_ARG;
    std::vector<const disc_map_config*> cfgs;
    std::vector<std::pair<const disc_frame*, int>> fr;
    for (int i = 0; i < n_maps; i++) {
        if (!maps[i] || !frames[i] || counts[i] <= 0) return DISC_ERR_INVALID_ARG;
        cfgs.push_back(&maps[i]->cfg);
        fr.push_back({frames[i], counts[i]});
    }
    CK(cudaSetDevice(g->cfg.device));
    finish_all(g->run);
    for (int i = 0; i < n_maps; i++) wait_pending(maps[i]);
    return autotune(g->run, cfgs, fr, reps, report);
}

void disc_group_destroy(disc_group* g)
{
    if (!g) return;
    cudaSetDevice(g->cfg.device);
    finish_all(g->run);
    cudaStream_t st = g->run.stream;
    runner_release(g->run);
    if (g->own_stream) cudaStreamDestroy(st);
    delete g;
}

int64_t disc_group_kernel_launches(disc_group* g) { return g ? g->run.launches : 0; }

int64_t disc_group_device_bytes(disc_group* g) { return g ? g->run.mem.bytes : 0; }

disc_status disc_group_set_phase_timing(disc_group* g, int32_t enable)
{
    if (!g) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(g->cfg.device));
    finish_all(g->run);
    CK(cudaStreamSynchronize(g->run.stream));
    reset_timing(g->run, enable != 0);
    return DISC_OK;
}

disc_status disc_group_phase_times(disc_group* g, double* ms, int64_t* launches, int64_t* calls, int32_t n)
{
    if (!g || n < 0) return DISC_ERR_INVALID_ARG;
    for (int i = 0; i < n && i < PH_COUNT; i++) {
        if (ms) ms[i] = g->run.phase_ms[i];
        if (launches) launches[i] = g->run.phase_launches[i];
        if (calls) calls[i] = g->run.phase_calls[i];
    }
    return DISC_OK;
}

disc_status disc_map_counts(disc_map* m, int64_t* nv, int32_t* nid)
{
    if (!m) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    wait_pending(m);
    CK(cudaStreamSynchronize(m->stream));
    if (nv) *nv = (int64_t)read_used(m, m->stream);
    if (nid) *nid = read_next_id(m, m->stream);
    return DISC_OK;
}

disc_status disc_map_export_voxels(disc_map* m, uint64_t* keys, int32_t* ids, int64_t cap)
{
    if (!m || (cap > 0 && (!keys || !ids))) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    wait_pending(m);
    CK(cudaStreamSynchronize(m->stream));
    const uint64_t tc = m->vt.mask + 1;
    std::vector<unsigned long long> k(tc);
    std::vector<int32_t> l(tc);
    const int nid = read_next_id(m, m->stream);
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

disc_status disc_map_export_assoc(disc_map* m, float* A, int32_t cap)
{
    if (!m || !A || m->cfg.assoc_dim <= 0) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    wait_pending(m);
    CK(cudaStreamSynchronize(m->stream));
    const int n = read_next_id(m, m->stream);
    if (n > cap) return DISC_ERR_INVALID_ARG;
    if (n > 0) CK(cudaMemcpy(A, m->inst.A, sizeof(float) * (size_t)n * m->inst.Da, cudaMemcpyDeviceToHost));
    return DISC_OK;
}

disc_status disc_map_export_instances(disc_map* m, int32_t* parent, int64_t* count, float* Q, float* E,
                                      int32_t* n_obs, int32_t cap)
{
    if (!m) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    wait_pending(m);
    CK(cudaStreamSynchronize(m->stream));
    const int n = read_next_id(m, m->stream);
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
    wait_pending(m);
    CK(cudaStreamSynchronize(m->stream));
    const int nid = read_next_id(m, m->stream);
    const int D = m->D;
    if (nid == 0) {
        for (int64_t i = 0; i < (int64_t)nq * k; i++) {
            ids[i] = -1;
            scores[i] = -INFINITY;
        }
        return DISC_OK;
    }
    const size_t b_q = align256(sizeof(float) * (size_t)nq * D), b_s = align256(sizeof(float) * (size_t)nq * nid);
    const size_t b_o = align256(sizeof(float) * (size_t)nq * k);
    unsigned char* base = query_scratch(m, b_q + b_s + 2 * b_o);
    if (!base) return DISC_ERR_OOM;
    float* dq = (float*)base;
    float* dsc = (float*)(base + b_q);
    float* dout = (float*)(base + b_q + b_s);
    int* dids = (int*)(base + b_q + b_s + b_o);
    CK(cudaMemcpyAsync(dq, q, sizeof(float) * (size_t)nq * D, cudaMemcpyHostToDevice, m->stream));
    launch_query_topk(dq, nq, D, m->inst, nid, dsc, k, dids, dout, m->stream);
    CK(cudaMemcpyAsync(ids, dids, sizeof(int) * (size_t)nq * k, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaMemcpyAsync(scores, dout, sizeof(float) * (size_t)nq * k, cudaMemcpyDeviceToHost, m->stream));
    return cuda_status(cudaStreamSynchronize(m->stream));
}

disc_status disc_query_points(disc_map* m, const float* xyz, int64_t n, int32_t* ids)
{
    if (!m || n < 0 || (n > 0 && (!xyz || !ids))) return DISC_ERR_INVALID_ARG;
    if (n == 0) return DISC_OK;
    CK(cudaSetDevice(m->cfg.device));
    wait_pending(m);
    const size_t b_x = align256(sizeof(float) * 3 * (size_t)n);
    unsigned char* base = query_scratch(m, b_x + sizeof(int) * (size_t)n);
    if (!base) return DISC_ERR_OOM;
    float* dx = (float*)base;
    int* di = (int*)(base + b_x);
    CK(cudaMemcpyAsync(dx, xyz, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, m->stream));
    launch_query_points(dx, n, m->cfg.voxel_size, m->vt, m->inst, di, m->stream);
    CK(cudaMemcpyAsync(ids, di, sizeof(int) * n, cudaMemcpyDeviceToHost, m->stream));
    return cuda_status(cudaStreamSynchronize(m->stream));
}

// checkpoint file: magic, config, counts, voxels (key, label), instance table
// A checkpoint's arrays as the device code expects them:
//   voxel keys packed (three 18-bit fields, below 2^54), hence never the
//     table's empty marker, and pairwise distinct;
//   voxel labels in [0, nid) (-1 too in a finalised map, whose dropped
//     instances leave unlabelled voxels);
//   parents in [0, nid) and flat (the parent of a parent is itself);
//   voxel counts and observation counts non-negative;
//   Q and every embedding entry finite, |entry| <= 1024 (a stored embedding
//     is a weighted mean of tokens, which obey that bound).
static bool checkpoint_contents_ok(const uint64_t* keys, const int32_t* ids, int64_t nv, const int32_t* parent,
                                   const int64_t* count, const float* Q, const float* E, const int32_t* obs,
                                   int32_t nid, int D, const float* A, int Da, bool finalized)
{
    for (int64_t i = 0; i < nv; i++) {
        if (keys[i] >> 54) return false;
        if (ids[i] >= nid || ids[i] < (finalized ? -1 : 0)) return false;
    }
    std::vector<uint64_t> sorted(keys, keys + nv);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return false;
    auto entry_ok = [](float x) { return std::isfinite(x) && std::fabs(x) <= 1024.0f; };
    for (int32_t i = 0; i < nid; i++) {
        if (parent[i] < 0 || parent[i] >= nid || parent[parent[i]] != parent[i]) return false;
        if (count[i] < 0 || obs[i] < 0 || !std::isfinite(Q[i])) return false;
    }
    for (size_t i = 0; i < (size_t)nid * D; i++)
        if (!entry_ok(E[i])) return false;
    for (size_t i = 0; A && i < (size_t)nid * Da; i++)
        if (!entry_ok(A[i])) return false;
    return true;
}

static const char kMagic[8] = {'D', 'I', 'S', 'C', 'M', 'A', 'P', '1'};
static const char kMagicFinal[8] = {'D', 'I', 'S', 'C', 'M', 'A', 'P', 'F'};  // a finalised map

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
    const int Da = m->cfg.assoc_dim;
    std::vector<float> A((size_t)std::max(nid, 1) * std::max(Da, 1));
    if (Da > 0) s = disc_map_export_assoc(m, A.data(), nid);
    if (s != DISC_OK) return s;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return DISC_ERR_INVALID_ARG;
    disc_map_config c = m->cfg;
    c.cuda_stream = nullptr;
    bool ok = std::fwrite(m->finalized ? kMagicFinal : kMagic, 1, 8, fp) == 8 && std::fwrite(&c, sizeof(c), 1, fp) == 1 &&
              std::fwrite(&nv, sizeof(nv), 1, fp) == 1 && std::fwrite(&nid, sizeof(nid), 1, fp) == 1;
    if (ok && nv) ok = std::fwrite(keys.data(), 8, nv, fp) == (size_t)nv && std::fwrite(ids.data(), 4, nv, fp) == (size_t)nv;
    if (ok && nid)
        ok = std::fwrite(parent.data(), 4, nid, fp) == (size_t)nid && std::fwrite(count.data(), 8, nid, fp) == (size_t)nid &&
             std::fwrite(Q.data(), 4, nid, fp) == (size_t)nid &&
             std::fwrite(E.data(), 4, (size_t)nid * D, fp) == (size_t)nid * D && std::fwrite(obs.data(), 4, nid, fp) == (size_t)nid;
    if (ok && nid && Da > 0) ok = std::fwrite(A.data(), 4, (size_t)nid * Da, fp) == (size_t)nid * Da;
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
    bool ok = std::fread(magic, 1, 8, fp) == 8 &&
              (std::memcmp(magic, kMagic, 8) == 0 || std::memcmp(magic, kMagicFinal, 8) == 0) &&
              std::fread(&c, sizeof(c), 1, fp) == 1 && std::fread(&nv, sizeof(nv), 1, fp) == 1 &&
              std::fread(&nid, sizeof(nid), 1, fp) == 1 && nv >= 0 && nv <= (int64_t(1) << 40) && nid >= 0 &&
              config_ok(c);
    // the header's sizes must account for the whole file before anything is
    // allocated from them
    if (ok) {
        const long here = std::ftell(fp);
        const uint64_t per_id = 4 + 8 + 4 + 4 * (uint64_t)c.embed_dim + 4 + 4 * (uint64_t)c.assoc_dim;
        const uint64_t want = (uint64_t)here + 12 * (uint64_t)nv + per_id * (uint64_t)nid;
        ok = here > 0 && std::fseek(fp, 0, SEEK_END) == 0 && (uint64_t)std::ftell(fp) == want &&
             std::fseek(fp, here, SEEK_SET) == 0;
    }
    if (!ok) {
        std::fclose(fp);
        return DISC_ERR_INVALID_ARG;
    }
    try {
    const int D = c.embed_dim;
    std::vector<uint64_t> keys(std::max<int64_t>(nv, 1));
    std::vector<int32_t> ids(std::max<int64_t>(nv, 1));
    std::vector<int32_t> parent(std::max(nid, 1)), obs(std::max(nid, 1));
    std::vector<int64_t> count(std::max(nid, 1));
    std::vector<float> Q(std::max(nid, 1)), E((size_t)std::max(nid, 1) * D);
    const int Da = c.assoc_dim;
    const int Ds = Da > 0 ? Da : D;  // length of the scoring master's rows
    std::vector<uint16_t> Eb(c.precision == DISC_BF16 ? (size_t)std::max(nid, 1) * Ds : 0);
    std::vector<float> A((size_t)std::max(nid, 1) * std::max(Da, 1));
    if (ok && nv) ok = std::fread(keys.data(), 8, nv, fp) == (size_t)nv && std::fread(ids.data(), 4, nv, fp) == (size_t)nv;
    if (ok && nid)
        ok = std::fread(parent.data(), 4, nid, fp) == (size_t)nid && std::fread(count.data(), 8, nid, fp) == (size_t)nid &&
             std::fread(Q.data(), 4, nid, fp) == (size_t)nid &&
             std::fread(E.data(), 4, (size_t)nid * D, fp) == (size_t)nid * D && std::fread(obs.data(), 4, nid, fp) == (size_t)nid;
    if (ok && nid && Da > 0) ok = std::fread(A.data(), 4, (size_t)nid * Da, fp) == (size_t)nid * Da;
    std::fclose(fp);
    fp = nullptr;
    if (!ok) return DISC_ERR_INVALID_ARG;
    // the contents too, before anything reaches a device: the kernels index
    // the instance arrays with voxel labels and parents, and the voxel table
    // needs distinct keys that differ from its empty marker
    if (!checkpoint_contents_ok(keys.data(), ids.data(), nv, parent.data(), count.data(), Q.data(), E.data(),
                                obs.data(), nid, D, Da > 0 ? A.data() : nullptr, Da,
                                std::memcmp(magic, kMagicFinal, 8) == 0))
        return DISC_ERR_INVALID_ARG;
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
        if (m->inst.A) cudaMemcpyAsync(m->inst.A, A.data(), 4 * (size_t)nid * Da, cudaMemcpyHostToDevice, m->stream);
        if (m->inst.Eb) {
            // bf16 scoring copy of the scoring master, rounded to nearest even
            // as on the device
            const std::vector<float>& Sm = Da > 0 ? A : E;
            for (size_t i = 0; i < (size_t)nid * Ds; i++) {
                uint32_t b;
                std::memcpy(&b, &Sm[i], 4);
                Eb[i] = (uint16_t)((b + 0x7fffu + ((b >> 16) & 1u)) >> 16);
            }
            cudaMemcpyAsync(m->inst.Eb, Eb.data(), 2 * (size_t)nid * Ds, cudaMemcpyHostToDevice, m->stream);
        }
        if (m->inst.E8) launch_e4m3_copies(m->inst, nid, D, m->stream);  // from the scoring master
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
    m->finalized = std::memcmp(magic, kMagicFinal, 8) == 0;
    *out = m;
    return DISC_OK;
    } catch (const std::bad_alloc&) {
        if (fp) std::fclose(fp);
        return DISC_ERR_OOM;
    }
}

disc_status disc_map_finalize(disc_map* m, const disc_finalize_config* cfg, disc_finalize_report* rep)
{
    if (!m || !cfg || cfg->contact_den <= 0 || cfg->contact_num < 0 || cfg->min_voxels < 0) return DISC_ERR_INVALID_ARG;
    if (m->finalized) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    wait_pending(m);
    CK(cudaStreamSynchronize(m->stream));
    const int nid = read_next_id(m, m->stream);
    cudaStream_t st = m->stream;
    uint64_t pcap = next_pow2(std::max<uint64_t>(4096, 16 * (uint64_t)nid));
    int32_t ctr[FIN_NCTR] = {};
    unsigned long long removed_voxels = 0;
    for (int attempt = 0; attempt < 4; attempt++, pcap *= 4) {
        DevAlloc a;
        FinalizeScratch fs{};
        fs.pkeys = a.get<unsigned long long>(pcap);
        fs.pcnt = a.get<int32_t>(pcap);
        fs.plist = a.get<int32_t>(pcap);
        fs.pmask = pcap - 1;
        fs.ea = a.get<int32_t>(pcap);
        fs.eb = a.get<int32_t>(pcap);
        fs.comp = a.get<int32_t>(std::max(nid, 1));
        fs.win = a.get<unsigned long long>(std::max(nid, 1));
        fs.drop = a.get<unsigned char>(std::max(nid, 1));
        fs.ctr = a.get<int32_t>(FIN_NCTR);
        fs.removed_voxels = a.get<unsigned long long>(1);
        if (a.failed) {
            a.free_all();
            return DISC_ERR_OOM;
        }
        disc_status s = DISC_OK;
        auto run = [&](int phase) {
            if (s != DISC_OK) return;
            launch_finalize(phase, m->vt, m->inst, nid, m->D, fs, cfg->min_voxels, cfg->contact_num,
                            cfg->contact_den, cfg->tau_cos, st);
            s = cuda_status(cudaMemcpyAsync(ctr, fs.ctr, sizeof(ctr), cudaMemcpyDeviceToHost, st));
            if (s == DISC_OK) s = cuda_status(cudaStreamSynchronize(st));
            if (s == DISC_OK && ctr[FIN_ERR]) s = (disc_status)ctr[FIN_ERR];
        };
        s = cuda_status(cudaMemsetAsync(fs.pkeys, 0xFF, sizeof(unsigned long long) * pcap, st));
        if (s == DISC_OK) s = cuda_status(cudaMemsetAsync(fs.pcnt, 0, sizeof(int32_t) * pcap, st));
        if (s == DISC_OK) s = cuda_status(cudaMemsetAsync(fs.ctr, 0, sizeof(int32_t) * FIN_NCTR, st));
        if (s == DISC_OK) s = cuda_status(cudaMemsetAsync(fs.removed_voxels, 0, sizeof(unsigned long long), st));
        run(0);  // contacts: the map is untouched until phase 2
        if (s == DISC_ERR_TABLE_FULL) {
            a.free_all();
            continue;  // more distinct contact pairs than slots: a larger pair table
        }
        run(1);
        run(2);
        if (s == DISC_OK)
            s = cuda_status(cudaMemcpy(&removed_voxels, fs.removed_voxels, sizeof(removed_voxels), cudaMemcpyDeviceToHost));
        a.free_all();
        if (s != DISC_OK) return s;
        m->finalized = true;
        if (rep) {
            rep->contact_pairs = ctr[FIN_PAIRS];
            rep->merged = ctr[FIN_MERGED];
            rep->removed = ctr[FIN_REMOVED];
            rep->removed_voxels = (int64_t)removed_voxels;
        }
        return DISC_OK;
    }
    return DISC_ERR_TABLE_FULL;
}

uint64_t disc_pack_key(int32_t kx, int32_t ky, int32_t kz)
{
    const uint64_t mask = (1ull << KEY_BITS) - 1;
    return (((uint64_t)(kx + KEY_BIAS) & mask) << (2 * KEY_BITS)) | (((uint64_t)(ky + KEY_BIAS) & mask) << KEY_BITS) |
           ((uint64_t)(kz + KEY_BIAS) & mask);
}

int64_t disc_map_device_bytes(disc_map* m) { return m ? m->mem.bytes + (m->run ? m->run->mem.bytes : 0) : 0; }

int64_t disc_map_kernel_launches(disc_map* m) { return m && m->run ? m->run->launches : 0; }

disc_status disc_map_set_phase_timing(disc_map* m, int32_t enable)
{
    if (!m) return DISC_ERR_INVALID_ARG;
    CK(cudaSetDevice(m->cfg.device));
    wait_pending(m);
    CK(cudaStreamSynchronize(m->stream));
    m->timing_wanted = enable != 0;
    if (m->run) reset_timing(*m->run, enable != 0);
    return DISC_OK;
}

disc_status disc_map_phase_times(disc_map* m, double* ms, int64_t* launches, int64_t* calls, int32_t n)
{
    if (!m || n < 0) return DISC_ERR_INVALID_ARG;
    for (int i = 0; i < n && i < PH_COUNT; i++) {
        if (ms) ms[i] = m->run ? m->run->phase_ms[i] : 0.0;
        if (launches) launches[i] = m->run ? m->run->phase_launches[i] : 0;
        if (calls) calls[i] = m->run ? m->run->phase_calls[i] : 0;
    }
    return DISC_OK;
}

const char* disc_phase_name(int32_t i)
{
    static const char* names[PH_COUNT] = {"clear",     "token_stats", "coverage",    "weights", "pool_exact",
                                          "pool_gemm", "dbscan",      "backproject", "entries", "overlap",
                                          "score",     "union",       "apply",       "lookup",  "associate",
                                          "commit"};
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
