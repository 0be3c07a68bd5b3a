// Host runtime of the wave path tracer: contexts, scene upload with a binned-SAH BVH build,
// render validation, launch slots, and the C-ABI entry points declared in include/hpt.h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "hpt.h"
#include "hpt_internal.h"

namespace hpt {
cudaError_t wave_gen(int prec, const JobTable *, const WaveDesc &, const PathBufs &, SlotScratch *, cudaStream_t);
cudaError_t wave_trace(int prec, bool stats, const JobTable *, const WaveDesc &, const PathBufs &, SlotScratch *, int it,
                       int grid, cudaStream_t);
cudaError_t wave_shade(int prec, bool stats, const JobTable *, const WaveDesc &, const PathBufs &, SlotScratch *, int it,
                       int grid, cudaStream_t);
cudaError_t wave_accum(int prec, const JobTable *, const WaveDesc &, const PathBufs &, SlotScratch *, cudaStream_t);
int wave_occupancy(int prec, int which);
cudaError_t wave_preload(int prec);
void fixed_scratch_setup(int dev);
cudaError_t fixed_scratch_status(int dev, unsigned *bits);
}  // namespace hpt

using namespace hpt;

// ------------------------------------------------------------------------------ errors
static thread_local std::string g_err;

static hpt_status fail(hpt_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CUDA_TRY(call)                                                                             \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? HPT_ERR_OOM : HPT_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                        \
    } while (0)

static RC make_rc(double x)
{
    RC r;
    r.d = x;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}

// ------------------------------------------------------------------------- BVH builder
namespace {

struct Box {
    float lo[3], hi[3];
    void reset()
    {
        for (int k = 0; k < 3; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    }
    void grow(const Box &b)
    {
        for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], b.lo[k]); hi[k] = std::max(hi[k], b.hi[k]); }
    }
    void grow(const float *p)
    {
        for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], p[k]); hi[k] = std::max(hi[k], p[k]); }
    }
};

struct BuildNode {
    Box box;
    int left = -1, right = -1;   // build-node indices (inner)
    int start = 0, count = 0;    // leaf range in the primitive order
};

struct Builder {
    const std::vector<Box> &pb;
    const std::vector<float> &cent;   // 3 per primitive
    std::vector<int> idx;
    std::vector<BuildNode> nodes;
    int max_depth_seen = 0;
    // depth <= TSTACK - 1: a near-first traversal then never holds more than TSTACK entries
#ifndef HPT_SAH_CT
#define HPT_SAH_CT 0.5
#endif
#ifndef HPT_LEAF_MAX
#define HPT_LEAF_MAX 2
#endif
#ifndef HPT_LEAF_CAP
#define HPT_LEAF_CAP 4
#endif
#ifndef HPT_PRIMARY_SIDE_W
#define HPT_PRIMARY_SIDE_W 0.2
#endif
    // SAH in units of one triangle test: a split costs CT (one node visit) times the node's area
    // plus the children's area-weighted triangle counts; a leaf costs its area times its count.
    // Nodes of at most LEAF_MAX triangles are always leaves, nodes of up to LEAF_CAP become
    // leaves when no split is cheaper.
    static constexpr int BINS = 32, LEAF_MAX = HPT_LEAF_MAX, LEAF_CAP = HPT_LEAF_CAP, DEPTH_LIMIT = TSTACK - 1;
    static constexpr double CT = HPT_SAH_CT;
    // weights of the box faces normal to x, y and z in the surface-area heuristic: all 1 for
    // rays in every direction; rays along one axis meet a box in proportion to its face across
    // that axis, so a tree for them weights the other two faces down
    double wface[3] = {1.0, 1.0, 1.0};

    Builder(const std::vector<Box> &pb_, const std::vector<float> &c_, std::vector<int> prims)
        : pb(pb_), cent(c_), idx(std::move(prims)) {}

    double area(const Box &b) const
    {
        double dx = b.hi[0] - b.lo[0], dy = b.hi[1] - b.lo[1], dz = b.hi[2] - b.lo[2];
        if (dx < 0 || dy < 0 || dz < 0) return 0.0;
        return 2.0 * (wface[0] * dy * dz + wface[1] * dz * dx + wface[2] * dx * dy);
    }

    int make_leaf(const Box &b, int start, int count)
    {
        BuildNode n;
        n.box = b;
        n.start = start;
        n.count = count;
        nodes.push_back(n);
        return (int)nodes.size() - 1;
    }

    int build(int start, int count, int depth)
    {
        max_depth_seen = std::max(max_depth_seen, depth);
        Box b, cb;
        b.reset();
        cb.reset();
        for (int i = start; i < start + count; ++i) {
            b.grow(pb[idx[i]]);
            cb.grow(&cent[3 * idx[i]]);
        }
        if (count <= LEAF_MAX || (depth >= DEPTH_LIMIT && count <= 255)) return make_leaf(b, start, count);
        // binned SAH over the three axes
        double best_cost = INFINITY;
        int best_axis = -1, best_split = -1;
        for (int ax = 0; ax < 3; ++ax) {
            float ext = cb.hi[ax] - cb.lo[ax];
            if (!(ext > 0.0f)) continue;
            Box bb[BINS];
            int bc[BINS] = {0};
            for (int k = 0; k < BINS; ++k) bb[k].reset();
            double scale = BINS / (double)ext;
            for (int i = start; i < start + count; ++i) {
                int k = std::min(BINS - 1, (int)((cent[3 * idx[i] + ax] - cb.lo[ax]) * scale));
                bc[k]++;
                bb[k].grow(pb[idx[i]]);
            }
            double la[BINS];
            int ln[BINS];
            Box acc;
            acc.reset();
            int n = 0;
            for (int k = 0; k < BINS - 1; ++k) {
                acc.grow(bb[k]);
                n += bc[k];
                la[k] = area(acc);
                ln[k] = n;
            }
            acc.reset();
            n = 0;
            for (int k = BINS - 1; k > 0; --k) {
                acc.grow(bb[k]);
                n += bc[k];
                if (ln[k - 1] == 0 || n == 0) continue;
                double cost = CT * area(b) + la[k - 1] * ln[k - 1] + area(acc) * n;
                if (cost < best_cost) { best_cost = cost; best_axis = ax; best_split = k; }
            }
        }
        double leaf_cost = area(b) * count;
        if (depth < DEPTH_LIMIT && count <= 255 && (best_axis < 0 || (best_cost >= leaf_cost && count <= LEAF_CAP)))
            return make_leaf(b, start, count);
        if (depth >= DEPTH_LIMIT) best_axis = -1;   // forced median split of an oversized deep node
        int mid;
        if (best_axis >= 0) {
            double scale = BINS / (double)(cb.hi[best_axis] - cb.lo[best_axis]);
            float lo = cb.lo[best_axis];
            int ax = best_axis, sp = best_split;
            auto it = std::partition(idx.begin() + start, idx.begin() + start + count, [&](int p) {
                int k = std::min(BINS - 1, (int)((cent[3 * p + ax] - lo) * scale));
                return k < sp;
            });
            mid = (int)(it - idx.begin());
            if (mid == start || mid == start + count) mid = start + count / 2;
        } else {
            mid = start + count / 2;   // identical centroids: split the list
        }
        int id = (int)nodes.size();
        nodes.push_back(BuildNode());
        nodes[id].box = b;
        int l = build(start, mid - start, depth + 1);
        int r = build(mid, start + count - mid, depth + 1);
        nodes[id].left = l;
        nodes[id].right = r;
        return id;
    }
};

}  // namespace

// ------------------------------------------------------------------------------ context
struct SceneRec {
    void *arena = nullptr;
    void *cache_buf = nullptr;      // a cache set after upload (hpt_scene_set_cache)
    size_t bytes = 0;
    DevScene dev{};
    int n_nodes = 0, depth = 0;
    std::atomic<int> users{0};
};

struct Slot {
    JobTable *d_table = nullptr;
    JobTable *h_table = nullptr;   // pinned
    cudaEvent_t done = nullptr;
    bool used = false;
};

struct Request {
    uint64_t id = 0;
    SceneRec *scene = nullptr;
    DevJob job{};
    int prec = 1;
    long long next = 0;          // next work item to schedule
    size_t out_bytes = 0;
    bool lib_out = false;        // the output is allocated by the library at admission
    void *out_lib = nullptr;     // that output (device), until hpt_request_release
    double t_submit = 0, t_admit = -1, t_done = -1;
    bool admitted = false;
    bool stopped = false;        // no more waves: cancelled or a wave failed to issue
    int waves = 0;               // issued waves carrying its items that have not completed
    unsigned dev_bits = 0;       // kernel status bits of those waves
    hpt_status status = HPT_OK;  // final status once done
    std::string err;             // message of a failed status
    bool done = false;
};

struct InflightWave {
    cudaEvent_t ev = nullptr;
    int status_slot = -1;                               // pinned word holding the wave's status bits
    std::vector<std::shared_ptr<Request>> carried;      // requests with items in this wave
};

struct hpt_ctx {
    int device = 0;
    int sm_count = 0;
    int grid_trace[2] = {1, 1}, grid_shade[2] = {1, 1};
    int occ_trace[2] = {1, 1}, occ_shade[2] = {1, 1};   // resident blocks per SM of the two kernels
    int lanes = HPT_LANES;                               // wave lanes of a trace (1 .. HPT_MAX_LANES)
    int trace_mult = 1, shade_mult = 1;                  // grid = SMs x resident blocks x mult
    struct Shape {
        int cap, lanes, tm, sm;
    };
    Shape tuned[HPT_SCENE_CLASSES]{};                    // hpt_autotune results per scene-size class
    bool tuned_valid[HPT_SCENE_CLASSES] = {};
    // path state of one wave (capacity paths), all wave work runs on wstream
    PathBufs pb{};
    void *pb_arena = nullptr;
    // wave lanes: consecutive waves of a trace rotate over lane 0 (pb, d_scr, wstream) and the
    // extra lanes below, so that one wave's kernels fill the others' launch gaps and tails
    static constexpr int EXTRA_LANES = HPT_MAX_LANES - 1;
    void *pb_arena_x[EXTRA_LANES > 0 ? EXTRA_LANES : 1] = {};
    PathBufs pb_x[EXTRA_LANES > 0 ? EXTRA_LANES : 1]{};
    SlotScratch *d_scr_x[EXTRA_LANES > 0 ? EXTRA_LANES : 1] = {};
    cudaStream_t wstream_x[EXTRA_LANES > 0 ? EXTRA_LANES : 1] = {};
    cudaEvent_t ev_fork = nullptr, ev_join_x[EXTRA_LANES > 0 ? EXTRA_LANES : 1] = {};
    // the serving scheduler's own lanes (allocated at its first wave): its waves rotate over
    // them independently of the trace calls' lanes
    void *spb_arena[HPT_LANES] = {};
    PathBufs spb[HPT_LANES]{};
    SlotScratch *sscr[HPT_LANES] = {};
    cudaStream_t slane_stream[HPT_LANES] = {};
    cudaEvent_t slane_ev[HPT_LANES] = {};   // end of the lane's latest wave
    int sched_next = 0;
    int capacity = 1 << 23;   // paths per wave of a trace (~1.7 GB of path state per lane)
    int sched_capacity = 1 << 23;   // paths per serving wave (fixed when the context is created)
    int debug_waves = 0;
    // captured frames of hpt_trace, keyed by what fixes the launch sequence
    // A captured frame reads its job table from d_table; each replay first copies the
    // caller's descriptor there from one of TABLE_RING pinned buffers, so the host only waits
    // when it runs TABLE_RING copies ahead of the device.
    static constexpr int TABLE_RING = 4;
    struct FrameGraph {
        int prec = 0, spp = 0, max_depth = 0, capacity = 0;
        long long n_items = 0;
        void *out = nullptr;
        JobTable *d_table = nullptr;
        JobTable *h_ring[TABLE_RING] = {};
        cudaEvent_t copied[TABLE_RING] = {};
        bool ring_used[TABLE_RING] = {};
        int ring_next = 0;
        cudaGraphExec_t exec = nullptr;
        cudaEvent_t done = nullptr;
        uint64_t last_use = 0;
    };
    std::vector<FrameGraph> graphs;
    bool use_graphs = true;
    uint64_t graph_clock = 0;
    // per-kernel timing (hpt_trace_timed): an event before every launch of a wave, one kind each
    struct KernelTimer {
        std::vector<cudaEvent_t> ev;
        std::vector<int> kind;
        size_t used = 0;
    };
    KernelTimer *timer = nullptr;
    SlotScratch *d_scr = nullptr;
    cudaStream_t wstream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::mutex mu;
    std::map<uint64_t, std::unique_ptr<SceneRec>> scenes;
    uint64_t next_scene = 1;
    static constexpr int NSLOTS = 16;
    Slot slots[NSLOTS];
    int next_slot = 0;
    void *host_out_dev = nullptr;
    // hpt_trace_host into pinned memory: finished rows leave on their own stream while later
    // waves run
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_wave = nullptr, ev_copied = nullptr;
    float4 *d_sincos = nullptr;
    size_t host_out_bytes = 0;
    std::chrono::steady_clock::time_point t0;
    // serving
    uint64_t budget = 0;                 // device bytes of in-flight request outputs
    int max_inflight = 8;                // requests on the device at once
    size_t max_queue = 4096;             // pending requests before hpt_submit says BUSY
    int flags = 0;                       // HPT_CTX_* of the descriptor
    std::mutex smu;
    std::condition_variable scv, dcv;
    std::deque<std::shared_ptr<Request>> pending;
    std::vector<std::shared_ptr<Request>> active;
    std::map<uint64_t, std::shared_ptr<Request>> reqs;
    std::deque<uint64_t> finished;       // ids of finished requests, oldest first (bounded retention)
    std::deque<InflightWave> inflight;
    std::vector<cudaEvent_t> free_events;
    static constexpr int STATUS_SLOTS = 16;
    unsigned *h_wave_status = nullptr;   // pinned, one word per in-flight serving wave
    bool status_slot_used[STATUS_SLOTS] = {};
    cudaStream_t ostream = nullptr;      // allocation, copy-out and release of library-owned outputs
    uint64_t next_req = 1;
    uint64_t bytes_active = 0;           // outputs of admitted, not yet finished requests
    int live = 0;                        // admitted, not yet finished requests
    size_t rr = 0;
    bool stop = false;
    std::thread sched;
    double now_us() const
    {
        return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
    }
};

static hpt_status check_ctx(hpt_ctx *ctx)
{
    if (!ctx) return fail(HPT_ERR_INVALID_ARG, "ctx is NULL");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail(HPT_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return HPT_OK;
}

static void sched_loop(hpt_ctx *ctx);

extern "C" const char *hpt_last_error(void) { return g_err.c_str(); }

extern "C" hpt_status hpt_create(hpt_ctx **out, int device, const hpt_ctx_desc *desc)
{
    g_err.clear();
    if (!out) return fail(HPT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(HPT_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, ndev);
    CUDA_TRY(cudaSetDevice(device));
    auto ctx = std::make_unique<hpt_ctx>();
    ctx->device = device;
    ctx->t0 = std::chrono::steady_clock::now();
    CUDA_TRY(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device));
    for (int prec = 0; prec < 2; ++prec) {
        CUDA_TRY(wave_preload(prec));   // all wave kernels loaded now, not at a first launch
        ctx->occ_trace[prec] = wave_occupancy(prec, 0);
        ctx->occ_shade[prec] = wave_occupancy(prec, 1);
        ctx->grid_trace[prec] = ctx->sm_count * ctx->occ_trace[prec];
        ctx->grid_shade[prec] = ctx->sm_count * ctx->occ_shade[prec];
    }
    if (const char *e = getenv("HPT_WAVE_PATHS")) ctx->capacity = std::max(1 << 12, std::min(atoi(e), 1 << 26));
    ctx->sched_capacity = ctx->capacity;
    if (const char *e = getenv("HPT_DEBUG_WAVES")) ctx->debug_waves = atoi(e);
    if (desc) ctx->flags = desc->flags;
    if (desc && (desc->flags & HPT_CTX_NO_GRAPHS)) ctx->use_graphs = false;
    if (const char *e = getenv("HPT_GRAPHS")) ctx->use_graphs = atoi(e) != 0;
    CUDA_TRY(cudaMalloc(&ctx->d_scr, sizeof(SlotScratch)));
    CUDA_TRY(cudaMemset(ctx->d_scr, 0, sizeof(SlotScratch)));
    CUDA_TRY(cudaStreamCreateWithFlags(&ctx->wstream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    for (int l = 0; l < hpt_ctx::EXTRA_LANES; ++l) {
        CUDA_TRY(cudaStreamCreateWithFlags(&ctx->wstream_x[l], cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_join_x[l], cudaEventDisableTiming));
        CUDA_TRY(cudaMalloc(&ctx->d_scr_x[l], sizeof(SlotScratch)));
        CUDA_TRY(cudaMemset(ctx->d_scr_x[l], 0, sizeof(SlotScratch)));
    }
    CUDA_TRY(cudaMallocHost(&ctx->h_wave_status, sizeof(unsigned) * hpt_ctx::STATUS_SLOTS));
    CUDA_TRY(cudaStreamCreateWithFlags(&ctx->ostream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming));
    // cos/sin(2 pi k / 256) split into float pairs for the double-float cone sampler
    float4 tab[256];
    for (int k = 0; k < 256; ++k) {
        double a = 2.0 * M_PI * k / 256.0;
        double c = cos(a), s = sin(a);
        float ch = (float)c, sh = (float)s;
        tab[k] = make_float4(ch, (float)(c - ch), sh, (float)(s - sh));
    }
    CUDA_TRY(cudaMalloc(&ctx->d_sincos, sizeof tab));
    CUDA_TRY(cudaMemcpy(ctx->d_sincos, tab, sizeof tab, cudaMemcpyHostToDevice));
    for (int i = 0; i < hpt_ctx::NSLOTS; ++i) {
        Slot &s = ctx->slots[i];
        CUDA_TRY(cudaMalloc(&s.d_table, sizeof(JobTable)));
        CUDA_TRY(cudaMallocHost(&s.h_table, sizeof(JobTable)));
        CUDA_TRY(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
    }
    if (desc) {
        ctx->budget = desc->hbm_budget_bytes;
        if (desc->max_inflight > 0) ctx->max_inflight = desc->max_inflight;
        if (desc->max_queue > 0) ctx->max_queue = (size_t)desc->max_queue;
    }
    if (ctx->budget == 0) {
        size_t fr = 0, tot = 0;
        CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        ctx->budget = (uint64_t)(fr * 0.6);
    }
    // the fixed-scratch entry point's array on this device (see hpt_trace_fixed_scratch)
    fixed_scratch_setup(device);
    hpt_ctx *raw = ctx.release();
    raw->sched = std::thread(sched_loop, raw);
    *out = raw;
    return HPT_OK;
}

static void free_frame(hpt_ctx::FrameGraph &g);

extern "C" void hpt_destroy(hpt_ctx *ctx)
{
    if (!ctx) return;
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        ctx->stop = true;
    }
    ctx->scv.notify_all();
    if (ctx->sched.joinable()) ctx->sched.join();
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &w : ctx->inflight)
        if (w.ev) cudaEventDestroy(w.ev);
    for (auto &kv : ctx->reqs)
        if (kv.second->out_lib) cudaFree(kv.second->out_lib);
    if (ctx->h_wave_status) cudaFreeHost(ctx->h_wave_status);
    if (ctx->ostream) cudaStreamDestroy(ctx->ostream);
    for (auto &g : ctx->graphs) free_frame(g);
    for (auto e : ctx->free_events) cudaEventDestroy(e);
    for (auto &kv : ctx->scenes) {
        cudaFree(kv.second->arena);
        if (kv.second->cache_buf) cudaFree(kv.second->cache_buf);
    }
    for (auto &s : ctx->slots) {
        cudaFree(s.d_table);
        cudaFreeHost(s.h_table);
        cudaEventDestroy(s.done);
    }
    if (ctx->pb_arena) cudaFree(ctx->pb_arena);
    if (ctx->d_scr) cudaFree(ctx->d_scr);
    if (ctx->wstream) cudaStreamDestroy(ctx->wstream);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    for (int l = 0; l < HPT_LANES; ++l) {
        if (ctx->slane_stream[l]) cudaStreamDestroy(ctx->slane_stream[l]);
        if (ctx->slane_ev[l]) cudaEventDestroy(ctx->slane_ev[l]);
        if (ctx->spb_arena[l]) cudaFree(ctx->spb_arena[l]);
        if (ctx->sscr[l]) cudaFree(ctx->sscr[l]);
    }
    for (int l = 0; l < hpt_ctx::EXTRA_LANES; ++l) {
        if (ctx->wstream_x[l]) cudaStreamDestroy(ctx->wstream_x[l]);
        if (ctx->ev_join_x[l]) cudaEventDestroy(ctx->ev_join_x[l]);
        if (ctx->pb_arena_x[l]) cudaFree(ctx->pb_arena_x[l]);
        if (ctx->d_scr_x[l]) cudaFree(ctx->d_scr_x[l]);
    }
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    if (ctx->host_out_dev) cudaFree(ctx->host_out_dev);
    if (ctx->cstream) cudaStreamDestroy(ctx->cstream);
    if (ctx->ev_wave) cudaEventDestroy(ctx->ev_wave);
    if (ctx->ev_copied) cudaEventDestroy(ctx->ev_copied);
    if (ctx->d_sincos) cudaFree(ctx->d_sincos);
    delete ctx;
}

// ------------------------------------------------------------------------ scene upload
static bool finite3(const float *p) { return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]); }

extern "C" hpt_status hpt_scene_upload(hpt_ctx *ctx, const hpt_scene_desc *d, uint64_t *scene_id)
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    if (!d || !scene_id) return fail(HPT_ERR_INVALID_ARG, "scene or scene_id is NULL");
    if (d->nv <= 0 || d->nt <= 0 || d->nm <= 0 || d->ntex < 0 || d->nl < 0 || d->np < 0)
        return fail(HPT_ERR_INVALID_ARG, "bad counts nv=%d nt=%d nm=%d", d->nv, d->nt, d->nm);
    if (!d->verts || !d->normals || !d->uvs || !d->tris || !d->tri_mat || !d->materials)
        return fail(HPT_ERR_INVALID_ARG, "missing geometry array");
    if (d->nt >= (1 << 23)) return fail(HPT_ERR_UNSUPPORTED, "more than 2^23 triangles");
    for (int i = 0; i < d->nv; ++i) {
        if (!finite3(d->verts + 3 * i) || !finite3(d->normals + 3 * i) || !std::isfinite(d->uvs[2 * i]) ||
            !std::isfinite(d->uvs[2 * i + 1]))
            return fail(HPT_ERR_INVALID_ARG, "non-finite vertex data at vertex %d", i);
    }
    for (int t = 0; t < d->nt; ++t) {
        for (int k = 0; k < 3; ++k)
            if (d->tris[3 * t + k] >= (uint32_t)d->nv) return fail(HPT_ERR_INVALID_ARG, "triangle %d index out of range", t);
        if (d->tri_mat[t] >= (uint32_t)d->nm) return fail(HPT_ERR_INVALID_ARG, "triangle %d material out of range", t);
    }
    for (int m = 0; m < d->nm; ++m) {
        const hpt_material &M = d->materials[m];
        if (M.kind < 0 || M.kind > 4) return fail(HPT_ERR_INVALID_ARG, "material %d: bad kind %d", m, M.kind);
        if (M.tex >= d->ntex) return fail(HPT_ERR_INVALID_ARG, "material %d: texture %d out of range", m, M.tex);
        if (M.light >= d->nl) return fail(HPT_ERR_INVALID_ARG, "material %d: light %d out of range", m, M.light);
        if (!finite3(M.albedo) || !finite3(M.Le) || !std::isfinite(M.roughness) || !std::isfinite(M.ior))
            return fail(HPT_ERR_INVALID_ARG, "material %d: non-finite value", m);
        if (M.kind == HPT_GGX && !(M.roughness > 0.0f)) return fail(HPT_ERR_INVALID_ARG, "material %d: GGX roughness must be > 0", m);
        if (M.kind == HPT_DIELECTRIC && !(M.ior > 0.0f)) return fail(HPT_ERR_INVALID_ARG, "material %d: ior must be > 0", m);
    }
    for (int i = 0; i < d->ntex; ++i) {
        const int32_t *ti = d->tex_info + 3 * i;
        if (ti[0] < 0 || ti[1] <= 0 || ti[2] <= 0 || (int64_t)ti[0] + (int64_t)ti[1] * ti[2] * 3 > d->tex_floats)
            return fail(HPT_ERR_INVALID_ARG, "texture %d out of bounds", i);
    }
    if (d->nl > 0 && !d->lights) return fail(HPT_ERR_INVALID_ARG, "lights is NULL");
    if (d->np > 0 && !d->points) return fail(HPT_ERR_INVALID_ARG, "points is NULL");
    if (d->cache_res < 0 || (d->cache_res > 0 && !d->cache_E)) return fail(HPT_ERR_INVALID_ARG, "bad cache");

    const int nt = d->nt, nv = d->nv;
    // primitive boxes and centroids; degenerate triangles never intersect and are left out
    std::vector<Box> pb(nt);
    std::vector<float> cent(3 * nt);
    std::vector<int> prims;
    prims.reserve(nt);
    float max_abs = 0.0f;
    for (int t = 0; t < nt; ++t) {
        const float *p[3] = {d->verts + 3 * d->tris[3 * t], d->verts + 3 * d->tris[3 * t + 1],
                             d->verts + 3 * d->tris[3 * t + 2]};
        pb[t].reset();
        for (int k = 0; k < 3; ++k) {
            pb[t].grow(p[k]);
            for (int c = 0; c < 3; ++c) max_abs = std::max(max_abs, std::fabs(p[k][c]));
        }
        for (int c = 0; c < 3; ++c) cent[3 * t + c] = (p[0][c] + p[1][c] + p[2][c]) / 3.0f;
        double e1[3], e2[3];
        for (int c = 0; c < 3; ++c) { e1[c] = (double)p[1][c] - p[0][c]; e2[c] = (double)p[2][c] - p[0][c]; }
        double n0 = e1[1] * e2[2] - e1[2] * e2[1], n1 = e1[2] * e2[0] - e1[0] * e2[2], n2 = e1[0] * e2[1] - e1[1] * e2[0];
        if (n0 * n0 + n1 * n1 + n2 * n2 > 0.0) prims.push_back(t);
    }
    if (prims.empty()) return fail(HPT_ERR_INVALID_ARG, "all triangles are degenerate");
    // a tree: kernel nodes (both child boxes of an inner node; leaves encoded in the parent's
    // link) and the triangle records in its leaf order
    struct Tree {
        std::vector<float4> knodes, tri4;
        int n_nodes = 0, n_tri4 = 0, depth = 0;
    };
    const float pad = 2e-6f * max_abs + 1e-12f;
    auto make_tree = [&](const double wface[3], Tree &T) {
        Builder B(pb, cent, prims);
        for (int k = 0; k < 3; ++k) B.wface[k] = wface[k];
        int root = B.build(0, (int)B.idx.size(), 0);
        std::vector<float4> &knodes = T.knodes;
        std::vector<int> order;   // triangle ids in leaf order
        order.reserve(B.idx.size());
        auto emit_leaf_link = [&](const BuildNode &n) {
            int start = (int)order.size();
            for (int i = n.start; i < n.start + n.count; ++i) order.push_back(B.idx[i]);
            return ~((start << 8) | n.count);
        };
        auto box_of = [&](const BuildNode *n, float lo[3], float hi[3]) {
            for (int k = 0; k < 3; ++k) {
                if (n) {
                    lo[k] = n->box.lo[k] - pad;
                    hi[k] = n->box.hi[k] + pad;
                } else {
                    lo[k] = 1e30f;   // far-away point box: no ray with t < 1e30 enters it
                    hi[k] = 1e30f;
                }
            }
        };
        // kernel nodes in depth-first order (a node's first child follows it in memory): the
        // root is an inner node whose children are the build root's children (or the root leaf)
        std::function<int(const BuildNode *, const BuildNode *)> emit = [&](const BuildNode *c0,
                                                                            const BuildNode *c1) -> int {
            const int kn = (int)(knodes.size() / 4);
            knodes.resize(knodes.size() + 4);
            const BuildNode *c[2] = {c0, c1};
            float lo[2][3], hi[2][3];
            int link[2];
            for (int s2 = 0; s2 < 2; ++s2) {
                box_of(c[s2], lo[s2], hi[s2]);
                if (!c[s2]) link[s2] = ~0;   // empty leaf, never entered
                else if (c[s2]->count) link[s2] = emit_leaf_link(*c[s2]);
                else link[s2] = emit(&B.nodes[c[s2]->left], &B.nodes[c[s2]->right]);
            }
            float4 *o = &knodes[4 * kn];
            o[0] = make_float4(lo[0][0], hi[0][0], lo[0][1], hi[0][1]);
            o[1] = make_float4(lo[1][0], hi[1][0], lo[1][1], hi[1][1]);
            o[2] = make_float4(lo[0][2], hi[0][2], lo[1][2], hi[1][2]);
            float l0, l1;
            memcpy(&l0, &link[0], 4);
            memcpy(&l1, &link[1], 4);
            o[3] = make_float4(l0, l1, 0.0f, 0.0f);
            return kn;
        };
        {
            const BuildNode &r = B.nodes[root];
            if (r.count) emit(&r, nullptr);
            else emit(&B.nodes[r.left], &B.nodes[r.right]);
        }
        const int n_knodes = (int)(knodes.size() / 4);
        const int n_order = (int)order.size();
        {
            // the first TOP_ORDER inner nodes breadth-first from the root, the others in their
            // depth-first order; the links are renumbered (the tree itself is unchanged)
            const int ntop = std::min(n_knodes, TOP_ORDER);
            std::vector<int> bfs;
            std::vector<char> top(n_knodes, 0);
            bfs.reserve(ntop);
            bfs.push_back(0);
            top[0] = 1;
            for (size_t h = 0; h < bfs.size() && (int)bfs.size() < ntop; ++h) {
                int link[2];
                memcpy(&link[0], &knodes[4 * (size_t)bfs[h] + 3].x, 4);
                memcpy(&link[1], &knodes[4 * (size_t)bfs[h] + 3].y, 4);
                for (int c = 0; c < 2; ++c)
                    if (link[c] >= 0 && (int)bfs.size() < ntop) {
                        bfs.push_back(link[c]);
                        top[link[c]] = 1;
                    }
            }
            std::vector<int> nid(n_knodes);
            int k = 0;
            for (int n : bfs) nid[n] = k++;
            for (int n = 0; n < n_knodes; ++n)
                if (!top[n]) nid[n] = k++;
            std::vector<float4> re(knodes.size());
            for (int n = 0; n < n_knodes; ++n) {
                float4 *o = &re[4 * (size_t)nid[n]];
                for (int j = 0; j < 4; ++j) o[j] = knodes[4 * (size_t)n + j];
                int link[2];
                memcpy(&link[0], &o[3].x, 4);
                memcpy(&link[1], &o[3].y, 4);
                for (int c = 0; c < 2; ++c)
                    if (link[c] >= 0) link[c] = nid[link[c]];
                memcpy(&o[3].x, &link[0], 4);
                memcpy(&o[3].y, &link[1], 4);
            }
            knodes.swap(re);
        }
        // triangle records
        std::vector<float4> &tri4 = T.tri4;
        tri4.assign(3 * (size_t)std::max(n_order, 1), make_float4(0.0f, 0.0f, 0.0f, 0.0f));
        for (int i = 0; i < n_order; ++i) {
            int t = order[i];
            const float *p0 = d->verts + 3 * d->tris[3 * t], *p1 = d->verts + 3 * d->tris[3 * t + 1],
                        *p2 = d->verts + 3 * d->tris[3 * t + 2];
            float idf;
            memcpy(&idf, &t, 4);
            // barycentric slack of the float test on incoherent rays: a band of 1e-6 x the scene's
            // largest coordinate (a few float ulps of a hit point) across the triangle's shortest
            // altitude, at most 2e-5
            double a[3] = {(double)p1[0] - p0[0], (double)p1[1] - p0[1], (double)p1[2] - p0[2]};
            double b[3] = {(double)p2[0] - p0[0], (double)p2[1] - p0[1], (double)p2[2] - p0[2]};
            double cr[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
            double area2 = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            double c3[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
            double lmax = sqrt(std::max({a[0] * a[0] + a[1] * a[1] + a[2] * a[2], b[0] * b[0] + b[1] * b[1] + b[2] * b[2],
                                         c3[0] * c3[0] + c3[1] * c3[1] + c3[2] * c3[2]}));
            double hmin = lmax > 0.0 ? area2 / lmax : 0.0;
            float slack = hmin > 0.0 ? (float)std::min(2e-5, 1e-6 * (double)max_abs / hmin) : 2e-5f;
            tri4[3 * i] = make_float4(p0[0], p0[1], p0[2], idf);
            tri4[3 * i + 1] = make_float4(p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2], slack);
            tri4[3 * i + 2] = make_float4(p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2], 0.0f);
        }
        T.n_nodes = n_knodes;
        T.n_tri4 = n_order;
        T.depth = B.max_depth_seen;
    };
    // the tree for rays in every direction, and one for the pixels' first rays, which leave the
    // hologram plane along +z inside a cone of a few degrees (the faces across z weighted 5:1)
    Tree tree, tree_p;
    {
        const double w_all[3] = {1.0, 1.0, 1.0};
        make_tree(w_all, tree);
        const double w_z[3] = {HPT_PRIMARY_SIDE_W, HPT_PRIMARY_SIDE_W, 1.0};
        make_tree(w_z, tree_p);
    }
    std::vector<double> ref64((size_t)nt * REF_N, 0.0);
    std::vector<float2> refdf((size_t)nt * REF_N);
    std::vector<uint4> attr(nt);
    std::vector<float4> tng(nt);
    for (int t = 0; t < nt; ++t) {
        const float *p0 = d->verts + 3 * d->tris[3 * t], *p1 = d->verts + 3 * d->tris[3 * t + 1],
                    *p2 = d->verts + 3 * d->tris[3 * t + 2];
        double e1[3], e2[3], v0[3];
        for (int c = 0; c < 3; ++c) { v0[c] = p0[c]; e1[c] = (double)p1[c] - p0[c]; e2[c] = (double)p2[c] - p0[c]; }
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
        double *r = &ref64[(size_t)t * REF_N];
        if (nn > 0.0) {
            r[0] = n[0]; r[1] = n[1]; r[2] = n[2];
            r[3] = n[0] * v0[0] + n[1] * v0[1] + n[2] * v0[2];
            // m1 = (e2 x n) / |n|^2, m2 = (n x e1) / |n|^2
            r[4] = (e2[1] * n[2] - e2[2] * n[1]) / nn;
            r[5] = (e2[2] * n[0] - e2[0] * n[2]) / nn;
            r[6] = (e2[0] * n[1] - e2[1] * n[0]) / nn;
            r[7] = (n[1] * e1[2] - n[2] * e1[1]) / nn;
            r[8] = (n[2] * e1[0] - n[0] * e1[2]) / nn;
            r[9] = (n[0] * e1[1] - n[1] * e1[0]) / nn;
            double ln = sqrt(nn);
            tng[t] = make_float4((float)(n[0] / ln), (float)(n[1] / ln), (float)(n[2] / ln), 0.0f);
        } else {
            tng[t] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
            r[2] = 1.0;
        }
        for (int k = 0; k < REF_N; ++k) {
            float h = (float)r[k];
            refdf[(size_t)t * REF_N + k] = make_float2(h, (float)(r[k] - (double)h));
        }
        attr[t] = make_uint4(d->tris[3 * t], d->tris[3 * t + 1], d->tris[3 * t + 2], d->tri_mat[t]);
    }
    std::vector<MatDev> mats(d->nm);
    for (int m = 0; m < d->nm; ++m) {
        const hpt_material &M = d->materials[m];
        MatDev &o = mats[m];
        o.kind = M.kind;
        o.tex = M.tex;
        o.emit_tex = M.emit_tex;
        o.light = M.light;
        for (int c = 0; c < 3; ++c) { o.albedo[c] = M.albedo[c]; o.Le[c] = M.Le[c]; }
        o.rough = M.roughness;
        o.ior = M.ior;
    }
    std::vector<LightDev> lights(std::max(d->nl, 1));
    for (int l = 0; l < d->nl; ++l) {
        const float *L = d->lights + 12 * l;
        LightDev &o = lights[l];
        for (int c = 0; c < 3; ++c) { o.corner[c] = L[c]; o.eu[c] = L[3 + c]; o.ev[c] = L[6 + c]; o.Le[c] = L[9 + c]; }
        double eu[3] = {L[3], L[4], L[5]}, ev[3] = {L[6], L[7], L[8]};
        double n[3] = {eu[1] * ev[2] - eu[2] * ev[1], eu[2] * ev[0] - eu[0] * ev[2], eu[0] * ev[1] - eu[1] * ev[0]};
        double a = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(a > 0.0)) return fail(HPT_ERR_INVALID_ARG, "light %d has zero area", l);
        for (int c = 0; c < 3; ++c) o.n[c] = (float)(n[c] / a);
        o.area = (float)a;
    }
    // one arena for everything
    struct Part { const void *src; size_t bytes; size_t off; };
    std::vector<Part> parts;
    size_t off = 0;
    auto add = [&](const void *src, size_t bytes) {
        size_t o = off;
        parts.push_back({src, bytes, o});
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    size_t o_nodes = add(tree.knodes.data(), tree.knodes.size() * sizeof(float4));
    size_t o_tri4 = add(tree.tri4.data(), tree.tri4.size() * sizeof(float4));
    size_t o_nodes_p = add(tree_p.knodes.data(), tree_p.knodes.size() * sizeof(float4));
    size_t o_tri4_p = add(tree_p.tri4.data(), tree_p.tri4.size() * sizeof(float4));
    size_t o_r64 = add(ref64.data(), ref64.size() * sizeof(double));
    size_t o_rdf = add(refdf.data(), refdf.size() * sizeof(float2));
    size_t o_attr = add(attr.data(), attr.size() * sizeof(uint4));
    size_t o_ng = add(tng.data(), tng.size() * sizeof(float4));
    size_t o_v = add(d->verts, (size_t)nv * 3 * sizeof(float));
    size_t o_n = add(d->normals, (size_t)nv * 3 * sizeof(float));
    size_t o_uv = add(d->uvs, (size_t)nv * 2 * sizeof(float));
    size_t o_m = add(mats.data(), mats.size() * sizeof(MatDev));
    float zero3[3] = {0, 0, 0};
    int zero_i[3] = {0, 0, 0};
    size_t o_tex = d->ntex > 0 ? add(d->tex_data, (size_t)d->tex_floats * sizeof(float)) : add(zero3, sizeof zero3);
    size_t o_ti = d->ntex > 0 ? add(d->tex_info, (size_t)d->ntex * 3 * sizeof(int)) : add(zero_i, sizeof zero_i);
    size_t o_l = add(lights.data(), lights.size() * sizeof(LightDev));
    double zero4[4] = {0, 0, 0, 0};
    size_t o_p = d->np > 0 ? add(d->points, (size_t)d->np * 4 * sizeof(double)) : add(zero4, sizeof zero4);
    size_t cache_elems = (size_t)d->cache_res * d->cache_res * d->cache_res * 3;
    uint16_t zero_h[4] = {0, 0, 0, 0};
    size_t o_c = d->cache_res > 0 ? add(d->cache_E, cache_elems * sizeof(uint16_t)) : add(zero_h, sizeof zero_h);

    auto rec = std::make_unique<SceneRec>();
    CUDA_TRY(cudaMalloc(&rec->arena, off));
    rec->bytes = off;
    char *base = (char *)rec->arena;
    for (auto &p : parts) {
        cudaError_t e = cudaMemcpy(base + p.off, p.src, p.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(rec->arena);
            return fail(HPT_ERR_CUDA, "scene copy: %s", cudaGetErrorString(e));
        }
    }
    DevScene &s = rec->dev;
    s.nodes = (const float4 *)(base + o_nodes);
    s.tri4 = (const float4 *)(base + o_tri4);
    s.nodes_p = (const float4 *)(base + o_nodes_p);
    s.tri4_p = (const float4 *)(base + o_tri4_p);
    s.ref64 = (const double *)(base + o_r64);
    s.refdf = (const float2 *)(base + o_rdf);
    s.tri_attr = (const uint4 *)(base + o_attr);
    s.tri_ng = (const float4 *)(base + o_ng);
    s.verts = (const float *)(base + o_v);
    s.normals = (const float *)(base + o_n);
    s.uvs = (const float *)(base + o_uv);
    s.mats = (const MatDev *)(base + o_m);
    s.tex = (const float *)(base + o_tex);
    s.tex_info = (const int *)(base + o_ti);
    s.lights = (const LightDev *)(base + o_l);
    s.points = (const double *)(base + o_p);
    s.cache = (const unsigned short *)(base + o_c);
    for (int c = 0; c < 3; ++c) { s.cache_bmin[c] = d->cache_bmin[c]; s.cache_bmax[c] = d->cache_bmax[c]; }
    s.cache_res = d->cache_res;
    s.n_tris = nt;
    s.n_tri4 = tree.n_tri4;
    s.n_nodes = tree.n_nodes;
    s.bvh_depth = tree.depth;
    s.n_tri4_p = tree_p.n_tri4;
    s.n_nodes_p = tree_p.n_nodes;
    s.bvh_depth_p = tree_p.depth;
    s.n_lights = d->nl;
    s.n_points = d->np;
    rec->n_nodes = tree.n_nodes;
    rec->depth = tree.depth;
    std::lock_guard<std::mutex> lk(ctx->mu);
    uint64_t id = ctx->next_scene++;
    ctx->scenes[id] = std::move(rec);
    *scene_id = id;
    return HPT_OK;
}

extern "C" hpt_status hpt_scene_release(hpt_ctx *ctx, uint64_t scene_id)
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    std::unique_ptr<SceneRec> rec;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->scenes.find(scene_id);
        if (it == ctx->scenes.end()) return fail(HPT_ERR_NOT_FOUND, "unknown scene %llu", (unsigned long long)scene_id);
        if (it->second->users.load() > 0) return fail(HPT_ERR_BUSY, "scene %llu is used by queued requests", (unsigned long long)scene_id);
        rec = std::move(it->second);
        ctx->scenes.erase(it);
    }
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaFree(rec->arena));
    if (rec->cache_buf) CUDA_TRY(cudaFree(rec->cache_buf));
    return HPT_OK;
}

extern "C" hpt_status hpt_scene_info(hpt_ctx *ctx, uint64_t scene_id, uint64_t *bytes, int32_t *n_nodes, int32_t *depth)
{
    g_err.clear();
    if (!ctx) return fail(HPT_ERR_INVALID_ARG, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->scenes.find(scene_id);
    if (it == ctx->scenes.end()) return fail(HPT_ERR_NOT_FOUND, "unknown scene %llu", (unsigned long long)scene_id);
    if (bytes) *bytes = it->second->bytes;
    if (n_nodes) *n_nodes = it->second->n_nodes;
    if (depth) *depth = it->second->depth;
    return HPT_OK;
}

// ---------------------------------------------------------------------- render -> job
static hpt_status make_job(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *r, void *out, size_t out_bytes,
                           DevJob &J, SceneRec **rec_out)
{
    if (!r) return fail(HPT_ERR_INVALID_ARG, "render desc is NULL");
    if (r->W <= 0 || r->H <= 0 || (int64_t)r->W * r->H > (1ll << 31))
        return fail(HPT_ERR_INVALID_ARG, "bad SLM size %dx%d", r->W, r->H);
    if (!(r->pitch > 0.0) || !std::isfinite(r->pitch)) return fail(HPT_ERR_INVALID_ARG, "bad pitch");
    if (r->n_lambda < 1 || r->n_lambda > 3) return fail(HPT_ERR_INVALID_ARG, "n_lambda must be 1..3");
    if (r->spp < 1 || r->max_depth < 1 || r->max_depth > 64) return fail(HPT_ERR_INVALID_ARG, "bad spp or max_depth");
    if (r->K < 1 || r->K > KMAX) return fail(HPT_ERR_INVALID_ARG, "K must be 1..%d", KMAX);
    if (r->hologram_offset < 0 || r->hologram_offset + r->K > (1 << 18)) return fail(HPT_ERR_INVALID_ARG, "bad hologram_offset");
    if (r->phase_mode != HPT_PHASE_HASH && r->phase_mode != HPT_PHASE_ZERO && r->phase_mode != HPT_PHASE_GRF)
        return fail(HPT_ERR_INVALID_ARG, "bad phase_mode");
    if (r->phase_mode == HPT_PHASE_GRF && (!r->grf_phi || r->grf_nx < 1 || r->grf_ny < 1 || r->grf_nx > (1 << 16) ||
                                           r->grf_ny > (1 << 16)))
        return fail(HPT_ERR_INVALID_ARG, "phase_mode GRF needs grf_phi and 1 <= grf_nx, grf_ny <= 65536");
    if (r->precision != HPT_PREC_FP64 && r->precision != HPT_PREC_DF32) return fail(HPT_ERR_INVALID_ARG, "bad precision");
    if (!(r->facet_size > 0.0) || !std::isfinite(r->facet_size)) return fail(HPT_ERR_INVALID_ARG, "bad facet_size");
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(r->T[i])) return fail(HPT_ERR_INVALID_ARG, "non-finite T");
    // rigid: orthonormal rotation block, last row (0, 0, 0, 1)
    const double *T = r->T;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double dp = T[4 * a] * T[4 * b] + T[4 * a + 1] * T[4 * b + 1] + T[4 * a + 2] * T[4 * b + 2];
            if (std::fabs(dp - (a == b ? 1.0 : 0.0)) > 1e-9) return fail(HPT_ERR_INVALID_ARG, "T is not rigid");
        }
    if (T[12] != 0.0 || T[13] != 0.0 || T[14] != 0.0 || T[15] != 1.0) return fail(HPT_ERR_INVALID_ARG, "T last row must be 0 0 0 1");
    const double det = T[0] * (T[5] * T[10] - T[6] * T[9]) - T[1] * (T[4] * T[10] - T[6] * T[8]) + T[2] * (T[4] * T[9] - T[5] * T[8]);
    if (det < 0.0) return fail(HPT_ERR_INVALID_ARG, "T must be a proper rotation");
    size_t need = (size_t)8 * r->n_lambda * r->K * (size_t)r->W * r->H;
    if (out && out_bytes < need) return fail(HPT_ERR_INVALID_ARG, "out_bytes %zu < %zu", out_bytes, need);
    SceneRec *rec;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->scenes.find(scene_id);
        if (it == ctx->scenes.end()) return fail(HPT_ERR_NOT_FOUND, "unknown scene %llu", (unsigned long long)scene_id);
        rec = it->second.get();
    }
    if (r->use_cache && rec->dev.cache_res <= 0) return fail(HPT_ERR_INVALID_ARG, "use_cache set but the scene has no cache");
    memset(&J, 0, sizeof J);
    J.sc = rec->dev;
    J.out = (float2 *)out;
    J.W = r->W;
    J.H = r->H;
    J.n_lambda = r->n_lambda;
    J.spp = r->spp;
    J.max_depth = r->max_depth;
    J.K = r->K;
    J.hologram_offset = r->hologram_offset;
    J.phase_mode = r->phase_mode;
    J.grf = r->phase_mode == HPT_PHASE_GRF ? r->grf_phi : nullptr;
    J.grf_nx = r->phase_mode == HPT_PHASE_GRF ? r->grf_nx : 0;
    J.grf_ny = r->phase_mode == HPT_PHASE_GRF ? r->grf_ny : 0;
    J.use_cache = r->use_cache ? 1 : 0;
    J.obliquity = r->omit_obliquity ? 0 : 1;
    J.n_tiles_x = (r->W + TILE_W - 1) / TILE_W;
    J.n_tiles = J.n_tiles_x * ((r->H + TILE_H - 1) / TILE_H);
    J.n_items = (long long)r->n_lambda * J.n_tiles * 32;
    J.seed_lo = (unsigned)r->seed;
    J.seed_hi = (unsigned)(r->seed >> 32);
    J.pseed_lo = (unsigned)r->phase_seed;
    J.pseed_hi = (unsigned)(r->phase_seed >> 32);
    for (int c = 0; c < r->n_lambda; ++c) {
        double lam = r->lambda[c];
        if (!(lam > 0.0) || !(lam < 2.0 * r->pitch)) return fail(HPT_ERR_INVALID_ARG, "lambda[%d] must be in (0, 2 pitch)", c);
        if (r->channel[c] < 0 || r->channel[c] > 2) return fail(HPT_ERR_INVALID_ARG, "channel[%d] must be 0..2", c);
        double thmax = asin(lam / (2.0 * r->pitch));
        double sh = sin(0.5 * thmax);
        double h = 2.0 * sh * sh;
        J.channel[c] = r->channel[c];
        J.lambda_f[c] = (float)lam;
        J.pdf_w[c] = (float)(1.0 / (2.0 * M_PI * h));
        J.cos_max[c] = (float)cos(thmax);
        J.lambda[c] = make_rc(lam);
        J.inv_lambda[c] = make_rc(1.0 / lam);
        J.h_cone[c] = make_rc(h);
    }
    J.pitch = make_rc(r->pitch);
    J.inv_facet = make_rc(1.0 / r->facet_size);
    J.inv_pitch = make_rc(1.0 / r->pitch);
    bool ident = true;
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
            J.R[3 * a + b] = make_rc(T[4 * a + b]);
            if (T[4 * a + b] != (a == b ? 1.0 : 0.0)) ident = false;
        }
        J.t[a] = make_rc(T[4 * a + 3]);
        if (T[4 * a + 3] != 0.0) ident = false;
    }
    J.t_identity = ident ? 1 : 0;
    J.sincos_tab = ctx->d_sincos;
    if (rec_out) *rec_out = rec;
    return HPT_OK;
}

// ---------------------------------------------------------------------------- launches
static Slot *acquire_slot(hpt_ctx *ctx)
{
    Slot *s = &ctx->slots[ctx->next_slot];
    ctx->next_slot = (ctx->next_slot + 1) % hpt_ctx::NSLOTS;
    if (s->used) cudaEventSynchronize(s->done);
    s->used = true;
    return s;
}

// bytes of path state per path (see PathBufs)
static size_t path_bytes() { return 7 * 8 + 3 * 4 + 4 + 6 * 4 + 3 * 16 + 16 + 4 + 3 * 4 + 3 * 4 + 6 * 4; }

static void carve_paths(void *arena, size_t B, PathBufs &b)
{
    char *p = (char *)arena;
    auto take = [&](size_t bytes) {
        void *r = p;
        p += (bytes + 255) & ~(size_t)255;
        return r;
    };
    b.cs0 = (uint4 *)take(16 * B);
    b.cs1 = (uint4 *)take(16 * B);
    b.cs2 = (uint4 *)take(16 * B);
    b.cs3 = (uint2 *)take(8 * B);
    b.coh4 = (float4 *)take(16 * B);
    b.inc = (float4 *)take(16 * B);
    b.inc2 = (float2 *)take(8 * B);
    b.ray_o = (float4 *)take(16 * B);
    b.ray_d = (float4 *)take(16 * B);
    b.sh_d = (float4 *)take(16 * B);
    b.hit = (float4 *)take(16 * B);
    b.occl = (int *)take(4 * B);
    b.amp = (float *)take(4 * B);
    b.fturn = (float *)take(4 * B);
    b.basep = (float *)take(4 * B);
    b.cx = (int *)take(4 * B);
    b.cy = (int *)take(4 * B);
    b.cz = (int *)take(4 * B);
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 2; ++j) b.q[k][j] = (int *)take(4 * B);
    b.capacity = (int)B;
}

static hpt_status ensure_paths(hpt_ctx *ctx)
{
    if (ctx->pb_arena) return HPT_OK;
    const size_t B = (size_t)ctx->capacity;
    CUDA_TRY(cudaMalloc(&ctx->pb_arena, B * path_bytes() + 64 * 256));
    for (int l = 0; l < ctx->lanes - 1; ++l) {
        cudaError_t e = cudaMalloc(&ctx->pb_arena_x[l], B * path_bytes() + 64 * 256);
        if (e != cudaSuccess) {
            cudaFree(ctx->pb_arena);
            ctx->pb_arena = nullptr;
            for (int k = 0; k < l; ++k) {
                cudaFree(ctx->pb_arena_x[k]);
                ctx->pb_arena_x[k] = nullptr;
            }
            return fail(HPT_ERR_OOM, "wave state: %s", cudaGetErrorString(e));
        }
        carve_paths(ctx->pb_arena_x[l], B, ctx->pb_x[l]);
    }
    carve_paths(ctx->pb_arena, B, ctx->pb);
    return HPT_OK;
}

// the serving scheduler's lanes; caller holds ctx->mu
static hpt_status ensure_sched_paths(hpt_ctx *ctx)
{
    if (ctx->spb_arena[0]) return HPT_OK;
    const size_t B = (size_t)ctx->sched_capacity;
    for (int l = 0; l < HPT_LANES; ++l) {
        if (!ctx->slane_stream[l]) CUDA_TRY(cudaStreamCreateWithFlags(&ctx->slane_stream[l], cudaStreamNonBlocking));
        if (!ctx->slane_ev[l]) CUDA_TRY(cudaEventCreateWithFlags(&ctx->slane_ev[l], cudaEventDisableTiming));
        if (!ctx->sscr[l]) {
            CUDA_TRY(cudaMalloc(&ctx->sscr[l], sizeof(SlotScratch)));
            CUDA_TRY(cudaMemset(ctx->sscr[l], 0, sizeof(SlotScratch)));
        }
        cudaError_t e = cudaMalloc(&ctx->spb_arena[l], B * path_bytes() + 64 * 256);
        if (e != cudaSuccess) {
            for (int k = 0; k <= l; ++k) {
                if (ctx->spb_arena[k]) cudaFree(ctx->spb_arena[k]);
                ctx->spb_arena[k] = nullptr;
            }
            return fail(HPT_ERR_OOM, "serving wave state: %s", cudaGetErrorString(e));
        }
        carve_paths(ctx->spb_arena[l], B, ctx->spb[l]);
    }
    return HPT_OK;
}

// Called after each wave's accumulation is queued, with the wave and the stream it ran on.
using AfterWave = std::function<hpt_status(const WaveDesc &, cudaStream_t)>;

// Queue the waves that cover all items of 'jobs' (job table already on the device) on ws.
// Waves take the items of each job in increasing order.  Caller holds ctx->mu.
static hpt_status enqueue_waves(hpt_ctx *ctx, const DevJob *jobs, int n, int prec, bool stats, const JobTable *jt,
                                cudaStream_t ws, bool allow_debug, const AfterWave *after_wave = nullptr)
{
    const int B = ctx->capacity;
    WaveDesc wd;
    memset(&wd, 0, sizeof wd);
    int max_depth = 1;
    hpt_status st = HPT_OK;
    // waves rotate over ctx->lanes lanes (path state, scratch, stream); the extra lanes fork from
    // ws at the start and join ws at the end.  Per-kernel timing keeps one lane.
    const int lanes = ctx->timer == nullptr ? ctx->lanes : 1;
    int n_waves = 0;
    bool forked = false;
    auto mark = [&](int kind) -> cudaError_t {
        hpt_ctx::KernelTimer *tm = ctx->timer;
        if (!tm) return cudaSuccess;
        if (tm->used == tm->ev.size()) {
            cudaEvent_t e;
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
            tm->ev.push_back(e);
            tm->kind.push_back(0);
        }
        tm->kind[tm->used] = kind;
        return cudaEventRecord(tm->ev[tm->used++], ws);
    };
    auto flush = [&]() -> hpt_status {
        if (wd.n_seg == 0) return HPT_OK;
        const int lane = n_waves % lanes;
        ++n_waves;
        const PathBufs &pb = lane ? ctx->pb_x[lane - 1] : ctx->pb;
        SlotScratch *scr = lane ? ctx->d_scr_x[lane - 1] : ctx->d_scr;
        cudaStream_t s = lane ? ctx->wstream_x[lane - 1] : ws;
        const int n_iter = max_depth + 1;
        CUDA_TRY(mark(HPT_K_GEN));
        CUDA_TRY(cudaMemsetAsync(scr->qcount, 0, sizeof(int) * 3 * (n_iter + 1), s));
        CUDA_TRY(wave_gen(prec, jt, wd, pb, scr, s));
        for (int it = 0; it < n_iter; ++it) {
            CUDA_TRY(mark(HPT_K_TRACE));
            CUDA_TRY(wave_trace(prec, stats, jt, wd, pb, scr, it, ctx->grid_trace[prec], s));
            CUDA_TRY(mark(HPT_K_SHADE));
            CUDA_TRY(wave_shade(prec, stats, jt, wd, pb, scr, it, ctx->grid_shade[prec], s));
        }
        CUDA_TRY(mark(HPT_K_ACCUM));
        CUDA_TRY(wave_accum(prec, jt, wd, pb, scr, s));
        CUDA_TRY(mark(-1));
        if (after_wave) {
            hpt_status st2 = (*after_wave)(wd, s);
            if (st2) return st2;
        }
        if (allow_debug && ctx->debug_waves > 0) {
            // diagnostic: queue lengths per iteration of the first waves (HPT_DEBUG_WAVES=n)
            --ctx->debug_waves;
            int q[MAX_ITER + 1][3];
            CUDA_TRY(cudaStreamSynchronize(s));
            CUDA_TRY(cudaMemcpy(q, scr->qcount, sizeof(int) * 3 * (n_iter + 1), cudaMemcpyDeviceToHost));
            fprintf(stderr, "wave paths=%d items=%d:", wd.n_paths, wd.n_items);
            for (int it = 0; it <= n_iter; ++it) fprintf(stderr, " [%d|%d|%d]", q[it][0], q[it][1], q[it][2]);
            fprintf(stderr, "\n");
        }
        memset(&wd, 0, sizeof wd);
        max_depth = 1;
        return HPT_OK;
    };
    if (lanes > 1) {
        CUDA_TRY(cudaEventRecord(ctx->ev_fork, ws));
        for (int l = 0; l < lanes - 1; ++l) CUDA_TRY(cudaStreamWaitEvent(ctx->wstream_x[l], ctx->ev_fork, 0));
        forked = true;
    }
    for (int j = 0; j < n; ++j) {
        const int spp = jobs[j].spp;
        if (spp > B) return fail(HPT_ERR_UNSUPPORTED, "spp %d exceeds the wave capacity %d", spp, B);
        long long c = 0;
        while (c < jobs[j].n_items) {
            int cap = (B - wd.n_paths) / spp;
            if (cap <= 0 || wd.n_seg == MAX_SEG) {
                st = flush();
                if (st) return st;
                continue;
            }
            const int take = (int)std::min<long long>(jobs[j].n_items - c, cap);
            WaveSeg &g = wd.seg[wd.n_seg++];
            g.job = j;
            g.spp = spp;
            g.item_begin = c;
            g.item_count = take;
            g.path_offset = wd.n_paths;
            wd.n_paths += take * spp;
            wd.n_items += take;
            wd.stack_n = std::max(wd.stack_n, scene_stack_entries(jobs[j].sc));
            max_depth = std::max(max_depth, jobs[j].max_depth);
            c += take;
        }
    }
    st = flush();
    if (st) return st;
    if (forked) {
        for (int l = 0; l < lanes - 1; ++l) {
            CUDA_TRY(cudaEventRecord(ctx->ev_join_x[l], ctx->wstream_x[l]));
            CUDA_TRY(cudaStreamWaitEvent(ws, ctx->ev_join_x[l], 0));
        }
    }
    return HPT_OK;
}

// One launch group: the waves covering all items of 'jobs', queued on the context's wave
// stream after the caller's stream, which then waits for them.  Caller holds ctx->mu.
static hpt_status run_jobs(hpt_ctx *ctx, const DevJob *jobs, int n, int prec, bool stats, cudaStream_t user,
                           const AfterWave *after_wave = nullptr)
{
    hpt_status st = ensure_paths(ctx);
    if (st) return st;
    Slot *slot = acquire_slot(ctx);
    JobTable *h = slot->h_table;
    h->n_jobs = n;
    for (int i = 0; i < n; ++i) h->jobs[i] = jobs[i];
    cudaStream_t ws = ctx->wstream;
    CUDA_TRY(cudaEventRecord(ctx->ev_in, user));
    CUDA_TRY(cudaStreamWaitEvent(ws, ctx->ev_in, 0));
    const size_t bytes = offsetof(JobTable, jobs) + sizeof(DevJob) * n;
    CUDA_TRY(cudaMemcpyAsync(slot->d_table, h, bytes, cudaMemcpyHostToDevice, ws));
    if (stats) {
        CUDA_TRY(cudaMemsetAsync(ctx->d_scr->counters, 0, sizeof(ctx->d_scr->counters), ws));
        for (int l = 0; l < hpt_ctx::EXTRA_LANES; ++l)
            CUDA_TRY(cudaMemsetAsync(ctx->d_scr_x[l]->counters, 0, sizeof(ctx->d_scr->counters), ws));
    }
    st = enqueue_waves(ctx, jobs, n, prec, stats, slot->d_table, ws, true, after_wave);
    if (st) return st;
    CUDA_TRY(cudaEventRecord(slot->done, ws));
    CUDA_TRY(cudaEventRecord(ctx->ev_out, ws));
    CUDA_TRY(cudaStreamWaitEvent(user, ctx->ev_out, 0));
    return HPT_OK;
}

// A frame of one job as a captured CUDA graph: the first call with a given launch shape
// (arithmetic, output buffer, items, spp, depth, wave capacity) captures every wave launch;
// each call copies its job table to the frame's device table and replays.  Caller holds
// ctx->mu.
static void free_frame(hpt_ctx::FrameGraph &g)
{
    if (g.done) cudaEventSynchronize(g.done);
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.done) cudaEventDestroy(g.done);
    for (int k = 0; k < hpt_ctx::TABLE_RING; ++k) {
        if (g.copied[k]) cudaEventDestroy(g.copied[k]);
        if (g.h_ring[k]) cudaFreeHost(g.h_ring[k]);
    }
    if (g.d_table) cudaFree(g.d_table);
    g = hpt_ctx::FrameGraph();
}

static hpt_status apply_tuned(hpt_ctx *ctx, const SceneRec *rec);

static hpt_status run_graph(hpt_ctx *ctx, const DevJob &J, int prec, cudaStream_t user)
{
    hpt_status st = ensure_paths(ctx);
    if (st) return st;
    hpt_ctx::FrameGraph *g = nullptr;
    for (auto &x : ctx->graphs)
        if (x.prec == prec && x.out == (void *)J.out && x.n_items == J.n_items && x.spp == J.spp &&
            x.max_depth == J.max_depth && x.capacity == ctx->capacity)
            g = &x;
    cudaStream_t ws = ctx->wstream;
    const size_t bytes = offsetof(JobTable, jobs) + sizeof(DevJob);
    if (!g) {
        if (ctx->graphs.size() >= 8) {   // evict the least recently used frame
            auto lru = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                        [](const hpt_ctx::FrameGraph &a, const hpt_ctx::FrameGraph &b) {
                                            return a.last_use < b.last_use;
                                        });
            free_frame(*lru);
            ctx->graphs.erase(lru);
        }
        hpt_ctx::FrameGraph x;
        x.prec = prec;
        x.out = (void *)J.out;
        x.n_items = J.n_items;
        x.spp = J.spp;
        x.max_depth = J.max_depth;
        x.capacity = ctx->capacity;
        cudaError_t e0 = cudaMalloc(&x.d_table, sizeof(JobTable));
        if (e0 == cudaSuccess) e0 = cudaEventCreateWithFlags(&x.done, cudaEventDisableTiming);
        for (int k = 0; k < hpt_ctx::TABLE_RING && e0 == cudaSuccess; ++k) {
            e0 = cudaMallocHost(&x.h_ring[k], sizeof(JobTable));
            if (e0 == cudaSuccess) e0 = cudaEventCreateWithFlags(&x.copied[k], cudaEventDisableTiming);
        }
        if (e0 != cudaSuccess) {
            free_frame(x);
            return fail(HPT_ERR_CUDA, "frame resources: %s", cudaGetErrorString(e0));
        }
        cudaGraph_t graph = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(ws, cudaStreamCaptureModeThreadLocal));
        hpt_status st2 = enqueue_waves(ctx, &J, 1, prec, false, x.d_table, ws, false);
        cudaError_t e2 = cudaStreamEndCapture(ws, &graph);
        cudaError_t e3 = cudaErrorUnknown;
        if (!st2 && e2 == cudaSuccess) e3 = cudaGraphInstantiate(&x.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (st2 || e2 != cudaSuccess || e3 != cudaSuccess) {
            free_frame(x);
            return st2 ? st2 : fail(HPT_ERR_CUDA, "frame capture failed: %s", cudaGetErrorString(e2 ? e2 : e3));
        }
        ctx->graphs.push_back(x);
        g = &ctx->graphs.back();
    }
    // this replay's job table: a free pinned ring buffer, copied ahead of the replay on ws
    const int k = g->ring_next;
    g->ring_next = (k + 1) % hpt_ctx::TABLE_RING;
    if (g->ring_used[k]) CUDA_TRY(cudaEventSynchronize(g->copied[k]));
    g->ring_used[k] = true;
    g->h_ring[k]->n_jobs = 1;
    g->h_ring[k]->pad = 0;
    g->h_ring[k]->jobs[0] = J;
    g->last_use = ++ctx->graph_clock;
    CUDA_TRY(cudaEventRecord(ctx->ev_in, user));
    CUDA_TRY(cudaStreamWaitEvent(ws, ctx->ev_in, 0));
    CUDA_TRY(cudaMemcpyAsync(g->d_table, g->h_ring[k], bytes, cudaMemcpyHostToDevice, ws));
    CUDA_TRY(cudaEventRecord(g->copied[k], ws));
    CUDA_TRY(cudaGraphLaunch(g->exec, ws));
    CUDA_TRY(cudaEventRecord(g->done, ws));
    CUDA_TRY(cudaEventRecord(ctx->ev_out, ws));
    CUDA_TRY(cudaStreamWaitEvent(user, ctx->ev_out, 0));
    return HPT_OK;
}

extern "C" hpt_status hpt_trace(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc, void *out_dev,
                                size_t out_bytes, void *stream)
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    if (!out_dev) return fail(HPT_ERR_INVALID_ARG, "out_dev is NULL");
    DevJob J;
    SceneRec *rec = nullptr;
    st = make_job(ctx, scene_id, desc, out_dev, out_bytes, J, &rec);
    if (st) return st;
    std::lock_guard<std::mutex> lk(ctx->mu);
    st = apply_tuned(ctx, rec);
    if (st) return st;
    nvtxRangePushA("hpt_trace frame");
    st = ctx->use_graphs && ctx->debug_waves == 0 ? run_graph(ctx, J, desc->precision, (cudaStream_t)stream)
                                                  : run_jobs(ctx, &J, 1, desc->precision, false, (cudaStream_t)stream);
    nvtxRangePop();
    return st;
}

extern "C" hpt_status hpt_trace_host(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc, void *out_host,
                                     size_t out_bytes, void *stream)
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    if (!out_host || !desc) return fail(HPT_ERR_INVALID_ARG, "out_host or desc is NULL");
    DevJob J;
    SceneRec *rec = nullptr;
    st = make_job(ctx, scene_id, desc, nullptr, 0, J, &rec);
    if (st) return st;
    size_t need = (size_t)8 * desc->n_lambda * desc->K * (size_t)desc->W * desc->H;
    if (out_bytes < need) return fail(HPT_ERR_INVALID_ARG, "out_bytes %zu < %zu", out_bytes, need);
    std::lock_guard<std::mutex> lk(ctx->mu);
    st = apply_tuned(ctx, rec);
    if (st) return st;
    if (ctx->host_out_bytes < need) {
        CUDA_TRY(cudaDeviceSynchronize());
        if (ctx->host_out_dev) cudaFree(ctx->host_out_dev);
        ctx->host_out_dev = nullptr;
        ctx->host_out_bytes = 0;
        CUDA_TRY(cudaMalloc(&ctx->host_out_dev, need));
        ctx->host_out_bytes = need;
    }
    J.out = (float2 *)ctx->host_out_dev;
    cudaStream_t s = (cudaStream_t)stream;
    struct Range {
        Range() { nvtxRangePushA("hpt_trace_host frame + copy"); }
        ~Range() { nvtxRangePop(); }
    } range;
    cudaPointerAttributes pa{};
    const bool pinned = cudaPointerGetAttributes(&pa, out_host) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    if (!pinned) (void)cudaGetLastError();   // an unregistered pointer is not an error here
    if (!pinned || ctx->debug_waves > 0) {
        // pageable memory: a copy into it would hold the host until it ends, so the whole frame
        // runs first (the staging buffer is the context's, so its captured graph is reused)
        st = ctx->use_graphs && ctx->debug_waves == 0 ? run_graph(ctx, J, desc->precision, s)
                                                      : run_jobs(ctx, &J, 1, desc->precision, false, s);
        if (st) return st;
        CUDA_TRY(cudaMemcpyAsync(out_host, ctx->host_out_dev, need, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return HPT_OK;
    }
    // pinned memory: the fields' rows are final once every pixel of their tile row has been
    // accumulated, and waves take the items (lambda-major, tile rows in order) in increasing
    // order, so after each wave the rows it completed are copied on the copy stream, behind an
    // event of that wave (the copy stream has waited for every earlier wave as well); only the
    // last wave's rows are copied after the trace
    if (!ctx->cstream) CUDA_TRY(cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking));
    if (!ctx->ev_wave) CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_wave, cudaEventDisableTiming));
    if (!ctx->ev_copied) CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_copied, cudaEventDisableTiming));
    const long long per_lam = (long long)J.n_tiles * 32, row_items = (long long)J.n_tiles_x * 32;
    const int n_rows = J.n_tiles / J.n_tiles_x;   // tile rows of one wavelength
    long long copied = 0;                         // tile rows (lambda * n_rows + row) copied so far
    char *dst = (char *)out_host;
    const char *src = (const char *)ctx->host_out_dev;
    const AfterWave after = [&](const WaveDesc &wd, cudaStream_t ls) -> hpt_status {
        long long end = 0;
        for (int i = 0; i < wd.n_seg; ++i) end = std::max(end, wd.seg[i].item_begin + wd.seg[i].item_count);
        CUDA_TRY(cudaEventRecord(ctx->ev_wave, ls));
        CUDA_TRY(cudaStreamWaitEvent(ctx->cstream, ctx->ev_wave, 0));
        const long long done = (end / per_lam) * n_rows + (end % per_lam) / row_items;
        while (copied < done) {
            const int lam = (int)(copied / n_rows), r0 = (int)(copied % n_rows);
            const int r1 = (int)std::min<long long>(n_rows, r0 + (done - copied));
            const int y0 = r0 * TILE_H, y1 = std::min(r1 * TILE_H, J.H);
            for (int k = 0; k < J.K; ++k) {
                const size_t off = (((size_t)lam * J.K + k) * J.H + y0) * J.W * sizeof(float2);
                CUDA_TRY(cudaMemcpyAsync(dst + off, src + off, (size_t)(y1 - y0) * J.W * sizeof(float2),
                                         cudaMemcpyDeviceToHost, ctx->cstream));
            }
            copied += r1 - r0;
        }
        return HPT_OK;
    };
    st = run_jobs(ctx, &J, 1, desc->precision, false, s, &after);
    if (st) {
        cudaStreamSynchronize(ctx->cstream);   // no copy lands in out_host after the call returns
        return st;
    }
    if (copied != (long long)desc->n_lambda * n_rows) {
        cudaStreamSynchronize(ctx->cstream);
        return fail(HPT_ERR_CUDA, "copy-out covered %lld of %lld tile rows", copied, (long long)desc->n_lambda * n_rows);
    }
    CUDA_TRY(cudaEventRecord(ctx->ev_copied, ctx->cstream));
    CUDA_TRY(cudaStreamWaitEvent(s, ctx->ev_copied, 0));
    CUDA_TRY(cudaStreamSynchronize(s));
    return HPT_OK;
}

static hpt_status read_status(hpt_ctx *ctx)
{
    unsigned bits = 0;
    CUDA_TRY(cudaMemcpy(&bits, &ctx->d_scr->status, sizeof bits, cudaMemcpyDeviceToHost));
    for (int l = 0; l < hpt_ctx::EXTRA_LANES; ++l) {
        unsigned b2 = 0;
        CUDA_TRY(cudaMemcpy(&b2, &ctx->d_scr_x[l]->status, sizeof b2, cudaMemcpyDeviceToHost));
        bits |= b2;
    }
    {
        unsigned b2 = 0;
        CUDA_TRY(fixed_scratch_status(ctx->device, &b2));
        bits |= b2;
    }
    if (bits) {
        CUDA_TRY(cudaMemset(&ctx->d_scr->status, 0, sizeof bits));
        for (int l = 0; l < hpt_ctx::EXTRA_LANES; ++l) CUDA_TRY(cudaMemset(&ctx->d_scr_x[l]->status, 0, sizeof bits));
        return fail(HPT_ERR_DEVICE, "kernel status 0x%x:%s%s%s%s", bits, (bits & ST_STACK_OVERFLOW) ? " traversal-stack-overflow" : "",
                    (bits & ST_BAD_JOB) ? " bad-job" : "", (bits & ST_FALLBACK_STACK) ? " fp64-stack-overflow" : "",
                    (bits & ST_BOUNDS) ? " index-out-of-bounds" : "");
    }
    return HPT_OK;
}

extern "C" hpt_status hpt_sync(hpt_ctx *ctx)
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    CUDA_TRY(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(ctx->mu);
    return read_status(ctx);
}

extern "C" hpt_status hpt_trace_counters(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc, void *out_dev,
                                         size_t out_bytes, uint64_t counters[HPT_NCOUNTERS])
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    if (!out_dev || !counters) return fail(HPT_ERR_INVALID_ARG, "out_dev or counters is NULL");
    DevJob J;
    st = make_job(ctx, scene_id, desc, out_dev, out_bytes, J, nullptr);
    if (st) return st;
    std::lock_guard<std::mutex> lk(ctx->mu);
    st = run_jobs(ctx, &J, 1, desc->precision, true, 0);
    if (st) return st;
    CUDA_TRY(cudaStreamSynchronize(0));
    unsigned long long c[8];
    CUDA_TRY(cudaMemcpy(c, ctx->d_scr->counters, sizeof c, cudaMemcpyDeviceToHost));
    for (int k = 0; k < HPT_NCOUNTERS; ++k) counters[k] = c[k];
    for (int l = 0; l < hpt_ctx::EXTRA_LANES; ++l) {
        CUDA_TRY(cudaMemcpy(c, ctx->d_scr_x[l]->counters, sizeof c, cudaMemcpyDeviceToHost));
        for (int k = 0; k < HPT_NCOUNTERS; ++k) counters[k] += c[k];
    }
    counters[0] = (uint64_t)desc->n_lambda * desc->W * (uint64_t)desc->H * desc->spp;   // path samples
    return read_status(ctx);
}

extern "C" hpt_status hpt_trace_timed(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc, void *out_dev,
                                      size_t out_bytes, float kernel_ms[HPT_NKERNELS],
                                      uint32_t launches[HPT_NKERNELS])
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    if (!out_dev || !kernel_ms || !launches) return fail(HPT_ERR_INVALID_ARG, "out_dev, kernel_ms or launches is NULL");
    DevJob J;
    st = make_job(ctx, scene_id, desc, out_dev, out_bytes, J, nullptr);
    if (st) return st;
    std::lock_guard<std::mutex> lk(ctx->mu);
    hpt_ctx::KernelTimer tm;
    ctx->timer = &tm;
    st = run_jobs(ctx, &J, 1, desc->precision, false, 0);
    ctx->timer = nullptr;
    cudaError_t e = cudaStreamSynchronize(ctx->wstream);
    for (int k = 0; k < HPT_NKERNELS; ++k) kernel_ms[k] = 0.0f, launches[k] = 0;
    if (!st && e == cudaSuccess) {
        // trace and shade each launch a coherent and an incoherent kernel back to back
        static const uint32_t per_call[HPT_NKERNELS] = {1, 2, 2, 1};
        for (size_t i = 0; i + 1 < tm.used && e == cudaSuccess; ++i) {
            const int k = tm.kind[i];
            if (k < 0) continue;
            float ms = 0.0f;
            e = cudaEventElapsedTime(&ms, tm.ev[i], tm.ev[i + 1]);
            kernel_ms[k] += ms;
            launches[k] += per_call[k];
        }
    }
    for (cudaEvent_t x : tm.ev) cudaEventDestroy(x);
    if (st) return st;
    if (e != cudaSuccess) return fail(HPT_ERR_CUDA, "kernel timing: %s", cudaGetErrorString(e));
    return read_status(ctx);
}

// ---------------------------------------------------------------------- cache construction
__global__ void k_to_half(const float *__restrict__ in, unsigned short *__restrict__ out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __half_as_ushort(__float2half_rn(in[i]));
}

extern "C" hpt_status hpt_cache_bake(hpt_ctx *ctx, uint64_t scene_id, const hpt_bake_desc *b, float *E_dev,
                                     size_t E_bytes, void *stream)
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    if (!b || !E_dev) return fail(HPT_ERR_INVALID_ARG, "desc or E_dev is NULL");
    if (b->res < 1 || b->res > 1024) return fail(HPT_ERR_INVALID_ARG, "res must be 1..1024");
    if (b->spp < 1 || b->max_depth < 1 || b->max_depth > 64) return fail(HPT_ERR_INVALID_ARG, "bad spp or max_depth");
    for (int k = 0; k < 3; ++k)
        if (!(b->bmax[k] > b->bmin[k]) || !std::isfinite(b->bmin[k]) || !std::isfinite(b->bmax[k]))
            return fail(HPT_ERR_INVALID_ARG, "need bmin < bmax");
    const size_t need = (size_t)b->res * b->res * b->res * 3 * sizeof(float);
    if (E_bytes < need) return fail(HPT_ERR_INVALID_ARG, "E_bytes %zu < %zu", E_bytes, need);
    // the cells as a res x res^2 image, the channels as three wavelengths
    hpt_render_desc r;
    memset(&r, 0, sizeof r);
    r.W = b->res;
    r.H = b->res * b->res;
    r.pitch = 1.0;
    r.n_lambda = 3;
    for (int c = 0; c < 3; ++c) {
        r.lambda[c] = 1.0;
        r.channel[c] = c;
    }
    r.spp = b->spp;
    r.max_depth = b->max_depth;
    r.K = 1;
    r.seed = b->seed;
    r.phase_mode = HPT_PHASE_ZERO;
    r.facet_size = 1.0;
    for (int k = 0; k < 4; ++k) r.T[5 * k] = 1.0;
    r.precision = HPT_PREC_DF32;
    DevJob J;
    st = make_job(ctx, scene_id, &r, nullptr, 0, J, nullptr);
    if (st) return st;
    J.kind = 1;
    J.bake_out = E_dev;
    for (int k = 0; k < 3; ++k) {
        J.bake_lo[k] = b->bmin[k];
        J.bake_h[k] = (b->bmax[k] - b->bmin[k]) / (float)b->res;
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    return run_jobs(ctx, &J, 1, HPT_PREC_DF32, false, (cudaStream_t)stream);
}

// replace the cache from a device float grid (E_dev) or a host binary16 grid (E_half)
static hpt_status set_cache(hpt_ctx *ctx, uint64_t scene_id, int32_t res, const float bmin[3], const float bmax[3],
                            const float *E_dev, const uint16_t *E_half)
{
    if (!bmin || !bmax || (res > 0 && !E_dev && !E_half)) return fail(HPT_ERR_INVALID_ARG, "bmin, bmax or the grid is NULL");
    if (res < 0 || res > 1024) return fail(HPT_ERR_INVALID_ARG, "res must be 0..1024");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(bmin[k]) || !std::isfinite(bmax[k]) || !(bmax[k] > bmin[k]))
            return fail(HPT_ERR_INVALID_ARG, "need finite bmin < bmax");
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->scenes.find(scene_id);
    if (it == ctx->scenes.end()) return fail(HPT_ERR_NOT_FOUND, "unknown scene %llu", (unsigned long long)scene_id);
    SceneRec *rec = it->second.get();
    if (rec->users.load() > 0) return fail(HPT_ERR_BUSY, "scene %llu is used by queued requests", (unsigned long long)scene_id);
    // traces already launched may still read the old cache
    CUDA_TRY(cudaDeviceSynchronize());
    if (rec->cache_buf) {
        CUDA_TRY(cudaFree(rec->cache_buf));
        rec->cache_buf = nullptr;
    }
    if (res > 0) {
        const size_t n = (size_t)res * res * res * 3;
        CUDA_TRY(cudaMalloc(&rec->cache_buf, n * sizeof(unsigned short)));
        if (E_dev) {
            k_to_half<<<(int)std::min<size_t>((n + 255) / 256, 152 * 32), 256>>>(E_dev, (unsigned short *)rec->cache_buf, n);
            CUDA_TRY(cudaGetLastError());
        } else {
            CUDA_TRY(cudaMemcpy(rec->cache_buf, E_half, n * sizeof(unsigned short), cudaMemcpyHostToDevice));
        }
        CUDA_TRY(cudaDeviceSynchronize());
        rec->dev.cache = (const unsigned short *)rec->cache_buf;
    }
    rec->dev.cache_res = res;
    for (int k = 0; k < 3; ++k) {
        rec->dev.cache_bmin[k] = bmin[k];
        rec->dev.cache_bmax[k] = bmax[k];
    }
    return HPT_OK;
}

extern "C" hpt_status hpt_cache_upload(hpt_ctx *ctx, uint64_t scene_id, int32_t res, const float bmin[3],
                                       const float bmax[3], const uint16_t *E_half_host)
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    return set_cache(ctx, scene_id, res, bmin, bmax, nullptr, E_half_host);
}

extern "C" hpt_status hpt_scene_set_cache(hpt_ctx *ctx, uint64_t scene_id, int32_t res, const float bmin[3],
                                          const float bmax[3], const float *E_dev)
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    return set_cache(ctx, scene_id, res, bmin, bmax, E_dev, nullptr);
}


// ---------------------------------------------------------------------------- autotune
static void drop_graphs(hpt_ctx *ctx)
{
    for (auto &g : ctx->graphs) free_frame(g);
    ctx->graphs.clear();
}

static int scene_class(int n_tris)
{
    return n_tris < (1 << 12) ? 0 : n_tris < (1 << 16) ? 1 : n_tris < (1 << 20) ? 2 : 3;
}

// Switch the trace launch shape: wave size, lanes and grid multipliers.  Caller holds ctx->mu.
static hpt_status set_shape(hpt_ctx *ctx, int cap, int lanes, int tm, int sm)
{
    const bool realloc = cap != ctx->capacity || lanes != ctx->lanes || !ctx->pb_arena;
    if (realloc || tm != ctx->trace_mult || sm != ctx->shade_mult) drop_graphs(ctx);   // frames embed the shape
    if (realloc) {
        CUDA_TRY(cudaDeviceSynchronize());   // waves in flight use the wave state
        if (ctx->pb_arena) CUDA_TRY(cudaFree(ctx->pb_arena));
        ctx->pb_arena = nullptr;
        for (int l = 0; l < hpt_ctx::EXTRA_LANES; ++l) {
            if (ctx->pb_arena_x[l]) CUDA_TRY(cudaFree(ctx->pb_arena_x[l]));
            ctx->pb_arena_x[l] = nullptr;
        }
        ctx->capacity = cap;
        ctx->lanes = lanes;
    }
    ctx->trace_mult = tm;
    ctx->shade_mult = sm;
    for (int prec = 0; prec < 2; ++prec) {
        ctx->grid_trace[prec] = ctx->sm_count * ctx->occ_trace[prec] * tm;
        ctx->grid_shade[prec] = ctx->sm_count * ctx->occ_shade[prec] * sm;
    }
    return realloc ? ensure_paths(ctx) : HPT_OK;
}

// the tuned shape of the scene's size class, if hpt_autotune recorded one; caller holds ctx->mu
static hpt_status apply_tuned(hpt_ctx *ctx, const SceneRec *rec)
{
    const int c = scene_class(rec->dev.n_tris);
    if (!ctx->tuned_valid[c]) return HPT_OK;
    const hpt_ctx::Shape &t = ctx->tuned[c];
    if (t.cap == ctx->capacity && t.lanes == ctx->lanes && t.tm == ctx->trace_mult && t.sm == ctx->shade_mult &&
        ctx->pb_arena)
        return HPT_OK;
    return set_shape(ctx, t.cap, t.lanes, t.tm, t.sm);
}

extern "C" hpt_status hpt_autotune(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc, hpt_tuning *out)
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    if (!desc) return fail(HPT_ERR_INVALID_ARG, "desc is NULL");
    hpt_render_desc band = *desc;
    const double per_row = (double)desc->W * std::max(desc->n_lambda, 1) * std::max(desc->spp, 1);
    band.H = (int)std::min<double>(desc->H, std::max(1.0, std::ceil(50e6 / per_row)));
    DevJob J;
    SceneRec *rec = nullptr;
    st = make_job(ctx, scene_id, &band, nullptr, 0, J, &rec);
    if (st) return st;
    const size_t out_b = (size_t)8 * band.n_lambda * band.K * (size_t)band.W * band.H;
    std::lock_guard<std::mutex> lk(ctx->mu);
    void *dout = nullptr;
    CUDA_TRY(cudaMalloc(&dout, out_b));
    J.out = (float2 *)dout;
    size_t fr = 0, tot = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaMemGetInfo(&fr, &tot);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaFree(dout);
        return fail(HPT_ERR_CUDA, "autotune set-up: %s", cudaGetErrorString(ce));
    }
    const size_t avail = fr + (ctx->pb_arena ? (size_t)ctx->lanes * ctx->capacity * path_bytes() : 0);
    hpt_ctx::Shape cur = {ctx->capacity, ctx->lanes, ctx->trace_mult, ctx->shade_mult};
    const hpt_ctx::Shape start = cur;
    int n_cand = 0;
    auto fits = [&](const hpt_ctx::Shape &x) {
        return (size_t)x.lanes * x.cap * path_bytes() <= avail / 2 && x.cap >= J.spp;
    };
    // band time of one shape: three runs, the first a warm-up, the best of the other two
    auto measure = [&](const hpt_ctx::Shape &x, double &ms_out) -> hpt_status {
        hpt_status s2 = set_shape(ctx, x.cap, x.lanes, x.tm, x.sm);
        if (s2) return s2;
        ++n_cand;
        double best = 1e30;
        for (int rep = 0; rep < 3; ++rep) {
            CUDA_TRY(cudaEventRecord(e0, ctx->wstream));
            s2 = run_jobs(ctx, &J, 1, band.precision, false, ctx->wstream);
            if (s2) return s2;
            CUDA_TRY(cudaEventRecord(e1, ctx->wstream));
            CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.0f;
            CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) best = std::min(best, (double)ms);
        }
        ms_out = best;
        return HPT_OK;
    };
    double best_ms = 0.0, start_ms = 0.0;
    if (!fits(cur)) cur.cap = std::max(J.spp, 1 << 21);
    st = measure(cur, best_ms);
    start_ms = best_ms;
    auto consider = [&](hpt_ctx::Shape x) {
        if (st || !fits(x)) return;
        if (x.cap == cur.cap && x.lanes == cur.lanes && x.tm == cur.tm && x.sm == cur.sm) return;
        double ms = 0.0;
        st = measure(x, ms);
        if (!st && ms < best_ms * 0.99) {
            best_ms = ms;
            cur = x;
        }
    };
    const hpt_ctx::Shape c0 = cur;
    for (int cap : {1 << 21, 1 << 22, 1 << 23, 1 << 24}) consider({cap, c0.lanes, c0.tm, c0.sm});
    const hpt_ctx::Shape c1 = cur;
    for (int lanes = 1; lanes <= HPT_MAX_LANES; ++lanes) consider({c1.cap, lanes, c1.tm, c1.sm});
    const hpt_ctx::Shape c2 = cur;
    for (int tm : {1, 2, 4}) consider({c2.cap, c2.lanes, tm, c2.sm});
    const hpt_ctx::Shape c3 = cur;
    for (int sm : {1, 2, 4}) consider({c3.cap, c3.lanes, c3.tm, sm});
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dout);
    if (st) {
        const std::string msg = g_err;
        set_shape(ctx, start.cap, start.lanes, start.tm, start.sm);
        return fail(st, "%s", msg.c_str());
    }
    st = set_shape(ctx, cur.cap, cur.lanes, cur.tm, cur.sm);
    if (st) return st;
    const int cls = scene_class(rec->dev.n_tris);
    ctx->tuned[cls] = cur;
    ctx->tuned_valid[cls] = true;
    if (out) {
        out->paths_per_wave = cur.cap;
        out->lanes = cur.lanes;
        out->trace_blocks_per_sm = ctx->occ_trace[band.precision] * cur.tm;
        out->shade_blocks_per_sm = ctx->occ_shade[band.precision] * cur.sm;
        out->scene_class = cls;
        out->candidates = n_cand;
        out->band_ms = best_ms;
        out->band_ms_start = start_ms;
        out->band_path_samples = (int64_t)band.n_lambda * band.W * (int64_t)band.H * band.spp;
    }
    return read_status(ctx);
}

// ------------------------------------------------------------------------------ serving
// Continuous batching.  A scheduler thread admits queued requests while fewer than
// max_inflight are active and their outputs fit in memory (caller-owned outputs: the HBM budget;
// library-owned outputs: allocated at admission, only while the device's free memory minus a
// reserve holds them), then keeps the device busy with waves: each wave takes an equal share of
// its paths from every active request of one arithmetic (round robin), so requests that arrive
// while others are running join the next wave and their work overlaps on the device.  A wave
// records its lane's kernel status bits into a pinned word of its own; a request is complete
// when the last wave carrying its items has completed, with the status bits of all of them.
// Per-pixel results do not depend on how items are grouped into waves, so a request's fields are
// the same alone and in the mix.
constexpr size_t FINISHED_KEPT = 4096;     // finished requests kept queryable (oldest dropped)

static size_t out_reserve_bytes(size_t total) { return std::max<size_t>(size_t(1) << 30, total / 20); }

// a request leaves the device's books; caller holds smu
static void finish_request(hpt_ctx *ctx, const std::shared_ptr<Request> &r, double now)
{
    r->done = true;
    r->t_done = now;
    if (r->status == HPT_OK && r->dev_bits) {
        char m[192];
        snprintf(m, sizeof m, "request %llu: kernel status 0x%x%s%s%s%s", (unsigned long long)r->id, r->dev_bits,
                 (r->dev_bits & ST_STACK_OVERFLOW) ? " traversal-stack-overflow" : "",
                 (r->dev_bits & ST_BAD_JOB) ? " bad-job" : "", (r->dev_bits & ST_FALLBACK_STACK) ? " fp64-stack-overflow" : "",
                 (r->dev_bits & ST_BOUNDS) ? " index-out-of-bounds" : "");
        r->status = HPT_ERR_DEVICE;
        r->err = m;
    }
    if (r->admitted) {
        ctx->bytes_active -= r->out_bytes;
        ctx->live--;
    }
    r->scene->users--;
    ctx->finished.push_back(r->id);
    while (ctx->finished.size() > FINISHED_KEPT) {
        auto it = ctx->reqs.find(ctx->finished.front());
        ctx->finished.pop_front();
        if (it == ctx->reqs.end()) continue;
        if (it->second->out_lib) cudaFreeAsync(it->second->out_lib, ctx->ostream);
        ctx->reqs.erase(it);
    }
}

static void retire_oldest(hpt_ctx *ctx)
{
    InflightWave w;
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        if (ctx->inflight.empty()) return;
        w = ctx->inflight.front();
    }
    cudaEventSynchronize(w.ev);
    const double now = ctx->now_us();
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        ctx->inflight.pop_front();
        ctx->free_events.push_back(w.ev);
        const unsigned bits = ctx->h_wave_status[w.status_slot];
        ctx->status_slot_used[w.status_slot] = false;
        for (auto &r : w.carried) {
            r->dev_bits |= bits;
            if (--r->waves == 0 && (r->stopped || r->next >= r->job.n_items)) finish_request(ctx, r, now);
        }
    }
    ctx->dcv.notify_all();
    ctx->scv.notify_all();
}

// the requests of a wave that could not be issued stop here; caller holds smu
static void stop_requests(hpt_ctx *ctx, const std::vector<std::pair<std::shared_ptr<Request>, int>> &picks, hpt_status st,
                          const std::string &msg)
{
    const double now = ctx->now_us();
    for (auto &pk : picks) {
        auto &r = pk.first;
        if (r->stopped) continue;
        r->stopped = true;
        r->status = st;
        r->err = msg;
        auto it = std::find(ctx->active.begin(), ctx->active.end(), r);
        if (it != ctx->active.end()) ctx->active.erase(it);
        if (r->waves == 0) finish_request(ctx, r, now);
    }
}

// admission of the oldest pending request; caller holds smu
static bool try_admit(hpt_ctx *ctx)
{
    if (ctx->pending.empty() || ctx->live >= ctx->max_inflight) return false;
    auto r = ctx->pending.front();
    if (ctx->live > 0 && ctx->bytes_active + r->out_bytes > ctx->budget) return false;
    if (r->lib_out) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return false;
        const size_t reserve = out_reserve_bytes(tot);
        if (fr < reserve || fr - reserve < r->out_bytes) {
            // nothing else on the device will free memory for it: refuse it rather than wait
            if (ctx->live > 0) return false;
            ctx->pending.pop_front();
            r->status = HPT_ERR_OOM;
            r->err = "request output does not fit in the device's free memory";
            r->stopped = true;
            finish_request(ctx, r, ctx->now_us());
            return true;
        }
        void *p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, r->out_bytes, ctx->ostream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->ostream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (p) cudaFreeAsync(p, ctx->ostream);
            if (ctx->live > 0) return false;
            ctx->pending.pop_front();
            r->status = HPT_ERR_OOM;
            r->err = std::string("request output: ") + cudaGetErrorString(e);
            r->stopped = true;
            finish_request(ctx, r, ctx->now_us());
            return true;
        }
        r->out_lib = p;
        r->job.out = (float2 *)p;
    }
    ctx->pending.pop_front();
    r->t_admit = ctx->now_us();
    r->admitted = true;
    ctx->bytes_active += r->out_bytes;
    ctx->live++;
    if (r->job.n_items == 0) {
        finish_request(ctx, r, r->t_admit);
        return true;
    }
    ctx->active.push_back(r);
    return true;
}

static void sched_loop(hpt_ctx *ctx)
{
    cudaSetDevice(ctx->device);
    for (;;) {
        std::vector<std::pair<std::shared_ptr<Request>, int>> picks;
        int prec = -1;
        bool idle_wait = false;
        int slot_idx = -1;
        {
            std::unique_lock<std::mutex> lk(ctx->smu);
            auto schedulable = [&] {
                for (auto &r : ctx->active)
                    if (r->next < r->job.n_items) return true;
                return false;
            };
            ctx->scv.wait(lk, [&] {
                return ctx->stop || !ctx->pending.empty() || schedulable() || !ctx->inflight.empty();
            });
            if (ctx->stop && ctx->inflight.empty()) break;
            if (ctx->stop) {
                idle_wait = true;   // drain what is in flight, start nothing new
                goto unlocked;
            }
            bool admitted_any = false;
            while (!ctx->stop && try_admit(ctx)) admitted_any = true;
            if (admitted_any) ctx->dcv.notify_all();
            // one wave: equal path shares of the active requests that use one arithmetic
            std::vector<std::shared_ptr<Request>> cand;
            const size_t na = ctx->active.size();
            for (size_t k = 0; k < na; ++k) {
                auto &r = ctx->active[(ctx->rr + k) % na];
                if (r->next >= r->job.n_items) continue;
                if (prec < 0) prec = r->prec;
                if (r->prec == prec && (int)cand.size() < MAX_SEG) cand.push_back(r);
            }
            if (!cand.empty()) {
                for (int k = 0; k < hpt_ctx::STATUS_SLOTS; ++k)
                    if (!ctx->status_slot_used[k]) { slot_idx = k; break; }
            }
            if (!cand.empty() && slot_idx >= 0) {
                ctx->status_slot_used[slot_idx] = true;
                ctx->rr = (ctx->rr + 1) % std::max<size_t>(na, 1);
                const long long share = std::max<long long>(1, (long long)ctx->sched_capacity / (long long)cand.size());
                for (auto &r : cand) {
                    long long take = std::max<long long>(1, share / r->job.spp);
                    take = std::min<long long>(take, r->job.n_items - r->next);
                    picks.push_back({r, (int)take});
                }
            } else {
                idle_wait = !ctx->inflight.empty();
            }
        }
    unlocked:
        if (!picks.empty()) {
            hpt_status st = HPT_OK;
            std::string msg;
            InflightWave w;
            w.status_slot = slot_idx;
            {
                std::lock_guard<std::mutex> lk(ctx->mu);
                nvtxRangePushA("hpt serving wave");
                if (ctx->flags & HPT_CTX_FAIL_SERVING_WAVES) st = fail(HPT_ERR_OOM, "serving wave state: injected failure");
                if (!st) st = ensure_sched_paths(ctx);
                Slot *slot = st ? nullptr : acquire_slot(ctx);
                WaveDesc wd;
                memset(&wd, 0, sizeof wd);
                int max_depth = 1;
                if (slot) {
                    JobTable *h = slot->h_table;
                    h->n_jobs = 0;
                    for (auto &pk : picks) {
                        Request &r = *pk.first;
                        const int j = h->n_jobs++;
                        h->jobs[j] = r.job;
                        WaveSeg &g = wd.seg[wd.n_seg++];
                        g.job = j;
                        g.spp = r.job.spp;
                        g.item_begin = r.next;
                        g.item_count = pk.second;
                        g.path_offset = wd.n_paths;
                        wd.n_paths += pk.second * r.job.spp;
                        wd.n_items += pk.second;
                        wd.stack_n = std::max(wd.stack_n, scene_stack_entries(r.job.sc));
                        max_depth = std::max(max_depth, r.job.max_depth);
                    }
                    // this wave's lane: path state, scratch and stream of its own
                    const int lane = ctx->sched_next++ % HPT_LANES;
                    cudaStream_t ws = ctx->slane_stream[lane];
                    const PathBufs &lpb = ctx->spb[lane];
                    SlotScratch *lscr = ctx->sscr[lane];
                    const int n_iter = max_depth + 1;
                    cudaError_t e = cudaMemcpyAsync(slot->d_table, h, offsetof(JobTable, jobs) + sizeof(DevJob) * h->n_jobs,
                                                    cudaMemcpyHostToDevice, ws);
                    if (e == cudaSuccess) e = cudaMemsetAsync(lscr->qcount, 0, sizeof(int) * 3 * (n_iter + 1), ws);
                    if (e == cudaSuccess) e = wave_gen(prec, slot->d_table, wd, lpb, lscr, ws);
                    for (int it = 0; e == cudaSuccess && it < n_iter; ++it) {
                        e = wave_trace(prec, false, slot->d_table, wd, lpb, lscr, it, ctx->grid_trace[prec], ws);
                        if (e == cudaSuccess) e = wave_shade(prec, false, slot->d_table, wd, lpb, lscr, it, ctx->grid_shade[prec], ws);
                    }
                    if (e == cudaSuccess) e = wave_accum(prec, slot->d_table, wd, lpb, lscr, ws);
                    if (e == cudaSuccess) e = cudaEventRecord(slot->done, ws);
                    // the wave's status bits: copied to its own pinned word, then cleared on the lane
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(ctx->h_wave_status + slot_idx, &lscr->status, sizeof(unsigned),
                                            cudaMemcpyDeviceToHost, ws);
                    if (e == cudaSuccess) e = cudaMemsetAsync(&lscr->status, 0, sizeof(unsigned), ws);
                    {
                        std::lock_guard<std::mutex> lk2(ctx->smu);
                        if (!ctx->free_events.empty()) {
                            w.ev = ctx->free_events.back();
                            ctx->free_events.pop_back();
                        }
                    }
                    if (!w.ev && e == cudaSuccess) e = cudaEventCreateWithFlags(&w.ev, cudaEventDisableTiming);
                    if (e == cudaSuccess) e = cudaEventRecord(w.ev, ws);
                    if (e == cudaSuccess) e = cudaEventRecord(ctx->slane_ev[lane], ws);
                    if (e != cudaSuccess) {
                        // nothing of a failed wave may still run once its requests are reported
                        cudaStreamSynchronize(ws);
                        st = fail(HPT_ERR_CUDA, "serving wave: %s", cudaGetErrorString(e));
                        cudaGetLastError();
                    }
                }
                if (st) msg = g_err;
                nvtxRangePop();
            }
            {
                std::lock_guard<std::mutex> lk(ctx->smu);
                if (st) {
                    if (w.ev) ctx->free_events.push_back(w.ev);
                    ctx->status_slot_used[slot_idx] = false;
                    stop_requests(ctx, picks, st, msg);
                } else {
                    for (auto &pk : picks) {
                        Request &r = *pk.first;
                        r.next += pk.second;
                        r.waves++;
                        w.carried.push_back(pk.first);
                        if (r.next >= r.job.n_items) {
                            auto it = std::find(ctx->active.begin(), ctx->active.end(), pk.first);
                            if (it != ctx->active.end()) ctx->active.erase(it);
                        }
                    }
                    ctx->inflight.push_back(w);
                }
            }
            if (st) {
                ctx->dcv.notify_all();
                continue;
            }
        }
        // keep at most one wave per lane queued ahead; retire finished ones
        size_t nin;
        {
            std::lock_guard<std::mutex> lk(ctx->smu);
            nin = ctx->inflight.size();
        }
        if (nin > HPT_LANES || (picks.empty() && (idle_wait || nin > 0))) retire_oldest(ctx);
    }
    // shutting down: nothing left in flight; pending requests are dropped
}

extern "C" hpt_status hpt_submit(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc, void *out_dev,
                                 size_t out_bytes, uint64_t *req_id)
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    if (!req_id) return fail(HPT_ERR_INVALID_ARG, "req_id is NULL");
    auto r = std::make_shared<Request>();
    SceneRec *rec = nullptr;
    st = make_job(ctx, scene_id, desc, out_dev, out_dev ? out_bytes : 0, r->job, &rec);
    if (st) return st;
    if (r->job.spp > ctx->sched_capacity) return fail(HPT_ERR_UNSUPPORTED, "spp exceeds the wave capacity");
    r->scene = rec;
    r->prec = desc->precision;
    r->out_bytes = (size_t)8 * desc->n_lambda * desc->K * (size_t)desc->W * desc->H;
    r->lib_out = out_dev == nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        if (ctx->stop) return fail(HPT_ERR_BUSY, "context is shutting down");
        if (ctx->pending.size() >= ctx->max_queue) return fail(HPT_ERR_BUSY, "request queue full (%zu)", ctx->max_queue);
        r->id = ctx->next_req++;
        r->t_submit = ctx->now_us();
        rec->users++;
        ctx->pending.push_back(r);
        ctx->reqs[r->id] = r;
        *req_id = r->id;
    }
    ctx->scv.notify_all();
    return HPT_OK;
}

static std::shared_ptr<Request> find_req(hpt_ctx *ctx, uint64_t id)
{
    auto it = ctx->reqs.find(id);
    return it == ctx->reqs.end() ? nullptr : it->second;
}

// the final status of a finished request, with its message for this thread
static hpt_status req_status(const Request &r)
{
    if (r.status != HPT_OK) return fail(r.status, "%s", r.err.c_str());
    return HPT_OK;
}

extern "C" hpt_status hpt_poll(hpt_ctx *ctx, uint64_t req_id, int *done)
{
    g_err.clear();
    if (!ctx || !done) return fail(HPT_ERR_INVALID_ARG, "ctx or done is NULL");
    std::lock_guard<std::mutex> lk(ctx->smu);
    auto r = find_req(ctx, req_id);
    if (!r) return fail(HPT_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
    *done = r->done ? 1 : 0;
    return r->done ? req_status(*r) : HPT_OK;
}

extern "C" hpt_status hpt_wait(hpt_ctx *ctx, uint64_t req_id, uint32_t timeout_ms)
{
    g_err.clear();
    if (!ctx) return fail(HPT_ERR_INVALID_ARG, "ctx is NULL");
    std::unique_lock<std::mutex> lk(ctx->smu);
    auto r = find_req(ctx, req_id);
    if (!r) return fail(HPT_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
    if (timeout_ms == 0) ctx->dcv.wait(lk, [&] { return r->done; });
    else if (!ctx->dcv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; }))
        return fail(HPT_ERR_TIMEOUT, "request %llu not done after %u ms", (unsigned long long)req_id, timeout_ms);
    return req_status(*r);
}

extern "C" hpt_status hpt_cancel(hpt_ctx *ctx, uint64_t req_id)
{
    g_err.clear();
    if (!ctx) return fail(HPT_ERR_INVALID_ARG, "ctx is NULL");
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        auto r = find_req(ctx, req_id);
        if (!r) return fail(HPT_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
        if (r->done || r->stopped) return HPT_OK;
        r->stopped = true;
        r->status = HPT_ERR_CANCELLED;
        r->err = "request cancelled";
        auto pit = std::find(ctx->pending.begin(), ctx->pending.end(), r);
        if (pit != ctx->pending.end()) ctx->pending.erase(pit);
        auto ait = std::find(ctx->active.begin(), ctx->active.end(), r);
        if (ait != ctx->active.end()) ctx->active.erase(ait);
        if (r->waves == 0) finish_request(ctx, r, ctx->now_us());   // else when its last wave completes
    }
    ctx->dcv.notify_all();
    ctx->scv.notify_all();
    return HPT_OK;
}

extern "C" hpt_status hpt_request_times(hpt_ctx *ctx, uint64_t req_id, double t[3])
{
    g_err.clear();
    if (!ctx || !t) return fail(HPT_ERR_INVALID_ARG, "ctx or t is NULL");
    std::lock_guard<std::mutex> lk(ctx->smu);
    auto r = find_req(ctx, req_id);
    if (!r) return fail(HPT_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
    t[0] = r->t_submit;
    t[1] = r->t_admit;
    t[2] = r->t_done;
    return r->done ? HPT_OK : fail(HPT_ERR_BUSY, "request %llu not done", (unsigned long long)req_id);
}

extern "C" hpt_status hpt_request_output(hpt_ctx *ctx, uint64_t req_id, void *dst, size_t bytes)
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    if (!dst) return fail(HPT_ERR_INVALID_ARG, "dst is NULL");
    void *src = nullptr;
    size_t n = 0;
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        auto r = find_req(ctx, req_id);
        if (!r) return fail(HPT_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
        if (!r->done) return fail(HPT_ERR_BUSY, "request %llu not done", (unsigned long long)req_id);
        if (r->status != HPT_OK) return req_status(*r);
        if (!r->out_lib) return fail(HPT_ERR_INVALID_ARG, "request %llu has no library-owned output", (unsigned long long)req_id);
        src = r->out_lib;
        n = r->out_bytes;
    }
    if (bytes < n) return fail(HPT_ERR_INVALID_ARG, "bytes %zu < %zu", bytes, n);
    // the output stays until hpt_request_release, which this copy precedes on the same stream
    CUDA_TRY(cudaMemcpyAsync(dst, src, n, cudaMemcpyDefault, ctx->ostream));
    CUDA_TRY(cudaStreamSynchronize(ctx->ostream));
    return HPT_OK;
}

extern "C" hpt_status hpt_request_release(hpt_ctx *ctx, uint64_t req_id)
{
    g_err.clear();
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    std::lock_guard<std::mutex> lk(ctx->smu);
    auto r = find_req(ctx, req_id);
    if (!r) return fail(HPT_ERR_NOT_FOUND, "unknown request %llu", (unsigned long long)req_id);
    if (!r->done) return fail(HPT_ERR_BUSY, "request %llu not done (cancel it first)", (unsigned long long)req_id);
    if (r->out_lib) CUDA_TRY(cudaFreeAsync(r->out_lib, ctx->ostream));
    r->out_lib = nullptr;
    ctx->reqs.erase(req_id);
    ctx->scv.notify_all();
    return HPT_OK;
}

// ------------------------------------------------------------ accessors for hpt_static.cu
namespace hpt {
hpt_status internal_make_job(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc, void *out, size_t out_bytes,
                             DevJob &J)
{
    hpt_status st = check_ctx(ctx);
    if (st) return st;
    return make_job(ctx, scene_id, desc, out, out_bytes, J, nullptr);
}
int internal_ctx_device(const hpt_ctx *ctx) { return ctx->device; }
void internal_grids(hpt_ctx *ctx, int prec, int &grid_trace, int &grid_shade)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    grid_trace = ctx->grid_trace[prec];
    grid_shade = ctx->grid_shade[prec];
}
hpt_status internal_fail(hpt_status st, const char *msg) { return fail(st, "%s", msg); }
hpt_status internal_check(hpt_ctx *ctx)
{
    g_err.clear();
    return check_ctx(ctx);
}
}  // namespace hpt
