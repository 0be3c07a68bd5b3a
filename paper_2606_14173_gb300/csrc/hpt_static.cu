// hpt_trace_fixed_scratch: the trace of hpt_trace with all of its scratch memory (wave path
// state, ray queues, queue counters, the job table) carved out of one fixed device array that
// exists for the lifetime of the process, so that the call itself allocates nothing.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "hpt.h"
#include "hpt_internal.h"

namespace hpt {
cudaError_t wave_gen(int prec, const JobTable *, const WaveDesc &, const PathBufs &, SlotScratch *, cudaStream_t);
cudaError_t wave_trace(int prec, bool stats, const JobTable *, const WaveDesc &, const PathBufs &, SlotScratch *, int it,
                       int grid, cudaStream_t);
cudaError_t wave_shade(int prec, bool stats, const JobTable *, const WaveDesc &, const PathBufs &, SlotScratch *, int it,
                       int grid, cudaStream_t);
cudaError_t wave_accum(int prec, const JobTable *, const WaveDesc &, const PathBufs &, SlotScratch *, cudaStream_t);
hpt_status internal_make_job(hpt_ctx *, uint64_t, const hpt_render_desc *, void *, size_t, DevJob &);
int internal_ctx_device(const hpt_ctx *);
void internal_grids(hpt_ctx *, int prec, int &grid_trace, int &grid_shade);
hpt_status internal_fail(hpt_status st, const char *msg);
hpt_status internal_check(hpt_ctx *ctx);
}  // namespace hpt

using namespace hpt;

// The fixed scratch: HPT_FIXED_SCRATCH_BYTES (64 MiB) on every device where this module is loaded
// (hpt_create loads it on the context's device), held until the process exits.  Host code must not
// use this name as a device address: it takes the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_fixed_scratch[HPT_FIXED_SCRATCH_BYTES];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;                          // serialises the host side of all calls
void *g_base[MAX_DEVICES] = {nullptr};    // device address of g_fixed_scratch, per device
cudaError_t g_setup_err[MAX_DEVICES] = {};  // why the set-up of a device failed (cudaSuccess: not tried or done)

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t PATH_BYTES = 7 * 8 + 3 * 4 + 4 + 6 * 4 + 3 * 16 + 16 + 4 + 3 * 4 + 3 * 4 + 6 * 4;
constexpr size_t HEAD_BYTES = ((sizeof(JobTable) + 255) & ~(size_t)255) + ((sizeof(SlotScratch) + 255) & ~(size_t)255);
// paths per wave that fit next to the job table and the counters (26 arrays, each 256-aligned)
constexpr int FIXED_CAPACITY = (int)(((HPT_FIXED_SCRATCH_BYTES - HEAD_BYTES - 26 * 256) / PATH_BYTES) & ~(size_t)255);

struct Layout {
    JobTable *table;
    SlotScratch *scr;
    PathBufs pb;
};

Layout carve(void *base)
{
    char *p = (char *)base;
    auto take = [&](size_t bytes) {
        void *r = p;
        p += round256(bytes);
        return r;
    };
    Layout L;
    L.table = (JobTable *)take(sizeof(JobTable));
    L.scr = (SlotScratch *)take(sizeof(SlotScratch));
    const size_t B = (size_t)FIXED_CAPACITY;
    PathBufs &b = L.pb;
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
    return L;
}
}  // namespace

static_assert(FIXED_CAPACITY >= 4096, "fixed scratch too small");

// The one-job table of a call, written on the device from a kernel parameter: the launch copies
// the parameter by value, so no host staging buffer is read after the call returns.
__global__ void k_put_job(JobTable *t, const DevJob job)
{
    t->n_jobs = 1;
    t->pad = 0;
    t->jobs[0] = job;
}

namespace hpt {
// Set-up of the fixed scratch on 'dev', called by hpt_create with that device current: looks up
// the array's device address (which loads this module and so places the array in device memory)
// and clears the status word once.  A failure is recorded and reported by the entry point only.
void fixed_scratch_setup(int dev)
{
    if (dev < 0 || dev >= MAX_DEVICES) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_base[dev]) return;
    void *ptr = nullptr;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_fixed_scratch);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_put_job);   // loaded now, not at a first call
    if (e == cudaSuccess) e = cudaMemset(&carve(ptr).scr->status, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        g_setup_err[dev] = e;
        cudaGetLastError();
        return;
    }
    g_base[dev] = ptr;
}

// The status bits the entry point's kernels left on 'dev' since the last read (then cleared);
// 0 when the array was never set up there.  Called by hpt_sync after the device synchronised.
cudaError_t fixed_scratch_status(int dev, unsigned *bits)
{
    *bits = 0;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaSuccess;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) return cudaSuccess;
    SlotScratch *scr = carve(g_base[dev]).scr;
    cudaError_t e = cudaMemcpy(bits, &scr->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && *bits) e = cudaMemset(&scr->status, 0, sizeof(unsigned));
    return e;
}
}  // namespace hpt

#define FS_TRY(call)                                                                              \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            char m_[256];                                                                         \
            snprintf(m_, sizeof m_, "%s: %s", #call, cudaGetErrorString(e_));                     \
            return internal_fail(HPT_ERR_CUDA, m_);                                               \
        }                                                                                         \
    } while (0)

extern "C" hpt_status hpt_trace_fixed_scratch(hpt_ctx *ctx, uint64_t scene_id, const hpt_render_desc *desc,
                                              void *out_dev, size_t out_bytes, void *cuda_stream)
{
    hpt_status st = internal_check(ctx);   // clears the thread's last error, sets the device
    if (st) return st;
    if (!out_dev) return internal_fail(HPT_ERR_INVALID_ARG, "out_dev is NULL");
    DevJob J;
    st = internal_make_job(ctx, scene_id, desc, out_dev, out_bytes, J);
    if (st) return st;
    if (J.spp > FIXED_CAPACITY) {
        char m[160];
        snprintf(m, sizeof m, "spp %d exceeds the fixed scratch: at most %d samples per pixel", J.spp, FIXED_CAPACITY);
        return internal_fail(HPT_ERR_INVALID_ARG, m);
    }
    const int dev = internal_ctx_device(ctx);
    if (dev < 0 || dev >= MAX_DEVICES) return internal_fail(HPT_ERR_UNSUPPORTED, "device index out of range");
    int grid_trace = 1, grid_shade = 1;
    const int prec = desc->precision;
    internal_grids(ctx, prec, grid_trace, grid_shade);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
        char m[200];
        snprintf(m, sizeof m, "the fixed scratch array is not available on device %d: %s", dev,
                 g_setup_err[dev] != cudaSuccess ? cudaGetErrorString(g_setup_err[dev]) : "not set up");
        return internal_fail(HPT_ERR_UNSUPPORTED, m);
    }
    const Layout L = carve(g_base[dev]);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    k_put_job<<<1, 1, 0, s>>>(L.table, J);
    FS_TRY(cudaGetLastError());
    // the array keeps the previous call's contents: the queue counters are cleared before every
    // wave; the status word is sticky until hpt_sync reads it
    const int n_iter = J.max_depth + 1;
    long long c = 0;
    while (c < J.n_items) {
        WaveDesc wd;
        memset(&wd, 0, sizeof wd);
        const int take = (int)std::min<long long>(J.n_items - c, FIXED_CAPACITY / J.spp);
        wd.n_seg = 1;
        wd.seg[0].job = 0;
        wd.seg[0].spp = J.spp;
        wd.seg[0].item_begin = c;
        wd.seg[0].item_count = take;
        wd.seg[0].path_offset = 0;
        wd.n_paths = take * J.spp;
        wd.n_items = take;
        wd.stack_n = scene_stack_entries(J.sc);
        FS_TRY(cudaMemsetAsync(L.scr->qcount, 0, sizeof(int) * 3 * (n_iter + 1), s));
        FS_TRY(wave_gen(prec, L.table, wd, L.pb, L.scr, s));
        for (int it = 0; it < n_iter; ++it) {
            FS_TRY(wave_trace(prec, false, L.table, wd, L.pb, L.scr, it, grid_trace, s));
            FS_TRY(wave_shade(prec, false, L.table, wd, L.pb, L.scr, it, grid_shade, s));
        }
        FS_TRY(wave_accum(prec, L.table, wd, L.pb, L.scr, s));
        c += take;
    }
    return HPT_OK;
}
