// Host-side launchers of the wavefront kernels for one coherent arithmetic R.
#pragma once
#include <algorithm>
#include <atomic>

#include "hpt_wave.cuh"

namespace hpt {

template <class R> struct WaveLaunch {
    static cudaError_t gen(const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr, cudaStream_t s)
    {
        const int g = (wd.n_paths + GEN_BLOCK - 1) / GEN_BLOCK;
        if (g > 0) k_gen<R><<<g, GEN_BLOCK, 0, s>>>(jt, wd, pb, scr);
        return cudaGetLastError();
    }
    // the coherent-ray kernel and the incoherent / shadow-ray kernel of one iteration; 'grid' is
    // sized for the first, the second gets the same multiple of its own resident blocks per SM
    static cudaError_t trace(bool stats, const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr,
                             int it, int grid, cudaStream_t s)
    {
        static const int occ_c = resident(k_trace<R, false, true>), occ_i = resident(k_trace<R, false, false>);
        const int grid_i = std::max(1, (int)((long long)grid * occ_i / std::max(occ_c, 1)));
        const size_t smem = stack_bytes(wd.stack_n);
        carve_for(wd.stack_n);
        if (stats) {
            k_trace<R, true, true><<<grid, TRACE_BLOCK, smem, s>>>(jt, wd, pb, scr, it);
            k_trace<R, true, false><<<grid_i, TRACE_BLOCK, smem, s>>>(jt, wd, pb, scr, it);
        } else {
            k_trace<R, false, true><<<grid, TRACE_BLOCK, smem, s>>>(jt, wd, pb, scr, it);
            k_trace<R, false, false><<<grid_i, TRACE_BLOCK, smem, s>>>(jt, wd, pb, scr, it);
        }
        return cudaGetLastError();
    }
    static size_t stack_bytes(int entries) { return (size_t)entries * TRACE_BLOCK * sizeof(int); }
    // blocks per SM the trace kernels can keep resident with the deepest stack
    template <class F> static int resident(F f)
    {
        int nb = 0;
        return (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, TRACE_BLOCK, stack_bytes(TSTACK)) == cudaSuccess &&
                nb > 0)
                   ? nb
                   : 1;
    }
    // the trace kernels ask for no more shared memory than their traversal stacks need, leaving
    // the rest of the SM's on-chip memory to the L1 cache that holds the BVH (set again whenever
    // the stack depth of a launch differs from the last one)
    static void carve_for(int entries)
    {
        static std::atomic<int> last{-1};
        if (last.exchange(entries) == entries) return;
        int dev = 0, smem_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        auto carve = [&](auto f, int minb) {
            const int need = minb * ((int)stack_bytes(entries) + 1024);
            const int pct = smem_sm > 0 ? std::min(100, (need * 100 + smem_sm - 1) / smem_sm) : 100;
            cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
        };
        carve(k_trace<R, false, true>, HPT_TRACE_MINB);
        carve(k_trace<R, true, true>, HPT_TRACE_MINB);
        carve(k_trace<R, false, false>, HPT_TRACE_INC_MINB);
        carve(k_trace<R, true, false>, HPT_TRACE_INC_MINB);
    }
    static cudaError_t shade(bool stats, const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr,
                             int it, int grid, cudaStream_t s)
    {
        if (stats) {
            k_shade<R, true, true><<<grid, SHADE_BLOCK, 0, s>>>(jt, wd, pb, scr, it);
            k_shade<R, true, false><<<grid, SHADE_BLOCK, 0, s>>>(jt, wd, pb, scr, it);
        } else {
            k_shade<R, false, true><<<grid, SHADE_BLOCK, 0, s>>>(jt, wd, pb, scr, it);
            k_shade<R, false, false><<<grid, SHADE_BLOCK, 0, s>>>(jt, wd, pb, scr, it);
        }
        return cudaGetLastError();
    }
    static cudaError_t accum(const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr, cudaStream_t s)
    {
        const int g = (wd.n_items + ACCUM_BLOCK - 1) / ACCUM_BLOCK;
        if (g > 0) k_accum<R><<<g, ACCUM_BLOCK, 0, s>>>(jt, wd, pb, scr);
        return cudaGetLastError();
    }
    // load every kernel of this arithmetic now (with lazy module loading a kernel is otherwise
    // loaded, and its code placed in device memory, at its first launch)
    static cudaError_t preload()
    {
        cudaFuncAttributes a;
        cudaError_t e = cudaFuncGetAttributes(&a, k_gen<R>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_trace<R, false, true>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_trace<R, false, false>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_trace<R, true, true>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_trace<R, true, false>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_shade<R, false, true>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_shade<R, false, false>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_shade<R, true, true>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_shade<R, true, false>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_accum<R>);
        return e;
    }
    // resident blocks per SM of the trace (0) and shade (1) kernels; the trace kernel asks for
    // no more shared memory than its traversal stacks need, leaving the rest of the SM's on-chip
    // memory to the L1 cache that holds the BVH
    static int occupancy(int which)
    {
        if (which == 0) {
            carve_for(TSTACK);
            return resident(k_trace<R, false, true>);
        }
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shade<R, false, true>, SHADE_BLOCK, 0);
        return (e == cudaSuccess && nb > 0) ? nb : 1;
    }
};

}  // namespace hpt
