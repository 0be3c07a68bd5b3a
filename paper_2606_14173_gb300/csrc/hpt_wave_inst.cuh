// Host-side launchers of the wavefront kernels for one coherent arithmetic R.
#pragma once
#include <algorithm>

#include "hpt_wave.cuh"

namespace hpt {

template <class R> struct WaveLaunch {
    static cudaError_t gen(const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr, cudaStream_t s)
    {
        const int g = (wd.n_paths + GEN_BLOCK - 1) / GEN_BLOCK;
        if (g > 0) k_gen<R><<<g, GEN_BLOCK, 0, s>>>(jt, wd, pb, scr);
        return cudaGetLastError();
    }
    static cudaError_t trace(bool stats, const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr,
                             int it, int grid, cudaStream_t s)
    {
        if (stats) k_trace<R, true><<<grid, TRACE_BLOCK, 0, s>>>(jt, wd, pb, scr, it);
        else k_trace<R, false><<<grid, TRACE_BLOCK, 0, s>>>(jt, wd, pb, scr, it);
        return cudaGetLastError();
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
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_trace<R, false>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_trace<R, true>);
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
            int dev = 0, smem_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            const int need = HPT_TRACE_MINB * (TSTACK * TRACE_BLOCK * 4 + 1024);
            const int pct = smem_sm > 0 ? std::min(100, (need * 100 + smem_sm - 1) / smem_sm) : 100;
            cudaFuncSetAttribute(k_trace<R, false>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
            cudaFuncSetAttribute(k_trace<R, true>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
        }
        int nb = 0;
        cudaError_t e = which == 0
                            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_trace<R, false>, TRACE_BLOCK, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_shade<R, false, true>, SHADE_BLOCK, 0);
        return (e == cudaSuccess && nb > 0) ? nb : 1;
    }
};

}  // namespace hpt
