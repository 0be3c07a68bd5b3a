// Dispatch of the wavefront kernels over the two coherent arithmetics (FP64 = 0, DF32 = 1);
// each arithmetic lives in its own translation unit so that they compile in parallel.
#include <cuda_runtime.h>
#include "hpt_internal.h"

namespace hpt {
#define HPT_DECL(n)                                                                                              \
    cudaError_t wave_gen_##n(const JobTable *, const WaveDesc &, const PathBufs &, SlotScratch *, cudaStream_t);  \
    cudaError_t wave_trace_##n(bool, const JobTable *, const WaveDesc &, const PathBufs &, SlotScratch *, int, int, \
                               cudaStream_t);                                                                    \
    cudaError_t wave_shade_##n(bool, const JobTable *, const WaveDesc &, const PathBufs &, SlotScratch *, int, int, \
                               cudaStream_t);                                                                    \
    cudaError_t wave_accum_##n(const JobTable *, const WaveDesc &, const PathBufs &, SlotScratch *, cudaStream_t); \
    int wave_occupancy_##n(int);                                                                                 \
    cudaError_t wave_preload_##n();
HPT_DECL(f64)
HPT_DECL(df)
#undef HPT_DECL

cudaError_t wave_gen(int prec, const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr,
                     cudaStream_t s)
{
    return prec == 0 ? wave_gen_f64(jt, wd, pb, scr, s) : wave_gen_df(jt, wd, pb, scr, s);
}
cudaError_t wave_trace(int prec, bool st, const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr,
                       int it, int grid, cudaStream_t s)
{
    return prec == 0 ? wave_trace_f64(st, jt, wd, pb, scr, it, grid, s) : wave_trace_df(st, jt, wd, pb, scr, it, grid, s);
}
cudaError_t wave_shade(int prec, bool st, const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr,
                       int it, int grid, cudaStream_t s)
{
    return prec == 0 ? wave_shade_f64(st, jt, wd, pb, scr, it, grid, s) : wave_shade_df(st, jt, wd, pb, scr, it, grid, s);
}
cudaError_t wave_accum(int prec, const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr,
                       cudaStream_t s)
{
    return prec == 0 ? wave_accum_f64(jt, wd, pb, scr, s) : wave_accum_df(jt, wd, pb, scr, s);
}
int wave_occupancy(int prec, int which) { return prec == 0 ? wave_occupancy_f64(which) : wave_occupancy_df(which); }
cudaError_t wave_preload(int prec) { return prec == 0 ? wave_preload_f64() : wave_preload_df(); }
}  // namespace hpt
