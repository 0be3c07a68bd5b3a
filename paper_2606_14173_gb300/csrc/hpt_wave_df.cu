// Wavefront kernels instantiated for the coherent arithmetic 'df'.
#include "hpt_wave_inst.cuh"

namespace hpt {
cudaError_t wave_gen_df(const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr, cudaStream_t s)
{
    return WaveLaunch<df>::gen(jt, wd, pb, scr, s);
}
cudaError_t wave_trace_df(bool st, const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr, int it,
                          int grid, cudaStream_t s)
{
    return WaveLaunch<df>::trace(st, jt, wd, pb, scr, it, grid, s);
}
cudaError_t wave_shade_df(bool st, const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr, int it,
                          int grid, cudaStream_t s)
{
    return WaveLaunch<df>::shade(st, jt, wd, pb, scr, it, grid, s);
}
cudaError_t wave_accum_df(const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr, cudaStream_t s)
{
    return WaveLaunch<df>::accum(jt, wd, pb, scr, s);
}
int wave_occupancy_df(int which) { return WaveLaunch<df>::occupancy(which); }
cudaError_t wave_preload_df() { return WaveLaunch<df>::preload(); }
}  // namespace hpt
