// Wavefront kernels instantiated for the coherent arithmetic 'double'.
#include "hpt_wave_inst.cuh"

namespace hpt {
cudaError_t wave_gen_f64(const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr, cudaStream_t s)
{
    return WaveLaunch<double>::gen(jt, wd, pb, scr, s);
}
cudaError_t wave_trace_f64(bool st, const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr, int it,
                          int grid, cudaStream_t s)
{
    return WaveLaunch<double>::trace(st, jt, wd, pb, scr, it, grid, s);
}
cudaError_t wave_shade_f64(bool st, const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr, int it,
                          int grid, cudaStream_t s)
{
    return WaveLaunch<double>::shade(st, jt, wd, pb, scr, it, grid, s);
}
cudaError_t wave_accum_f64(const JobTable *jt, const WaveDesc &wd, const PathBufs &pb, SlotScratch *scr, cudaStream_t s)
{
    return WaveLaunch<double>::accum(jt, wd, pb, scr, s);
}
int wave_occupancy_f64(int which) { return WaveLaunch<double>::occupancy(which); }
cudaError_t wave_preload_f64() { return WaveLaunch<double>::preload(); }
}  // namespace hpt
