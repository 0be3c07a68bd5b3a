// Instantiation of the trace kernel: coherent arithmetic double, counters true.
#include "hpt_trace.cuh"

namespace hpt {
const void *kernel_f64_stats() { return (const void *)trace_kernel<double, true>; }
void launch_f64_stats(const JobTable *t, SlotScratch *s, int grid, cudaStream_t st)
{
    trace_kernel<double, true><<<grid, BLOCK, 0, st>>>(t, s);
}
}  // namespace hpt
