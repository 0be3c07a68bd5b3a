// Instantiation of the trace kernel: coherent arithmetic double, counters false.
#include "hpt_trace.cuh"

namespace hpt {
const void *kernel_f64() { return (const void *)trace_kernel<double, false>; }
void launch_f64(const JobTable *t, SlotScratch *s, int grid, cudaStream_t st)
{
    trace_kernel<double, false><<<grid, BLOCK, 0, st>>>(t, s);
}
}  // namespace hpt
