// Instantiation of the trace kernel: coherent arithmetic df, counters false.
#include "hpt_trace.cuh"

namespace hpt {
const void *kernel_df() { return (const void *)trace_kernel<df, false>; }
void launch_df(const JobTable *t, SlotScratch *s, int grid, cudaStream_t st)
{
    trace_kernel<df, false><<<grid, BLOCK, 0, st>>>(t, s);
}
}  // namespace hpt
