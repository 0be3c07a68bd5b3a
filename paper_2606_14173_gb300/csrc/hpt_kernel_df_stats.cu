// Instantiation of the trace kernel: coherent arithmetic df, counters true.
#include "hpt_trace.cuh"

namespace hpt {
const void *kernel_df_stats() { return (const void *)trace_kernel<df, true>; }
void launch_df_stats(const JobTable *t, SlotScratch *s, int grid, cudaStream_t st)
{
    trace_kernel<df, true><<<grid, BLOCK, 0, st>>>(t, s);
}
}  // namespace hpt
