// Dispatch over the trace-kernel variants (one translation unit per variant).
#include <cuda_runtime.h>
#include "hpt_internal.h"

namespace hpt {
const void *kernel_f64();
const void *kernel_f64_stats();
const void *kernel_df();
const void *kernel_df_stats();
void launch_f64(const JobTable *, SlotScratch *, int, cudaStream_t);
void launch_f64_stats(const JobTable *, SlotScratch *, int, cudaStream_t);
void launch_df(const JobTable *, SlotScratch *, int, cudaStream_t);
void launch_df_stats(const JobTable *, SlotScratch *, int, cudaStream_t);

static const void *kernel_ptr(int prec, bool stats)
{
    if (prec == 0) return stats ? kernel_f64_stats() : kernel_f64();
    return stats ? kernel_df_stats() : kernel_df();
}

int trace_blocks_per_sm(int prec, bool stats)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_ptr(prec, stats), BLOCK, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_trace(int prec, bool stats, const JobTable *d_table, SlotScratch *d_scratch, int grid,
                         cudaStream_t s)
{
    if (prec == 0) {
        if (stats) launch_f64_stats(d_table, d_scratch, grid, s);
        else launch_f64(d_table, d_scratch, grid, s);
    } else {
        if (stats) launch_df_stats(d_table, d_scratch, grid, s);
        else launch_df(d_table, d_scratch, grid, s);
    }
    return cudaGetLastError();
}
}  // namespace hpt
