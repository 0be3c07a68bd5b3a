// Throughput probes of this GPU: FP32 and FP64 fused multiply-add rates and the L2 read
// bandwidth, each timed with CUDA events.  They give the measured denominators of the
// ALU-bound roofline next to the peak derived from the unit counts and clocks.
#include <algorithm>
#include <cstdio>

#include <cuda_runtime.h>

#include "hpt.h"

namespace hpt {
int internal_ctx_device(const hpt_ctx *);
hpt_status internal_fail(hpt_status st, const char *msg);
hpt_status internal_check(hpt_ctx *ctx);
}  // namespace hpt

using namespace hpt;

namespace {

// eight independent FMA chains per thread; 'n' runtime iterations
template <class T>
__global__ void k_fma(T *out, int n, T a, T b)
{
    T x0 = (T)threadIdx.x, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3, x4 = x0 + (T)4, x5 = x0 + (T)5,
      x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int i = 0; i < n; ++i) {
        x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
        x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
    const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == (T)-12345.678) out[blockIdx.x] = s;   // keeps the chains alive, never true in practice
}

// every thread reads float4s of an L2-resident buffer 'reps' times
__global__ void k_l2(const float4 *__restrict__ buf, size_t n4, int reps, float *out)
{
    float acc = 0.0f;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc += v.x + v.y + v.z + v.w;
        }
    if (acc == -12345.678f) out[0] = acc;
}

}  // namespace

#define PROBE_TRY(x)                                                                               \
    do {                                                                                           \
        cudaError_t e_ = (x);                                                                      \
        if (e_ != cudaSuccess) {                                                                   \
            char m_[256];                                                                          \
            snprintf(m_, sizeof m_, "%s: %s", #x, cudaGetErrorString(e_));                         \
            return internal_fail(HPT_ERR_CUDA, m_);                                                \
        }                                                                                          \
    } while (0)

extern "C" hpt_status hpt_probe_peaks(hpt_ctx *ctx, double peaks[HPT_NPEAKS])
{
    hpt_status st = internal_check(ctx);
    if (st) return st;
    if (!peaks) return internal_fail(HPT_ERR_INVALID_ARG, "peaks is NULL");
    PROBE_TRY(cudaSetDevice(internal_ctx_device(ctx)));
    int dev = 0, sms = 0;
    PROBE_TRY(cudaGetDevice(&dev));
    PROBE_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s;
    PROBE_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    PROBE_TRY(cudaEventCreate(&e0));
    PROBE_TRY(cudaEventCreate(&e1));
    const size_t l2_bytes = 64ull << 20;
    void *buf = nullptr;
    PROBE_TRY(cudaMalloc(&buf, l2_bytes + 4096));
    PROBE_TRY(cudaMemsetAsync(buf, 0, l2_bytes + 4096, s));
    float ms = 0.0f;
    const int blocks = sms * 8, threads = 256;
    // FP32: 8 chains x 2 flops x n per thread
    const int n32 = 1 << 16;
    k_fma<float><<<blocks, threads, 0, s>>>((float *)buf, 256, 0.999f, 1e-3f);   // warm-up
    PROBE_TRY(cudaEventRecord(e0, s));
    k_fma<float><<<blocks, threads, 0, s>>>((float *)buf, n32, 0.999f, 1e-3f);
    PROBE_TRY(cudaEventRecord(e1, s));
    PROBE_TRY(cudaEventSynchronize(e1));
    PROBE_TRY(cudaEventElapsedTime(&ms, e0, e1));
    peaks[0] = 16.0 * n32 * (double)blocks * threads / (ms * 1e-3) / 1e12;
    // FP64
    const int n64 = 1 << 11;
    k_fma<double><<<blocks, threads, 0, s>>>((double *)buf, 16, 0.999, 1e-3);
    PROBE_TRY(cudaEventRecord(e0, s));
    k_fma<double><<<blocks, threads, 0, s>>>((double *)buf, n64, 0.999, 1e-3);
    PROBE_TRY(cudaEventRecord(e1, s));
    PROBE_TRY(cudaEventSynchronize(e1));
    PROBE_TRY(cudaEventElapsedTime(&ms, e0, e1));
    peaks[1] = 16.0 * n64 * (double)blocks * threads / (ms * 1e-3) / 1e12;
    // L2 read bandwidth over a 64 MiB buffer (below the 129 MB L2)
    const int reps = 100;
    const size_t n4 = l2_bytes / sizeof(float4);
    k_l2<<<blocks, threads, 0, s>>>((const float4 *)buf, n4, 2, (float *)((char *)buf + l2_bytes));
    PROBE_TRY(cudaEventRecord(e0, s));
    k_l2<<<blocks, threads, 0, s>>>((const float4 *)buf, n4, reps, (float *)((char *)buf + l2_bytes));
    PROBE_TRY(cudaEventRecord(e1, s));
    PROBE_TRY(cudaEventSynchronize(e1));
    PROBE_TRY(cudaEventElapsedTime(&ms, e0, e1));
    peaks[2] = (double)reps * l2_bytes / (ms * 1e-3) / 1e9;
    peaks[3] = sms;
    PROBE_TRY(cudaGetLastError());
    cudaFree(buf);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    return HPT_OK;
}
