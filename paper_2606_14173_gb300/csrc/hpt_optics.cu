// Wave optics around the tracer: the band-limited Gaussian random field phase maps of Eq. 4
// (hpt_grf_build) and the angular spectrum method of the two-stage scheme (hpt_asm_propagate).
//
// Both rest on one 2-D FFT of power-of-two sizes: every row transformed in shared memory by
// one block (radix-2 decimation in time, bit-reversed load), a tiled transpose, the rows
// again, and the transpose back.  The data are complex64; the twiddle factors are rounded
// from double-precision values.  The transfer function's phase 2 pi z sqrt(1/lambda^2 - f^2),
// ~1e5 turns, is formed in double before its fraction is taken.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include <cuda_runtime.h>

#include "hpt.h"
#include "hpt_device.cuh"

namespace hpt {
int internal_ctx_device(const hpt_ctx *);
hpt_status internal_fail(hpt_status st, const char *msg);
hpt_status internal_check(hpt_ctx *ctx);
}  // namespace hpt

using namespace hpt;

namespace {

constexpr int FFT_MAX_LOG = 13;          // 8192 points: 64 KB of shared memory per row
constexpr int FFT_THREADS = 512;
constexpr unsigned GRF_TAG = 0x47524600u;

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// tw[k] = exp(-2 pi i k / n), k < n / 2
__global__ void k_twiddles(float2 *tw, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n / 2) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)n, &s, &c);
    tw[k] = make_float2((float)c, (float)s);
}

// In-place FFT of 'rows' consecutive rows of n = 2^logn points.  sign = -1: forward
// (exp(-2 pi i k j / n)), +1: inverse without the 1/n; the result is multiplied by 'scale'.
__global__ void __launch_bounds__(FFT_THREADS) k_fft_rows(float2 *data, int logn, int rows, float sign,
                                                          const float2 *__restrict__ tw, float scale)
{
    extern __shared__ float2 sm[];
    const int n = 1 << logn;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        float2 *d = data + (size_t)row * n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) sm[__brev((unsigned)i) >> (32 - logn)] = d[i];
        __syncthreads();
        for (int s = 1; s <= logn; ++s) {
            const int half = 1 << (s - 1), tstride = n >> s;
            for (int j = threadIdx.x; j < n / 2; j += blockDim.x) {
                const int pos = j & (half - 1);
                const int i0 = ((j >> (s - 1)) << s) + pos, i1 = i0 + half;
                float2 w = __ldg(tw + pos * tstride);
                w.y *= -sign;
                const float2 a = sm[i0], t = cmul(w, sm[i1]);
                sm[i0] = make_float2(a.x + t.x, a.y + t.y);
                sm[i1] = make_float2(a.x - t.x, a.y - t.y);
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const float2 v = sm[i];
            d[i] = make_float2(v.x * scale, v.y * scale);
        }
        __syncthreads();
    }
}

// out[x][y] = in[y][x], in is h x w
__global__ void k_transpose(const float2 *__restrict__ in, float2 *__restrict__ out, int w, int h)
{
    __shared__ float2 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int x = bx + threadIdx.x, y = by + k;
        if (x < w && y < h) tile[k][threadIdx.x] = in[(size_t)y * w + x];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int x = by + threadIdx.x, y = bx + k;
        if (x < h && y < w) out[(size_t)y * h + x] = tile[threadIdx.x][k];
    }
}

// Eq. 4: exp(i xi_m) on the circular passband, 0 elsewhere; [ny][nx] in FFT order
__global__ void k_grf_spectrum(float2 *spec, int nx, int ny, unsigned m, unsigned seed_lo, unsigned seed_hi)
{
    const size_t n = (size_t)nx * ny;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nx), iy = (int)(i / nx);
        const long long kx = ix < nx / 2 ? ix : ix - nx, ky = iy < ny / 2 ? iy : iy - ny;
        const long long NX = nx, NY = ny;
        float2 v = make_float2(0.0f, 0.0f);
        if (4 * (kx * kx * NY * NY + ky * ky * NX * NX) <= NX * NX * NY * NY) {
            const uint4 o = philox(make_uint4((unsigned)ix, (unsigned)iy, m, GRF_TAG), seed_lo, seed_hi);
            float s, c;
            sincospif(2.0f * u24(o.x), &s, &c);
            v = make_float2(c, s);
        }
        spec[i] = v;
    }
}

__global__ void k_arg(const float2 *__restrict__ r, float *__restrict__ phi, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 v = r[i];
        phi[i] = atan2f(v.y, v.x);
    }
}

// exp(i 2 pi z sqrt(1/lambda^2 - fx^2 - fy^2)) on the padded grid (FFT order), times 'scale'
__global__ void k_transfer(float2 *Hf, int Wp, int Hp, double pitch, double lambda, double z, float scale)
{
    const size_t n = (size_t)Wp * Hp;
    const double il2 = 1.0 / (lambda * lambda);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % Wp), iy = (int)(i / Wp);
        const double fx = (double)(ix < Wp / 2 ? ix : ix - Wp) / (Wp * pitch);
        const double fy = (double)(iy < Hp / 2 ? iy : iy - Hp) / (Hp * pitch);
        const double a = il2 - fx * fx - fy * fy;
        float2 v = make_float2(0.0f, 0.0f);
        if (a > 0.0) {
            const double turns = z * sqrt(a);
            const float f = (float)(turns - floor(turns));
            float s, c;
            sincospif(2.0f * f, &s, &c);
            v = make_float2(c * scale, s * scale);
        }
        Hf[i] = v;
    }
}

__global__ void k_pad(const float2 *__restrict__ in, float2 *__restrict__ P, int W, int H, int Wp, int Hp, int ox, int oy)
{
    const size_t n = (size_t)Wp * Hp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % Wp) - ox, y = (int)(i / Wp) - oy;
        P[i] = (x >= 0 && x < W && y >= 0 && y < H) ? in[(size_t)y * W + x] : make_float2(0.0f, 0.0f);
    }
}

__global__ void k_mul(float2 *__restrict__ P, const float2 *__restrict__ Hf, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        P[i] = cmul(P[i], Hf[i]);
}

__global__ void k_crop(const float2 *__restrict__ P, float2 *__restrict__ out, int W, int H, int Wp, int ox, int oy)
{
    const size_t n = (size_t)W * H;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % W), y = (int)(i / W);
        out[i] = P[(size_t)(y + oy) * Wp + x + ox];
    }
}

int ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

bool pow2_in_range(int n) { return n >= 2 && n <= (1 << FFT_MAX_LOG) && (n & (n - 1)) == 0; }

int grid_for(size_t n)
{
    return (int)std::min<size_t>((n + 255) / 256, 152 * 32);
}

// 2-D FFT of A [ny][nx] in place, B as scratch of the same size
cudaError_t fft2d(float2 *A, float2 *B, int nx, int ny, const float2 *twx, const float2 *twy, float sign, float scale,
                  cudaStream_t s)
{
    const int lx = ilog2(nx), ly = ilog2(ny);
    const dim3 tb(32, 8);
    k_fft_rows<<<std::min(ny, 152 * 8), std::min(FFT_THREADS, std::max(32, nx / 2)), sizeof(float2) * nx, s>>>(
        A, lx, ny, sign, twx, 1.0f);
    k_transpose<<<dim3((nx + 31) / 32, (ny + 31) / 32), tb, 0, s>>>(A, B, nx, ny);
    k_fft_rows<<<std::min(nx, 152 * 8), std::min(FFT_THREADS, std::max(32, ny / 2)), sizeof(float2) * ny, s>>>(
        B, ly, nx, sign, twy, scale);
    k_transpose<<<dim3((ny + 31) / 32, (nx + 31) / 32), tb, 0, s>>>(B, A, ny, nx);
    return cudaGetLastError();
}

cudaError_t fft_setup()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(float2) << FFT_MAX_LOG);
    if (e == cudaSuccess) done = true;
    return e;
}

}  // namespace

#define OPT_TRY(x)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (x);                                                                      \
        if (e_ != cudaSuccess) {                                                                   \
            char m_[256];                                                                          \
            snprintf(m_, sizeof m_, "%s: %s", #x, cudaGetErrorString(e_));                         \
            return internal_fail(HPT_ERR_CUDA, m_);                                                \
        }                                                                                          \
    } while (0)

extern "C" hpt_status hpt_grf_build(hpt_ctx *ctx, uint64_t phase_seed, int32_t hologram_offset, int32_t K, int32_t nx,
                                    int32_t ny, double pitch, float *phi_dev, void *stream)
{
    hpt_status st = internal_check(ctx);
    if (st) return st;
    if (!phi_dev) return internal_fail(HPT_ERR_INVALID_ARG, "phi_dev is NULL");
    if (K < 1 || hologram_offset < 0) return internal_fail(HPT_ERR_INVALID_ARG, "K must be >= 1, hologram_offset >= 0");
    if (!pow2_in_range(nx) || !pow2_in_range(ny))
        return internal_fail(HPT_ERR_INVALID_ARG, "nx and ny must be powers of two in 2 .. 8192");
    if (!(pitch > 0.0)) return internal_fail(HPT_ERR_INVALID_ARG, "pitch must be > 0");
    OPT_TRY(cudaSetDevice(internal_ctx_device(ctx)));
    OPT_TRY(fft_setup());
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)nx * ny;
    char *buf = nullptr;
    const size_t bytes = 2 * n * sizeof(float2) + (size_t)(nx / 2 + ny / 2) * sizeof(float2);
    OPT_TRY(cudaMallocAsync((void **)&buf, bytes, s));
    float2 *A = (float2 *)buf, *B = A + n, *twx = B + n, *twy = twx + nx / 2;
    cudaError_t e = cudaSuccess;
    k_twiddles<<<(nx / 2 + 255) / 256, 256, 0, s>>>(twx, nx);
    k_twiddles<<<(ny / 2 + 255) / 256, 256, 0, s>>>(twy, ny);
    for (int k = 0; k < K && e == cudaSuccess; ++k) {
        k_grf_spectrum<<<grid_for(n), 256, 0, s>>>(A, nx, ny, (unsigned)(hologram_offset + k), (unsigned)phase_seed,
                                                   (unsigned)(phase_seed >> 32));
        e = fft2d(A, B, nx, ny, twx, twy, +1.0f, 1.0f, s);
        if (e == cudaSuccess) {
            k_arg<<<grid_for(n), 256, 0, s>>>(A, phi_dev + (size_t)k * n, n);
            e = cudaGetLastError();
        }
    }
    cudaError_t e2 = cudaFreeAsync(buf, s);
    OPT_TRY(e);
    OPT_TRY(e2);
    return HPT_OK;
}

extern "C" hpt_status hpt_asm_propagate(hpt_ctx *ctx, const void *in_dev, void *out_dev, int32_t W, int32_t H,
                                        int32_t n_lambda, int32_t K, const double *lambdas, double pitch, double z,
                                        void *stream)
{
    hpt_status st = internal_check(ctx);
    if (st) return st;
    if (!in_dev || !out_dev || !lambdas) return internal_fail(HPT_ERR_INVALID_ARG, "in_dev, out_dev or lambdas is NULL");
    if (W < 1 || H < 1 || n_lambda < 1 || n_lambda > 3 || K < 1)
        return internal_fail(HPT_ERR_INVALID_ARG, "need W, H, K >= 1 and 1 <= n_lambda <= 3");
    int Wp = 1, Hp = 1;
    while (Wp < 2 * W) Wp <<= 1;
    while (Hp < 2 * H) Hp <<= 1;
    if (!pow2_in_range(Wp) || !pow2_in_range(Hp))
        return internal_fail(HPT_ERR_UNSUPPORTED, "padded size above 8192 x 8192 (W, H <= 4096)");
    if (!(pitch > 0.0)) return internal_fail(HPT_ERR_INVALID_ARG, "pitch must be > 0");
    for (int l = 0; l < n_lambda; ++l)
        if (!(lambdas[l] > 0.0)) return internal_fail(HPT_ERR_INVALID_ARG, "wavelengths must be > 0");
    OPT_TRY(cudaSetDevice(internal_ctx_device(ctx)));
    OPT_TRY(fft_setup());
    cudaStream_t s = (cudaStream_t)stream;
    const size_t np = (size_t)Wp * Hp;
    const size_t bytes = (2 + (size_t)n_lambda) * np * sizeof(float2) + (size_t)(Wp / 2 + Hp / 2) * sizeof(float2);
    char *buf = nullptr;
    OPT_TRY(cudaMallocAsync((void **)&buf, bytes, s));
    float2 *A = (float2 *)buf, *B = A + np, *Hf = B + np, *twx = Hf + (size_t)n_lambda * np, *twy = twx + Wp / 2;
    const int ox = (Wp - W) / 2, oy = (Hp - H) / 2;
    cudaError_t e = cudaSuccess;
    k_twiddles<<<(Wp / 2 + 255) / 256, 256, 0, s>>>(twx, Wp);
    k_twiddles<<<(Hp / 2 + 255) / 256, 256, 0, s>>>(twy, Hp);
    for (int l = 0; l < n_lambda; ++l)
        k_transfer<<<grid_for(np), 256, 0, s>>>(Hf + (size_t)l * np, Wp, Hp, pitch, lambdas[l], z, 1.0f / (float)np);
    const float2 *in = (const float2 *)in_dev;
    float2 *out = (float2 *)out_dev;
    for (int f = 0; f < n_lambda * K && e == cudaSuccess; ++f) {
        const size_t fo = (size_t)f * W * H;
        k_pad<<<grid_for(np), 256, 0, s>>>(in + fo, A, W, H, Wp, Hp, ox, oy);
        e = fft2d(A, B, Wp, Hp, twx, twy, -1.0f, 1.0f, s);
        if (e != cudaSuccess) break;
        k_mul<<<grid_for(np), 256, 0, s>>>(A, Hf + (size_t)(f / K) * np, np);
        e = fft2d(A, B, Wp, Hp, twx, twy, +1.0f, 1.0f, s);
        if (e != cudaSuccess) break;
        k_crop<<<grid_for((size_t)W * H), 256, 0, s>>>(A, out + fo, W, H, Wp, ox, oy);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(buf, s);
    OPT_TRY(e);
    OPT_TRY(e2);
    return HPT_OK;
}
