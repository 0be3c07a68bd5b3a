// Wave optics around the tracer: the band-limited Gaussian random field phase maps of Eq. 4
// (hpt_grf_build) and the angular spectrum method of the two-stage scheme (hpt_asm_propagate).
//
// Both rest on one 2-D FFT of power-of-two sizes: every row transformed in shared memory by
// one block (Stockham autosort: radix-16 passes in registers, the remainder radix first, the
// first pass reading global memory and the last writing it in natural order, shared buffers
// in between), a tiled
// transpose, the rows again, and the transpose back.  The data are complex64; the twiddle factors are rounded
// from double-precision values.  The transfer function's phase 2 pi z sqrt(1/lambda^2 - f^2),
// ~1e5 turns, is formed in double before its fraction is taken.
#include <algorithm>
#include <cmath>
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

constexpr int FFT_MAX_LOG = 13;          // 8192 points: 2 (3 for the ASM pass) x 64 KB of shared memory
constexpr int FFT_THREADS = 512;
constexpr unsigned GRF_TAG = 0x47524600u;

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// tw[k] = exp(-2 pi i k / n), k < n
__global__ void k_twiddles(float2 *tw, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)n, &s, &c);
    tw[k] = make_float2((float)c, (float)s);
}

// exp(-2 pi i m / 16), m < 8: the constants of the in-register radix-16 DFT
__device__ __forceinline__ float2 w16(int m)
{
    const float c[8] = {1.0f, 0.923879533f, 0.707106781f, 0.382683432f, 0.0f, -0.382683432f, -0.707106781f, -0.923879533f};
    const float s[8] = {0.0f, 0.382683432f, 0.707106781f, 0.923879533f, 1.0f, 0.923879533f, 0.707106781f, 0.382683432f};
    return make_float2(c[m], -s[m]);
}

// R-point DFT of v in registers (R = 2, 4, 8, 16): bit-reversed order, then log2 R radix-2
// stages; sign = -1 forward, +1 inverse
template <int R>
__device__ __forceinline__ void dft_reg(float2 *v, float sign)
{
    constexpr int B = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
    float2 t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        int r = 0;
#pragma unroll
        for (int b = 0; b < B; ++b) r |= ((i >> b) & 1) << (B - 1 - b);
        t[r] = v[i];
    }
#pragma unroll
    for (int half = 1; half < R; half *= 2) {
#pragma unroll
        for (int g = 0; g < R; g += 2 * half) {
#pragma unroll
            for (int pos = 0; pos < half; ++pos) {
                float2 w = w16(pos * (8 / half));
                w.y *= -sign;
                const float2 a = t[g + pos], b = cmul(w, t[g + pos + half]);
                t[g + pos] = make_float2(a.x + b.x, a.y + b.y);
                t[g + pos + half] = make_float2(a.x - b.x, a.y - b.y);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = t[i];
}

// One Stockham pass of radix R over n points: element j of the pass reads x[j + r n/R]
// (r < R) through 'ld', multiplies it by exp(sign 2 pi i r (j mod Ns) / (Ns R)) (the n-point
// twiddle table), takes the R-point DFT and writes y[(j - j mod Ns) R + j mod Ns + r Ns]
// through 'st'.
template <int R, class LD, class ST>
__device__ __forceinline__ void stockham_pass(int n, int Ns, float sign, const float2 *__restrict__ tw, LD ld, ST st)
{
    const int q = n / R, tws = n / (Ns * R);
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        const int k = j & (Ns - 1);
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 a = ld(j + r * q);
            if (r > 0 && Ns > 1) {
                float2 w = __ldg(tw + r * k * tws);
                w.y *= -sign;
                a = cmul(a, w);
            }
            v[r] = a;
        }
        dft_reg<R>(v, sign);
        const int o = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) st(o + r * Ns, v[r]);
    }
}

template <class LD, class ST>
__device__ __forceinline__ void pass_any(int R, int n, int Ns, float sign, const float2 *tw, LD ld, ST st)
{
    switch (R) {
    case 2: stockham_pass<2>(n, Ns, sign, tw, ld, st); break;
    case 4: stockham_pass<4>(n, Ns, sign, tw, ld, st); break;
    case 8: stockham_pass<8>(n, Ns, sign, tw, ld, st); break;
    default: stockham_pass<16>(n, Ns, sign, tw, ld, st); break;
    }
}

// FFT of one row of n = 2^logn points: radix 16 passes (the remainder radix first), input
// through 'gld' (global memory or shared), output through 'gst', the passes in between in the
// shared buffers a and b.  The first pass reads gld, the last writes gst; a one-pass transform
// goes through a.  Ends with a barrier.
template <class LD, class ST>
__device__ __forceinline__ void row_fft(int logn, float sign, const float2 *tw, float2 *a, float2 *b, LD gld, ST gst)
{
    const int n = 1 << logn, rem = logn & 3;
    const int npass = (logn >> 2) + (rem ? 1 : 0);
    int Ns = 1;
    for (int p = 0; p < npass; ++p) {
        const int R = (p == 0 && rem) ? (1 << rem) : 16;
        float2 *dst = (p & 1) ? b : a;
        const float2 *src = (p & 1) ? a : b;
        const bool first = p == 0, last = p == npass - 1 && npass > 1;
        auto sld = [&](int i) { return src[i]; };
        auto sst = [&](int i, float2 v) { dst[i] = v; };
        if (first) pass_any(R, n, Ns, sign, tw, gld, sst);
        else if (last) pass_any(R, n, Ns, sign, tw, sld, gst);
        else pass_any(R, n, Ns, sign, tw, sld, sst);
        __syncthreads();
        Ns *= R;
    }
    if (npass == 1) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) gst(i, a[i]);
        __syncthreads();
    }
}

__host__ __device__ constexpr int fft_threads(int n) { return n / 16 > 32 ? (n / 16 < FFT_THREADS ? n / 16 : FFT_THREADS) : 32; }

// In-place FFT of 'rows' consecutive rows of n = 2^logn points, times 'scale'.
__global__ void __launch_bounds__(FFT_THREADS) k_fft_rows(float2 *data, int logn, int rows, float sign,
                                                          const float2 *__restrict__ tw, float scale)
{
    extern __shared__ float2 sm[];
    const int n = 1 << logn;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        float2 *d = data + (size_t)row * n;
        row_fft(logn, sign, tw, sm, sm + n, [&](int i) { return d[i]; },
                [&](int i, float2 v) { d[i] = make_float2(v.x * scale, v.y * scale); });
    }
}

// ASM pass 1: forward FFT of the rows of the zero-padded field.  Row r of the padded grid holds
// in[r - oy][c - ox] for the window, 0 elsewhere; rows outside the window transform to 0.
__global__ void __launch_bounds__(FFT_THREADS) k_asm_rows_in(const float2 *__restrict__ in, float2 *__restrict__ out,
                                                             int logn, int rows, int W, int H, int ox, int oy,
                                                             const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    const int n = 1 << logn;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        float2 *d = out + (size_t)row * n;
        const int y = row - oy;
        if (y < 0 || y >= H) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = make_float2(0.0f, 0.0f);
            continue;
        }
        const float2 *src = in + (size_t)y * W;
        row_fft(logn, -1.0f, tw, sm, sm + n,
                [&](int i) {
                    const int x = i - ox;
                    return (x >= 0 && x < W) ? src[x] : make_float2(0.0f, 0.0f);
                },
                [&](int i, float2 v) { d[i] = v; });
    }
}

// ASM pass 2, on the transposed spectrum (one row per spatial frequency fx): forward FFT of the
// row, multiplication by the transfer function's row (scale folded in) on the way into shared
// memory, inverse FFT.
__global__ void __launch_bounds__(FFT_THREADS) k_asm_rows_conv(float2 *data, int logn, int rows,
                                                               const float2 *__restrict__ Ht,
                                                               const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    const int n = 1 << logn;
    float2 *a = sm, *b = sm + n, *c = sm + 2 * n;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        float2 *d = data + (size_t)row * n;
        const float2 *h = Ht + (size_t)row * n;
        row_fft(logn, -1.0f, tw, a, b, [&](int i) { return d[i]; },
                [&](int i, float2 v) { c[i] = cmul(v, __ldg(h + i)); });
        row_fft(logn, +1.0f, tw, a, b, [&](int i) { return c[i]; }, [&](int i, float2 v) { d[i] = v; });
    }
}

// ASM pass 3: inverse FFT of the rows that hold the window, cropped into the output field.
__global__ void __launch_bounds__(FFT_THREADS) k_asm_rows_out(const float2 *__restrict__ data, float2 *__restrict__ out,
                                                              int logn, int W, int H, int ox, int oy,
                                                              const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    const int n = 1 << logn;
    for (int y = blockIdx.x; y < H; y += gridDim.x) {
        const float2 *d = data + (size_t)(y + oy) * n;
        float2 *dst = out + (size_t)y * W;
        row_fft(logn, +1.0f, tw, sm, sm + n, [&](int i) { return d[i]; },
                [&](int i, float2 v) {
                    const int x = i - ox;
                    if (x >= 0 && x < W) dst[x] = v;
                });
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

// exp(i 2 pi z sqrt(1/lambda^2 - fx^2 - fy^2)) on the padded grid (FFT order), times 'scale',
// stored transposed: Ht[ix][iy]
__global__ void k_transfer(float2 *Hf, int Wp, int Hp, double pitch, double lambda, double z, float scale)
{
    const size_t n = (size_t)Wp * Hp;
    const double il2 = 1.0 / (lambda * lambda);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int iy = (int)(i % Hp), ix = (int)(i / Hp);
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
    k_fft_rows<<<std::min(ny, 152 * 8), fft_threads(nx), 2 * sizeof(float2) * nx, s>>>(
        A, lx, ny, sign, twx, 1.0f);
    k_transpose<<<dim3((nx + 31) / 32, (ny + 31) / 32), tb, 0, s>>>(A, B, nx, ny);
    k_fft_rows<<<std::min(nx, 152 * 8), fft_threads(ny), 2 * sizeof(float2) * ny, s>>>(
        B, ly, nx, sign, twy, scale);
    k_transpose<<<dim3((ny + 31) / 32, (nx + 31) / 32), tb, 0, s>>>(B, A, ny, nx);
    return cudaGetLastError();
}

cudaError_t fft_setup()
{
    static bool done = false;
    if (done) return cudaSuccess;
    const int smem = (int)(3 * sizeof(float2)) << FFT_MAX_LOG;
    cudaError_t e = cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_asm_rows_in, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_asm_rows_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_asm_rows_out, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
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
    const size_t bytes = 2 * n * sizeof(float2) + (size_t)(nx + ny) * sizeof(float2);
    OPT_TRY(cudaMallocAsync((void **)&buf, bytes, s));
    float2 *A = (float2 *)buf, *B = A + n, *twx = B + n, *twy = twx + nx;
    cudaError_t e = cudaSuccess;
    k_twiddles<<<(nx + 255) / 256, 256, 0, s>>>(twx, nx);
    k_twiddles<<<(ny + 255) / 256, 256, 0, s>>>(twy, ny);
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

namespace {

// One padded angular-spectrum step of a W x H field: the sizes and the scratch it needs.
struct AsmPlan {
    int W, H, Wp, Hp, lx, ly, ox, oy;
    float2 *A, *B, *twx, *twy;
};

cudaError_t asm_field(const AsmPlan &P, const float2 *in, float2 *out, const float2 *Ht, cudaStream_t s)
{
    // rows of the padded field -> transpose -> per-frequency rows: FFT, transfer, inverse FFT
    // -> transpose -> inverse FFT of the window's rows, cropped
    const dim3 tb(32, 8);
    k_asm_rows_in<<<std::min(P.Hp, 152 * 8), fft_threads(P.Wp), 2 * sizeof(float2) * P.Wp,
                    s>>>(in, P.A, P.lx, P.Hp, P.W, P.H, P.ox, P.oy, P.twx);
    k_transpose<<<dim3((P.Wp + 31) / 32, (P.Hp + 31) / 32), tb, 0, s>>>(P.A, P.B, P.Wp, P.Hp);
    k_asm_rows_conv<<<std::min(P.Wp, 152 * 8), fft_threads(P.Hp), 3 * sizeof(float2) * P.Hp, s>>>(P.B, P.ly, P.Wp,
                                                                                                   Ht, P.twy);
    k_transpose<<<dim3((P.Hp + 31) / 32, (P.Wp + 31) / 32), tb, 0, s>>>(P.B, P.A, P.Hp, P.Wp);
    k_asm_rows_out<<<std::min(P.H, 152 * 8), fft_threads(P.Wp), 2 * sizeof(float2) * P.Wp,
                     s>>>(P.A, out, P.lx, P.W, P.H, P.ox, P.oy, P.twx);
    return cudaGetLastError();
}

bool asm_sizes(int W, int H, AsmPlan &P)
{
    P.W = W;
    P.H = H;
    P.Wp = P.Hp = 1;
    while (P.Wp < 2 * W) P.Wp <<= 1;
    while (P.Hp < 2 * H) P.Hp <<= 1;
    if (!pow2_in_range(P.Wp) || !pow2_in_range(P.Hp)) return false;
    P.lx = ilog2(P.Wp);
    P.ly = ilog2(P.Hp);
    P.ox = (P.Wp - W) / 2;
    P.oy = (P.Hp - H) / 2;
    return true;
}

// ---- phase-only encoding -----------------------------------------------------------------
constexpr int RED_BLOCKS = 304, RED_THREADS = 256;

__global__ void k_phase_field(const float *__restrict__ phi, float2 *__restrict__ u, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float sn, cs;
        sincosf(phi[i], &sn, &cs);
        u[i] = make_float2(cs, sn);
    }
}

// per-block partial sums (double) of <A, T> = sum conj(A) T and <A, A>
__global__ void __launch_bounds__(RED_THREADS) k_dots(const float2 *__restrict__ A, const float2 *__restrict__ T, size_t n,
                                                      double *__restrict__ part)
{
    __shared__ double sre[RED_THREADS], sim[RED_THREADS], saa[RED_THREADS];
    double re = 0.0, im = 0.0, aa = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 a = A[i], t = T[i];
        re += (double)a.x * t.x + (double)a.y * t.y;
        im += (double)a.x * t.y - (double)a.y * t.x;
        aa += (double)a.x * a.x + (double)a.y * a.y;
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    saa[threadIdx.x] = aa;
    __syncthreads();
    for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sre[threadIdx.x] += sre[threadIdx.x + o];
            sim[threadIdx.x] += sim[threadIdx.x + o];
            saa[threadIdx.x] += saa[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = sre[0];
        part[3 * blockIdx.x + 1] = sim[0];
        part[3 * blockIdx.x + 2] = saa[0];
    }
}

// s = <A, T> / <A, A>, from the partial sums in a fixed order
__global__ void k_scale(const double *__restrict__ part, int nb, double *__restrict__ sc)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double re = 0.0, im = 0.0, aa = 0.0;
    for (int b = 0; b < nb; ++b) {
        re += part[3 * b];
        im += part[3 * b + 1];
        aa += part[3 * b + 2];
    }
    sc[0] = aa > 0.0 ? re / aa : 0.0;
    sc[1] = aa > 0.0 ? im / aa : 0.0;
}

// V = conj(s) (s A - T), with per-block partial sums of |s A - T|^2
__global__ void __launch_bounds__(RED_THREADS) k_residual(const float2 *__restrict__ A, const float2 *__restrict__ T,
                                                          const double *__restrict__ sc, float2 *__restrict__ V, size_t n,
                                                          double *__restrict__ part)
{
    __shared__ double sl[RED_THREADS];
    const float sr = (float)sc[0], si = (float)sc[1];
    double l = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 a = A[i], t = T[i];
        const float rr = sr * a.x - si * a.y - t.x, ri = sr * a.y + si * a.x - t.y;
        l += (double)rr * rr + (double)ri * ri;
        V[i] = make_float2(sr * rr + si * ri, sr * ri - si * rr);
    }
    sl[threadIdx.x] = l;
    __syncthreads();
    for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sl[threadIdx.x] += sl[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sl[0];
}

__global__ void k_loss(const double *__restrict__ part, int nb, double *__restrict__ loss)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double l = 0.0;
    for (int b = 0; b < nb; ++b) l += part[b];
    *loss = l;
}

// phi <- phi - lr dL/dphi, dL/dphi = -2 Im(u conj(G))
__global__ void k_phase_step(float *__restrict__ phi, const float2 *__restrict__ u, const float2 *__restrict__ G, size_t n,
                             float lr)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 a = u[i], g = G[i];
        phi[i] += 2.0f * lr * (a.y * g.x - a.x * g.y);
    }
}

}  // namespace

extern "C" hpt_status hpt_asm_propagate(hpt_ctx *ctx, const void *in_dev, void *out_dev, int32_t W, int32_t H,
                                        int32_t n_lambda, int32_t K, const double *lambdas, double pitch, double z,
                                        void *stream)
{
    hpt_status st = internal_check(ctx);
    if (st) return st;
    if (!in_dev || !out_dev || !lambdas) return internal_fail(HPT_ERR_INVALID_ARG, "in_dev, out_dev or lambdas is NULL");
    if (W < 1 || H < 1 || n_lambda < 1 || n_lambda > 3 || K < 1)
        return internal_fail(HPT_ERR_INVALID_ARG, "need W, H, K >= 1 and 1 <= n_lambda <= 3");
    AsmPlan P;
    if (!asm_sizes(W, H, P)) return internal_fail(HPT_ERR_UNSUPPORTED, "padded size above 8192 x 8192 (W, H <= 4096)");
    const int Wp = P.Wp, Hp = P.Hp;
    if (!(pitch > 0.0)) return internal_fail(HPT_ERR_INVALID_ARG, "pitch must be > 0");
    for (int l = 0; l < n_lambda; ++l)
        if (!(lambdas[l] > 0.0)) return internal_fail(HPT_ERR_INVALID_ARG, "wavelengths must be > 0");
    OPT_TRY(cudaSetDevice(internal_ctx_device(ctx)));
    OPT_TRY(fft_setup());
    cudaStream_t s = (cudaStream_t)stream;
    const size_t np = (size_t)Wp * Hp;
    const size_t bytes = (2 + (size_t)n_lambda) * np * sizeof(float2) + (size_t)(Wp + Hp) * sizeof(float2);
    char *buf = nullptr;
    OPT_TRY(cudaMallocAsync((void **)&buf, bytes, s));
    P.A = (float2 *)buf;
    P.B = P.A + np;
    float2 *Hf = P.B + np;
    P.twx = Hf + (size_t)n_lambda * np;
    P.twy = P.twx + Wp;
    cudaError_t e = cudaSuccess;
    k_twiddles<<<(Wp + 255) / 256, 256, 0, s>>>(P.twx, Wp);
    k_twiddles<<<(Hp + 255) / 256, 256, 0, s>>>(P.twy, Hp);
    for (int l = 0; l < n_lambda; ++l)
        k_transfer<<<grid_for(np), 256, 0, s>>>(Hf + (size_t)l * np, Wp, Hp, pitch, lambdas[l], z, 1.0f / (float)np);
    const float2 *in = (const float2 *)in_dev;
    float2 *out = (float2 *)out_dev;
    for (int f = 0; f < n_lambda * K && e == cudaSuccess; ++f) {
        const size_t fo = (size_t)f * W * H;
        e = asm_field(P, in + fo, out + fo, Hf + (size_t)(f / K) * np, s);
    }
    cudaError_t e2 = cudaFreeAsync(buf, s);
    OPT_TRY(e);
    OPT_TRY(e2);
    return HPT_OK;
}

extern "C" hpt_status hpt_phase_encode(hpt_ctx *ctx, const void *target_dev, float *phi_dev, int32_t W, int32_t H,
                                       double lambda, double pitch, double z, int32_t iters, float lr, double *losses,
                                       void *stream)
{
    hpt_status st = internal_check(ctx);
    if (st) return st;
    if (!target_dev || !phi_dev) return internal_fail(HPT_ERR_INVALID_ARG, "target_dev or phi_dev is NULL");
    if (W < 1 || H < 1 || iters < 0) return internal_fail(HPT_ERR_INVALID_ARG, "need W, H >= 1 and iters >= 0");
    if (!(pitch > 0.0) || !(lambda > 0.0) || !std::isfinite(z) || !std::isfinite(lr))
        return internal_fail(HPT_ERR_INVALID_ARG, "bad pitch, lambda, z or lr");
    AsmPlan P;
    if (!asm_sizes(W, H, P)) return internal_fail(HPT_ERR_UNSUPPORTED, "padded size above 8192 x 8192 (W, H <= 4096)");
    OPT_TRY(cudaSetDevice(internal_ctx_device(ctx)));
    OPT_TRY(fft_setup());
    cudaStream_t s = (cudaStream_t)stream;
    const size_t np = (size_t)P.Wp * P.Hp, n = (size_t)W * H;
    const size_t bytes = 4 * np * sizeof(float2) + (size_t)(P.Wp + P.Hp) * sizeof(float2) + 3 * n * sizeof(float2) +
                         (3 * RED_BLOCKS + 2 + (size_t)std::max(iters, 1)) * sizeof(double);
    char *buf = nullptr;
    OPT_TRY(cudaMallocAsync((void **)&buf, bytes, s));
    P.A = (float2 *)buf;
    P.B = P.A + np;
    float2 *Hp_ = P.B + np, *Hm = Hp_ + np;          // transfer over +z and over -z (the adjoint)
    P.twx = Hm + np;
    P.twy = P.twx + P.Wp;
    float2 *U = P.twy + P.Hp, *Afield = U + n, *V = Afield + n;
    double *part = (double *)(V + n), *sc = part + 3 * RED_BLOCKS, *dloss = sc + 2;
    const float2 *T = (const float2 *)target_dev;
    k_twiddles<<<(P.Wp + 255) / 256, 256, 0, s>>>(P.twx, P.Wp);
    k_twiddles<<<(P.Hp + 255) / 256, 256, 0, s>>>(P.twy, P.Hp);
    k_transfer<<<grid_for(np), 256, 0, s>>>(Hp_, P.Wp, P.Hp, pitch, lambda, z, 1.0f / (float)np);
    k_transfer<<<grid_for(np), 256, 0, s>>>(Hm, P.Wp, P.Hp, pitch, lambda, -z, 1.0f / (float)np);
    cudaError_t e = cudaGetLastError();
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
        k_phase_field<<<grid_for(n), 256, 0, s>>>(phi_dev, U, n);
        e = asm_field(P, U, Afield, Hp_, s);
        if (e != cudaSuccess) break;
        k_dots<<<RED_BLOCKS, RED_THREADS, 0, s>>>(Afield, T, n, part);
        k_scale<<<1, 32, 0, s>>>(part, RED_BLOCKS, sc);
        k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(Afield, T, sc, V, n, part);
        k_loss<<<1, 32, 0, s>>>(part, RED_BLOCKS, dloss + it);
        e = asm_field(P, V, V, Hm, s);
        if (e != cudaSuccess) break;
        k_phase_step<<<grid_for(n), 256, 0, s>>>(phi_dev, U, V, n, lr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && losses && iters > 0)
        e = cudaMemcpyAsync(losses, dloss, sizeof(double) * iters, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && losses && iters > 0) e = cudaStreamSynchronize(s);
    cudaError_t e2 = cudaFreeAsync(buf, s);
    OPT_TRY(e);
    OPT_TRY(e2);
    return HPT_OK;
}
