// Wave optics around the tracer: the band-limited Gaussian random field phase maps of Eq. 4
// (hpt_grf_build) and the angular spectrum method of the two-stage scheme (hpt_asm_propagate).
//
// Both rest on one 2-D FFT of power-of-two sizes: every row transformed in shared memory by
// one block (Stockham autosort: radix-16 passes in registers, the remainder radix first, the
// first pass reading global memory and the last writing it in natural order, the passes in
// between in place in one bank-padded shared buffer), then every column the same way, a few
// adjacent columns per block read and written in place in the row-major array (no transposes).
// Work around the transforms is folded into them: the GRF spectrum is generated as the row
// pass loads it and the phase taken as the column pass stores it; the ASM's zero padding is
// never stored (see asm_field).  The data are complex64; the twiddle factors are rounded from
// double-precision values.  The transfer function's phase 2 pi z sqrt(1/lambda^2 - f^2),
// ~1e5 turns, is formed in double-float arithmetic before its fraction is taken.
#include <algorithm>
#include <type_traits>
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

constexpr int FFT_MAX_LOG = 13;          // 8192 points: 68 KB of shared memory
constexpr int FFT_THREADS = 512;
#ifndef HPT_FFT_REGS
#define HPT_FFT_REGS 64                  // registers per thread the row kernels are compiled for
#endif
#ifndef HPT_FFT_CONV_REGS
#define HPT_FFT_CONV_REGS 64             // the same for the ASM's y pass (two transforms per row)
#endif
constexpr unsigned GRF_TAG = 0x47524600u;
constexpr int ASM_BATCH = 8;             // fields of one wavelength propagated by one group of launches

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
// stages; SIGN = -1 forward, +1 inverse.  The butterflies whose twiddle is 1 or -+i take no
// multiplication.
template <int R, int SIGN>
__device__ __forceinline__ void dft_reg(float2 *v)
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
                const int m = pos * (8 / half);        // twiddle exp(SIGN 2 pi i m / 16)
                float2 b = t[g + pos + half];
                if (m == 4) {
                    b = SIGN > 0 ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
                } else if (m != 0) {
                    float2 w = w16(m);
                    if (SIGN > 0) w.y = -w.y;
                    b = cmul(w, b);
                }
                const float2 a = t[g + pos];
                t[g + pos] = make_float2(a.x + b.x, a.y + b.y);
                t[g + pos + half] = make_float2(a.x - b.x, a.y - b.y);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = t[i];
}

// Shared-memory index of point i of a row: one float2 of padding after every 16, so that the
// stride-16 stores of the first pass and the strided loads after it fall in distinct banks.
__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int fft_smem_bytes(int n) { return (n + n / 16 + 1) * (int)sizeof(float2); }
// threads of a row's block: n / 16 (each holds 16 points of a pass), at least one warp
__host__ __device__ constexpr int fft_threads(int n) { return n / 16 > 32 ? (n / 16 < FFT_THREADS ? n / 16 : FFT_THREADS) : 32; }
// resident blocks per SM the row kernels are compiled for: 'regs' registers per thread
__host__ __device__ constexpr int fft_minb(int n, int regs)
{
    return 65536 / (regs * fft_threads(n)) < 1 ? 1 : (65536 / (regs * fft_threads(n)) > 32 ? 32 : 65536 / (regs * fft_threads(n)));
}
// radix of pass p of a 2^logn-point transform (the remainder radix first, then 16s), the number
// of passes, and the span Ns of the sub-transforms pass p combines
__host__ __device__ constexpr int fft_radix(int logn, int p) { return (p == 0 && (logn & 3)) ? (1 << (logn & 3)) : 16; }
__host__ __device__ constexpr int fft_npass(int logn) { return (logn >> 2) + ((logn & 3) ? 1 : 0); }
__host__ __device__ constexpr int fft_ns(int logn, int p) { return p == 0 ? 1 : fft_ns(logn, p - 1) * fft_radix(logn, p - 1); }

// Pass P of the Stockham transform of N = 2^LOGN points (radix R, span NS): element j reads
// x[j + r N/R] (r < R) through 'ld', multiplies it by exp(SIGN 2 pi i r (j mod NS) / (NS R))
// (the N-point twiddle table), takes the R-point DFT and writes
// y[(j - j mod NS) R + j mod NS + r NS] through 'st'.  Thread t takes j = t + m T (T threads,
// m < J; t = tid, the thread's index within the transform); with 'inplace' every thread holds
// its values in registers across a barrier before it stores, so that x and y may be the same buffer.
template <int LOGN, int P, int SIGN, class LD, class ST>
__device__ __forceinline__ void stockham_pass(const float2 *__restrict__ tw, LD ld, ST st, bool inplace, int tid)
{
    constexpr int N = 1 << LOGN, R = fft_radix(LOGN, P), NS = fft_ns(LOGN, P), T = fft_threads(N);
    constexpr int Q = N / R, TWS = N / (NS * R), J = (Q + T - 1) / T;
    constexpr bool RAGGED = J * T > Q;
    float2 v[J][R];
#pragma unroll
    for (int m = 0; m < J; ++m) {
        // past the row (small N only) a thread repeats the last element's loads and stores nothing
        const int j = RAGGED ? min(tid + m * T, Q - 1) : tid + m * T;
        const int k = j & (NS - 1);
#pragma unroll
        for (int r = 0; r < R; ++r) v[m][r] = ld(j + r * Q);
        if (NS > 1) {
            // twiddles w^r, w = exp(SIGN 2 pi i k / (NS R)): w, w^2, w^3 formed from the loaded w,
            // w^(4c) loaded for c >= 1 and multiplied by them (at most three complex products
            // per twiddle, ~1e-7 relative)
            float2 w1 = __ldg(tw + k * TWS);
            if (SIGN > 0) w1.y = -w1.y;
            const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w;
                if (r % 4 == 0 || r < 4) {
                    w = r == 1 ? w1 : r == 2 ? w2 : r == 3 ? w3 : __ldg(tw + r * k * TWS);
                    if (r >= 4 && SIGN > 0) w.y = -w.y;
                } else {
                    float2 b = __ldg(tw + (r & ~3) * k * TWS);
                    if (SIGN > 0) b.y = -b.y;
                    w = cmul(b, (r & 3) == 1 ? w1 : (r & 3) == 2 ? w2 : w3);
                }
                v[m][r] = cmul(v[m][r], w);
            }
        }
        dft_reg<R, SIGN>(v[m]);
    }
    if (inplace) __syncthreads();
#pragma unroll
    for (int m = 0; m < J; ++m) {
        const int j = tid + m * T;
        if (!RAGGED || j < Q) {
            const int k = j & (NS - 1);
            const int o = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) st(o + r * NS, v[m][r]);
        }
    }
}

// FFT of one row of 2^LOGN points by fft_threads(2^LOGN) threads: the passes from P on, the
// first reading through 'gld', the last writing through 'gst', the ones in between in place in
// the shared buffer 'buf' (padded by spad).  IN_SMEM / OUT_SMEM say that gld / gst touch 'buf'
// themselves.  tid: the thread's index within the transform (threadIdx.x when a block takes one
// row).  Ends with a barrier of the whole block.
template <int LOGN, int SIGN, bool IN_SMEM, bool OUT_SMEM, int P = 0, class LD, class ST>
__device__ __forceinline__ void row_fft(const float2 *tw, float2 *buf, LD gld, ST gst, int tid = threadIdx.x)
{
    constexpr int NP = fft_npass(LOGN);
    constexpr bool first = P == 0, last = P == NP - 1;
    constexpr bool src_smem = first ? IN_SMEM : true, dst_smem = last ? OUT_SMEM : true;
    constexpr bool inplace = (src_smem && dst_smem) || NP == 1;
    auto sld = [&](int i) { return buf[spad(i)]; };
    auto sst = [&](int i, float2 v) { buf[spad(i)] = v; };
    if constexpr (first && last) stockham_pass<LOGN, P, SIGN>(tw, gld, gst, inplace, tid);
    else if constexpr (first) stockham_pass<LOGN, P, SIGN>(tw, gld, sst, inplace, tid);
    else if constexpr (last) stockham_pass<LOGN, P, SIGN>(tw, sld, gst, inplace, tid);
    else stockham_pass<LOGN, P, SIGN>(tw, sld, sst, inplace, tid);
    __syncthreads();
    if constexpr (P + 1 < NP) row_fft<LOGN, SIGN, IN_SMEM, OUT_SMEM, P + 1>(tw, buf, gld, gst, tid);
}

#define FFT_BOUNDS(L) __launch_bounds__(fft_threads(1 << (L)), fft_minb(1 << (L), HPT_FFT_REGS))
#define FFT_BOUNDS_CONV(L) __launch_bounds__(fft_threads(1 << (L)), fft_minb(1 << (L), HPT_FFT_CONV_REGS))

// GRF pass 1 (Eq. 4): for each spectrum row ky < ny, the unit-modulus random spectrum
// exp(i xi) inside the elliptic passband 4 (kx^2 ny^2 + ky^2 nx^2) <= nx^2 ny^2 (integers, FFT
// order) and 0 outside it, xi = 2 pi u24(Philox(ix, iy, m, 'GRF'; seed)), generated as the
// first pass loads it, and its unnormalised inverse FFT along x.
template <int LOGN>
__global__ void FFT_BOUNDS(LOGN) k_grf_rows(float2 *out, int ny, unsigned m, unsigned seed_lo, unsigned seed_hi,
                                            const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    constexpr int nx = 1 << LOGN;
    const long long NX = nx, NY = ny;
    {
        const int iy = blockIdx.x;    // one row per block
        const long long ky = iy < ny / 2 ? iy : iy - ny;
        const long long rest = NX * NX * NY * NY - 4 * ky * ky * NX * NX;
        float2 *d = out + ((size_t)iy << LOGN);
        row_fft<LOGN, +1, false, false>(tw, sm,
                                    [&](int ix) {
                                        const long long kx = ix < nx / 2 ? ix : ix - nx;
                                        float2 v = make_float2(0.0f, 0.0f);
                                        if (4 * kx * kx * NY * NY <= rest) {
                                            const uint4 o = philox(make_uint4((unsigned)ix, (unsigned)iy, m, GRF_TAG),
                                                                   seed_lo, seed_hi);
                                            float sn, cs;
                                            sincospif(2.0f * u24(o.x), &sn, &cs);
                                            v = make_float2(cs, sn);
                                        }
                                        return v;
                                    },
                                    [&](int i, float2 v) { d[i] = v; });
    }
}

// The ASM's 2-D transforms skip the zero padding: only the H rows of the window are transformed
// along x, kept compact (H rows of n_x, row-major); the column pass reads each column of that
// array in place, zero-extends it to n_y as it loads it and stores only its window rows after
// the inverse transform; the rows outside the window are never written nor read.

// ASM pass 1: forward FFT along x of the window's rows, zero-padded to 2^LOGN: out[y][k] for
// row y = blockIdx.x (the H rows of each of the fields, one field after the other), from
// in[y][k - ox] inside the window and 0 outside it.
template <int LOGN>
__global__ void FFT_BOUNDS(LOGN) k_asm_rows_in(const float2 *__restrict__ in, float2 *__restrict__ out, int W, int ox,
                                               const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    {
        const int y = blockIdx.x;     // one row per block
        float2 *d = out + ((size_t)y << LOGN);
        const float2 *src = in + (size_t)y * W;
        row_fft<LOGN, -1, false, false>(tw, sm,
                                    [&](int i) {
                                        const int x = i - ox;
                                        // only the window's points are loaded (a predicated load)
                                        return (x >= 0 && x < W) ? __ldg(src + x) : make_float2(0.0f, 0.0f);
                                    },
                                    [&](int i, float2 v) { d[i] = v; });
    }
}

// Column transforms without transposes: a block takes C adjacent columns of a row-major array,
// thread (c, t) = (threadIdx.x, threadIdx.y) being thread t of column c's transform, so that the
// lanes of a warp read and write C consecutive elements of each row (C x 8 bytes: whole 32-byte
// sectors for C >= 4).  Each column has its own shared buffer, C of them per block.
// columns per block by transform length, as measured on the GB300: two, except four for 2048
// points (the 4096x2048 GRF maps: 0.81 ms against 0.91 with two and 0.99 with eight); four
// columns of 4096 points (1024 threads, 139 KB per block, one block per SM) ran 19 % slower than
// two on the 1080p ASM, eight columns of 1024 points 24 % slower than two on the 1920x270 one
__host__ __device__ constexpr int cols_per_block(int logn) { return logn == 11 ? 4 : 2; }
// float2 elements between the shared buffers of two of C columns: at least the padded row, plus
// 8 (4 for eight columns), so that the columns a warp's lanes touch start in different banks
__host__ __device__ constexpr int col_stride(int n, int c) { return ((n + n / 16 + 1 + 15) / 16) * 16 + (c >= 8 ? 4 : 8); }
__host__ __device__ constexpr int cols_smem_bytes(int n, int c) { return c * col_stride(n, c) * (int)sizeof(float2); }
static_assert(cols_per_block(13) * fft_threads(1 << 13) <= 1024 && cols_smem_bytes(1 << 13, cols_per_block(13)) <= 227 * 1024,
              "column blocks of 8192 points exceed a block's threads or shared memory");

#define COLS_BOUNDS(L, C) __launch_bounds__((C) * fft_threads(1 << (L)), fft_minb(1 << (L), HPT_FFT_CONV_REGS * (C)))

// ASM pass 2, on the compact spectra A (per field H rows of Wp, row-major): for C spatial
// frequencies fx per block, the column of H values zero-extended to 2^LOGN rows (the window at
// rows oy .. oy + H - 1), forward FFT in shared memory, multiplication by the transfer
// function's row (scale folded in), inverse FFT, and the window's rows stored back in place.
// Consecutive blocks take the same frequencies of the nf fields in turn, so that the transfer
// function's rows are read from memory once.
template <int LOGN, int C>
__global__ void COLS_BOUNDS(LOGN, C) k_asm_cols(float2 *A, int Wp, int H, int oy, int nf,
                                                const float2 *__restrict__ Ht, const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    const int c = threadIdx.x, t = threadIdx.y;
    const int grp = blockIdx.x / nf, f = blockIdx.x - grp * nf;
    const int fx = grp * C + c;
    float2 *col = A + (size_t)f * H * Wp + fx;           // row y at col[y * Wp]
    float2 *buf = sm + c * col_stride(1 << LOGN, C);
    const float2 *h = Ht + ((size_t)fx << LOGN);
    constexpr int HSH = LOGN > 4 ? LOGN - 4 : 0;
    auto HALF = [](int i) { return ((i >> HSH) & 1) != 0; };
    row_fft<LOGN, -1, false, true>(tw, buf,
                                   [&](int i) {
                                       const int y = i - oy;
                                       // only the window's rows are loaded (a predicated load)
                                       return (y >= 0 && y < H) ? col[(size_t)y * Wp] : make_float2(0.0f, 0.0f);
                                   },
                                   // the transfer function, half of it applied as the forward
                                   // transform's last pass stores the spectrum ...
                                   [&](int i, float2 v) { buf[spad(i)] = HALF(i) ? v : cmul(v, __ldg(h + i)); }, t);
    // ... the other half as the inverse transform's first pass loads it (each point once; a
    // thread holds half as many transfer-function values at a time)
    row_fft<LOGN, +1, true, false>(tw, buf, [&](int i) { return HALF(i) ? cmul(buf[spad(i)], __ldg(h + i)) : buf[spad(i)]; },
                                   [&](int i, float2 v) {
                                       const int y = i - oy;
                                       if (y >= 0 && y < H) col[(size_t)y * Wp] = v;
                                   },
                                   t);
}

// GRF pass 2 (Eq. 4): the unnormalised inverse FFT along y of C columns of the row pass's output
// B [ny][nx] per block, its phase (atan2) stored to phi [ny][nx] row-major.
template <int LOGN, int C>
__global__ void COLS_BOUNDS(LOGN, C) k_grf_cols(const float2 *__restrict__ B, float *__restrict__ phi, int nx,
                                                const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    const int c = threadIdx.x, t = threadIdx.y;
    const int ix = blockIdx.x * C + c;
    const float2 *col = B + ix;
    float *out = phi + ix;
    float2 *buf = sm + c * col_stride(1 << LOGN, C);
    row_fft<LOGN, +1, false, false>(tw, buf, [&](int i) { return col[(size_t)i * nx]; },
                                    [&](int i, float2 v) { out[(size_t)i * nx] = atan2f(v.y, v.x); }, t);
}

// ASM pass 3: inverse FFT along x of the compact rows (H per field), cropped into the output
// fields.
template <int LOGN>
__global__ void FFT_BOUNDS(LOGN) k_asm_rows_out(const float2 *__restrict__ data, float2 *__restrict__ out, int W,
                                                int ox, const float2 *__restrict__ tw)
{
    extern __shared__ float2 sm[];
    {
        const int y = blockIdx.x;     // one row per block
        const float2 *d = data + ((size_t)y << LOGN);
        float2 *dst = out + (size_t)y * W;
        row_fft<LOGN, +1, false, false>(tw, sm, [&](int i) { return d[i]; },
                                    [&](int i, float2 v) {
                                        const int x = i - ox;
                                        if (x >= 0 && x < W) dst[x] = v;
                                    });
    }
}

// calls f(std::integral_constant<int, logn>) for logn in [1, FFT_MAX_LOG]
template <class F>
cudaError_t with_logn(int logn, F f)
{
    switch (logn) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 3: return f(std::integral_constant<int, 3>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 5: return f(std::integral_constant<int, 5>{});
    case 6: return f(std::integral_constant<int, 6>{});
    case 7: return f(std::integral_constant<int, 7>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 9: return f(std::integral_constant<int, 9>{});
    case 10: return f(std::integral_constant<int, 10>{});
    case 11: return f(std::integral_constant<int, 11>{});
    case 12: return f(std::integral_constant<int, 12>{});
    case 13: return f(std::integral_constant<int, 13>{});
    default: return cudaErrorInvalidValue;
    }
}

// exp(i 2 pi z sqrt(1/lambda^2 - fx^2 - fy^2)) on the padded grid (FFT order), times 'scale',
// stored transposed: Ht[ix][iy].  The value depends on fx^2 and fy^2 only, and the frequencies of
// ix and Wp - ix (iy and Hp - iy) are exact negatives of each other, so each value is computed
// once for ix <= Wp / 2, iy <= Hp / 2 (one block row per ix: grid Wp / 2 + 1 high) and stored
// at its up to four mirror positions.
__global__ void k_transfer(float2 *Hf, int Wp, int Hp, float2 fx_unit, float2 fy_unit, float2 inv_lambda2, float2 zdist,
                           float scale)
{
    // double-float arithmetic (~48-bit significands): the phase runs to ~1e5 turns and its
    // fraction must hold ~1e-7
    const int ix = blockIdx.y;                               // 0 .. Wp / 2
    const df fx = mul_f(mkdf(fx_unit.x, fx_unit.y), (float)(ix < Wp / 2 ? ix : ix - Wp));
    const df base = mkdf(inv_lambda2.x, inv_lambda2.y) - fx * fx;
    const df fyu = mkdf(fy_unit.x, fy_unit.y), z = mkdf(zdist.x, zdist.y);
    float2 *row = Hf + (size_t)ix * Hp;
    float2 *row2 = (ix > 0 && ix < Wp / 2) ? Hf + (size_t)(Wp - ix) * Hp : nullptr;
    for (int iy = blockIdx.x * blockDim.x + threadIdx.x; iy <= Hp / 2; iy += gridDim.x * blockDim.x) {
        const df fy = mul_f(fyu, (float)(iy < Hp / 2 ? iy : iy - Hp));
        const df a = base - fy * fy;
        float2 v = make_float2(0.0f, 0.0f);
        if (a.hi > 0.0f) {
            const float f = RealOps<df>::frac_f(z * df_sqrt(a));
            float sn, cs;
            sincospif(2.0f * f, &sn, &cs);
            v = make_float2(cs * scale, sn * scale);
        }
        const bool my = iy > 0 && iy < Hp / 2;
        row[iy] = v;
        if (my) row[Hp - iy] = v;
        if (row2) {
            row2[iy] = v;
            if (my) row2[Hp - iy] = v;
        }
    }
}

// the launch shape of k_transfer for a Wp x Hp grid
inline dim3 transfer_grid(int Wp, int Hp) { return dim3((Hp / 2 + 1 + 255) / 256, Wp / 2 + 1); }

// a double as a double-float pair (head, tail)
float2 to_df(double x)
{
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
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
cudaError_t fft_setup()
{
    static bool done = false;
    if (done) return cudaSuccess;
    for (int l = 1; l <= FFT_MAX_LOG; ++l) {
        cudaError_t e = with_logn(l, [&](auto L) {
            constexpr int ll = decltype(L)::value;
            const int smem = fft_smem_bytes(1 << ll);
            cudaError_t r = cudaFuncSetAttribute(k_grf_rows<ll>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (r == cudaSuccess) r = cudaFuncSetAttribute(k_asm_rows_in<ll>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            constexpr int cc = cols_per_block(ll);
            const int csmem = cols_smem_bytes(1 << ll, cc);
            if (r == cudaSuccess) r = cudaFuncSetAttribute(k_asm_cols<ll, cc>, cudaFuncAttributeMaxDynamicSharedMemorySize, csmem);
            if (r == cudaSuccess) r = cudaFuncSetAttribute(k_grf_cols<ll, cc>, cudaFuncAttributeMaxDynamicSharedMemorySize, csmem);
            if (r == cudaSuccess) r = cudaFuncSetAttribute(k_asm_cols<ll, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           cols_smem_bytes(1 << ll, 2));
            if (r == cudaSuccess) r = cudaFuncSetAttribute(k_grf_cols<ll, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           cols_smem_bytes(1 << ll, 2));
            if (r == cudaSuccess) r = cudaFuncSetAttribute(k_asm_rows_out<ll>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            return r;
        });
        if (e != cudaSuccess) return e;
    }
    done = true;
    return cudaSuccess;
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
    if (!(pitch > 0.0) || !std::isfinite(pitch)) return internal_fail(HPT_ERR_INVALID_ARG, "pitch must be finite and > 0");
    OPT_TRY(cudaSetDevice(internal_ctx_device(ctx)));
    OPT_TRY(fft_setup());
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)nx * ny;
    char *buf = nullptr;
    const size_t bytes = n * sizeof(float2) + (size_t)(nx + ny) * sizeof(float2);
    OPT_TRY(cudaMallocAsync((void **)&buf, bytes, s));
    float2 *A = (float2 *)buf, *twx = A + n, *twy = twx + nx;
    cudaError_t e = cudaSuccess;
    k_twiddles<<<(nx + 255) / 256, 256, 0, s>>>(twx, nx);
    k_twiddles<<<(ny + 255) / 256, 256, 0, s>>>(twy, ny);
    // per map: spectrum generated and transformed along x (row-major [ny][nx]), then the columns
    // transformed along y with the phase taken as they are stored
    const int ly = ilog2(ny);
    for (int k = 0; k < K && e == cudaSuccess; ++k) {
        e = with_logn(ilog2(nx), [&](auto L) {
            constexpr int l = decltype(L)::value;
            k_grf_rows<l><<<ny, fft_threads(1 << l), fft_smem_bytes(1 << l), s>>>(
                A, ny, (unsigned)(hologram_offset + k), (unsigned)phase_seed, (unsigned)(phase_seed >> 32), twx);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) break;
        e = with_logn(ly, [&](auto L) {
            constexpr int l = decltype(L)::value;
            constexpr int cc = cols_per_block(l);
            float *dst = phi_dev + (size_t)k * n;
            if (nx >= cc)
                k_grf_cols<l, cc><<<nx / cc, dim3(cc, fft_threads(1 << l)), cols_smem_bytes(1 << l, cc), s>>>(A, dst, nx, twy);
            else
                k_grf_cols<l, 2><<<nx / 2, dim3(2, fft_threads(1 << l)), cols_smem_bytes(1 << l, 2), s>>>(A, dst, nx, twy);
            return cudaGetLastError();
        });
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
    float2 *A, *twx, *twy;
};

// nf fields of one wavelength (consecutive W x H fields of 'in' and 'out'; P.A holds nf x Wp x H)
cudaError_t asm_field(const AsmPlan &P, const float2 *in, float2 *out, int nf, const float2 *Ht, cudaStream_t s)
{
    // the window's rows along x (H x Wp per field, compact, row-major) -> per-frequency columns
    // zero-extended to Hp, read and written in place: FFT, transfer, inverse FFT, window rows kept
    // -> inverse FFT along x, cropped
    const int rows = nf * P.H;
    cudaError_t e = with_logn(P.lx, [&](auto L) {
        constexpr int l = decltype(L)::value;
        k_asm_rows_in<l><<<rows, fft_threads(1 << l), fft_smem_bytes(1 << l), s>>>(in, P.A, P.W, P.ox, P.twx);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    e = with_logn(P.ly, [&](auto L) {
        constexpr int l = decltype(L)::value;
        constexpr int cc = cols_per_block(l);
        if (P.Wp >= cc)
            k_asm_cols<l, cc><<<(P.Wp / cc) * nf, dim3(cc, fft_threads(1 << l)), cols_smem_bytes(1 << l, cc), s>>>(
                P.A, P.Wp, P.H, P.oy, nf, Ht, P.twy);
        else
            k_asm_cols<l, 2><<<(P.Wp / 2) * nf, dim3(2, fft_threads(1 << l)), cols_smem_bytes(1 << l, 2), s>>>(
                P.A, P.Wp, P.H, P.oy, nf, Ht, P.twy);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    return with_logn(P.lx, [&](auto L) {
        constexpr int l = decltype(L)::value;
        k_asm_rows_out<l><<<rows, fft_threads(1 << l), fft_smem_bytes(1 << l), s>>>(P.A, out, P.W, P.ox, P.twx);
        return cudaGetLastError();
    });
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

// Reductions: each thread sums its elements in float in runs of RED_RUN, the runs and the
// block's threads in double (a fixed order: the result does not depend on timing).
constexpr int RED_RUN = 16;

// tree sum of v over the block's RED_THREADS threads (in place in the shared array)
__device__ __forceinline__ double block_sum(double *sh, double v)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// per-block partial sums of <A, T> = sum conj(A) T and <A, A>
__global__ void __launch_bounds__(RED_THREADS) k_dots(const float2 *__restrict__ A, const float2 *__restrict__ T, size_t n,
                                                      double *__restrict__ part)
{
    __shared__ double sh[RED_THREADS];
    double re = 0.0, im = 0.0, aa = 0.0;
    float fre = 0.0f, fim = 0.0f, faa = 0.0f;
    int c = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 a = __ldg(A + i), t = __ldg(T + i);
        fre += a.x * t.x + a.y * t.y;
        fim += a.x * t.y - a.y * t.x;
        faa += a.x * a.x + a.y * a.y;
        if (++c == RED_RUN) {
            re += fre; im += fim; aa += faa;
            fre = fim = faa = 0.0f;
            c = 0;
        }
    }
    re += fre; im += fim; aa += faa;
    re = block_sum(sh, re);
    im = block_sum(sh, im);
    aa = block_sum(sh, aa);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = re;
        part[3 * blockIdx.x + 1] = im;
        part[3 * blockIdx.x + 2] = aa;
    }
}

// s = <A, T> / <A, A> from the nb partial sums (one block)
__global__ void __launch_bounds__(RED_THREADS) k_scale(const double *__restrict__ part, int nb, double *__restrict__ sc)
{
    __shared__ double sh[RED_THREADS];
    double re = 0.0, im = 0.0, aa = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        re += part[3 * b];
        im += part[3 * b + 1];
        aa += part[3 * b + 2];
    }
    re = block_sum(sh, re);
    im = block_sum(sh, im);
    aa = block_sum(sh, aa);
    if (threadIdx.x == 0) {
        sc[0] = aa > 0.0 ? re / aa : 0.0;
        sc[1] = aa > 0.0 ? im / aa : 0.0;
    }
}

// V = conj(s) (s A - T), with per-block partial sums of |s A - T|^2
__global__ void __launch_bounds__(RED_THREADS) k_residual(const float2 *__restrict__ A, const float2 *__restrict__ T,
                                                          const double *__restrict__ sc, float2 *__restrict__ V, size_t n,
                                                          double *__restrict__ part)
{
    __shared__ double sh[RED_THREADS];
    const float sr = (float)sc[0], si = (float)sc[1];
    double l = 0.0;
    float fl = 0.0f;
    int c = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 a = A[i], t = __ldg(T + i);
        const float rr = sr * a.x - si * a.y - t.x, ri = sr * a.y + si * a.x - t.y;
        fl += rr * rr + ri * ri;
        if (++c == RED_RUN) {
            l += fl;
            fl = 0.0f;
            c = 0;
        }
        V[i] = make_float2(sr * rr + si * ri, sr * ri - si * rr);
    }
    l = block_sum(sh, l + fl);
    if (threadIdx.x == 0) part[blockIdx.x] = l;
}

// the loss from the nb partial sums (one block)
__global__ void __launch_bounds__(RED_THREADS) k_loss(const double *__restrict__ part, int nb, double *__restrict__ loss)
{
    __shared__ double sh[RED_THREADS];
    double l = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) l += part[b];
    l = block_sum(sh, l);
    if (threadIdx.x == 0) *loss = l;
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
    if (!(pitch > 0.0) || !std::isfinite(pitch) || !std::isfinite(z))
        return internal_fail(HPT_ERR_INVALID_ARG, "pitch must be finite and > 0, z finite");
    for (int l = 0; l < n_lambda; ++l)
        if (!(lambdas[l] > 0.0) || !std::isfinite(lambdas[l]))
            return internal_fail(HPT_ERR_INVALID_ARG, "wavelengths must be finite and > 0");
    OPT_TRY(cudaSetDevice(internal_ctx_device(ctx)));
    OPT_TRY(fft_setup());
    cudaStream_t s = (cudaStream_t)stream;
    const size_t np = (size_t)Wp * Hp;
    const int KB = std::min(K, ASM_BATCH);                 // fields per launch group
    const size_t na = (size_t)KB * Wp * H;
    const size_t bytes = (na + (size_t)n_lambda * np + (size_t)(Wp + Hp)) * sizeof(float2);
    char *buf = nullptr;
    OPT_TRY(cudaMallocAsync((void **)&buf, bytes, s));
    P.A = (float2 *)buf;
    float2 *Hf = P.A + na;
    P.twx = Hf + (size_t)n_lambda * np;
    P.twy = P.twx + Wp;
    cudaError_t e = cudaSuccess;
    k_twiddles<<<(Wp + 255) / 256, 256, 0, s>>>(P.twx, Wp);
    k_twiddles<<<(Hp + 255) / 256, 256, 0, s>>>(P.twy, Hp);
    for (int l = 0; l < n_lambda; ++l)
        k_transfer<<<transfer_grid(Wp, Hp), 256, 0, s>>>(Hf + (size_t)l * np, Wp, Hp, to_df(1.0 / (Wp * pitch)),
                                                              to_df(1.0 / (Hp * pitch)),
                                                              to_df(1.0 / (lambdas[l] * lambdas[l])), to_df(z),
                                                              1.0f / (float)np);
    const float2 *in = (const float2 *)in_dev;
    float2 *out = (float2 *)out_dev;
    for (int l = 0; l < n_lambda && e == cudaSuccess; ++l)
        for (int k = 0; k < K && e == cudaSuccess; k += KB) {
            const size_t fo = ((size_t)l * K + k) * W * H;
            e = asm_field(P, in + fo, out + fo, std::min(KB, K - k), Hf + (size_t)l * np, s);
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
    if (!(pitch > 0.0) || !(lambda > 0.0) || !std::isfinite(pitch) || !std::isfinite(lambda) || !std::isfinite(z) ||
        !std::isfinite(lr))
        return internal_fail(HPT_ERR_INVALID_ARG, "bad pitch, lambda, z or lr");
    AsmPlan P;
    if (!asm_sizes(W, H, P)) return internal_fail(HPT_ERR_UNSUPPORTED, "padded size above 8192 x 8192 (W, H <= 4096)");
    OPT_TRY(cudaSetDevice(internal_ctx_device(ctx)));
    OPT_TRY(fft_setup());
    cudaStream_t s = (cudaStream_t)stream;
    const size_t np = (size_t)P.Wp * P.Hp, n = (size_t)W * H, na = (size_t)P.Wp * H;
    const size_t bytes = (na + 2 * np) * sizeof(float2) + (size_t)(P.Wp + P.Hp) * sizeof(float2) + 3 * n * sizeof(float2) +
                         (3 * RED_BLOCKS + 2 + (size_t)std::max(iters, 1)) * sizeof(double);
    char *buf = nullptr;
    OPT_TRY(cudaMallocAsync((void **)&buf, bytes, s));
    P.A = (float2 *)buf;
    float2 *Hp_ = P.A + na, *Hm = Hp_ + np;          // transfer over +z and over -z (the adjoint)
    P.twx = Hm + np;
    P.twy = P.twx + P.Wp;
    float2 *U = P.twy + P.Hp, *Afield = U + n, *V = Afield + n;
    double *part = (double *)(V + n), *sc = part + 3 * RED_BLOCKS, *dloss = sc + 2;
    const float2 *T = (const float2 *)target_dev;
    k_twiddles<<<(P.Wp + 255) / 256, 256, 0, s>>>(P.twx, P.Wp);
    k_twiddles<<<(P.Hp + 255) / 256, 256, 0, s>>>(P.twy, P.Hp);
    const dim3 tg = transfer_grid(P.Wp, P.Hp);
    const float2 fxu = to_df(1.0 / (P.Wp * pitch)), fyu = to_df(1.0 / (P.Hp * pitch)), il2 = to_df(1.0 / (lambda * lambda));
    k_transfer<<<tg, 256, 0, s>>>(Hp_, P.Wp, P.Hp, fxu, fyu, il2, to_df(z), 1.0f / (float)np);
    k_transfer<<<tg, 256, 0, s>>>(Hm, P.Wp, P.Hp, fxu, fyu, il2, to_df(-z), 1.0f / (float)np);
    cudaError_t e = cudaGetLastError();
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
        k_phase_field<<<grid_for(n), 256, 0, s>>>(phi_dev, U, n);
        e = asm_field(P, U, Afield, 1, Hp_, s);
        if (e != cudaSuccess) break;
        k_dots<<<RED_BLOCKS, RED_THREADS, 0, s>>>(Afield, T, n, part);
        k_scale<<<1, RED_THREADS, 0, s>>>(part, RED_BLOCKS, sc);
        k_residual<<<RED_BLOCKS, RED_THREADS, 0, s>>>(Afield, T, sc, V, n, part);
        k_loss<<<1, RED_THREADS, 0, s>>>(part, RED_BLOCKS, dloss + it);
        e = asm_field(P, V, V, 1, Hm, s);
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
