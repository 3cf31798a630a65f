// Register-wavefront temporal blocking: host side, {0, 1}-probability instantiations and the
// surface check the height-bit representation relies on (kernel in sca_wave.cuh; dyadic
// instantiations in sca_wave_dyadic.cu).
#include "sca.h"
#include "sca_wave.cuh"

namespace sca {

// Dyadic instantiations (other translation unit, compiled in parallel); V words per lane.
cudaError_t launch_wave_dyadic(const WaveArgs &a, int K, int V, int grid, cudaStream_t st);
int wave_dyadic_blocks_per_sm(const Rule &R, int K, int V, uint32_t X, uint32_t Y);
// Per-site uniform instantiations (sca_wave_uniform.cu), one word per lane.
cudaError_t launch_wave_uniform(const WaveArgs &a, int K, int grid, cudaStream_t st);
int wave_uniform_blocks_per_sm(int K);

// Words per lane, when the row length allows four: dyadic draws take four (one Philox call per
// draw for the four words); {0, 1} probabilities take four at 1 or 2 MCS per launch, where the
// launch streams at memory speed: a tile then owns 120 words, whole 32-byte sectors starting on
// a sector, so no sector is written by two tiles (with one word per lane the 30-word tiles
// share edge sectors that L2 evicted half-written and refilled from DRAM: 0.9 GB read per launch
// at L = 65536 against 0.54 GB), and its loads are 16 bytes a lane.  At 4 MCS per launch on rows
// of 1024 words or more they take four too (161 registers against 64, but the launch still moves
// the state once per 4 MCS: 0.17 ms less per benchmark step at L = 65536, whose run to t = 8 is
// one such launch).  Else one.
static int wave_V(uint32_t L, int mode, uint32_t k)
{
    if ((L / 64) % 4 != 0) return 1;
    if (mode == 1) return 4;
    if (mode == 0 && (k <= 2 || (k == 4 && L / 64 >= 1024))) return 4;
    return 1;
}

template <int K, int V, bool DP, bool DQ>
static int blocks_per_sm()
{
    static int n = 0;
    if (n == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, wave01_kernel<K, V, DP, DQ>(), 32 * kWaveWarps, 0) !=
                cudaSuccess || b <= 0)
            b = 1;
        n = b;
    }
    return n;
}

template <int K, int V>
static int blocks_mode0(bool dp, bool dq)
{
    if (dp && dq) return blocks_per_sm<K, V, true, true>();
    if (dp) return blocks_per_sm<K, V, true, false>();
    if (dq) return blocks_per_sm<K, V, false, true>();
    return blocks_per_sm<K, V, false, false>();
}

template <int K, int V>
static cudaError_t launch_mode0(const WaveArgs &a, int grid, cudaStream_t st)
{
    const bool dp = a.R.Pp != 0, dq = a.R.Pq != 0;
    if (dp && dq) wave01_kernel<K, V, true, true>()<<<grid, 32 * kWaveWarps, 0, st>>>(a);
    else if (dp) wave01_kernel<K, V, true, false>()<<<grid, 32 * kWaveWarps, 0, st>>>(a);
    else if (dq) wave01_kernel<K, V, false, true>()<<<grid, 32 * kWaveWarps, 0, st>>>(a);
    else wave01_kernel<K, V, false, false>()<<<grid, 32 * kWaveWarps, 0, st>>>(a);
    return cudaGetLastError();
}

int wave_max_k(int mode) { return mode == 0 ? 16 : mode == 1 ? 4 : mode == 2 ? 2 : 0; }

uint32_t wave_pick_k(uint32_t want, int mode)
{
    uint32_t k = 1;
    const uint32_t cap = (uint32_t)wave_max_k(mode);
    while (2 * k <= want && 2 * k <= cap) k *= 2;
    return cap ? k : 0;
}

static int blocks_for(int K, int V, const Rule &R, uint32_t X, uint32_t Y)
{
    if (R.mode == 1) return wave_dyadic_blocks_per_sm(R, K, V, X, Y);
    if (R.mode == 2) return wave_uniform_blocks_per_sm(K);
    const bool dp = R.Pp != 0, dq = R.Pq != 0;
    switch (K) {
    case 1: return V == 4 ? blocks_mode0<1, 4>(dp, dq) : blocks_mode0<1, 1>(dp, dq);
    case 2: return V == 4 ? blocks_mode0<2, 4>(dp, dq) : blocks_mode0<2, 1>(dp, dq);
    case 4: return V == 4 ? blocks_mode0<4, 4>(dp, dq) : blocks_mode0<4, 1>(dp, dq);
    case 8: return blocks_mode0<8, 1>(dp, dq);
    default: return blocks_mode0<16, 1>(dp, dq);
    }
}

// Bands of rows: enough tiles (warps) for one full wave of resident warps, but bands of at
// least 8K rows so the recomputed halo stays at most half of the streamed rows.  X sites per
// row (the tiles' columns of words), Y rows (the bands).
static bool wave_plan(uint32_t X, uint32_t Y, uint32_t k, int mode, uint32_t bands, int blocks_per_sm,
                      uint32_t *nbands, uint32_t *ncols)
{
    if (X < 64 || X % 64 != 0 || Y < 2 || Y % 2 != 0 || k == 0 || (k & (k - 1)) != 0) return false;
    if ((int)k > wave_max_k(mode)) return false;
    if ((uint64_t)Y * (X / 64) >= (1ull << 32)) return false;   // word indices are 32-bit
    const uint32_t W = X / 64, tw = kWaveTileWords * (uint32_t)wave_V(X, mode, k);
    const uint32_t nc = (W + tw - 1) / tw;
    uint32_t nb = bands;
    if (nb == 0) {
        const uint64_t warps = (uint64_t)sm_count() * blocks_per_sm * kWaveWarps;
        nb = (uint32_t)(warps / nc);            // every tile resident at once: no tail wave
        const uint32_t cap = Y / (8u * k);
        if (nb > cap) nb = cap;
        if (nb == 0) nb = 1;
    }
    if (nb > Y / 2) return false;
    *nbands = nb;
    *ncols = nc;
    return true;
}

#ifndef SCA_WAVE_TAIL_PCT
#define SCA_WAVE_TAIL_PCT 10
#endif
#ifndef SCA_WAVE_TAIL_DIV
#define SCA_WAVE_TAIL_DIV 2
#endif

// Two tiers of bands for the planned one-wave launch of the {0, 1}-probability kernel: warps
// with equal work finish unevenly (an SM quarter's schedulers favour its oldest warps), so the
// first wave's nb bands share all rows but SCA_WAVE_TAIL_PCT percent of them, and bands
// SCA_WAVE_TAIL_DIV times shorter, queued after them, take the rest and start in the slots the
// first finishers free.  10 % in half-height bands: +2.9 % per benchmark step at L = 65536 and
// +3.4 % at L = 131072 (8 % or 12 % of the rows, or third-height bands, lose against it); at
// L <= 32768 the short bands would fall under 8 MCS-lengths of rows and the plan stays one
// tier.  With random draws the kernels run several waves of shorter launches, and a second
// tier lost 1-7 % (p = 1/2), so they keep one tier.
static void wave_tiers(uint32_t Y, uint32_t k, int mode, uint32_t *nb, uint32_t *ntall, uint32_t *ytall)
{
    if (SCA_WAVE_TAIL_PCT <= 0 || mode != 0) return;
    const uint32_t rest = 2u * (uint32_t)((uint64_t)Y * SCA_WAVE_TAIL_PCT / 200u);
    const uint32_t top = Y - rest;
    const uint32_t tall_h = top / *nb, short_h = tall_h / SCA_WAVE_TAIL_DIV;
    if (rest == 0 || short_h < 8u * k || short_h < 2) return;
    const uint32_t nshort = (rest + short_h - 1) / short_h;
    *ntall = *nb;
    *ytall = top;
    *nb += nshort;
}

bool wave_supported(uint32_t L, uint32_t k, int mode) { return wave_supported_xy(L, L, k, mode); }

bool wave_supported_xy(uint32_t X, uint32_t Y, uint32_t k, int mode)
{
    uint32_t nb, nc;
    return wave_plan(X, Y, wave_pick_k(k, mode), mode, 0, 1, &nb, &nc);
}

cudaError_t launch_wave(const uint32_t *src, uint32_t *dst, uint32_t L, uint64_t t0, uint32_t k,
                        const Rule &R, cudaStream_t st, const uint64_t *t_dev, uint32_t bands)
{
    return launch_wave_xy(src, dst, L, L, t0, k, R, st, t_dev, bands);
}

cudaError_t launch_wave_xy(const uint32_t *src, uint32_t *dst, uint32_t X, uint32_t Y, uint64_t t0, uint32_t k,
                           const Rule &R, cudaStream_t st, const uint64_t *t_dev, uint32_t bands, bool sx_all)
{
    const int mode = (int)R.mode;
    uint32_t nb, nc;
    if (!wave_plan(X, Y, k, mode, bands, 1, &nb, &nc)) return cudaErrorInvalidValue;
    const int V = wave_V(X, mode, k);
    if (!wave_plan(X, Y, k, mode, bands, blocks_for((int)k, V, R, X, Y), &nb, &nc)) return cudaErrorInvalidValue;
    uint32_t ntall = nb, ytall = Y;
    if (bands == 0) wave_tiers(Y, k, mode, &nb, &ntall, &ytall);
    // the row a band keeps sx- words for must be one of its final rows: bands of at least
    // 2k + 2 rows (the planner's are at least 8k; an explicit band count may cut shorter ones)
    if (2u * (ytall / 2 / ntall) < 2u * k + 2u) sx_all = true;
    if (nb > ntall && 2u * ((Y - ytall) / 2 / (nb - ntall)) < 2u * k + 2u) sx_all = true;
    const WaveArgs a{src, dst, X, X / 64, Y, nb, nc, ntall, ytall, sx_all ? 1u : 0u, t0, t_dev, R};
    const uint64_t tiles = (uint64_t)nb * nc;
    const int grid = (int)((tiles + kWaveWarps - 1) / kWaveWarps);
    count_launches(1);
    if (mode == 1) return launch_wave_dyadic(a, (int)k, V, grid, st);
    if (mode == 2) return launch_wave_uniform(a, (int)k, grid, st);
    switch (k) {
    case 1: return V == 4 ? launch_mode0<1, 4>(a, grid, st) : launch_mode0<1, 1>(a, grid, st);
    case 2: return V == 4 ? launch_mode0<2, 4>(a, grid, st) : launch_mode0<2, 1>(a, grid, st);
    case 4: return V == 4 ? launch_mode0<4, 4>(a, grid, st) : launch_mode0<4, 1>(a, grid, st);
    case 8: return launch_mode0<8, 1>(a, grid, st);
    case 16: return launch_mode0<16, 1>(a, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------------------ surface check
// A state is a surface when every plaquette closes and the slopes sum to zero around the torus
// along row 0 and column 0 (then along every row and column).  For the plaquette with corners
// (x-1, y-1) and (x, y): sx-(x, y) - sx-(x, y-1) == sy-(x, y) - sy-(x-1, y), i.e. with slope
// bits a, b, c, d: a + d == b + c.  One thread per canonical word of sublattice s, row y; Y rows
// of W words per sublattice.
__global__ void k_surface_check(const uint32_t *A, uint32_t Y, uint32_t W, uint32_t *out)
{
    const size_t plane = (size_t)Y * W;
    const size_t n = 2 * plane;
    for (size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += (size_t)gridDim.x * blockDim.x) {
        const uint32_t s = (uint32_t)(w / plane);
        const size_t rem = w - (size_t)s * plane;
        const uint32_t y = (uint32_t)(rem / W), j = (uint32_t)(rem - (size_t)y * W);
        const uint32_t ns = s ^ 1u, yp = y == 0 ? Y - 1 : y - 1, jp = j == 0 ? W - 1 : j - 1;
        const uint32_t *SXs = A + (size_t)(2 * s) * plane, *SYs = A + (size_t)(2 * s + 1) * plane;
        const uint32_t *SXn = A + (size_t)(2 * ns) * plane, *SYn = A + (size_t)(2 * ns + 1) * plane;
        const uint32_t a = SXs[(size_t)y * W + j];
        const uint32_t b = SXn[(size_t)yp * W + j];
        const uint32_t c = SYs[(size_t)y * W + j];
        const uint32_t dn = SYn[(size_t)y * W + j];
        // the site left of x is bit k of the other sublattice when this row sits right
        // ((s + y) odd), else bit k - 1
        const uint32_t d = ((s + y) & 1u) ? dn : __funnelshift_l(SYn[(size_t)y * W + jp], dn, 1);
        const uint32_t bad = ((a ^ d) ^ (b ^ c)) | ((a & d) ^ (b & c));
        if (bad) atomicOr(out, 1u);
        if (y == 0) atomicAdd(out + 1, (uint32_t)__popc(a));
        if (j == 0 && s == (y & 1u)) atomicAdd(out + 2, c & 1u);
    }
}

// Row 0 holds X/2 sx- ones and column 0 Y/2 sy- ones when both close.
bool surface_from(const uint32_t *h, uint32_t X, uint32_t Y) { return h[0] == 0 && h[1] == X / 2 && h[2] == Y / 2; }

cudaError_t surface_check_async(const uint32_t *A, uint32_t X, uint32_t Y, uint32_t *scratch, uint32_t *host3,
                                cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(scratch, 0, 3 * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const uint32_t W = X / 64;
    const size_t n = 2 * (size_t)Y * W;
    int grid = (int)((n + 255) / 256);
    if (grid > sm_count() * 8) grid = sm_count() * 8;
    k_surface_check<<<grid, 256, 0, st>>>(A, Y, W, scratch);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(host3, scratch, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
}

cudaError_t surface_check(const uint32_t *A, uint32_t X, uint32_t Y, uint32_t *scratch, cudaStream_t st,
                          bool *is_surface)
{
    cudaError_t e = cudaMemsetAsync(scratch, 0, 3 * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const uint32_t W = X / 64;
    const size_t n = 2 * (size_t)Y * W;
    int grid = (int)((n + 255) / 256);
    if (grid > sm_count() * 8) grid = sm_count() * 8;
    k_surface_check<<<grid, 256, 0, st>>>(A, Y, W, scratch);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint32_t h[3];
    e = cudaMemcpyAsync(h, scratch, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *is_surface = surface_from(h, X, Y);
    return cudaSuccess;
}

}  // namespace sca

// ------------------------------------------------------------------------- logic-rate probe
// Issue rate of 32-bit three-input logic instructions (the unit the height-bit update is bound
// by) on this GPU: every thread runs eight independent LOP3 chains, every SM is filled.
namespace sca {

__global__ void __launch_bounds__(256) k_logic_rate(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    uint32_t a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed * (threadIdx.x + 1u) + (uint32_t)k;
    const uint32_t b = seed ^ threadIdx.x, c = ~seed + blockIdx.x;
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) asm("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[k]) : "r"(b), "r"(c));
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) x ^= a[k];
    if (x == 0x9E3779B9u) *sink = x;      // keeps the chains live; practically never taken
}

// Issue rate of 32 x 32 -> 64-bit multiplies (the product a Philox round takes twice): eight
// independent chains per thread, each step d = lo(d) * M + d in one wide multiply-add.
__global__ void __launch_bounds__(256) k_mul_rate(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    uint64_t d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) d[k] = (uint64_t)(seed * (threadIdx.x + 1u) + (uint32_t)k) << 7;
    const uint32_t M = 0xD2511F53u ^ (seed & 0xF0u);
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k)
                asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(d[k]) : "r"((uint32_t)d[k]), "r"(M));
    }
    uint64_t x = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) x ^= d[k];
    if ((uint32_t)x == 0x9E3779B9u) *sink = (uint32_t)(x >> 32);
}

// Philox4x32-10 calls per second as the update kernels compute them (philox4x32_10_rk with the
// round keys in kernel parameters): four independent counters per thread and iteration.
struct PhiloxKeys { uint32_t rk[20]; };
__global__ void __launch_bounds__(256) k_philox_rate(uint32_t iters, PhiloxKeys K, uint32_t *sink)
{
    uint32_t acc = 0;
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const Ctr4 o = philox4x32_10_rk(Ctr4{g, i, (uint32_t)c, 0u}, K.rk);
            acc ^= o.x ^ o.y ^ o.z ^ o.w;
        }
    }
    if (acc == 0x9E3779B9u) *sink = acc;
}

}  // namespace sca

// Multiply-pipe and Philox rates (see sca.h).
extern "C" int sca_measure_mul_rate(double *wide_mul_per_s, double *philox_calls_per_s)
{
    using namespace sca;
    if (!wide_mul_per_s || !philox_calls_per_s) return fail(SCA_EINVAL, "NULL argument");
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    uint32_t *sink = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventCreate(&e2);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(uint32_t));
    PhiloxKeys K;
    for (int r = 0; r < 10; ++r) {
        K.rk[2 * r] = 0x1234567u + (uint32_t)r * 0x9E3779B9u;
        K.rk[2 * r + 1] = 0x89ABCDEu + (uint32_t)r * 0xBB67AE85u;
    }
    const uint32_t blocks = (uint32_t)sm_count() * 8u, threads = 256u, iters_m = 8000u, iters_p = 8000u;
    float ms_m = 0.f, ms_p = 0.f;
    if (e == cudaSuccess) {
        k_mul_rate<<<blocks, threads, 0, st>>>(100u, 0x1234567u, sink);       // warm-up
        k_philox_rate<<<blocks, threads, 0, st>>>(20u, K, sink);
        count_launches(2);
        e = cudaEventRecord(e0, st);
    }
    if (e == cudaSuccess) {
        k_mul_rate<<<blocks, threads, 0, st>>>(iters_m, 0x7654321u, sink);
        k_philox_rate<<<blocks, threads, 0, st>>>(1u, K, sink);               // keeps e1 after e0's work
        count_launches(2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) {
        k_philox_rate<<<blocks, threads, 0, st>>>(iters_p, K, sink);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e2, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e2);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_m, e0, e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_p, e1, e2);
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e2) cudaEventDestroy(e2);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return cuda_fail(e, "multiply-rate probe");
    *wide_mul_per_s = (double)blocks * threads * iters_m * 128.0 / (ms_m * 1e-3);
    *philox_calls_per_s = (double)blocks * threads * iters_p * 4.0 / (ms_p * 1e-3);
    return SCA_OK;
}

extern "C" int sca_measure_logic_rate(double *ops_per_s)
{
    using namespace sca;
    if (!ops_per_s) return fail(SCA_EINVAL, "NULL argument");
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    uint32_t *sink = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(uint32_t));
    const uint32_t blocks = (uint32_t)sm_count() * 8u, threads = 256u, iters = 20000u;
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_logic_rate<<<blocks, threads, 0, st>>>(200u, 0x1234567u, sink);     // warm-up
        count_launches(1);
        e = cudaEventRecord(e0, st);
    }
    if (e == cudaSuccess) {
        k_logic_rate<<<blocks, threads, 0, st>>>(iters, 0x7654321u, sink);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return cuda_fail(e, "logic-rate probe");
    *ops_per_s = (double)blocks * threads * iters * 128.0 / (ms * 1e-3);
    return SCA_OK;
}
