// Absolute height of the origin site, carried through the updates (growth velocity).
//
// The slopes fix the heights only up to a constant, which the roughness sets by h(0,0) = 0.
// The growth velocity, the rate of change of the absolute mean height <h>, needs one absolute
// height carried along: the origin's, which changes by +2 at each deposition there and by -2
// at each removal (Eq. 1).  With it, <h> = h(0,0) + S1 / N, S1 being the roughness sum.
//
// The update kernels are left as they are.  Instead, before each update launch of K MCS, one
// block re-runs those K MCS on the patch of sites within R = 2K + 2 of the origin (heights
// integrated from the canonical words with the origin at 0), with the same random numbers,
// and adds the origin's height change to a device counter.  A site's update reads its four
// neighbours only, so a wrong value spreads by one site per half-step: the patch's frozen
// edge never reaches the origin in 2K half-steps, and the origin's history is exact.  Patches
// larger than the lattice wrap around it (the periodic lattice unrolled), which is exact for a
// surface since every row and column closes.
#include "sca_internal.h"

namespace sca {

constexpr int kOriginMaxK = 16;                  // MCS per tracked launch, at most
constexpr int kOriginR = 2 * kOriginMaxK + 2;    // patch radius
constexpr int kOriginP = 2 * kOriginR;           // patch side: x, y in [-R, R)
constexpr int kOriginThreads = 1024;

// slope bit d (0: sx-, 1: sy-) of site (x, y) in the canonical words (X sites per row, Y rows)
__device__ __forceinline__ uint32_t origin_slope_bit(const uint32_t *A, uint32_t X, uint32_t Y, uint32_t x,
                                                     uint32_t y, int d)
{
    const uint32_t W = X / 64, s = (x + y) & 1u, k = x >> 1;
    return (A[((size_t)(s * 2 + d) * Y + y) * W + (k >> 5)] >> (k & 31)) & 1u;
}

// Is the flip of site (x, y) of sublattice s at MCS t accepted?  removal: the q side.  The same
// draws as the update kernels: the packed word's xi for dyadic rules, the site's 32-bit
// uniform for per-site rules.
__device__ __forceinline__ bool origin_accept(const Rule &R, uint32_t X, uint32_t x, uint32_t y, int s,
                                              uint64_t t, bool removal)
{
    if (R.mode == 0) return removal ? R.Pq != 0 : R.Pp != 0;
    const uint32_t k = x >> 1;
    if (R.mode == 1) {
        uint32_t xp[1], xq[1];
        xi_dyadic<1>(R, R.rk, (uint64_t)y * (X / 64) + (k >> 5), t, s, xp, xq);
        return (((removal ? xq[0] : xp[0]) >> (k & 31)) & 1u) != 0;
    }
    const uint64_t u = (uint64_t)y * (X / 2) + k;
    const uint32_t r = lane_of(philox4x32_10_rk(draw_counter(u >> 2, t, s, 1, 1), R.rk), (uint32_t)(u & 3));
    const uint64_t T = removal ? R.Tq : R.Tp;
    return (uint64_t)r < T;
}

__global__ void __launch_bounds__(kOriginThreads) k_origin_track(const uint32_t *A, uint32_t X, uint32_t Y,
                                                                 uint64_t t0, uint32_t K, const Rule R,
                                                                 int64_t *h00)
{
    __shared__ int32_t h[kOriginP][kOriginP];     // h[j][i]: site x = i - R, y = j - R
    const int tid = threadIdx.x;
    auto wx = [&](int i) { return (uint32_t)(((int64_t)i - kOriginR + 64 * (int64_t)X) % X); };
    auto wy = [&](int j) { return (uint32_t)(((int64_t)j - kOriginR + 64 * (int64_t)Y) % Y); };
    // heights relative to the origin: along row y = 0, then up and down every column
    if (tid == 0) {
        int32_t v = 0;
        h[kOriginR][kOriginR] = 0;
        for (int i = kOriginR + 1; i < kOriginP; ++i) {
            v += 2 * (int32_t)origin_slope_bit(A, X, Y, wx(i), 0, 0) - 1;
            h[kOriginR][i] = v;
        }
        v = 0;
        for (int i = kOriginR; i > 0; --i) {
            v -= 2 * (int32_t)origin_slope_bit(A, X, Y, wx(i), 0, 0) - 1;
            h[kOriginR][i - 1] = v;
        }
    }
    __syncthreads();
    if (tid < kOriginP) {
        const int i = tid;
        const uint32_t x = wx(i);
        int32_t v = h[kOriginR][i];
        for (int j = kOriginR + 1; j < kOriginP; ++j) {
            v += 2 * (int32_t)origin_slope_bit(A, X, Y, x, wy(j), 1) - 1;
            h[j][i] = v;
        }
        v = h[kOriginR][i];
        for (int j = kOriginR; j > 0; --j) {
            v -= 2 * (int32_t)origin_slope_bit(A, X, Y, x, wy(j), 1) - 1;
            h[j - 1][i] = v;
        }
    }
    __syncthreads();
    // K MCS on the patch (edge sites frozen), even sublattice then odd
    int64_t dh = 0;
    for (uint32_t m = 0; m < K; ++m) {
        for (int s = 0; s < 2; ++s) {
            for (int c = tid; c < (kOriginP - 2) * (kOriginP - 2); c += blockDim.x) {
                const int j = 1 + c / (kOriginP - 2), i = 1 + c % (kOriginP - 2);
                if (((i + j) & 1) != s) continue;        // X, Y even: parity of x + y is that of i + j
                const int32_t v = h[j][i];
                const int32_t a = h[j][i - 1], b = h[j][i + 1], cc = h[j - 1][i], d = h[j + 1][i];
                const bool mn = a == v + 1 && b == v + 1 && cc == v + 1 && d == v + 1;
                const bool mx = a == v - 1 && b == v - 1 && cc == v - 1 && d == v - 1;
                if (!mn && !mx) continue;
                if (origin_accept(R, X, wx(i), wy(j), s, t0 + m, mx)) {
                    h[j][i] = v + (mn ? 2 : -2);
                    if (i == kOriginR && j == kOriginR) dh += mn ? 2 : -2;
                }
            }
            __syncthreads();
        }
    }
    if (tid == (((kOriginP - 2) * (kOriginR - 1) + (kOriginR - 1)) % kOriginThreads)) *h00 += dh;
}

int origin_max_k() { return kOriginMaxK; }

cudaError_t launch_origin_track(const uint32_t *A, uint32_t X, uint32_t Y, uint64_t t0, uint32_t K, const Rule &R,
                                int64_t *h00, cudaStream_t st)
{
    if (K == 0) return cudaSuccess;
    if (K > (uint32_t)kOriginMaxK) return cudaErrorInvalidValue;
    k_origin_track<<<1, kOriginThreads, 0, st>>>(A, X, Y, t0, K, R, h00);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sca
