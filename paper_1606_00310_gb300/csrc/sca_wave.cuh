// Register-wavefront temporal blocking on height bits (kernel template; host code in
// sca_wave.cu).
//
// Representation.  The canonical words hold two slope bits per site (Sec. II.B).  In the
// octahedron model every slope is +-1 and h(x, y) has the parity of x + y, so h mod 4 is one
// bit per site: b = ((h - ((x + y) & 1)) / 2) mod 2.  For a site of parity s and a neighbour n
// the slope h(n) - h(x) is +1 exactly when b(n) xor b(x) == s, so the local-minimum condition
// of Eq. (2) (all four neighbours one higher) is "b xor b(n) == s for all four neighbours",
// the local maximum of Eq. (3) is "== 1 - s for all four", and an update (h += 2 or h -= 2)
// flips b alone.  Inside the kernel the state is therefore one height-bit word per sublattice
// per row; a half-step reads the other sublattice's words of rows r-1, r, r+1 and writes only
// its own word of row r.  The conversion is exact for a surface (every plaquette closes):
// loading a row needs only its sy- words, b(x, y) = b(x, y-1) xor sy-bit(x, y) xor s, after
// the first row of a tile has been integrated along x (a prefix xor across the warp); storing
// a row recovers all four canonical slope words from b and its left and upper neighbours.
//
// Wavefront.  Half-step i at row r needs half-step i-1 at rows r-1, r, r+1, so one warp
// streams a band of rows: when row R arrives, half-step 1 runs on row R-1, ..., half-step 2K
// on row R-2K, and row R-2K is final for all K MCS.  The 2K+2 live rows stay in registers; the
// loop is unrolled by the window length so every row slot is a fixed register, and because the
// half-step index and the row advance together, all half-steps of one position agree on which
// side the shifted x-neighbour word comes from (a compile-time fact after unrolling).
//
// Tiles.  Lane l of a warp owns one packed word of every row of its band; lanes 0 and 31 hold
// halo words (the x light cone grows by at most one bit per half-step, so one word on each side
// covers K <= 16) and bands carry 2K + 2 halo rows above and 2K below.  Halos are recomputed by the
// neighbouring tiles from the same counter-based random bits, so tiles never communicate;
// they read the source buffer and write only their own words of the destination buffer.
#pragma once
#include "sca_internal.h"

namespace sca {

struct WaveArgs {
    const uint32_t *src;
    uint32_t *dst;
    uint32_t L, W;
    uint32_t nbands, ncols;  // tiles: bands of rows x columns of words
    uint64_t t0;             // MCS index of the first step, or offset from *t_dev
    const uint64_t *t_dev;
    Rule R;
};

constexpr int kWaveWarps = 4;          // warps (independent tiles) per CTA
constexpr int kWaveRaw = 3;            // rows of sy- words loaded ahead of the wavefront
constexpr uint32_t kWaveTileWords = 30; // words a warp tile owns (32 lanes minus two halos)

__device__ __forceinline__ uint32_t wave_xor_prefix(uint32_t g)
{
    g ^= g << 1;
    g ^= g << 2;
    g ^= g << 4;
    g ^= g << 8;
    g ^= g << 16;
    return g;
}

// MODE 0: p, q in {0, 1} with DP = (p == 1), DQ = (q == 1); MODE 1: dyadic draws.
template <int K, int MODE, bool DP, bool DQ>
__global__ void __launch_bounds__(32 * kWaveWarps) k_wave(const WaveArgs a)
{
    constexpr int S = 2 * K;                                // half-steps per launch
    constexpr int NH = ((S + 2 + 2 * kWaveRaw - 1) / (2 * kWaveRaw)) * (2 * kWaveRaw);  // rows of height bits
    constexpr int NRAW = kWaveRaw;
    static_assert(NH % 2 == 0 && NH % NRAW == 0 && NH >= S + 2, "window");
    const uint32_t FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const uint32_t tile = blockIdx.x * kWaveWarps + threadIdx.x / 32;
    if (tile >= a.nbands * a.ncols) return;
    const uint32_t band = tile / a.ncols, col = tile - band * a.ncols;
    const uint32_t L = a.L, W = a.W;
    // band rows [y0, y1), y0 even: the first streamed row is even, so band-row parity is
    // lattice-row parity
    const uint32_t y0 = 2u * (uint32_t)(((uint64_t)band * (L / 2)) / a.nbands);
    const uint32_t y1 = 2u * (uint32_t)(((uint64_t)(band + 1) * (L / 2)) / a.nbands);
    // halo: 2K rows below, 2K + 2 above (the top row's sy- words need the row above it, and
    // the first streamed row stays even)
    const uint32_t NR = y1 - y0 + 4u * K + 2u;
    const uint32_t first = (y0 + 2u * L - 2u * K - 2u) % L;
    const size_t plane = (size_t)L * W;
    const uint32_t *SX0 = a.src, *SY0 = a.src + plane, *SX1 = a.src + 2 * plane, *SY1 = a.src + 3 * plane;
    uint32_t *DX0 = a.dst, *DY0 = a.dst + plane, *DX1 = a.dst + 2 * plane, *DY1 = a.dst + 3 * plane;
    const uint64_t t0 = a.t_dev ? *a.t_dev + a.t0 : a.t0;

    const int64_t jj = (int64_t)col * kWaveTileWords - 1 + lane;
    const uint32_t j = (uint32_t)(((jj % (int64_t)W) + W) % (int64_t)W);
    const bool own = lane >= 1 && lane <= 30 && jj < (int64_t)W;

    uint32_t h[NH][2];              // height bits, row slot = band row mod NH, [sublattice]
    uint32_t raw[NRAW][2];          // sy- words of rows loaded ahead, slot = band row mod NRAW
#pragma unroll
    for (int i = 0; i < NH; ++i) h[i][0] = h[i][1] = 0u;

    // First row (even lattice row: sublattice 0 at even x): integrate along x.  With e(x) =
    // b(x) xor b(x-1) = sx-bit(x) xor (x & 1), the even-x bits obey b_e(k) = b_e(k-1) xor
    // ~sx1(k-1) xor sx0(k); the prefix xor runs over the whole warp (lane 0's reference bit is
    // arbitrary: flipping every bit of a connected region changes no slope).
    {
        const size_t o = (size_t)first * W + j;
        const uint32_t sx0 = __ldg(SX0 + o), nsx1 = ~__ldg(SX1 + o);
        const uint32_t prev = __shfl_up_sync(FULL, nsx1, 1);
        uint32_t pre = wave_xor_prefix(sx0 ^ __funnelshift_l(prev, nsx1, 1));
        uint32_t par = pre >> 31, incl = par;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl ^= t;
        }
        pre ^= 0u - (incl ^ par);
        h[0][0] = pre;
        h[0][1] = pre ^ nsx1;
    }
    uint32_t yl = first + 1 >= L ? first + 1 - L : first + 1;     // next row to load
#pragma unroll
    for (int d = 1; d <= NRAW; ++d) {
        if ((uint32_t)d < NR) {
            raw[d % NRAW][0] = __ldg(SY0 + (size_t)yl * W + j);
            raw[d % NRAW][1] = __ldg(SY1 + (size_t)yl * W + j);
        }
        if (++yl == L) yl = 0;
    }
    uint32_t yu = first;                                          // lattice row of row R

    for (uint32_t R0 = 0; R0 < NR; R0 += NH) {
#pragma unroll
        for (int u = 0; u < NH; ++u) {
            const uint32_t R = R0 + (uint32_t)u;
            if (R >= NR) break;
            if (R > 0) {
                // b(x, y) = b(x, y-1) xor sy-bit(x, y) xor s (sites of sublattice s have parity s)
                uint32_t(&hr)[2] = h[u];
                const uint32_t(&hp)[2] = h[(u + NH - 1) % NH];
                hr[0] = hp[1] ^ raw[u % NRAW][0];
                hr[1] = ~(hp[0] ^ raw[u % NRAW][1]);
                if (R + NRAW < NR) {
                    raw[u % NRAW][0] = __ldg(SY0 + (size_t)yl * W + j);
                    raw[u % NRAW][1] = __ldg(SY1 + (size_t)yl * W + j);
                }
                if (++yl == L) yl = 0;
            }
            // rows of sublattice s at parity (s + y) & 1 == 1 sit one site right; for every
            // half-step of this position (s + y) & 1 == (R + 1) & 1
            const bool right_shift = ((u + 1) & 1) != 0;
#pragma unroll
            for (int i = 1; i <= S; ++i) {
                const int s = (i - 1) & 1, ns = s ^ 1;
                uint32_t &b = h[(u - i + 2 * NH) % NH][s];
                const uint32_t up = h[(u - i - 1 + 2 * NH) % NH][ns];
                const uint32_t dn = h[(u - i + 1 + 2 * NH) % NH][ns];
                const uint32_t mid = h[(u - i + 2 * NH) % NH][ns];
                uint32_t side;
                if (right_shift) side = __funnelshift_r(mid, __shfl_down_sync(FULL, mid, 1), 1);
                else side = __funnelshift_l(__shfl_up_sync(FULL, mid, 1), mid, 1);
                // e(n) = b xor b(n) for the four neighbours
                const uint32_t e_or = (b ^ up) | (b ^ dn) | (b ^ mid) | (b ^ side);
                const uint32_t e_and = (b ^ up) & (b ^ dn) & (b ^ mid) & (b ^ side);
                // local minimum: every e == s; local maximum: every e == 1 - s
                const uint32_t is_min = s == 0 ? ~e_or : e_and;
                const uint32_t is_max = s == 0 ? e_and : ~e_or;
                uint32_t m;
                if constexpr (MODE == 0) {
                    m = (DP ? is_min : 0u) | (DQ ? is_max : 0u);
                } else {
                    const uint32_t y = (yu + 2 * L - (uint32_t)i) % L;
                    uint32_t xp[1], xq[1];
                    xi_dyadic<1>(a.R, a.R.rk, (uint64_t)y * W + j, t0 + (uint32_t)((i - 1) >> 1), s, xp, xq);
                    m = (xp[0] & is_min) | (xq[0] & is_max);
                }
                b ^= m;
            }
            if (R >= 4u * K + 2u) {                 // band row R - 2K (lattice row y) is final
                const uint32_t(&hr)[2] = h[(u - S + 2 * NH) % NH];
                const uint32_t(&hp)[2] = h[(u - S - 1 + 2 * NH) % NH];
                const uint32_t y = y0 + R - 4u * K - 2u;
                // sy-bit = b xor b(x, y-1) xor s and sx-bit = b xor b(x-1, y) xor s.  In even
                // rows sublattice 0 sits at even x, so its left neighbour is bit k-1 of the
                // sublattice-1 word and sublattice 1's is bit k of the sublattice-0 word; odd
                // rows the other way round (y has the parity of u).
                const uint32_t sy0 = hr[0] ^ hp[1], sy1 = ~(hr[1] ^ hp[0]);
                uint32_t sx0, sx1;
                if ((u & 1) == 0) {
                    sx0 = hr[0] ^ __funnelshift_l(__shfl_up_sync(FULL, hr[1], 1), hr[1], 1);
                    sx1 = ~(hr[1] ^ hr[0]);
                } else {
                    sx0 = hr[0] ^ hr[1];
                    sx1 = ~(hr[1] ^ __funnelshift_l(__shfl_up_sync(FULL, hr[0], 1), hr[0], 1));
                }
                if (own) {
                    const size_t o = (size_t)y * W + j;
                    DX0[o] = sx0;
                    DY0[o] = sy0;
                    DX1[o] = sx1;
                    DY1[o] = sy1;
                }
            }
            if (++yu == L) yu = 0;
        }
    }
}

}  // namespace sca
