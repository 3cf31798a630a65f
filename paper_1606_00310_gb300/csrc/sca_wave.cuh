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
// on row R-2K, and row R-2K is final for all K MCS.  The live rows stay in registers: the row
// loop is unrolled by a block of U rows, so every row slot is a fixed register, and the window
// slides by U slots after each block.  Because the half-step index and the row advance
// together, all half-steps of one position agree on which side the shifted x-neighbour word
// comes from (a compile-time fact after unrolling).
//
// Tiles.  Lane l of a warp owns V consecutive packed words of every row of its band (V = 1, or
// 4 where one Philox call serves four words or the launch streams at memory speed); lanes 0 and
// 31 hold halo words (the x light cone grows by at most one bit per half-step, so one word on
// each side covers K <= 16) and bands carry 2K + 2 halo rows above and 2K below.  Halos are
// recomputed by the neighbouring tiles from the same counter-based random bits, so tiles never
// communicate; they read the source buffer and write only their own words of the destination.
#pragma once
#include "sca_internal.h"

namespace sca {

struct WaveArgs {
    const uint32_t *src;
    uint32_t *dst;
    uint32_t L, W;           // sites per row (X) and words per sublattice row
    uint32_t Y;              // rows
    uint32_t nbands, ncols;  // tiles: bands of rows x columns of words
    uint32_t ntall, ytall;   // the first ntall bands share rows [0, ytall), the rest [ytall, Y)
    uint32_t sx_all;         // 0: sx- planes only on each band's row y1 - 2K - 2 (see below)
    uint64_t t0;             // MCS index of the first step, or offset from *t_dev
    const uint64_t *t_dev;
    Rule R;
};

// Warps (independent tiles) per CTA: one.  The register file then fills warp by warp rather
// than four warps at a time, and with a 32-thread launch bound the compiler fits the 16-MCS
// {0, 1}-probability instantiation in 128 registers (16 warps per SM) where 128-thread CTAs got
// 150 (12 warps per SM).
constexpr int kWaveWarps = 1;
constexpr uint32_t kWaveTileWords = 30; // words a warp tile owns (32 lanes minus two halos)
// Rows per loop iteration (even): larger blocks shift the row window less often, smaller ones
// keep the unrolled loop inside the instruction cache; the dyadic update carries a Philox
// call per half-step, so it takes the smaller block.
#ifndef SCA_WAVE_U0
#define SCA_WAVE_U0 4
#endif
#ifndef SCA_WAVE_U1
#define SCA_WAVE_U1 2
#endif
#ifndef SCA_WAVE_MINB
#define SCA_WAVE_MINB 16
#endif
#ifndef SCA_WAVE_P0
#define SCA_WAVE_P0 SCA_WAVE_U0
#endif
constexpr int kWaveU0 = SCA_WAVE_U0;   // {0, 1} probabilities
constexpr int kWaveU1 = SCA_WAVE_U1;   // dyadic draws

// Prefetch distance in rows (the sy- ring's entries) for U rows per block: a divisor of U, so
// that the ring entry of every row of a block is a compile-time index.
__host__ __device__ constexpr int wave_ring(int U, int MODE) { return MODE == 0 ? SCA_WAVE_P0 : U; }
static_assert(SCA_WAVE_U0 % SCA_WAVE_P0 == 0, "the ring length divides the rows per block");

// Resident CTAs per SM the compiler must allow.  The 16-MCS {0, 1}-probability kernel is held to
// 128 registers, 16 warps per SM: it then takes 124, and runs 11 % faster than with no bound (96
// registers, 20 warps per SM) or a bound of 20.  The others get 0, no bound: even a bound of 1
// changes the compiler's register choice for them.
__host__ __device__ constexpr int wave_min_blocks(int K, int V, int MODE)
{
    return (MODE == 0 && V == 1 && K == 16) ? SCA_WAVE_MINB : 0;
}

// Three-input bitwise function given by its truth table (bit 4a + 2b + c of LUT is f(a, b, c)).
template <uint32_t LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
}

__device__ __forceinline__ uint32_t wave_xor_prefix(uint32_t g)
{
    g ^= g << 1;
    g ^= g << 2;
    g ^= g << 4;
    g ^= g << 8;
    g ^= g << 16;
    return g;
}

template <int V>
__device__ __forceinline__ void wave_ld(const uint32_t *p, uint32_t (&r)[V])
{
    if constexpr (V == 4) {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
        r[0] = q.x; r[1 % V] = q.y; r[2 % V] = q.z; r[3 % V] = q.w;
    } else if constexpr (V == 2) {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p));
        r[0] = q.x; r[1 % V] = q.y;
    } else {
        r[0] = __ldg(p);
    }
}

template <int V>
__device__ __forceinline__ void wave_st(uint32_t *p, const uint32_t (&r)[V])
{
    if constexpr (V == 4) *reinterpret_cast<uint4 *>(p) = make_uint4(r[0], r[1 % V], r[2 % V], r[3 % V]);
    else if constexpr (V == 2) *reinterpret_cast<uint2 *>(p) = make_uint2(r[0], r[1 % V]);
    else *p = r[0];
}

// Philox key sources: the rule's precomputed round keys (one lattice per launch, kernel
// parameters) or a key pair per lane group (many lattices per warp), schedule computed inline.
struct KeysRk {
    const uint32_t *rk;
    __device__ __forceinline__ Ctr4 operator()(Ctr4 c) const { return philox4x32_10_rk(c, rk); }
};
struct KeysLane {
    uint32_t k0, k1;
    __device__ __forceinline__ Ctr4 operator()(Ctr4 c) const { return philox4x32_10(c, k0, k1); }
};

// Dyadic xi words (Sec. III construction, as xi_dyadic) for V words starting at word unit u0,
// where u0 is a multiple of 4 when V == 4 (one Philox call per draw gives all four words).
template <int V, class KEYS>
__device__ __forceinline__ void wave_xi(const Rule &R, const KEYS &key, uint64_t u0, uint64_t t, int s, uint32_t (&xp)[V],
                                        uint32_t (&xq)[V])
{
#pragma unroll
    for (int v = 0; v < V; ++v) {
        xp[v] = (R.np == 0 && R.Pp) ? 0xFFFFFFFFu : 0u;
        xq[v] = (R.nq == 0 && R.Pq) ? 0xFFFFFFFFu : 0u;
    }
#pragma unroll 1
    for (int i = (int)R.n_draws; i >= 1; --i) {
        uint32_t r[V];
        if constexpr (V == 4) {
            const Ctr4 o = key(draw_counter(u0 >> 2, t, s, i, 0));
            r[0] = o.x; r[1 % V] = o.y; r[2 % V] = o.z; r[3 % V] = o.w;
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const uint64_t u = u0 + v;
                r[v] = lane_of(key(draw_counter(u >> 2, t, s, i, 0)), (uint32_t)(u & 3));
            }
        }
        if (i <= (int)R.np) {
            const bool first = (i == (int)R.np);
            const bool bit = (R.Pp >> (R.np - i)) & 1u;
#pragma unroll
            for (int v = 0; v < V; ++v) xp[v] = first ? r[v] : (bit ? (r[v] | xp[v]) : (r[v] & xp[v]));
        }
        if (i <= (int)R.nq) {
            const bool first = (i == (int)R.nq);
            const bool bit = (R.Pq >> (R.nq - i)) & 1u;
#pragma unroll
            for (int v = 0; v < V; ++v) xq[v] = first ? r[v] : (bit ? (r[v] | xq[v]) : (r[v] & xq[v]));
        }
    }
}

// The same construction with the number of draws ND fixed at compile time, so the ND Philox
// chains are independent straight-line code the scheduler interleaves; DP / DQ false when
// p / q is exactly 0 (that word is then 0 and its test drops out of the update).
template <int V, int ND, bool DP, bool DQ, class KEYS>
__device__ __forceinline__ void wave_xi_fixed(const Rule &R, const KEYS &key, uint64_t u0, uint64_t t, int s,
                                              uint32_t (&xp)[V], uint32_t (&xq)[V])
{
#pragma unroll
    for (int v = 0; v < V; ++v) {
        xp[v] = (R.np == 0 && R.Pp) ? 0xFFFFFFFFu : 0u;
        xq[v] = (R.nq == 0 && R.Pq) ? 0xFFFFFFFFu : 0u;
    }
#pragma unroll
    for (int i = ND; i >= 1; --i) {
        uint32_t r[V];
        if constexpr (V == 4) {
            const Ctr4 o = key(draw_counter(u0 >> 2, t, s, i, 0));
            r[0] = o.x; r[1 % V] = o.y; r[2 % V] = o.z; r[3 % V] = o.w;
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const uint64_t u = u0 + v;
                r[v] = lane_of(key(draw_counter(u >> 2, t, s, i, 0)), (uint32_t)(u & 3));
            }
        }
        if (DP && i <= (int)R.np) {
            const bool first = (i == (int)R.np);
            const bool bit = (R.Pp >> (R.np - i)) & 1u;
#pragma unroll
            for (int v = 0; v < V; ++v) xp[v] = first ? r[v] : (bit ? (r[v] | xp[v]) : (r[v] & xp[v]));
        }
        if (DQ && i <= (int)R.nq) {
            const bool first = (i == (int)R.nq);
            const bool bit = (R.Pq >> (R.nq - i)) & 1u;
#pragma unroll
            for (int v = 0; v < V; ++v) xq[v] = first ? r[v] : (bit ? (r[v] | xq[v]) : (r[v] & xq[v]));
        }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        if (!DP) xp[v] = 0u;
        if (!DQ) xq[v] = 0u;
    }
}

// One site word after a half-step of its sublattice s (Eqs. 2 and 3 in height bits): with
// e(n) = b xor b(n) for the four neighbours, a site is a local minimum when every e == s and a
// local maximum when every e == 1 - s; xp / xq gate deposition / removal (MODE 0: DP / DQ).
template <int MODE, bool DP, bool DQ>
__device__ __forceinline__ uint32_t wave_update(uint32_t b, uint32_t up, uint32_t dn, uint32_t mid, uint32_t side,
                                                int s, uint32_t xp, uint32_t xq)
{
    if constexpr (MODE == 0 && DP != DQ) {
        // one kind of flip in three three-input operations: the flip set is "every e == 0" (the
        // OR of the e's is 0) or "every e == 1" (their AND is 1); minima of even sites and
        // maxima of odd sites are the first kind
        if ((s == 0) == DP) {
            const uint32_t t1 = lop3<0x7E>(b, up, dn);       // (b ^ up) | (b ^ dn)
            const uint32_t t2 = lop3<0x7E>(b, mid, side);    // (b ^ mid) | (b ^ side)
            return lop3<0xE1>(b, t1, t2);                    // b ^ ~(t1 | t2)
        } else {
            const uint32_t t1 = lop3<0x18>(b, up, dn);       // (b ^ up) & (b ^ dn)
            const uint32_t t2 = lop3<0x18>(b, mid, side);    // (b ^ mid) & (b ^ side)
            return lop3<0x78>(b, t1, t2);                    // b ^ (t1 & t2)
        }
    } else if constexpr (MODE == 1) {
        // with draws: "every e == 0" as ~(t1o | t2o), "every e == 1" as t1a & t2a (three-input
        // ops), gated by the draw words; minima are the first kind on even sites.  Written as
        // plain C the compiler took more operations (p = q = 1/2: 1.85e13 against 1.98e13,
        // p = 3/4, q = 1/4: 1.19e13 against 1.26e13 at L = 65536)
        const bool min_is_or = s == 0;
        if constexpr (DP != DQ) {
            const uint32_t x = DP ? xp : xq;
            const bool gate_or = min_is_or == DP;        // the flip set is "every e == 0"
            if (gate_or) {
                const uint32_t t1 = lop3<0x7E>(b, up, dn), t2 = lop3<0x7E>(b, mid, side);
                return b ^ lop3<0x10>(x, t1, t2);        // x & ~t1 & ~t2
            } else {
                const uint32_t t1 = lop3<0x18>(b, up, dn), t2 = lop3<0x18>(b, mid, side);
                return b ^ lop3<0x80>(x, t1, t2);        // x & t1 & t2
            }
        } else {
            const uint32_t t1o = lop3<0x7E>(b, up, dn), t2o = lop3<0x7E>(b, mid, side);
            const uint32_t t1a = lop3<0x18>(b, up, dn), t2a = lop3<0x18>(b, mid, side);
            const uint32_t g_or = lop3<0x10>(min_is_or ? xp : xq, t1o, t2o);
            const uint32_t g_and = lop3<0x80>(min_is_or ? xq : xp, t1a, t2a);
            return lop3<0x1E>(b, g_or, g_and);           // b ^ (g_or | g_and)
        }
    } else {
        const uint32_t e_or = (b ^ up) | (b ^ dn) | (b ^ mid) | (b ^ side);
        const uint32_t e_and = (b ^ up) & (b ^ dn) & (b ^ mid) & (b ^ side);
        const uint32_t is_min = s == 0 ? ~e_or : e_and;
        const uint32_t is_max = s == 0 ? e_and : ~e_or;
        uint32_t m;
        if constexpr (MODE == 0) m = (DP ? is_min : 0u) | (DQ ? is_max : 0u);
        else m = (xp & is_min) | (xq & is_max);
        return b ^ m;
    }
}

// The 2K half-steps of the wavefront when row R arrives in slot S + 1 + u: half-step i on row
// R - i (slot S + 1 + u - i).  yu is the lattice row of row R (used by the random draws).
template <int K, int V, int U, int MODE, bool DP, bool DQ, int ND>
__device__ __forceinline__ void wave_half_steps(const Rule &Rl, uint32_t (&h)[2 * K + 1 + U][2][V], const int u,
                                                const uint32_t yu, const uint32_t L, const uint32_t Y,
                                                const uint32_t W, const uint32_t j, const uint64_t t0)
{
    constexpr int S = 2 * K;
    constexpr int base = S + 1;
    const uint32_t FULL = 0xFFFFFFFFu;
    // rows of sublattice s at parity (s + y) & 1 == 1 sit one site right; for every half-step
    // of this position (s + y) & 1 == (R + 1) & 1, and the first row of a block is even
    const bool right_shift = ((u + 1) & 1) != 0;
#pragma unroll
    for (int i = 1; i <= S; ++i) {
        const int s = (i - 1) & 1, ns = s ^ 1;
        const int c = base + u - i;             // slot of row R - i
        uint32_t(&b)[V] = h[c][s];
        const uint32_t(&up)[V] = h[c - 1][ns];
        const uint32_t(&dn)[V] = h[c + 1][ns];
        const uint32_t(&mid)[V] = h[c][ns];
        // the x-neighbour that is not in the same bit position: bit k+1 of the other
        // sublattice when this row sits right, else bit k-1
        uint32_t side[V];
        if (right_shift) {
            const uint32_t nx = __shfl_down_sync(FULL, mid[0], 1);
#pragma unroll
            for (int v = 0; v < V; ++v)
                side[v] = __funnelshift_r(mid[v], v + 1 < V ? mid[(v + 1) % V] : nx, 1);
        } else {
            const uint32_t pv = __shfl_up_sync(FULL, mid[V - 1], 1);
#pragma unroll
            for (int v = 0; v < V; ++v)
                side[v] = __funnelshift_l(v ? mid[(v + V - 1) % V] : pv, mid[v], 1);
        }
        uint32_t xp[V] = {}, xq[V] = {};
        if constexpr (MODE == 2) {
            // one 32-bit uniform per site (Sec. II.B), four sites per Philox call
            const uint32_t y = yu >= (uint32_t)i ? yu - (uint32_t)i : yu + Y - (uint32_t)i;
#pragma unroll
            for (int v = 0; v < V; ++v)
                xi_uniform_word(Rl, Rl.rk, (uint64_t)y * (L / 2) + 32u * (j + v), t0 + (uint32_t)((i - 1) >> 1), s,
                                0u, xp[v], xq[v]);
        }
        if constexpr (MODE == 1) {
            const uint32_t y = yu >= (uint32_t)i ? yu - (uint32_t)i : yu + Y - (uint32_t)i;
            const KeysRk key{Rl.rk};
            // y W + j < 2^28 for every supported lattice (Y <= 2^17 rows, W <= 2^11 words, the
            // plan refuses more): a 32-bit multiply-add, and the counter's high word parts are
            // known to be zero (+4 % at p = 1/2 against the 64-bit product)
            const uint64_t g = (uint64_t)(y * W + j);
            if constexpr (ND == 0)
                wave_xi<V>(Rl, key, g, t0 + (uint32_t)((i - 1) >> 1), s, xp, xq);
            else
                wave_xi_fixed<V, ND, DP, DQ>(Rl, key, g, t0 + (uint32_t)((i - 1) >> 1), s, xp, xq);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            b[v] = wave_update<MODE, DP, DQ>(b[v], up[v], dn[v], mid[v], side[v], s, xp[v], xq[v]);
        }
    }
}

// Store a final row (height bits hr, the row above hp) as its four canonical slope words at
// word offset o: sy-bit = b xor b(x, y-1) xor s and sx-bit = b xor b(x-1, y) xor s.  In even
// rows sublattice 0 sits at even x, so its left neighbour is bit k-1 of the sublattice-1 word
// and sublattice 1's is bit k of the sublattice-0 word; odd rows (odd u) the other way round.
// with_sx false (warp-uniform): the sy- words only.
template <int V>
__device__ __forceinline__ void wave_store_row(const uint32_t (&hr)[2][V], const uint32_t (&hp)[2][V], const int u,
                                               const bool own, const bool with_sx, const uint32_t o, uint32_t *DX0,
                                               uint32_t *DY0, uint32_t *DX1, uint32_t *DY1)
{
    uint32_t sy[2][V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        sy[0][v] = hr[0][v] ^ hp[1][v];
        sy[1][v] = ~(hr[1][v] ^ hp[0][v]);
    }
    if (own) {
        wave_st<V>(DY0 + o, sy[0]);
        wave_st<V>(DY1 + o, sy[1]);
    }
    if (!with_sx) return;
    const int lo = (u & 1) ? 1 : 0;             // sublattice whose left neighbour is shifted
    const uint32_t pv = __shfl_up_sync(0xFFFFFFFFu, hr[lo ^ 1][V - 1], 1);
    uint32_t sx[2][V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const uint32_t left = __funnelshift_l(v ? hr[lo ^ 1][(v + V - 1) % V] : pv, hr[lo ^ 1][v], 1);
        sx[lo][v] = hr[lo][v] ^ left;
        sx[lo ^ 1][v] = hr[lo ^ 1][v] ^ hr[lo][v];
    }
#pragma unroll
    for (int v = 0; v < V; ++v) sx[1][v] = ~sx[1][v];
    if (own) {
        wave_st<V>(DX0 + o, sx[0]);
        wave_st<V>(DX1 + o, sx[1]);
    }
}

// b(x, y) = b(x, y-1) xor sy-bit(x, y) xor s for both sublattices of an arriving row (sites of
// sublattice s have parity s).
template <int V>
__device__ __forceinline__ void wave_convert_row(uint32_t (&hn)[2][V], const uint32_t (&hp)[2][V],
                                                 const uint32_t (&sy)[2][V])
{
#pragma unroll
    for (int v = 0; v < V; ++v) {
        hn[0][v] = hp[1][v] ^ sy[0][v];
        hn[1][v] = ~(hp[0][v] ^ sy[1][v]);
    }
}

// Slide the row window by U slots once a block of U rows has been processed.
template <int K, int V, int U>
__device__ __forceinline__ void wave_slide(uint32_t (&h)[2 * K + 1 + U][2][V])
{
#pragma unroll
    for (int c = 0; c <= 2 * K; ++c)
#pragma unroll
        for (int v = 0; v < V; ++v) {
            h[c][0][v] = h[c + U][0][v];
            h[c][1][v] = h[c + U][1][v];
        }
}

// Per-tile values the row blocks of the {0, 1}-probability kernels share.
struct WaveTile {
    const uint32_t *SY0, *SY1;
    uint32_t *DX0, *DY0, *DX1, *DY1;
    uint32_t L, W, plane, NR, j;
    uint32_t ol;     // word offset of the next row to load (32 bits: a plane holds <= 2^28 words)
    uint32_t os;     // word offset of the next final row to store
    uint32_t rsx;    // the one row R whose sx- words are stored (all rows: sx_all)
    bool sx_all;
    bool own;        // this lane stores its words
};

// One block of U arriving rows R0 .. R0 + U - 1 of a {0, 1}-probability tile.  CHK: some row of
// the block is the first one, lies past the band's end, has no row U further on to prefetch, or
// precedes the first final row, so every per-row step is guarded; blocks in the steady state
// skip the guards.
template <int K, int V, int U, int P, bool DP, bool DQ, bool CHK>
__device__ __forceinline__ void wave_block01(const Rule &Rl, WaveTile &T, uint32_t (&h)[2 * K + 1 + U][2][V],
                                             uint32_t (&rc)[P][2][V], const uint32_t R0)
{
    constexpr int S = 2 * K;
    constexpr int base = S + 1;                 // slot of row R0
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t R = R0 + (uint32_t)u;
        if (CHK && R >= T.NR) break;
        if (!CHK || R > 0) wave_convert_row<V>(h[base + u], h[base + u - 1], rc[u % P]);
        if (!CHK || R + P < T.NR) {             // row R + P into the ring entry just freed
            wave_ld<V>(T.SY0 + T.ol, rc[u % P][0]);
            wave_ld<V>(T.SY1 + T.ol, rc[u % P][1]);
        }
        T.ol += T.W;
        if (T.ol >= T.plane) T.ol -= T.plane;
        wave_half_steps<K, V, U, 0, DP, DQ, 0>(Rl, h, u, 0u, T.L, T.L, T.W, T.j, 0u);
        if (!CHK || R >= 4u * K + 2u) {         // row R - 2K is final
            wave_store_row<V>(h[base + u - S], h[base + u - S - 1], u, T.own, T.sx_all || R == T.rsx, T.os, T.DX0,
                              T.DY0, T.DX1, T.DY1);
            T.os += T.W;
        }
    }
}

// V consecutive words per lane (V = 1, 2 or 4; the lattice's words per row must be a multiple
// of V).  U rows per loop iteration: the loop body holds U x 2K half-step updates, and the row
// window (2K+1+U slots) shifts by U slots per iteration.  MODE 0: p, q in {0, 1} with
// DP = (p == 1), DQ = (q == 1); MODE 1: dyadic draws, ND of them fixed at compile time (0: the
// rule's count at run time), DP / DQ = (p != 0) / (q != 0); MODE 2: per-site uniforms.
// MINB: resident CTAs per SM the compiler must allow (negative: the policy above).
template <int K, int V, int U, int MODE, bool DP, bool DQ, int ND = 0, int MINB = -1>
__global__ void __launch_bounds__(32 * kWaveWarps, MINB >= 0 ? MINB : wave_min_blocks(K, V, MODE))
    k_wave(const WaveArgs a)
{
    constexpr int S = 2 * K;                    // half-steps per launch
    constexpr int NW = S + 1 + U;               // row slots: slot of row R = R - R0 + S + 1
    static_assert(U % 2 == 0, "U rows per iteration keeps the row parity of each slot");
    const uint32_t FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const uint32_t tile = blockIdx.x * kWaveWarps + threadIdx.x / 32;
    if (tile >= a.nbands * a.ncols) return;
    const uint32_t band = tile / a.ncols, col = tile - band * a.ncols;
    const uint32_t L = a.L, W = a.W, Y = a.Y;   // L sites per row, Y rows
    // band rows [y0, y1), y0 even: the first streamed row is even, so band-row parity is
    // lattice-row parity
    // two tiers: ntall bands over rows [0, ytall), then the rest, shorter, over [ytall, Y); the
    // short bands come later in launch order and fill the SM slots the tall ones free
    const bool tall = band < a.ntall;
    const uint32_t tb = tall ? band : band - a.ntall, tn = tall ? a.ntall : a.nbands - a.ntall;
    const uint32_t ty = tall ? 0u : a.ytall, th = (tall ? a.ytall : Y - a.ytall) / 2;
    const uint32_t y0 = ty + 2u * (uint32_t)(((uint64_t)tb * th) / tn);
    const uint32_t y1 = ty + 2u * (uint32_t)(((uint64_t)(tb + 1) * th) / tn);
    // halo: 2K rows below, 2K + 2 above (the top row's sy- words need the row above it, and
    // the first streamed row stays even); rows are taken modulo Y, so a band taller than the
    // lattice streams some rows twice, as the periodic lattice unrolled along y
    const uint32_t NR = y1 - y0 + 4u * K + 2u;
    const uint32_t first = (uint32_t)(((uint64_t)y0 + 64ull * Y - 2u * K - 2u) % Y);
    const size_t plane = (size_t)Y * W;
    const uint32_t *SX0 = a.src, *SY0 = a.src + plane, *SX1 = a.src + 2 * plane, *SY1 = a.src + 3 * plane;
    uint32_t *DX0 = a.dst, *DY0 = a.dst + plane, *DX1 = a.dst + 2 * plane, *DY1 = a.dst + 3 * plane;
    const uint64_t t0 = a.t_dev ? *a.t_dev + a.t0 : a.t0;

    // lane l owns words jj .. jj + V - 1 of every row; lanes 0 and 31 are halo
    const int64_t jj = (int64_t)col * (kWaveTileWords * V) - V + (int64_t)lane * V;
    const uint32_t j = (uint32_t)(((jj % (int64_t)W) + W) % (int64_t)W);
    const bool own = lane >= 1 && lane <= 30 && jj < (int64_t)W;

    uint32_t h[NW][2][V];           // height bits [slot][sublattice][word]
    // sy- words of rows R .. R + P - 1 (ring: row R sits in entry R mod P; once a row has been
    // converted its entry takes the row P further on, in flight while the next rows compute)
    constexpr int P = wave_ring(U, MODE);
    static_assert(U % P == 0, "the ring length divides the rows per block");
    uint32_t rc[P][2][V];
#pragma unroll
    for (int i = 0; i < NW; ++i)
#pragma unroll
        for (int v = 0; v < V; ++v) h[i][0][v] = h[i][1][v] = 0u;

    // First row (even lattice row: sublattice 0 at even x): integrate along x.  With e(x) =
    // b(x) xor b(x-1) = sx-bit(x) xor (x & 1), the even-x bits obey b_e(k) = b_e(k-1) xor
    // ~sx1(k-1) xor sx0(k); the prefix xor runs over the lane's words and then the warp (lane
    // 0's reference bit is arbitrary: flipping every bit of a connected region changes no slope).
    {
        const size_t o = (size_t)first * W + j;
        uint32_t sx0[V], nsx1[V];
        wave_ld<V>(SX0 + o, sx0);
        wave_ld<V>(SX1 + o, nsx1);
#pragma unroll
        for (int v = 0; v < V; ++v) nsx1[v] = ~nsx1[v];
        const uint32_t prev = __shfl_up_sync(FULL, nsx1[V - 1], 1);
        uint32_t pre[V], c = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            pre[v] = wave_xor_prefix(sx0[v] ^ __funnelshift_l(v ? nsx1[(v + V - 1) % V] : prev, nsx1[v], 1));
            pre[v] ^= 0u - c;
            c = pre[v] >> 31;
        }
        uint32_t incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl ^= t;
        }
        const uint32_t flip = 0u - (incl ^ c);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            h[S + 1][0][v] = pre[v] ^ flip;
            h[S + 1][1][v] = pre[v] ^ flip ^ nsx1[v];
        }
    }
    const uint32_t plane32 = Y * W;
    uint32_t ol = (first + 1 >= Y ? first + 1 - Y : first + 1) * W + j;     // next row to load
#pragma unroll
    for (int u = 1; u < P; ++u) {
        if ((uint32_t)u < NR) {
            wave_ld<V>(SY0 + ol, rc[u][0]);
            wave_ld<V>(SY1 + ol, rc[u][1]);
        }
        ol += W;
        if (ol >= plane32) ol -= plane32;
    }
    uint32_t os = y0 * W + j;                   // lattice row y0 is the first final row
    // The next launch of the same plan integrates band b's first row, y0(b) - 2K - 2, from its
    // sx- words; that row is this band's row y1 - 2K - 2 (the next band starts at y1, the first
    // at y1 = Y modulo Y), stored when R = y1 - y0 + 2K.  Every other row's sx- words can wait
    // for the last launch before the state is read (sx_all).
    const bool sx_all = a.sx_all != 0;
    const uint32_t rsx = y1 - y0 + 2u * K;
    constexpr int base = S + 1;                 // slot of the first row of a block

    if constexpr (MODE == 0) {
        WaveTile T;
        T.SY0 = SY0; T.SY1 = SY1;
        T.DX0 = DX0; T.DY0 = DY0; T.DX1 = DX1; T.DY1 = DY1;
        T.L = L; T.W = W; T.plane = plane32; T.NR = NR; T.j = j;
        T.ol = ol; T.os = os; T.own = own;
        T.rsx = rsx; T.sx_all = sx_all;
        for (uint32_t R0 = 0; R0 < NR; R0 += U) {
            if (R0 >= 4u * K + 2u && R0 + U + P <= NR)
                wave_block01<K, V, U, P, DP, DQ, false>(a.R, T, h, rc, R0);
            else
                wave_block01<K, V, U, P, DP, DQ, true>(a.R, T, h, rc, R0);
            wave_slide<K, V, U>(h);
        }
    } else {
        uint32_t yu = first;                    // lattice row of row R
        for (uint32_t R0 = 0; R0 < NR; R0 += U) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t R = R0 + (uint32_t)u;
                if (R >= NR) break;
                if (R > 0) wave_convert_row<V>(h[base + u], h[base + u - 1], rc[u % P]);
                if (R + P < NR) {               // row R + P into the ring entry just freed
                    wave_ld<V>(SY0 + ol, rc[u % P][0]);
                    wave_ld<V>(SY1 + ol, rc[u % P][1]);
                }
                ol += W;
                if (ol >= plane32) ol -= plane32;
                wave_half_steps<K, V, U, MODE, DP, DQ, ND>(a.R, h, u, yu, L, Y, W, j, t0);
                if (R >= 4u * K + 2u) {         // row R - 2K is final
                    wave_store_row<V>(h[base + u - S], h[base + u - S - 1], u, own, sx_all || R == rsx, os, DX0,
                                      DY0, DX1, DY1);
                    os += W;
                }
                if (++yu == Y) yu = 0;
            }
            wave_slide<K, V, U>(h);
        }
    }
}

// The kernel that runs K MCS per launch with {0, 1} probabilities, V words per lane.
template <int K, int V, bool DP, bool DQ>
constexpr void (*wave01_kernel())(WaveArgs)
{
    return k_wave<K, V, kWaveU0, 0, DP, DQ>;
}

}  // namespace sca
