// Counter-based random bits for the SCA update, evaluated in registers.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11): ten rounds of two 32x32->64 multiplies with the published round multipliers and
// Weyl key increments.  Replaces the paper's per-thread TinyMT (Sec. II.B) so that any word of
// any MCS can be drawn without stored generator state, which lets tile edges be recomputed.
#pragma once
#include <cstdint>

namespace sca {

struct Ctr4 { uint32_t x, y, z, w; };

__device__ __forceinline__ Ctr4 philox4x32_10(Ctr4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = Ctr4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same ten rounds with the key schedule precomputed: rk[2r], rk[2r+1] are the key words
// of round r (k0 + r * 0x9E3779B9, k1 + r * 0xBB67AE85 mod 2^32).  When rk points into kernel
// parameters the round keys are free operands; elsewhere they cost one load per round.
__device__ __forceinline__ Ctr4 philox4x32_10_rk(Ctr4 c, const uint32_t *rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = Ctr4{hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0};
    }
    return c;
}

// Counter layout: (g, t, s | (draw-1) << 1 | (t >> 32) << 6, tag | (g >> 32) << 1).
__device__ __forceinline__ Ctr4 draw_counter(uint64_t g, uint64_t t, int s, int draw, int tag)
{
    return Ctr4{(uint32_t)g, (uint32_t)t,
                (uint32_t)s | ((uint32_t)(draw - 1) << 1) | ((uint32_t)(t >> 32) << 6),
                (uint32_t)tag | ((uint32_t)(g >> 32) << 1)};
}

__device__ __forceinline__ uint32_t lane_of(const Ctr4 &o, uint32_t lane)
{
    return lane == 0 ? o.x : lane == 1 ? o.y : lane == 2 ? o.z : o.w;
}

// Per-launch rule: how xi_p and xi_q are produced.
struct Rule {
    uint32_t k0, k1;      // Philox key (seed low / high)
    uint32_t mode;        // 0: p, q in {0, 1} (no draws); 1: dyadic; 2: per-site uniform
    uint32_t n_draws;     // dyadic: max(n_p, n_q)
    uint32_t np, nq;      // dyadic exponents
    uint32_t Pp, Pq;      // dyadic odd numerators (p = Pp / 2^np); 0/1 when n = 0
    uint64_t Tp, Tq;      // per-site thresholds floor(p * 2^32), floor(q * 2^32)
    uint32_t rk[20];      // Philox round keys (see philox4x32_10_rk)
};

// xi words for V consecutive packed words starting at word unit u0 (= y * W + j) of
// sublattice s at MCS t; dyadic construction of Sec. III: xi = r_n, then for i = n-1 .. 1
// xi = b_i ? (r_i | xi) : (r_i & xi) where b_i is the i-th binary digit of the probability.
template <int V>
__device__ __forceinline__ void xi_dyadic(const Rule &R, const uint32_t *rk, uint64_t u0, uint64_t t,
                                          int s, uint32_t (&xp)[V], uint32_t (&xq)[V])
{
#pragma unroll
    for (int v = 0; v < V; ++v) {
        xp[v] = (R.np == 0 && R.Pp) ? 0xFFFFFFFFu : 0u;
        xq[v] = (R.nq == 0 && R.Pq) ? 0xFFFFFFFFu : 0u;
    }
    for (int i = (int)R.n_draws; i >= 1; --i) {
        uint32_t r[V];
        if (V == 4 && (u0 & 3) == 0) {
            const Ctr4 o = philox4x32_10_rk(draw_counter(u0 >> 2, t, s, i, 0), rk);
            r[0] = o.x; r[1 % V] = o.y; r[2 % V] = o.z; r[3 % V] = o.w;
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const uint64_t u = u0 + v;
                r[v] = lane_of(philox4x32_10_rk(draw_counter(u >> 2, t, s, i, 0), rk),
                               (uint32_t)(u & 3));
            }
        }
        if (i <= (int)R.np) {
            const bool first = (i == (int)R.np);
            const bool bit = (R.Pp >> (R.np - i)) & 1u;
#pragma unroll
            for (int v = 0; v < V; ++v)
                xp[v] = first ? r[v] : (bit ? (r[v] | xp[v]) : (r[v] & xp[v]));
        }
        if (i <= (int)R.nq) {
            const bool first = (i == (int)R.nq);
            const bool bit = (R.Pq >> (R.nq - i)) & 1u;
#pragma unroll
            for (int v = 0; v < V; ++v)
                xq[v] = first ? r[v] : (bit ? (r[v] | xq[v]) : (r[v] & xq[v]));
        }
    }
}

// The same construction with the number of draws ND known at compile time: all ND Philox
// calls are independent, so they are issued first (the compiler interleaves their round
// chains) and combined afterwards.  Requires R.n_draws == ND.
template <int V, int ND>
__device__ __forceinline__ void xi_dyadic_fixed(const Rule &R, const uint32_t *rk, uint64_t u0,
                                                uint64_t t, int s, uint32_t (&xp)[V],
                                                uint32_t (&xq)[V])
{
    uint32_t r[ND][V];
    if (V == 4 && (u0 & 3) == 0) {
#pragma unroll
        for (int i = 0; i < ND; ++i) {
            const Ctr4 o = philox4x32_10_rk(draw_counter(u0 >> 2, t, s, i + 1, 0), rk);
            r[i][0] = o.x; r[i][1 % V] = o.y; r[i][2 % V] = o.z; r[i][3 % V] = o.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < ND; ++i)
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const uint64_t u = u0 + v;
                r[i][v] = lane_of(philox4x32_10_rk(draw_counter(u >> 2, t, s, i + 1, 0), rk),
                                  (uint32_t)(u & 3));
            }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        xp[v] = (R.np == 0 && R.Pp) ? 0xFFFFFFFFu : 0u;
        xq[v] = (R.nq == 0 && R.Pq) ? 0xFFFFFFFFu : 0u;
    }
#pragma unroll
    for (int i = ND; i >= 1; --i) {
        if (i <= (int)R.np) {
            const bool first = (i == (int)R.np);
            const bool bit = (R.Pp >> (R.np - i)) & 1u;
#pragma unroll
            for (int v = 0; v < V; ++v)
                xp[v] = first ? r[i - 1][v] : (bit ? (r[i - 1][v] | xp[v]) : (r[i - 1][v] & xp[v]));
        }
        if (i <= (int)R.nq) {
            const bool first = (i == (int)R.nq);
            const bool bit = (R.Pq >> (R.nq - i)) & 1u;
#pragma unroll
            for (int v = 0; v < V; ++v)
                xq[v] = first ? r[i - 1][v] : (bit ? (r[i - 1][v] | xq[v]) : (r[i - 1][v] & xq[v]));
        }
    }
}

// MODE 1 with ND draws: ND in 1..4 uses the fixed-count form, 0 the runtime loop.
template <int V, int ND>
__device__ __forceinline__ void xi_dyadic_any(const Rule &R, const uint32_t *rk, uint64_t u0,
                                              uint64_t t, int s, uint32_t (&xp)[V],
                                              uint32_t (&xq)[V])
{
    if constexpr (ND == 0) xi_dyadic<V>(R, rk, u0, t, s, xp, xq);
    else xi_dyadic_fixed<V, ND>(R, rk, u0, t, s, xp, xq);
}

// xi words for one packed word from per-site uniforms (Sec. II.B: one random number per
// site).  Site unit u = y * (L/2) + k, k = 32 * word + bit; four sites per Philox call.  All
// eight calls of a word are made (skipping ineligible groups would diverge within a warp and
// save nothing); they run four at a time as independent chains.  Thresholds are 32-bit, with
// p = 1 (threshold 2^32) carried by the all_p / all_q masks.
__device__ __forceinline__ void xi_uniform_word(const Rule &R, const uint32_t *rk, uint64_t site0,
                                                uint64_t t, int s, uint32_t need, uint32_t &xp,
                                                uint32_t &xq)
{
    (void)need;
    const uint32_t Tp = R.Tp >= (1ull << 32) ? 0xFFFFFFFFu : (uint32_t)R.Tp;
    const uint32_t Tq = R.Tq >= (1ull << 32) ? 0xFFFFFFFFu : (uint32_t)R.Tq;
    const uint32_t all_p = R.Tp >= (1ull << 32) ? 0xFFFFFFFFu : 0u;
    const uint32_t all_q = R.Tq >= (1ull << 32) ? 0xFFFFFFFFu : 0u;
    xp = all_p;
    xq = all_q;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        Ctr4 o[4];
#pragma unroll
        for (int g = 0; g < 4; ++g)
            o[g] = philox4x32_10_rk(draw_counter((site0 >> 2) + 4 * half + g, t, s, 1, 1), rk);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int b = 16 * half + 4 * g;
            xp |= ((uint32_t)(o[g].x < Tp) << b) | ((uint32_t)(o[g].y < Tp) << (b + 1)) |
                  ((uint32_t)(o[g].z < Tp) << (b + 2)) | ((uint32_t)(o[g].w < Tp) << (b + 3));
            xq |= ((uint32_t)(o[g].x < Tq) << b) | ((uint32_t)(o[g].y < Tq) << (b + 1)) |
                  ((uint32_t)(o[g].z < Tq) << (b + 2)) | ((uint32_t)(o[g].w < Tq) << (b + 3));
        }
    }
}

// Update mask of Eqs. (2)-(4): m_p = xi_p & ~(sx- | sy-) & sx+ & sy+,
// m_q = xi_q & ~(sx+ | sy+) & sx- & sy-, m = m_p ^ m_q.
__device__ __forceinline__ uint32_t update_mask(uint32_t xm, uint32_t ym, uint32_t xpl, uint32_t ypl,
                                                uint32_t xi_p, uint32_t xi_q)
{
    const uint32_t mp = xi_p & ~(xm | ym) & xpl & ypl;
    const uint32_t mq = xi_q & ~(xpl | ypl) & xm & ym;
    return mp ^ mq;
}

// Sites of a word that can flip at all (a minimum or a maximum), before any draw.
__device__ __forceinline__ uint32_t eligible(uint32_t xm, uint32_t ym, uint32_t xpl, uint32_t ypl)
{
    return (~(xm | ym) & xpl & ypl) | (~(xpl | ypl) & xm & ym);
}

}  // namespace sca
