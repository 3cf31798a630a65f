// Streaming engine of the batched ensemble: the register wavefront of sca_wave.cuh applied to
// many small lattices at once.
//
// A lattice of the batch has at most 32 packed words per sublattice row, so a whole row fits a
// group of G = W / V lanes (V words per lane).  A warp holds 32 / G groups; each group streams
// one band of rows of one lattice through registers as height bits and advances it K MCS per
// launch.  Because a group holds the entire row, the x direction is exactly periodic through
// width-G shuffles: no halo words.  Bands carry 2K + 2 halo rows above and 2K below (periodic
// in y), read from the source buffer and recomputed, and write only their own rows of the
// destination buffer.  Each group has its own lattice's Philox key; all lattices of one launch
// share L and the rule (a "class" of the batch), so the control flow of a warp is uniform.
#include "sca_wave.cuh"

namespace sca {

struct WBArgs {
    const uint32_t *src;
    uint32_t *dst;
    const WBItem *items;
    uint32_t n_items;
    uint32_t L, W, n;   // class lattice size, words per row, rows per band (even)
    uint32_t G;         // lanes per row group (W / V, a power of two <= 32)
    uint64_t t0;
    uint32_t sx_all;    // 0: sx- words only on each band's row y0 + n - 2K - 2 (the row the next
                        // launch of the same K starts the following band from)
    Rule R;             // class rule; the keys come from the items
};

// One warp per CTA: the register file fills warp by warp (at 152 registers a thread 13 warps fit
// an SM, against 12 in 128-thread CTAs).
constexpr int kWBWarps = 1;

template <int K, int V, int U, int MODE, bool DP, bool DQ, int ND>
__global__ void __launch_bounds__(32 * kWBWarps) k_wave_batch(const WBArgs a)
{
    constexpr int S = 2 * K;
    constexpr int NW = S + 1 + U;
    static_assert(U % 2 == 0, "U rows per iteration keeps the row parity of each slot");
    const uint32_t FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const int G = (int)a.G, NG = 32 / G;
    const int lig = lane & (G - 1), grp = lane / G;
    const uint32_t warp = blockIdx.x * kWBWarps + threadIdx.x / 32;
    const uint32_t first_item = warp * (uint32_t)NG;
    if (first_item >= a.n_items) return;                       // whole warp idle
    const uint32_t item = first_item + (uint32_t)grp;
    const bool act = item < a.n_items;                         // idle groups shuffle only
    WBItem it{};
    if (act) it = a.items[item];
    const uint32_t L = a.L, W = a.W;
    const uint32_t y0 = it.y0;
    const uint32_t NR = a.n + 4u * K + 2u;
    const uint32_t first = (y0 + 2u * L - 2u * K - 2u) % L;
    const size_t plane = (size_t)L * W;
    const uint32_t *SX0 = a.src + it.off, *SY0 = SX0 + plane, *SX1 = SX0 + 2 * plane, *SY1 = SX0 + 3 * plane;
    uint32_t *DX0 = a.dst + it.off, *DY0 = DX0 + plane, *DX1 = DX0 + 2 * plane, *DY1 = DX0 + 3 * plane;
    const KeysLane key{it.k0, it.k1};
    const uint64_t t0 = a.t0;
    const uint32_t j = (uint32_t)lig * V;

    auto ld = [&](const uint32_t *p, uint32_t (&r)[V]) {
        if (act) wave_ld<V>(p, r);
        else {
#pragma unroll
            for (int v = 0; v < V; ++v) r[v] = 0u;
        }
    };

    uint32_t h[NW][2][V];
    uint32_t rc[U][2][V], rn[U][2][V];
#pragma unroll
    for (int i = 0; i < NW; ++i)
#pragma unroll
        for (int v = 0; v < V; ++v) h[i][0][v] = h[i][1][v] = 0u;

    // first row: integrate along x over the group (the row is complete, so the reference bit of
    // the group's first site is the only free choice)
    {
        const size_t o = (size_t)first * W + j;
        uint32_t sx0[V], nsx1[V];
        ld(SX0 + o, sx0);
        ld(SX1 + o, nsx1);
#pragma unroll
        for (int v = 0; v < V; ++v) nsx1[v] = ~nsx1[v];
        const uint32_t prev = __shfl_sync(FULL, nsx1[V - 1], lig + G - 1, G);
        uint32_t pre[V], c = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            pre[v] = wave_xor_prefix(sx0[v] ^ __funnelshift_l(v ? nsx1[(v + V - 1) % V] : prev, nsx1[v], 1));
            pre[v] ^= 0u - c;
            c = pre[v] >> 31;
        }
        uint32_t incl = c;
        for (int d = 1; d < G; d <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, d, G);
            if (lig >= d) incl ^= t;
        }
        const uint32_t flip = 0u - (incl ^ c);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            h[S + 1][0][v] = pre[v] ^ flip;
            h[S + 1][1][v] = pre[v] ^ flip ^ nsx1[v];
        }
    }
    uint32_t yl = first + 1 >= L ? first + 1 - L : first + 1;
#pragma unroll
    for (int u = 1; u < U; ++u) {
        if ((uint32_t)u < NR) {
            ld(SY0 + (size_t)yl * W + j, rc[u][0]);
            ld(SY1 + (size_t)yl * W + j, rc[u][1]);
        }
        if (++yl == L) yl = 0;
    }
    uint32_t yu = first;

    for (uint32_t R0 = 0; R0 < NR; R0 += U) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (R0 + U + u < NR) {
                ld(SY0 + (size_t)yl * W + j, rn[u][0]);
                ld(SY1 + (size_t)yl * W + j, rn[u][1]);
            }
            if (++yl == L) yl = 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t R = R0 + (uint32_t)u;
            if (R >= NR) break;
            constexpr int base = S + 1;
            if (R > 0) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    h[base + u][0][v] = h[base + u - 1][1][v] ^ rc[u][0][v];
                    h[base + u][1][v] = ~(h[base + u - 1][0][v] ^ rc[u][1][v]);
                }
            }
            const bool right_shift = ((u + 1) & 1) != 0;
#pragma unroll
            for (int i = 1; i <= S; ++i) {
                const int s = (i - 1) & 1, ns = s ^ 1;
                const int cc = base + u - i;
                uint32_t(&b)[V] = h[cc][s];
                const uint32_t(&up)[V] = h[cc - 1][ns];
                const uint32_t(&dn)[V] = h[cc + 1][ns];
                const uint32_t(&mid)[V] = h[cc][ns];
                uint32_t side[V];
                if (right_shift) {
                    const uint32_t nx = __shfl_sync(FULL, mid[0], lig + 1, G);
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        side[v] = __funnelshift_r(mid[v], v + 1 < V ? mid[(v + 1) % V] : nx, 1);
                } else {
                    const uint32_t pv = __shfl_sync(FULL, mid[V - 1], lig + G - 1, G);
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        side[v] = __funnelshift_l(v ? mid[(v + V - 1) % V] : pv, mid[v], 1);
                }
                uint32_t xp[V] = {}, xq[V] = {};
                if constexpr (MODE == 1) {
                    const uint32_t y = yu >= (uint32_t)i ? yu - (uint32_t)i : yu + L - (uint32_t)i;
                    // word index y W + j < 2^16 (L <= 2048): a 32-bit multiply-add
                    if constexpr (ND == 0)
                        wave_xi<V>(a.R, key, (uint64_t)(y * W + j), t0 + (uint32_t)((i - 1) >> 1), s, xp, xq);
                    else
                        wave_xi_fixed<V, ND, DP, DQ>(a.R, key, (uint64_t)(y * W + j), t0 + (uint32_t)((i - 1) >> 1),
                                                     s, xp, xq);
                }
#pragma unroll
                for (int v = 0; v < V; ++v)
                    b[v] = wave_update<MODE, DP, DQ>(b[v], up[v], dn[v], mid[v], side[v], s, xp[v], xq[v]);
            }
            if (R >= 4u * K + 2u) {
                const uint32_t(&hr)[2][V] = h[base + u - S];
                const uint32_t(&hp)[2][V] = h[base + u - S - 1];
                const uint32_t y = y0 + R - 4u * K - 2u;
                const size_t o = (size_t)y * W + j;
                uint32_t sy[2][V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    sy[0][v] = hr[0][v] ^ hp[1][v];
                    sy[1][v] = ~(hr[1][v] ^ hp[0][v]);
                }
                if (act) {
                    wave_st<V>(DY0 + o, sy[0]);
                    wave_st<V>(DY1 + o, sy[1]);
                }
                // every group of the warp is at the same R: the branch is warp-uniform
                if (a.sx_all || R == a.n + 2u * K) {
                    const int lo = (u & 1) ? 1 : 0;
                    const uint32_t pv = __shfl_sync(FULL, hr[lo ^ 1][V - 1], lig + G - 1, G);
                    uint32_t sx[2][V];
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const uint32_t left = __funnelshift_l(v ? hr[lo ^ 1][(v + V - 1) % V] : pv, hr[lo ^ 1][v], 1);
                        sx[lo][v] = hr[lo][v] ^ left;
                        sx[lo ^ 1][v] = hr[lo ^ 1][v] ^ hr[lo][v];
                    }
#pragma unroll
                    for (int v = 0; v < V; ++v) sx[1][v] = ~sx[1][v];
                    if (act) {
                        wave_st<V>(DX0 + o, sx[0]);
                        wave_st<V>(DX1 + o, sx[1]);
                    }
                }
            }
            if (++yu == L) yu = 0;
        }
#pragma unroll
        for (int c2 = 0; c2 <= S; ++c2)
#pragma unroll
            for (int v = 0; v < V; ++v) {
                h[c2][0][v] = h[c2 + U][0][v];
                h[c2][1][v] = h[c2 + U][1][v];
            }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int v = 0; v < V; ++v) {
                rc[u][0][v] = rn[u][0][v];
                rc[u][1][v] = rn[u][1][v];
            }
    }
}

// Copy whole lattices (those of the items whose band starts at row 0: one per lattice) from
// one state buffer to the other; one block per item at a time.
__global__ void k_wave_batch_copy(const uint32_t *src, uint32_t *dst, const WBItem *items, uint32_t n_items,
                                  uint32_t words_per_lattice)
{
    for (uint32_t i = blockIdx.x; i < n_items; i += gridDim.x) {
        const WBItem it = items[i];
        if (it.y0 != 0) continue;
        for (uint32_t w = threadIdx.x; w < words_per_lattice; w += blockDim.x)
            dst[it.off + w] = src[it.off + w];
    }
}

// ---------------------------------------------------------------------------------------- host
// The engine's class launch: K MCS (1, 2, 4 or 8 for {0, 1} probabilities; 1 or 2 for dyadic
// draws), V words per lane as the class was planned (1, or 4 for dyadic draws when W allows).
template <int K, int V, int MODE, bool DP, bool DQ, int ND>
static cudaError_t wb_go(const WBArgs &a, cudaStream_t st)
{
    const uint32_t groups_per_warp = 32u / a.G;
    const uint32_t warps = (a.n_items + groups_per_warp - 1) / groups_per_warp;
    const uint32_t grid = (warps + kWBWarps - 1) / kWBWarps;
    k_wave_batch<K, V, (MODE == 0 ? kWaveU0 : kWaveU1), MODE, DP, DQ, ND><<<grid, 32 * kWBWarps, 0, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int K>
static cudaError_t wb_mode0(const WBArgs &a, cudaStream_t st)
{
    const bool dp = a.R.Pp != 0, dq = a.R.Pq != 0;
    if (dp && dq) return wb_go<K, 1, 0, true, true, 0>(a, st);
    if (dp) return wb_go<K, 1, 0, true, false, 0>(a, st);
    if (dq) return wb_go<K, 1, 0, false, true, 0>(a, st);
    return wb_go<K, 1, 0, false, false, 0>(a, st);
}

template <int K>
static cudaError_t wb_mode1(const WBArgs &a, int V, cudaStream_t st)
{
    const Rule &R = a.R;
    const bool dp = !(R.np == 0 && R.Pp == 0), dq = !(R.nq == 0 && R.Pq == 0);
    if (V == 4 && dp && R.n_draws >= 1 && R.n_draws <= 3) {
        switch (R.n_draws * 2 + (dq ? 1 : 0)) {
        case 2: return wb_go<K, 4, 1, true, false, 1>(a, st);
        case 3: return wb_go<K, 4, 1, true, true, 1>(a, st);
        case 4: return wb_go<K, 4, 1, true, false, 2>(a, st);
        case 5: return wb_go<K, 4, 1, true, true, 2>(a, st);
        case 6: return wb_go<K, 4, 1, true, false, 3>(a, st);
        default: return wb_go<K, 4, 1, true, true, 3>(a, st);
        }
    }
    if (V == 4) return wb_go<K, 4, 1, true, true, 0>(a, st);
    return wb_go<K, 1, 1, true, true, 0>(a, st);
}

int wave_batch_max_k(const Rule &R)
{
    if (R.mode == 0) return 8;
    if (R.mode == 1) return R.n_draws <= 2 ? 2 : 1;
    return 0;
}

int wave_batch_V(uint32_t L, const Rule &R)
{
    const uint32_t W = L / 64;
    if (R.mode == 1 && W % 4 == 0) return 4;
    return 1;
}

bool wave_batch_supported(uint32_t L, const Rule &R)
{
    if (L < 64 || L % 64 != 0 || L > 2048 || (R.mode != 0 && R.mode != 1)) return false;
    const uint32_t G = (L / 64) / (uint32_t)wave_batch_V(L, R);
    return G >= 1 && G <= 32 && (G & (G - 1)) == 0;
}

cudaError_t launch_wave_batch(const uint32_t *src, uint32_t *dst, const WBItem *items, uint32_t n_items,
                              uint32_t L, uint32_t rows_per_band, uint64_t t0, uint32_t k, const Rule &R,
                              cudaStream_t st, bool sx_all)
{
    const int V = wave_batch_V(L, R);
    if (rows_per_band < 2 * k + 2) sx_all = true;     // the kept row must be one of the band's
    WBArgs a{src, dst, items, n_items, L, L / 64, rows_per_band, (L / 64) / (uint32_t)V, t0, sx_all ? 1u : 0u, R};
    if (R.mode == 0) {
        switch (k) {
        case 1: return wb_mode0<1>(a, st);
        case 2: return wb_mode0<2>(a, st);
        case 4: return wb_mode0<4>(a, st);
        case 8: return wb_mode0<8>(a, st);
        default: return cudaErrorInvalidValue;
        }
    }
    if (R.mode == 1) {
        if (k == 1) return wb_mode1<1>(a, V, st);
        if (k == 2) return wb_mode1<2>(a, V, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_wave_batch_copy(const uint32_t *src, uint32_t *dst, const WBItem *items, uint32_t n_items,
                                   uint32_t L, cudaStream_t st)
{
    const uint32_t words = L * (L / 16);
    const uint32_t grid = n_items < 4096u ? n_items : 4096u;
    k_wave_batch_copy<<<grid, 256, 0, st>>>(src, dst, items, n_items, words);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sca
