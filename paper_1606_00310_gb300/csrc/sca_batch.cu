// Batched ensemble: many independent lattices of uneven size in one persistent launch.
//
// Each lattice lives in shared memory for its whole run, so the dynamics never touch HBM
// after the first load (the paper's update, Sec. II.B Eqs. 2-4, applied to words held on
// chip).  A lattice too large for one CTA is split by rows over G CTAs of a thread-block
// cluster; the only coupling between parts is the sy+ plane row just below a part (Sec. II.A:
// sy+(x,y) = sy-(x,y+1)), which the part above reads and updates directly in its neighbour's
// shared memory (DSMEM).  Work units (the lattices of one cluster: one lattice over 8 CTAs,
// or a few smaller ones) are pulled from a device counter by whole clusters; all CTAs of a
// cluster run the same MCS count, so one cluster barrier after each half-step (Sec. I.A: all
// even sites, then all odd sites) keeps the parts of a lattice consistent.  Roughness is
// computed in shared memory at the requested times and written as exact per-part partials.
#include <cooperative_groups.h>
#include <mutex>

#include "sca_batch.h"

namespace cg = cooperative_groups;

namespace sca {

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

template <int V>
__device__ __forceinline__ void ldv(const uint32_t *p, uint32_t (&r)[V])
{
    if constexpr (V == 4) {
        const uint4 q = *reinterpret_cast<const uint4 *>(p);
        r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
    } else if constexpr (V == 2) {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        r[0] = q.x; r[1] = q.y;
    } else {
        r[0] = *p;
    }
}

template <int V>
__device__ __forceinline__ void stv(uint32_t *p, const uint32_t (&r)[V])
{
    if constexpr (V == 4) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(r[0], r[1], r[2], r[3]);
    } else if constexpr (V == 2) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(r[0], r[1]);
    } else {
        *p = r[0];
    }
}

// One item of a half-step in shared memory: V words of one row.  In a shifted row the mask
// enters the neighbour sublattice's sx- one bit up, and the top bit of the item's last word
// belongs in bit 0 of the next item's first word.  That bit is not written here: it goes to
// carry[] and the owner of that word applies it when it next loads the word as its own sx-
// (the next half-step, which updates that sublattice), so no two threads ever write one word.
template <int V, int MODE, int ND>
__device__ __forceinline__ void batch_item(uint32_t *own_x, uint32_t *own_y, uint32_t *nb_x,
                                           uint32_t *nb_yn, uint32_t j, uint32_t W, bool shifted,
                                           const Rule &R, const uint32_t *rk, uint32_t y, uint32_t L,
                                           uint64_t t, int s, uint32_t carry_in, uint8_t *carry_out)
{
    uint32_t xm[V], ym[V], nx[V], ny[V], xpl[V];
    ldv<V>(own_x + j, xm);                // one 128-bit access per plane for V = 4: consecutive
    ldv<V>(own_y + j, ym);                // threads touch consecutive 16-byte chunks, so the
    ldv<V>(nb_x + j, nx);                 // accesses are free of bank conflicts
    ldv<V>(nb_yn + j, ny);
    xm[0] ^= carry_in;                    // pending carry of the previous half-step
    if (shifted) {
        const uint32_t jn = (j + V == W) ? 0u : j + V;
        const uint32_t next = nb_x[jn];   // bit 0 only: settled, its pending carry was applied
#pragma unroll
        for (int v = 0; v < V; ++v) xpl[v] = (nx[v] >> 1) | ((v + 1 < V ? nx[(v + 1) % V] : next) << 31);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) xpl[v] = nx[v];
    }
    uint32_t xip[V], xiq[V];
    if constexpr (MODE == 0) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            xip[v] = R.Pp ? 0xFFFFFFFFu : 0u;
            xiq[v] = R.Pq ? 0xFFFFFFFFu : 0u;
        }
    } else if constexpr (MODE == 1) {
        xi_dyadic_any<V, ND>(R, rk, (uint64_t)y * W + j, t, s, xip, xiq);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const uint32_t need = eligible(xm[v], ym[v], xpl[v], ny[v]);
            xi_uniform_word(R, rk, (uint64_t)y * (L / 2) + 32u * (j + v), t, s, need, xip[v], xiq[v]);
        }
    }
    uint32_t m[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        m[v] = update_mask(xm[v], ym[v], xpl[v], ny[v], xip[v], xiq[v]);
        xm[v] ^= m[v];
        ym[v] ^= m[v];
        ny[v] ^= m[v];
    }
    stv<V>(own_x + j, xm);
    stv<V>(own_y + j, ym);
    stv<V>(nb_yn + j, ny);
    if (!shifted) {
#pragma unroll
        for (int v = 0; v < V; ++v) nx[v] ^= m[v];
        *carry_out = 0;
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) nx[v] ^= (m[v] << 1) | (v > 0 ? (m[(v + V - 1) % V] >> 31) : 0u);
        *carry_out = (uint8_t)(m[V - 1] >> 31);
    }
    stv<V>(nb_x + j, nx);
}

// Carries live in two byte arrays, one byte per item (row-major, W / V items per row): the
// half-step of sublattice s reads the carries pending for its own sx- words from cbuf[s] and
// writes the ones it produces into cbuf[s ^ 1], so reads and writes never meet.
// Update rows 0..R-1 of the CTA's rows held in shared memory (planes of plane_rows rows each);
// row r is lattice row (r0 + r) mod L; the row after the last updated row is remote_nb_y.
template <int V, int MODE, int ND>
__device__ void batch_half_step(uint32_t *sm, uint8_t *cbuf, const BatchLattice &lt, const uint32_t *rk,
                                uint32_t R, uint32_t r0, uint32_t *remote_nb_y, int s, uint64_t t,
                                uint32_t plane_rows)
{
    const uint32_t W = lt.W;
    const size_t P = (size_t)plane_rows * W;
    uint32_t *own_x = sm + (size_t)(s * 2 + 0) * P;
    uint32_t *own_y = sm + (size_t)(s * 2 + 1) * P;
    uint32_t *nbx = sm + (size_t)((s ^ 1) * 2 + 0) * P;
    uint32_t *nby = sm + (size_t)((s ^ 1) * 2 + 1) * P;
    const uint32_t per_row = W / V;
    const uint32_t items = R * per_row;
    const uint8_t *c_rd = cbuf + (size_t)s * items;
    uint8_t *c_wr = cbuf + (size_t)(s ^ 1) * items;
    const bool pow2 = (per_row & (per_row - 1)) == 0;
    const uint32_t sh = pow2 ? (uint32_t)__ffs(per_row) - 1 : 0;
    for (uint32_t it = threadIdx.x; it < items; it += blockDim.x) {
        const uint32_t r = pow2 ? it >> sh : it / per_row;
        const uint32_t q = it - r * per_row;
        const uint32_t y = (r0 + r < lt.L) ? r0 + r : r0 + r - lt.L;
        uint32_t *nyn = (r + 1 < R) ? nby + (size_t)(r + 1) * W : remote_nb_y;
        batch_item<V, MODE, ND>(own_x + (size_t)r * W, own_y + (size_t)r * W, nbx + (size_t)r * W, nyn,
                            q * V, W, ((uint32_t)s + y) & 1u, lt.R, rk, y, lt.L, t, s, c_rd[it],
                            &c_wr[r * per_row + (q + 1 == per_row ? 0 : q + 1)]);
    }
}

template <int V>
__device__ void batch_half_step_v(uint32_t *sm, uint8_t *cbuf, const BatchLattice &lt, const uint32_t *rk,
                                  uint32_t R, uint32_t r0, uint32_t *remote_nb_y, int s, uint64_t t,
                                  uint32_t plane_rows)
{
    if (lt.R.mode == 0) batch_half_step<V, 0, 0>(sm, cbuf, lt, rk, R, r0, remote_nb_y, s, t, plane_rows);
    else if (lt.R.mode == 1) {
        switch (lt.R.n_draws) {
        case 1: batch_half_step<V, 1, 1>(sm, cbuf, lt, rk, R, r0, remote_nb_y, s, t, plane_rows); break;
        case 2: batch_half_step<V, 1, 2>(sm, cbuf, lt, rk, R, r0, remote_nb_y, s, t, plane_rows); break;
        case 3: batch_half_step<V, 1, 3>(sm, cbuf, lt, rk, R, r0, remote_nb_y, s, t, plane_rows); break;
        case 4: batch_half_step<V, 1, 4>(sm, cbuf, lt, rk, R, r0, remote_nb_y, s, t, plane_rows); break;
        default: batch_half_step<V, 1, 0>(sm, cbuf, lt, rk, R, r0, remote_nb_y, s, t, plane_rows); break;
        }
    } else batch_half_step<V, 2, 0>(sm, cbuf, lt, rk, R, r0, remote_nb_y, s, t, plane_rows);
}

// Apply the carries pending after an odd half-step (they belong to sublattice 0's sx- words,
// read from cbuf[0]) and clear them; needed before the state is read as a whole.
__device__ void batch_flush_carry(uint32_t *sm, uint8_t *cbuf, const BatchLattice &lt, uint32_t R)
{
    const uint32_t W = lt.W, V = lt.V, per_row = W / V, items = R * per_row;
    for (uint32_t it = threadIdx.x; it < items; it += blockDim.x) {
        const uint32_t r = it / per_row, q = it - r * per_row;
        sm[(size_t)r * W + q * V] ^= cbuf[it];      // plane 0 = sublattice 0, sx-
        cbuf[it] = 0;
    }
}

__device__ __forceinline__ int64_t warp_scan_incl(int64_t v, int width)
{
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < width; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xFFFFFFFFu, v, o, width);
        if ((lane & (width - 1)) >= o) v += u;
    }
    return v;
}

// Exclusive prefix over the block of one value per thread (thread order); also the total.
__device__ int64_t block_excl_scan(int64_t v, int64_t *ws, int64_t &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t incl = warp_scan_incl(v, 32);
    __syncthreads();
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int64_t x = lane < nw ? ws[lane] : 0;
        x = warp_scan_incl(x, 32);
        ws[lane] = x;
    }
    __syncthreads();
    total = ws[nw - 1];
    return incl - v + (wid > 0 ? ws[wid - 1] : 0);
}

struct ObsShared {
    int64_t ws[32];
    int64_t red1[32];
    unsigned long long red2[32];
    uint32_t flag;
    int64_t colsum;          // this part's sum of sy-(0,y) over its rows with y >= 1
    int64_t colsum_all;      // including y = 0
};

// Roughness partial of this CTA's rows at one observation (all CTAs of the cluster call it).
__device__ void batch_observe(cg::cluster_group &cluster, bool multi, uint32_t *sm, int32_t *h0,
                              bool have, const BatchLattice &lt, int part, uint32_t R, int base_rank,
                              ObsShared &os, ObsPartial *out)
{
    const uint32_t W = have ? lt.W : 1;
    const size_t P = (size_t)R * W;
    const uint32_t r0 = have ? (uint32_t)((uint64_t)part * lt.L / lt.G) : 0;
    // column 0: site (0,y) is site 0 of sublattice y & 1; its sy- is bit 0 of word 0
    auto s0y = [&](uint32_t r) -> int64_t {
        const uint32_t y = r0 + r;
        return 2 * (int64_t)(sm[(size_t)((y & 1u) * 2 + 1) * P + (size_t)r * W] & 1u) - 1;
    };
    const uint32_t per = have ? (R + blockDim.x - 1) / blockDim.x : 0;
    const uint32_t ra = threadIdx.x * per;
    int64_t loc = 0, loc_all = 0;
    for (uint32_t r = ra; r < ra + per && r < R; ++r) {
        const int64_t v = s0y(r);
        loc_all += v;
        if (r0 + r > 0) loc += v;
    }
    if (threadIdx.x == 0) os.flag = 0;
    int64_t tot_all;
    block_excl_scan(loc_all, os.ws, tot_all);
    int64_t tot;
    const int64_t excl = block_excl_scan(loc, os.ws, tot);
    if (threadIdx.x == 0) {
        os.colsum = tot;
        os.colsum_all = tot_all;
    }
    if (multi) cluster.sync();
    else __syncthreads();
    int64_t offset = 0;
    if (have) {
        for (int q = 0; q < part; ++q)
            offset += cluster.map_shared_rank(&os, base_rank + q)->colsum;
        if (part == 0 && threadIdx.x == 0) {
            int64_t all = 0;
            for (uint32_t q = 0; q < lt.G; ++q) all += cluster.map_shared_rank(&os, base_rank + q)->colsum_all;
            if (all != 0) os.flag |= 1u;      // column 0 does not close around y
        }
        int64_t run = offset + excl;
        for (uint32_t r = ra; r < ra + per && r < R; ++r) {
            if (r0 + r > 0) run += s0y(r);
            h0[r] = (int32_t)run;
        }
    }
    __syncthreads();
    int64_t s1 = 0;
    unsigned long long s2 = 0;
    uint32_t flags = 0;
    if (have) {
        int TP = 1;
        while (TP < (int)W) TP <<= 1;
        const int teams = blockDim.x / TP;
        const int team = threadIdx.x / TP, lane = threadIdx.x - team * TP;
        const int wl = threadIdx.x & 31;
        const uint32_t rounds = (R + teams - 1) / teams;
        for (uint32_t k = 0; k < rounds; ++k) {
            const uint32_t r = k * teams + team;
            const bool act = r < R && lane < (int)W && team < teams;
            uint32_t e = 0, o = 0;
            int64_t c = 0;
            const uint32_t y = r0 + r;
            if (act) {
                e = sm[(size_t)((y & 1u) * 2) * P + (size_t)r * W + lane];
                o = sm[(size_t)(((y & 1u) ^ 1u) * 2) * P + (size_t)r * W + lane];
                c = 2 * (__popc(e) + __popc(o)) - 64;
            }
            const int64_t incl = warp_scan_incl(c, TP);
            const int64_t total = __shfl_sync(0xFFFFFFFFu, incl, (wl & ~(TP - 1)) + TP - 1);
            if (act) {
                if (lane == 0 && total != 0) flags |= 2u;   // row does not close around x
                const int64_t s0 = 2 * (int64_t)(sm[(size_t)((y & 1u) * 2) * P + (size_t)r * W] & 1u) - 1;
                const int64_t H = (int64_t)h0[r] + incl - c - s0;
                int32_t d = 0, sd = 0, sd2 = 0;
#pragma unroll 8
                for (int b = 0; b < 32; ++b) {
                    d += 2 * (int32_t)((e >> b) & 1u) - 1;
                    sd += d;
                    sd2 += d * d;
                    d += 2 * (int32_t)((o >> b) & 1u) - 1;
                    sd += d;
                    sd2 += d * d;
                }
                s1 += 64 * H + sd;
                s2 += (unsigned long long)(64 * H * H + 2 * H * (int64_t)sd + (int64_t)sd2);
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_down_sync(0xFFFFFFFFu, s1, off);
        s2 += __shfl_down_sync(0xFFFFFFFFu, s2, off);
    }
    if (flags) atomicOr(&os.flag, flags);
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        os.red1[wid] = s1;
        os.red2[wid] = s2;
    }
    __syncthreads();
    if (have && threadIdx.x == 0) {
        int64_t t1 = 0;
        unsigned long long t2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t1 += os.red1[w];
            t2 += os.red2[w];
        }
        out->s1 = t1;
        out->s2_lo = t2;
        out->s2_hi = 0;
        out->flags = os.flag;
    }
    if (multi) cluster.sync();   // the other parts are done reading colsum before it is reused
    else __syncthreads();
}

// ------------------------------------------------------------- height bits in shared memory
// The batch kernel keeps each lattice part as height bits (one bit of h mod 4 per site, two
// planes: sublattice 0 and 1, R rows x W words each), the representation of the register
// wavefront kernel: with b = ((h - ((x+y) & 1)) / 2) mod 2, a site of parity s is a local
// minimum (Eq. 2) when b xor b(n) == s for its four neighbours, a maximum (Eq. 3) when
// == 1 - s, and an update flips b alone.  A half-step of sublattice s therefore reads the
// other plane (rows r-1, r, r+1) and writes only its own words; the rows above and below a
// part are read from the neighbouring parts' shared memory.  The same xi words (same Philox
// counters) decide the flips as in the slope kernels, so results are bit-identical.

// One item of a height-bit half-step: V words of row r of plane s.
template <int V, int MODE, int ND>
__device__ __forceinline__ void hb_item(uint32_t *b_row, const uint32_t *mid_row, const uint32_t *up_row,
                                        const uint32_t *dn_row, uint32_t j, uint32_t W, bool right_shift,
                                        const Rule &R, const uint32_t *rk, uint32_t y, uint32_t L,
                                        uint64_t t, int s)
{
    uint32_t b[V], mid[V], up[V], dn[V], side[V];
    ldv<V>(b_row + j, b);
    ldv<V>(mid_row + j, mid);
    ldv<V>(up_row + j, up);
    ldv<V>(dn_row + j, dn);
    // the x-neighbour that is not at the same bit: bit k+1 of the other sublattice when this
    // row's sites sit at odd x, else bit k-1 (periodic in x)
    if (right_shift) {
        const uint32_t nx = mid_row[(j + V == W) ? 0u : j + V];
#pragma unroll
        for (int v = 0; v < V; ++v) side[v] = __funnelshift_r(mid[v], v + 1 < V ? mid[(v + 1) % V] : nx, 1);
    } else {
        const uint32_t pv = mid_row[j == 0 ? W - 1 : j - 1];
#pragma unroll
        for (int v = 0; v < V; ++v) side[v] = __funnelshift_l(v > 0 ? mid[(v + V - 1) % V] : pv, mid[v], 1);
    }
    uint32_t is_min[V], is_max[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const uint32_t e_or = (b[v] ^ up[v]) | (b[v] ^ dn[v]) | (b[v] ^ mid[v]) | (b[v] ^ side[v]);
        const uint32_t e_and = (b[v] ^ up[v]) & (b[v] ^ dn[v]) & (b[v] ^ mid[v]) & (b[v] ^ side[v]);
        is_min[v] = s == 0 ? ~e_or : e_and;
        is_max[v] = s == 0 ? e_and : ~e_or;
    }
    uint32_t xip[V], xiq[V];
    if constexpr (MODE == 0) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            xip[v] = R.Pp ? 0xFFFFFFFFu : 0u;
            xiq[v] = R.Pq ? 0xFFFFFFFFu : 0u;
        }
    } else if constexpr (MODE == 1) {
        xi_dyadic_any<V, ND>(R, rk, (uint64_t)y * W + j, t, s, xip, xiq);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v)
            xi_uniform_word(R, rk, (uint64_t)y * (L / 2) + 32u * (j + v), t, s, is_min[v] | is_max[v],
                            xip[v], xiq[v]);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) b[v] ^= (xip[v] & is_min[v]) | (xiq[v] & is_max[v]);
    stv<V>(b_row + j, b);
}

// Half-step of sublattice s over the part's R rows (row r is lattice row (r0 + r) mod L).
// hb: the two planes of R rows; up_remote / dn_remote: row r0 - 1 and row r0 + R of the other
// plane (a neighbouring part's, or this part's own last / first row when it holds the lattice).
template <int V, int MODE, int ND>
__device__ void hb_half_step(uint32_t *hb, const BatchLattice &lt, const uint32_t *rk, uint32_t R,
                             uint32_t r0, const uint32_t *up_remote, const uint32_t *dn_remote, int s,
                             uint64_t t)
{
    const uint32_t W = lt.W;
    const size_t P = (size_t)R * W;
    uint32_t *own = hb + (size_t)s * P;
    const uint32_t *oth = hb + (size_t)(s ^ 1) * P;
    const uint32_t per_row = W / V;
    const uint32_t items = R * per_row;
    const bool pow2 = (per_row & (per_row - 1)) == 0;
    const uint32_t sh = pow2 ? (uint32_t)__ffs(per_row) - 1 : 0;
    for (uint32_t it = threadIdx.x; it < items; it += blockDim.x) {
        const uint32_t r = pow2 ? it >> sh : it / per_row;
        const uint32_t q = it - r * per_row;
        const uint32_t y = (r0 + r < lt.L) ? r0 + r : r0 + r - lt.L;
        const uint32_t *up = r > 0 ? oth + (size_t)(r - 1) * W : up_remote;
        const uint32_t *dn = r + 1 < R ? oth + (size_t)(r + 1) * W : dn_remote;
        hb_item<V, MODE, ND>(own + (size_t)r * W, oth + (size_t)r * W, up, dn, q * V, W,
                             (((uint32_t)s + y) & 1u) != 0, lt.R, rk, y, lt.L, t, s);
    }
}

template <int V>
__device__ void hb_half_step_v(uint32_t *hb, const BatchLattice &lt, const uint32_t *rk, uint32_t R,
                               uint32_t r0, const uint32_t *up_remote, const uint32_t *dn_remote, int s,
                               uint64_t t)
{
    if (lt.R.mode == 0) hb_half_step<V, 0, 0>(hb, lt, rk, R, r0, up_remote, dn_remote, s, t);
    else if (lt.R.mode == 1) {
        switch (lt.R.n_draws) {
        case 1: hb_half_step<V, 1, 1>(hb, lt, rk, R, r0, up_remote, dn_remote, s, t); break;
        case 2: hb_half_step<V, 1, 2>(hb, lt, rk, R, r0, up_remote, dn_remote, s, t); break;
        case 3: hb_half_step<V, 1, 3>(hb, lt, rk, R, r0, up_remote, dn_remote, s, t); break;
        case 4: hb_half_step<V, 1, 4>(hb, lt, rk, R, r0, up_remote, dn_remote, s, t); break;
        default: hb_half_step<V, 1, 0>(hb, lt, rk, R, r0, up_remote, dn_remote, s, t); break;
        }
    } else hb_half_step<V, 2, 0>(hb, lt, rk, R, r0, up_remote, dn_remote, s, t);
}

// Slope words of row r recovered from the height bits: e = sx- of the even-x sites (sublattice
// y & 1), o = sx- of the odd-x sites.  sx-bit(x) = b(x) xor b(x-1) xor parity(x): the even-x
// site k's left neighbour is odd-x site k-1 (previous word's top bit at k = 0, periodic), the
// odd-x site k's is even-x site k.
__device__ __forceinline__ void hb_sx_words(const uint32_t *be_row, const uint32_t *bo_row, uint32_t j,
                                            uint32_t W, uint32_t se, uint32_t &e, uint32_t &o)
{
    const uint32_t be = be_row[j], bo = bo_row[j], bo_prev = bo_row[j == 0 ? W - 1 : j - 1];
    e = be ^ __funnelshift_l(bo_prev, bo, 1) ^ (0u - se);
    o = ~(bo ^ be ^ (0u - se));
}

// Load rows [r0, r0 + R) of a lattice from its canonical words into height bits.  The
// reference is global, so parts of one lattice agree: h(0,0) = 0, h(0,y) = sum of sy-(0,y')
// for y' = 1..y (the observation's definition), and b(0,y) = ((h(0,y) - (y & 1)) / 2) mod 2;
// along the row b(x) = b(x-1) xor sx-bit(x) xor parity(x).
__device__ void hb_load(uint32_t *hb, const uint32_t *g, const BatchLattice &lt, uint32_t r0, uint32_t R,
                        int64_t *ws)
{
    const uint32_t L = lt.L, W = lt.W;
    const size_t plane = (size_t)L * W, P = (size_t)R * W;
    auto col_slope = [&](uint32_t y) -> int64_t {        // sy-(0, y) as +-1
        return 2 * (int64_t)(g[(size_t)((y & 1u) * 2 + 1) * plane + (size_t)y * W] & 1u) - 1;
    };
    // h(0, r0): the column above the part
    int64_t above = 0;
    for (uint32_t y = 1 + threadIdx.x; y <= r0; y += blockDim.x) above += col_slope(y);
    int64_t tot;
    block_excl_scan(above, ws, tot);
    const int64_t h_r0 = tot;
    // rows of the part: each thread a contiguous run; h(0, y) from an exclusive scan
    const uint32_t per = (R + blockDim.x - 1) / blockDim.x;
    const uint32_t ra = threadIdx.x * per, rb = ra + per < R ? ra + per : R;
    int64_t loc = 0;
    for (uint32_t r = ra; r < rb; ++r)
        if (r > 0) loc += col_slope(r0 + r);
    int64_t all;
    int64_t h = h_r0 + block_excl_scan(loc, ws, all);
    for (uint32_t r = ra; r < rb; ++r) {
        const uint32_t y = r0 + r;
        if (r > 0) h += col_slope(y);
        const uint32_t se = y & 1u, so = se ^ 1u;
        const uint32_t *sxe = g + (size_t)(se * 2) * plane + (size_t)y * W;
        const uint32_t *sxo = g + (size_t)(so * 2) * plane + (size_t)y * W;
        uint32_t *be = hb + (size_t)se * P + (size_t)r * W;
        uint32_t *bo = hb + (size_t)so * P + (size_t)r * W;
        // even-x bits: b_e(k) = b_e(k-1) xor sx_e(k) xor ~sx_o(k-1); b_e(0) = b(0, y)
        uint32_t carry = (uint32_t)(((h - (int64_t)se) >> 1) & 1);    // b(0, y)
        uint32_t prev_no = 0;                                         // ~sx_o of the previous word
        for (uint32_t j = 0; j < W; ++j) {
            const uint32_t xe = sxe[j], no = ~sxo[j];
            uint32_t gk = xe ^ __funnelshift_l(prev_no, no, 1);
            if (j == 0) gk = (gk & ~1u) | carry;                      // bit 0: the reference itself
            uint32_t pre = gk;
            pre ^= pre << 1;
            pre ^= pre << 2;
            pre ^= pre << 4;
            pre ^= pre << 8;
            pre ^= pre << 16;
            if (j > 0) pre ^= 0u - carry;
            be[j] = pre;
            bo[j] = pre ^ sxo[j] ^ (0u - so);
            carry = pre >> 31;
            prev_no = no;
        }
    }
}

// Store the part's rows back as canonical words: sx- from the row (hb_sx_words), sy-bit =
// b xor b(x, y-1) xor parity, with row r0 - 1 from up0 / up1 (the other parts' or own rows).
__device__ void hb_store(const uint32_t *hb, uint32_t *g, const BatchLattice &lt, uint32_t r0, uint32_t R,
                         const uint32_t *up0, const uint32_t *up1)
{
    const uint32_t L = lt.L, W = lt.W;
    const size_t plane = (size_t)L * W, P = (size_t)R * W;
    for (uint32_t i = threadIdx.x; i < R * W; i += blockDim.x) {
        const uint32_t r = i / W, j = i - r * W;
        const uint32_t y = r0 + r;
        const uint32_t se = y & 1u, so = se ^ 1u;
        const uint32_t *be = hb + (size_t)se * P + (size_t)r * W;
        const uint32_t *bo = hb + (size_t)so * P + (size_t)r * W;
        uint32_t e, o;
        hb_sx_words(be, bo, j, W, se, e, o);
        g[(size_t)(se * 2) * plane + (size_t)y * W + j] = e;
        g[(size_t)(so * 2) * plane + (size_t)y * W + j] = o;
        // sy-: the site (x, y) of sublattice s sits above site (x, y-1) of sublattice s ^ 1, same bit
        const uint32_t *u0 = r > 0 ? hb + (size_t)0 * P + (size_t)(r - 1) * W : up0;
        const uint32_t *u1 = r > 0 ? hb + (size_t)1 * P + (size_t)(r - 1) * W : up1;
        g[(size_t)1 * plane + (size_t)y * W + j] = hb[(size_t)r * W + j] ^ u1[j];
        g[(size_t)3 * plane + (size_t)y * W + j] = ~(hb[P + (size_t)r * W + j] ^ u0[j]);
    }
}

// Roughness partial of this CTA's rows at one observation, from the height bits (the
// slope-word version above with the words recovered on the fly); up0 / up1: row r0 - 1.
__device__ void hb_observe(cg::cluster_group &cluster, bool multi, const uint32_t *hb, int32_t *h0,
                           bool have, const BatchLattice &lt, int part, uint32_t R, int base_rank,
                           ObsShared &os, ObsPartial *out, const uint32_t *up0, const uint32_t *up1)
{
    const uint32_t W = have ? lt.W : 1;
    const size_t P = (size_t)R * W;
    const uint32_t r0 = have ? (uint32_t)((uint64_t)part * lt.L / lt.G) : 0;
    // column 0: sy-(0,y) = b(0,y) xor b(0,y-1) xor (y & 1), site (0,y) being bit 0 of word 0 of
    // plane y & 1 and site (0,y-1) bit 0 of word 0 of plane (y-1) & 1
    auto s0y = [&](uint32_t r) -> int64_t {
        const uint32_t y = r0 + r;
        const uint32_t a = hb[(size_t)(y & 1u) * P + (size_t)r * W] & 1u;
        const uint32_t pp = (y & 1u) ^ 1u;
        const uint32_t c = (r > 0 ? hb[(size_t)pp * P + (size_t)(r - 1) * W] : (pp ? up1[0] : up0[0])) & 1u;
        return 2 * (int64_t)(a ^ c ^ (y & 1u)) - 1;
    };
    const uint32_t per = have ? (R + blockDim.x - 1) / blockDim.x : 0;
    const uint32_t ra = threadIdx.x * per;
    int64_t loc = 0, loc_all = 0;
    for (uint32_t r = ra; r < ra + per && r < R; ++r) {
        const int64_t v = s0y(r);
        loc_all += v;
        if (r0 + r > 0) loc += v;
    }
    if (threadIdx.x == 0) os.flag = 0;
    int64_t tot_all;
    block_excl_scan(loc_all, os.ws, tot_all);
    int64_t tot;
    const int64_t excl = block_excl_scan(loc, os.ws, tot);
    if (threadIdx.x == 0) {
        os.colsum = tot;
        os.colsum_all = tot_all;
    }
    if (multi) cluster.sync();
    else __syncthreads();
    int64_t offset = 0;
    if (have) {
        for (int q = 0; q < part; ++q)
            offset += cluster.map_shared_rank(&os, base_rank + q)->colsum;
        if (part == 0 && threadIdx.x == 0) {
            int64_t all = 0;
            for (uint32_t q = 0; q < lt.G; ++q) all += cluster.map_shared_rank(&os, base_rank + q)->colsum_all;
            if (all != 0) os.flag |= 1u;      // column 0 does not close around y
        }
        int64_t run = offset + excl;
        for (uint32_t r = ra; r < ra + per && r < R; ++r) {
            if (r0 + r > 0) run += s0y(r);
            h0[r] = (int32_t)run;
        }
    }
    __syncthreads();
    int64_t s1 = 0;
    unsigned long long s2 = 0;
    uint32_t flags = 0;
    if (have) {
        int TP = 1;
        while (TP < (int)W) TP <<= 1;
        const int teams = blockDim.x / TP;
        const int team = threadIdx.x / TP, lane = threadIdx.x - team * TP;
        const int wl = threadIdx.x & 31;
        const uint32_t rounds = (R + teams - 1) / teams;
        for (uint32_t k = 0; k < rounds; ++k) {
            const uint32_t r = k * teams + team;
            const bool act = r < R && lane < (int)W && team < teams;
            uint32_t e = 0, o = 0, e0 = 0;
            int64_t c = 0;
            const uint32_t y = r0 + r;
            if (act) {
                const uint32_t se = y & 1u;
                const uint32_t *be = hb + (size_t)se * P + (size_t)r * W;
                const uint32_t *bo = hb + (size_t)(se ^ 1u) * P + (size_t)r * W;
                hb_sx_words(be, bo, (uint32_t)lane, W, se, e, o);
                uint32_t o0;
                hb_sx_words(be, bo, 0, W, se, e0, o0);
                c = 2 * (__popc(e) + __popc(o)) - 64;
            }
            const int64_t incl = warp_scan_incl(c, TP);
            const int64_t total = __shfl_sync(0xFFFFFFFFu, incl, (wl & ~(TP - 1)) + TP - 1);
            if (act) {
                if (lane == 0 && total != 0) flags |= 2u;   // row does not close around x
                const int64_t s0 = 2 * (int64_t)(e0 & 1u) - 1;
                const int64_t H = (int64_t)h0[r] + incl - c - s0;
                int32_t d = 0, sd = 0, sd2 = 0;
#pragma unroll 8
                for (int bb = 0; bb < 32; ++bb) {
                    d += 2 * (int32_t)((e >> bb) & 1u) - 1;
                    sd += d;
                    sd2 += d * d;
                    d += 2 * (int32_t)((o >> bb) & 1u) - 1;
                    sd += d;
                    sd2 += d * d;
                }
                s1 += 64 * H + sd;
                s2 += (unsigned long long)(64 * H * H + 2 * H * (int64_t)sd + (int64_t)sd2);
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_down_sync(0xFFFFFFFFu, s1, off);
        s2 += __shfl_down_sync(0xFFFFFFFFu, s2, off);
    }
    if (flags) atomicOr(&os.flag, flags);
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        os.red1[wid] = s1;
        os.red2[wid] = s2;
    }
    __syncthreads();
    if (have && threadIdx.x == 0) {
        int64_t t1 = 0;
        unsigned long long t2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t1 += os.red1[w];
            t2 += os.red2[w];
        }
        out->s1 = t1;
        out->s2_lo = t2;
        out->s2_hi = 0;
        out->flags = os.flag;
    }
    if (multi) cluster.sync();   // the other parts are done reading colsum before it is reused
    else __syncthreads();
}

__global__ void __launch_bounds__(512, 1) k_batch(const BatchArgs a)
{
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ int s_unit;
    __shared__ ObsShared os;
    __shared__ uint32_t s_rk[20];      // Philox round keys of this CTA's lattice
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const uint64_t t_end = a.times[a.n_times - 1];

    for (;;) {
        if (rank == 0 && threadIdx.x == 0) s_unit = (int)atomicAdd(a.unit_counter, 1u);
        cluster.sync();
        const int unit = *cluster.map_shared_rank(&s_unit, 0);
        cluster.sync();
        if (unit >= a.n_units) break;
        if (rank == 0 && threadIdx.x == 0) a.unit_ns[2 * unit] = global_ns();
        const BatchSlot slot = a.slots[(size_t)unit * a.C + rank];
        const bool have = slot.lattice >= 0;
        // lattices split over CTAs need cluster barriers; a unit of one-CTA lattices runs each
        // CTA on its own with block barriers (the choice is the same for every CTA of the unit)
        const bool multi = slot.unit_G > 1;
        BatchLattice lt;
        if (have) lt = a.lat[slot.lattice];
        else { lt.L = 64; lt.W = 1; lt.G = 1; lt.V = 1; }
        // part p of a lattice split over G CTAs holds rows [p L / G, (p+1) L / G)
        const uint32_t r0 = have ? (uint32_t)((uint64_t)slot.part * lt.L / lt.G) : 0;
        const uint32_t R = have ? (uint32_t)((uint64_t)(slot.part + 1) * lt.L / lt.G) - r0 : 0;
        const uint32_t W = lt.W;
        const int base_rank = rank - (have ? slot.part : 0);
        const size_t P = (size_t)R * W;
        uint32_t *hb = sm;                                        // two planes of height bits
        int32_t *h0 = reinterpret_cast<int32_t *>(sm + 2 * P);
        // row r0 - 1 (the previous part's last row) and row r0 + R (the next part's first row)
        // of both planes; a lattice held by one CTA is its own neighbour (periodic in y)
        const uint32_t *up[2] = {nullptr, nullptr};
        const uint32_t *dn[2] = {nullptr, nullptr};
        if (have) {
            const uint32_t pp = (slot.part + lt.G - 1) % lt.G, np = (slot.part + 1) % lt.G;
            const uint32_t Rp = (uint32_t)((uint64_t)(pp + 1) * lt.L / lt.G) - (uint32_t)((uint64_t)pp * lt.L / lt.G);
            const uint32_t Rn = (uint32_t)((uint64_t)(np + 1) * lt.L / lt.G) - (uint32_t)((uint64_t)np * lt.L / lt.G);
            for (int pl = 0; pl < 2; ++pl) {
                up[pl] = cluster.map_shared_rank(sm + (size_t)pl * Rp * W + (size_t)(Rp - 1) * W, base_rank + (int)pp);
                dn[pl] = cluster.map_shared_rank(sm + (size_t)pl * Rn * W, base_rank + (int)np);
            }
            hb_load(hb, a.state + lt.state_off, lt, r0, R, os.ws);
            if (threadIdx.x < 20) s_rk[threadIdx.x] = a.lat[slot.lattice].R.rk[threadIdx.x];
        }
        if (multi) cluster.sync();
        else __syncthreads();
        int obs = 0;
        while (obs < a.n_times && a.times[obs] <= a.t0) ++obs;
        for (uint64_t t = a.t0; t < t_end; ++t) {
            for (int s = 0; s < 2; ++s) {
                if (have) {
                    if (lt.V == 4) hb_half_step_v<4>(hb, lt, s_rk, R, r0, up[s ^ 1], dn[s ^ 1], s, t);
                    else if (lt.V == 2) hb_half_step_v<2>(hb, lt, s_rk, R, r0, up[s ^ 1], dn[s ^ 1], s, t);
                    else hb_half_step_v<1>(hb, lt, s_rk, R, r0, up[s ^ 1], dn[s ^ 1], s, t);
                }
                if (multi) cluster.sync();
                else __syncthreads();
            }
            while (obs < a.n_times && a.times[obs] == t + 1) {
                ObsPartial *out = have ? a.partials + lt.part_off + (size_t)obs * lt.G + slot.part : nullptr;
                hb_observe(cluster, multi, hb, h0, have, lt, have ? slot.part : 0, R, base_rank, os, out,
                           up[0], up[1]);
                ++obs;
            }
        }
        if (have) hb_store(hb, a.state + lt.state_off, lt, r0, R, up[0], up[1]);
        __syncthreads();
        if (rank == 0 && threadIdx.x == 0) a.unit_ns[2 * unit + 1] = global_ns();
    }
}

// One thread per (lattice, observation): add the G part partials in 128-bit integers.
__global__ void k_batch_finalize(const BatchLattice *lat, int n_lat, const ObsPartial *part,
                                 const uint64_t *times, int n_times, ObsDev *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_lat * n_times) return;
    const int li = i / n_times, ob = i - li * n_times;
    const BatchLattice lt = lat[li];
    __int128 S1 = 0;
    unsigned __int128 S2 = 0;
    uint32_t flags = 0;
    for (uint32_t g = 0; g < lt.G; ++g) {
        const ObsPartial p = part[lt.part_off + (size_t)ob * lt.G + g];
        S1 += p.s1;
        S2 += ((unsigned __int128)p.s2_hi << 64) | p.s2_lo;
        flags |= p.flags;
    }
    const unsigned __int128 N = (unsigned __int128)lt.L * lt.L;
    const unsigned __int128 num = N * S2 - (unsigned __int128)(S1 * S1);
    ObsDev o;
    o.t = times[ob];
    o.N = (uint64_t)N;
    o.S1 = (int64_t)S1;
    o.S2_lo = (uint64_t)S2;
    o.S2_hi = (uint64_t)(S2 >> 64);
    o.num_lo = (uint64_t)num;
    o.num_hi = (uint64_t)(num >> 64);
    o.w2 = 0.0;
    o.status = flags ? -7 : 0;
    o.reserved = (int32_t)flags;
    o.h00 = 0;
    out[i] = o;
}

// ------------------------------------------------------------- single lattice, k MCS per pass
// Temporal blocking (multi-MCS per launch) for lattices whose state is too small to keep HBM
// busy but too large for one cluster's shared memory.  CTA b owns rows [y0, y1) and loads them
// with a halo of 2k rows on each side into shared memory; it then runs k MCS there (each
// half-step leaves one more row at each end of the loaded block stale, since an update at row
// r reads and writes rows r and r+1), so after k MCS exactly rows [y0, y1) are current and are
// written to the other state buffer.  The halo updates are recomputed by the neighbouring
// CTAs with the same counter-based random numbers.  Half-steps reuse the batch kernel's
// shared-memory update.
struct TBArgs {
    const uint32_t *src;
    uint32_t *dst;
    uint32_t L, W, V, k, nslabs;
    uint64_t t0;             // MCS index of the first step, or offset from *t_dev
    const uint64_t *t_dev;
    Rule R;
};

__global__ void __launch_bounds__(512, 1) k_tblock(const TBArgs a)
{
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ uint32_t s_rk[20];
    const uint32_t L = a.L, W = a.W, k = a.k;
    const uint32_t b = blockIdx.x;
    const uint32_t y0 = (uint32_t)((uint64_t)b * L / a.nslabs);
    const uint32_t y1 = (uint32_t)((uint64_t)(b + 1) * L / a.nslabs);
    const uint32_t n = y1 - y0, N = n + 4 * k;
    const uint32_t first = (y0 + L - 2 * k) % L;
    const size_t P = (size_t)N * W, plane = (size_t)L * W;
    const uint32_t items = (N - 1) * (W / a.V);
    uint8_t *cbuf = reinterpret_cast<uint8_t *>(sm + 4 * P);
    for (size_t i = threadIdx.x; i < 4 * P; i += blockDim.x) {
        const uint32_t pl = (uint32_t)(i / P);
        const size_t rem = i - (size_t)pl * P;
        const uint32_t r = (uint32_t)(rem / W), j = (uint32_t)(rem - (size_t)r * W);
        uint32_t y = first + r;
        if (y >= L) y -= L;
        sm[i] = a.src[(size_t)pl * plane + (size_t)y * W + j];
    }
    for (uint32_t i = threadIdx.x; i < 2 * items; i += blockDim.x) cbuf[i] = 0;
    if (threadIdx.x < 20) s_rk[threadIdx.x] = a.R.rk[threadIdx.x];
    BatchLattice lt;
    lt.L = L;
    lt.W = W;
    lt.V = a.V;
    lt.G = 1;
    lt.R = a.R;
    const uint64_t t0 = a.t_dev ? *a.t_dev + a.t0 : a.t0;
    __syncthreads();
    for (uint32_t m = 0; m < k; ++m) {
        for (int s = 0; s < 2; ++s) {
            // rows 0..N-2 are updated; row N-1 only supplies sy+ for row N-2
            uint32_t *last_y = sm + (size_t)((s ^ 1) * 2 + 1) * P + (size_t)(N - 1) * W;
            if (a.V == 4) batch_half_step_v<4>(sm, cbuf, lt, s_rk, N - 1, first, last_y, s, t0 + m, N);
            else if (a.V == 2) batch_half_step_v<2>(sm, cbuf, lt, s_rk, N - 1, first, last_y, s, t0 + m, N);
            else batch_half_step_v<1>(sm, cbuf, lt, s_rk, N - 1, first, last_y, s, t0 + m, N);
            __syncthreads();
        }
    }
    batch_flush_carry(sm, cbuf, lt, N - 1);
    __syncthreads();
    const size_t PN = (size_t)n * W;
    for (size_t i = threadIdx.x; i < 4 * PN; i += blockDim.x) {
        const uint32_t pl = (uint32_t)(i / PN);
        const size_t rem = i - (size_t)pl * PN;
        const uint32_t r = (uint32_t)(rem / W), j = (uint32_t)(rem - (size_t)r * W);
        a.dst[(size_t)pl * plane + (size_t)(y0 + r) * W + j] = sm[(size_t)pl * P + (size_t)(r + 2 * k) * W + j];
    }
}

size_t tblock_smem(uint32_t L, uint32_t n, uint32_t k)
{
    const uint32_t W = L / 64, V = (W % 4 == 0) ? 4 : (W % 2 == 0) ? 2 : 1, N = n + 4 * k;
    return 4 * (size_t)N * W * sizeof(uint32_t) + 2 * (size_t)(N - 1) * (W / V);
}

// Slab count: at least one CTA per SM, and slabs of at least 4k rows so the recomputed halo
// stays at most half of the work; shared memory must hold a slab with its halo.
bool tblock_plan(uint32_t L, uint32_t k, uint32_t *nslabs, size_t *smem)
{
    if (L < 128 || L % 64 != 0 || k == 0 || 4 * k >= L) return false;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t cap = (size_t)optin - 1024;
    uint32_t ns = (uint32_t)sm_count();
    if (ns > L / (4 * k)) ns = L / (4 * k);
    if (ns == 0) ns = 1;
    while (tblock_smem(L, (L + ns - 1) / ns, k) > cap && ns < L / 2) ns *= 2;
    if (tblock_smem(L, (L + ns - 1) / ns, k) > cap) return false;
    *nslabs = ns;
    *smem = tblock_smem(L, (L + ns - 1) / ns, k);
    return true;
}

cudaError_t launch_tblock(const uint32_t *src, uint32_t *dst, uint32_t L, uint64_t t0, uint32_t k,
                          const Rule &R, cudaStream_t st, const uint64_t *t_dev)
{
    uint32_t ns = 0;
    size_t smem = 0;
    if (!tblock_plan(L, k, &ns, &smem)) return cudaErrorInvalidValue;
    static int configured = 0;
    if (!configured) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, k_tblock);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_tblock, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
        configured = optin - (int)fa.sharedSizeBytes;
    }
    if ((int)smem > configured) return cudaErrorInvalidConfiguration;
    const uint32_t W = L / 64;
    TBArgs a{src, dst, L, W, (W % 4 == 0) ? 4u : (W % 2 == 0) ? 2u : 1u, k, ns, t0, t_dev, R};
    k_tblock<<<ns, 512, smem, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------- host
struct BatchPlan {
    int C = 8;            // cluster size
    int threads = 512;    // threads per CTA
    size_t smem = 0;      // dynamic shared memory per CTA
};

// Two planes of height bits and the observation's column-0 heights of the largest part.
size_t batch_part_smem(uint32_t L, uint32_t G)
{
    const uint32_t W = L / 64, R = (L + G - 1) / G;      // the largest part
    return 2 * (size_t)R * W * sizeof(uint32_t) + (size_t)R * sizeof(int32_t);
}

// Kernel attributes for a launch shape; call before launching or capturing.  The shared
// memory limit only ever grows, so batches with different needs can coexist in one process.
cudaError_t batch_prepare(int C, size_t smem)
{
    static std::mutex mu;
    static size_t granted = 0;
    static bool nonportable = false;
    std::lock_guard<std::mutex> lock(mu);
    auto kern = k_batch;
    cudaError_t e = cudaSuccess;
    if (smem > granted) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        granted = smem;
    }
    if (C > 8 && !nonportable) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) nonportable = true;
    }
    return e;
}

cudaError_t launch_batch(const BatchArgs &a, int n_clusters, int threads, size_t smem,
                         cudaStream_t st)
{
    auto kern = k_batch;
    cudaError_t e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_clusters * a.C), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, a);
    count_launches(1);
    return e;
}

cudaError_t batch_max_clusters(int C, int threads, size_t smem, int *out)
{
    auto kern = k_batch;
    cudaError_t e = batch_prepare(C, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(out, kern, &cfg);
}

cudaError_t launch_batch_finalize(const BatchLattice *lat, int n_lat, const ObsPartial *part,
                                  const uint64_t *times, int n_times, ObsDev *out, cudaStream_t st)
{
    const int n = n_lat * n_times;
    k_batch_finalize<<<(n + 255) / 256, 256, 0, st>>>(lat, n_lat, part, times, n_times, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sca
