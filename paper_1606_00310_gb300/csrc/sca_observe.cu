// Exact height reconstruction and roughness sums from the canonical packed words.
//
// The paper works with slopes only and names the roughness without defining it (Sec. I.A);
// the definition used here: h(0,0) = 0, h(0,y) = sum of sy-(0,y') for y' = 1..y, and
// h(x,y) = h(0,y) + sum of sx-(x',y) for x' = 1..x (slopes as +-1).  S1 = sum h,
// S2 = sum h^2 (128-bit), num = N * S2 - S1^2 (128-bit); W^2 = num / N^2.  Heights are never
// stored: one kernel scans column 0, one kernel scans every row in registers (popcounts of
// the interleaved even-x / odd-x words give each thread's offset) and reduces per block,
// and a last kernel combines the block partials in 128-bit integers.
#include "sca_internal.h"

namespace sca {

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v, int width)
{
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < width; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xFFFFFFFFu, v, o, width);
        if ((lane & (width - 1)) >= o) v += u;
    }
    return v;
}

// Column 0: site (0, y) is site k = 0 of sublattice y & 1, so sy-(0,y) is bit 0 of word 0 of
// row y in plane (y & 1, y).  One block of 1024 threads; each thread scans a run of rows.
__global__ void __launch_bounds__(1024) k_obs_col0(const uint32_t *A, uint32_t L, int64_t *h0,
                                                   ObsPartial *col_flag)
{
    __shared__ int64_t warp_tot[32];
    const uint32_t W = L / 64;
    const size_t plane = (size_t)L * W;
    const uint32_t per = (L + blockDim.x - 1) / blockDim.x;
    const uint32_t y0 = threadIdx.x * per;
    auto sy0 = [&](uint32_t y) -> int64_t {
        const uint32_t s = y & 1u;
        return 2 * (int64_t)(A[(size_t)(s * 2 + 1) * plane + (size_t)y * W] & 1u) - 1;
    };
    int64_t local = 0;
    // the rows of one thread are independent loads: issue them in batches so their latencies
    // overlap instead of adding up
    for (uint32_t yb = y0; yb < y0 + per && yb < L; yb += 8) {
        int64_t v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t y = yb + k;
            v[k] = (y < y0 + per && y < L && y > 0) ? sy0(y) : 0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) local += v[k];
    }
    int64_t incl = warp_incl_scan(local, 32);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int64_t v = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        v = warp_incl_scan(v, 32);
        warp_tot[lane] = v;
    }
    __syncthreads();
    int64_t run = incl - local + (wid > 0 ? warp_tot[wid - 1] : 0);
    for (uint32_t y = y0; y < y0 + per && y < L; ++y) {
        if (y > 0) run += sy0(y);
        h0[y] = run;
    }
    if (threadIdx.x == blockDim.x - 1) {
        // closure around the y cycle: h(0, L-1) + sy-(0, 0) must return to h(0, 0) = 0
        const int64_t total = warp_tot[(blockDim.x >> 5) - 1];
        col_flag->flags = (total + sy0(0) != 0) ? 1u : 0u;
    }
}

struct RowsArgs {
    const uint32_t *A;
    uint32_t L, W;
    int T, TP;
    const int64_t *h0;
    ObsPartial *part;
};

// Rows: a team of threads spans row y; thread `lane` owns words j = lane*V .. lane*V+V-1 of
// the even-x plane (sublattice y & 1) and the odd-x plane (sublattice (y & 1) ^ 1), i.e.
// x in [64 j, 64 (j + V)).
// Table over the 256 values of (4 even-x bits, 4 odd-x bits): for the 8 sites in x order
// (e0, o0, e1, o1, ...), slopes s = 2b - 1, running offsets d_k = s_0 + ... + s_k:
// bits 0-4: sum s + 8, bits 5-11: sum d + 36, bits 12-19: sum d^2.
__device__ __forceinline__ uint32_t nibble_pair_entry(uint32_t i)
{
    int d = 0, sd = 0, sd2 = 0;
    for (int k = 0; k < 4; ++k) {
        d += 2 * (int)((i >> k) & 1u) - 1;
        sd += d;
        sd2 += d * d;
        d += 2 * (int)((i >> (4 + k)) & 1u) - 1;
        sd += d;
        sd2 += d * d;
    }
    return (uint32_t)(d + 8) | ((uint32_t)(sd + 36) << 5) | ((uint32_t)sd2 << 12);
}

template <int V>
__global__ void __launch_bounds__(1024) k_obs_rows(const RowsArgs a)
{
    __shared__ uint32_t tab[256];
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) tab[i] = nibble_pair_entry(i);
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t red1[32];
    __shared__ unsigned long long red2[32][2];
    __shared__ uint32_t red_flag;
    const int tpb = blockDim.x / a.TP;
    const int team = threadIdx.x / a.TP;
    const int lane = threadIdx.x - team * a.TP;
    const int wid = threadIdx.x >> 5, wl = threadIdx.x & 31;
    const bool owner = lane < a.T;
    const uint32_t L = a.L, W = a.W;
    const size_t plane = (size_t)L * W;
    if (threadIdx.x == 0) red_flag = 0;
    __syncthreads();

    int64_t s1 = 0;
    unsigned __int128 s2 = 0;
    uint32_t flags = 0;
    for (uint32_t base = blockIdx.x * tpb; base < L; base += gridDim.x * tpb) {
        const uint32_t y = base + team;
        const bool active = owner && y < L;
        const uint32_t j = (uint32_t)lane * V;
        uint32_t e[V], o[V];
        int64_t csum = 0;
        if (active) {
            const uint32_t se = y & 1u, so = se ^ 1u;
            const uint32_t *pe = a.A + (size_t)(se * 2) * plane + (size_t)y * W + j;
            const uint32_t *po = a.A + (size_t)(so * 2) * plane + (size_t)y * W + j;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                e[v] = pe[v];
                o[v] = po[v];
                csum += 2 * (__popc(e[v]) + __popc(o[v])) - 64;
            }
        }
        // exclusive prefix of csum over the team, and the team total
        int64_t excl, total;
        if (a.TP <= 32) {
            const int64_t incl = warp_incl_scan(csum, a.TP);
            excl = incl - csum;
            total = __shfl_sync(0xFFFFFFFFu, incl, (wl & ~(a.TP - 1)) + a.TP - 1);
        } else {
            const int64_t incl = warp_incl_scan(csum, 32);
            if (wl == 31) warp_tot[wid] = incl;
            __syncthreads();
            const int w0 = (team * a.TP) >> 5;
            const int nw = a.TP >> 5;
            int64_t before = 0, all = 0;
            for (int w = 0; w < nw; ++w) {
                if (w0 + w < wid) before += warp_tot[w0 + w];
                all += warp_tot[w0 + w];
            }
            __syncthreads();
            excl = before + incl - csum;
            total = all;
        }
        if (active) {
            if (lane == 0 && total != 0) flags |= 2u;   // row does not close around x
            const int64_t s0 = 2 * (int64_t)(a.A[(size_t)((y & 1u) * 2) * plane + (size_t)y * W] & 1u) - 1;
            const int64_t H = a.h0[y] + excl - s0;      // h(x) = H + d(x), d summed from x0
            // 8 sites at a time: with D the offset before a block and (S, A, B) its table entry,
            // the block adds 8D + A to sum d, 8D^2 + 2DA + B to sum d^2, and S to D
            int32_t d = 0, sd = 0, sd2 = 0;
#pragma unroll
            for (int v = 0; v < V; ++v) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t ent = tab[((e[v] >> (4 * k)) & 0xFu) | (((o[v] >> (4 * k)) & 0xFu) << 4)];
                    const int32_t S = (int32_t)(ent & 31u) - 8;
                    const int32_t A = (int32_t)((ent >> 5) & 127u) - 36;
                    const int32_t B = (int32_t)(ent >> 12);
                    sd += 8 * d + A;
                    sd2 += 8 * d * d + 2 * d * A + B;
                    d += S;
                }
            }
            const int64_t n = 64 * V;
            s1 += n * H + sd;
            s2 += (unsigned __int128)(uint64_t)(n * H * H + 2 * H * (int64_t)sd + (int64_t)sd2);
        }
    }
    // block reduction
    for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_down_sync(0xFFFFFFFFu, s1, off);
        const uint64_t lo = (uint64_t)s2, hi = (uint64_t)(s2 >> 64);
        const uint64_t olo = __shfl_down_sync(0xFFFFFFFFu, lo, off);
        const uint64_t ohi = __shfl_down_sync(0xFFFFFFFFu, hi, off);
        s2 += ((unsigned __int128)ohi << 64) | olo;
    }
    if (flags) atomicOr(&red_flag, flags);
    if (wl == 0) {
        red1[wid] = s1;
        red2[wid][0] = (uint64_t)s2;
        red2[wid][1] = (uint64_t)(s2 >> 64);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t1 = 0;
        unsigned __int128 t2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t1 += red1[w];
            t2 += ((unsigned __int128)red2[w][1] << 64) | red2[w][0];
        }
        a.part[blockIdx.x].s1 = t1;
        a.part[blockIdx.x].s2_lo = (uint64_t)t2;
        a.part[blockIdx.x].s2_hi = (uint64_t)(t2 >> 64);
        a.part[blockIdx.x].flags = red_flag;
    }
}

__global__ void __launch_bounds__(256) k_obs_final(const ObsPartial *part, int n,
                                                   const ObsPartial *col_flag, uint32_t L,
                                                   uint64_t t, ObsDev *out)
{
    __shared__ long long s1w[8];
    __shared__ unsigned long long s2w[8][2];
    __shared__ uint32_t fw[8];
    int64_t s1 = 0;
    unsigned __int128 s2 = 0;
    uint32_t flags = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        s1 += part[i].s1;
        s2 += ((unsigned __int128)part[i].s2_hi << 64) | part[i].s2_lo;
        flags |= part[i].flags;
    }
    for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_down_sync(0xFFFFFFFFu, s1, off);
        const uint64_t lo = (uint64_t)s2, hi = (uint64_t)(s2 >> 64);
        s2 += ((unsigned __int128)__shfl_down_sync(0xFFFFFFFFu, hi, off) << 64) |
              __shfl_down_sync(0xFFFFFFFFu, lo, off);
        flags |= __shfl_down_sync(0xFFFFFFFFu, flags, off);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s1w[w] = s1;
        s2w[w][0] = (uint64_t)s2;
        s2w[w][1] = (uint64_t)(s2 >> 64);
        fw[w] = flags;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    __int128 S1 = 0;
    unsigned __int128 S2 = 0;
    flags = col_flag->flags;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        S1 += s1w[k];
        S2 += ((unsigned __int128)s2w[k][1] << 64) | s2w[k][0];
        flags |= fw[k];
    }
    const unsigned __int128 N = (unsigned __int128)L * L;
    const unsigned __int128 num = N * S2 - (unsigned __int128)(S1 * S1);
    out->t = t;
    out->N = (uint64_t)N;
    out->S1 = (int64_t)S1;
    out->S2_lo = (uint64_t)S2;
    out->S2_hi = (uint64_t)(S2 >> 64);
    out->num_lo = (uint64_t)num;
    out->num_hi = (uint64_t)(num >> 64);
    out->w2 = 0.0;
    out->status = flags ? -7 : 0;   // SCA_ESTATE
    out->reserved = (int32_t)flags;
}

int obs_partials(uint32_t L)
{
    const TeamShape ts = team_shape(L / 64, 256);
    const int grid = (int)((L + ts.teams - 1) / ts.teams);
    const int cap = sm_count() * 8 < kObsGridCap ? sm_count() * 8 : kObsGridCap;
    return grid < cap ? grid : cap;
}

cudaError_t launch_observe(const uint32_t *A, uint32_t L, int64_t *h0, ObsPartial *partials,
                           ObsDev *result, uint64_t t, cudaStream_t st)
{
    const uint32_t W = L / 64;
    const TeamShape ts = team_shape(W, 256);
    const int grid = obs_partials(L);
    ObsPartial *col_flag = partials + grid;
    k_obs_col0<<<1, 1024, 0, st>>>(A, L, h0, col_flag);
    RowsArgs ra{A, L, W, ts.T, ts.TP, h0, partials};
    if (ts.V == 4) k_obs_rows<4><<<grid, ts.block, 0, st>>>(ra);
    else if (ts.V == 2) k_obs_rows<2><<<grid, ts.block, 0, st>>>(ra);
    else k_obs_rows<1><<<grid, ts.block, 0, st>>>(ra);
    k_obs_final<<<1, 256, 0, st>>>(partials, grid, col_flag, L, t, result);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace sca
