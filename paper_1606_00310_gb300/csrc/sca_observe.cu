// Exact height reconstruction and roughness sums from the canonical packed words.
//
// The paper works with slopes only and names the roughness without defining it (Sec. I.A);
// the definition used here: h(0,0) = 0, h(0,y) = sum of sy-(0,y') for y' = 1..y, and
// h(x,y) = h(0,y) + sum of sx-(x',y) for x' = 1..x (slopes as +-1).  S1 = sum h,
// S2 = sum h^2 (128-bit), num = N * S2 - S1^2 (128-bit); W^2 = num / N^2.  Heights are never
// stored.  With g(x,y) = h(x,y) - h(0,y), every row y reduces to A_y = sum_x g and
// B_y = sum_x g^2 on its own, and
//   S1 = sum_y (L h(0,y) + A_y),   S2 = sum_y (L h(0,y)^2 + 2 h(0,y) A_y + B_y),
// so one kernel reduces every row independently (a warp per row: each lane walks a contiguous
// chunk of words with a table over 8 sites at a time, a warp scan of the chunk totals places
// the chunks) and writes A_y with the row's column-0 slope bit, and a second kernel integrates
// column 0 and combines everything in 128-bit integers.
#include "sca_internal.h"

namespace sca {

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

__device__ __forceinline__ int64_t warp_sum(int64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Table over the 256 values of (4 even-x bits, 4 odd-x bits): for the 8 sites in x order
// (e0, o0, e1, o1, ...), slopes s = 2b - 1, running offsets d_k = s_0 + ... + s_k: byte 0 holds
// S = d_7 + 8 (<= 16), bits 8-23 B = sum d_k^2 (<= 204, eight entries add to at most 1632),
// byte 3 A = sum d_k + 36 (<= 72).
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
    return (uint32_t)(d + 8) | ((uint32_t)sd2 << 8) | ((uint32_t)(sd + 36) << 24);
}

// 64 sites of the even-x word e and the odd-x word o (x order e0, o0, e1, o1, ...), appended to
// a chunk whose running offset is d: sd += sum of offsets, sd2 += sum of squared offsets.
// Block k (8 sites) has the entry (S_k, A_k, B_k) and starts at offset d + dl_k inside the pair,
// dl_k = S_0 + ... + S_{k-1}; the pair adds 64 d + X to sd and 64 d^2 + 2 d X + Z to sd2, with
//   X = 8 sum dl_k + sum A_k,   Z = 8 sum dl_k^2 + 2 sum dl_k A_k + sum B_k.
// The dl_k are formed four to a word as bytes, biased by 64 to lie in [8, 120]: the S bytes of
// four blocks times 0x01010101 are their inclusive prefix sums, shifted up one byte the
// exclusive ones; the sums over blocks are then byte dot products (dp4a), with the biases
// taken out in closed form.  sum B_k comes from one sum of the entries (no field carries).
// tab: the table replicated per lane, entry i of lane l at tab[32 i + l], so the 32 lanes of a
// warp always read 32 different banks.
__device__ __forceinline__ void obs_word_pair(const uint32_t *tab, uint32_t e, uint32_t o, int32_t &d,
                                              int32_t &sd, int64_t &sd2)
{
    // byte m of x0 indexes block 2m (nibble 2m of e and of o), byte m of x1 block 2m + 1
    const uint32_t x0 = (e & 0x0F0F0F0Fu) | ((o << 4) & 0xF0F0F0F0u);
    const uint32_t x1 = ((e >> 4) & 0x0F0F0F0Fu) | (o & 0xF0F0F0F0u);
    uint32_t ent[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        ent[k] = tab[32u * __byte_perm((k & 1) ? x1 : x0, 0u, 0x4440u + (uint32_t)(k >> 1))];
    uint32_t P = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) P += ent[k];
    // S bytes (S0, S1) and A bytes (A0, A1) of blocks 0-3 and 4-7
    const uint32_t l0 = __byte_perm(ent[0], ent[1], 0x7340u), h0 = __byte_perm(ent[2], ent[3], 0x7340u);
    const uint32_t l1 = __byte_perm(ent[4], ent[5], 0x7340u), h1 = __byte_perm(ent[6], ent[7], 0x7340u);
    const uint32_t S0 = __byte_perm(l0, h0, 0x5410u), A0 = __byte_perm(l0, h0, 0x7632u);
    const uint32_t S1 = __byte_perm(l1, h1, 0x5410u), A1 = __byte_perm(l1, h1, 0x7632u);
    const uint32_t I0 = S0 * 0x01010101u, I1 = S1 * 0x01010101u;   // inclusive sums of S + 8
    // byte j: dl + 64 of block j (the constant 64 - 8 j takes out the S biases), of block 4 + j
    const uint32_t D0 = (I0 << 8) + 0x28303840u;
    const uint32_t D1 = (I1 << 8) + (I0 >> 24) * 0x01010101u + 0x08101820u;
    const uint32_t q = __dp4a(D1, D1, __dp4a(D0, D0, 0u));   // sum (dl + 64)^2
    const uint32_t r = __dp4a(D1, A1, __dp4a(D0, A0, 0u));   // sum (dl + 64)(A + 36)
    const uint32_t u = __dp4a(D0 + D1, 0x01010101u, 0u);    // sum (dl + 64)
    const uint32_t a = __dp4a(A0 + A1, 0x01010101u, 0u);    // sum (A + 36)
    const int32_t SB = (int32_t)((P >> 8) & 0xFFFFu);
    const int32_t X = 8 * (int32_t)u + (int32_t)a - 4384;
    const int32_t Z = 8 * (int32_t)q + 2 * (int32_t)r - 1096 * (int32_t)u - 128 * (int32_t)a + 299008 + SB;
    sd += 64 * d + X;
    sd2 += (int64_t)d * (64 * d + 2 * X) + Z;
    d += (int32_t)(I0 >> 24) + (int32_t)(I1 >> 24) - 64;
}

constexpr int kObsRowsWarps = 8;
constexpr int kObsChunkRows = 256;            // rows of one block's chunk, at most
constexpr int kObsChunkCap = kObsGridCap / 2; // chunk records fit the partials scratch

// Column 0 is integrated chunk by chunk: with s(y) the sy- slope of site (0, y), U_c the sum of
// s over the chunk's rows y >= 1, P_c the sum of U over the chunks before c and hl(y) the
// chunk-local inclusive sum, h(0, y) = P_c + hl(y), so each chunk reports sums that only the
// chunk-level prefix P_c completes.
struct ObsChunk {
    int64_t U, SA, Sh, Sh2, ShA;   // slope total; sums of A_y, hl, hl^2, hl A_y over the chunk
    uint64_t SB_lo, SB_hi;         // sum of B_y (128-bit)
    uint32_t n, flags;             // rows; bit 1 a row does not close, bit 2: s(0) = +1
};
static_assert(sizeof(ObsChunk) == 2 * sizeof(ObsPartial), "chunk records fill two partial slots");

// One block reduces the contiguous rows [r0, r1) of the lattice A: one warp per row, lane l
// walks words [l W / 32, (l+1) W / 32) of the row's even-x plane (sublattice y & 1) and odd-x
// plane (sublattice (y & 1) ^ 1), i.e. x in [64 j, 64 j + 64) for each owned word j.
template <bool VEC>
__device__ void obs_rows_chunk(const uint32_t *A, uint32_t L, uint32_t Y, uint32_t r0, uint32_t r1,
                               ObsChunk *chunk)
{
    __shared__ __align__(16) uint32_t tabr[256 * 32];
    __shared__ uint32_t tab0[256];
    __shared__ int64_t sA[kObsChunkRows];
    __shared__ unsigned long long red2[kObsRowsWarps][2];
    __shared__ uint32_t sbits[kObsChunkRows / 32];
    __shared__ uint32_t red_flag;
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) tab0[i] = nibble_pair_entry(i);
    if (threadIdx.x < kObsChunkRows / 32) sbits[threadIdx.x] = 0;
    if (threadIdx.x == 0) red_flag = 0;
    __syncthreads();
    // the per-lane copies: consecutive threads write consecutive 16-byte groups (entry i fills
    // words 32 i .. 32 i + 31), so the stores meet no bank conflict
    for (uint32_t w = threadIdx.x; w < 256 * 8; w += blockDim.x) {
        const uint32_t v = tab0[w >> 3];
        reinterpret_cast<uint4 *>(tabr)[w] = make_uint4(v, v, v, v);
    }
    __syncthreads();
    const uint32_t W = L / 64;                  // L: sites per row; Y: rows
    const size_t plane = (size_t)Y * W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t *tab = tabr + lane;
    const uint32_t c0 = (uint32_t)(((uint64_t)lane * W) / 32), c1 = (uint32_t)(((uint64_t)(lane + 1) * W) / 32);
    const int64_t n = 64 * (int64_t)(c1 - c0);
    unsigned __int128 sB = 0;
    uint32_t flags = 0;
    for (uint32_t y = r0 + warp; y < r1; y += kObsRowsWarps) {
        const uint32_t se = y & 1u, so = se ^ 1u;
        const uint32_t *pe = A + (size_t)(se * 2) * plane + (size_t)y * W;
        const uint32_t *po = A + (size_t)(so * 2) * plane + (size_t)y * W;
        int32_t d = 0, sd = 0;
        int64_t sd2 = 0;
        if constexpr (VEC) {
            // chunks of a lane are a multiple of 4 words (at least 4): 16-byte loads, four word
            // pairs at a time, the next four loaded before these are reduced
            uint4 e = *reinterpret_cast<const uint4 *>(pe + c0);
            uint4 o = *reinterpret_cast<const uint4 *>(po + c0);
            for (uint32_t j = c0; j < c1; j += 4) {
                uint4 en = e, on = o;
                if (j + 4 < c1) {
                    en = *reinterpret_cast<const uint4 *>(pe + j + 4);
                    on = *reinterpret_cast<const uint4 *>(po + j + 4);
                }
                obs_word_pair(tab, e.x, o.x, d, sd, sd2);
                obs_word_pair(tab, e.y, o.y, d, sd, sd2);
                obs_word_pair(tab, e.z, o.z, d, sd, sd2);
                obs_word_pair(tab, e.w, o.w, d, sd, sd2);
                e = en;
                o = on;
            }
        } else {
            for (uint32_t j = c0; j < c1; ++j) obs_word_pair(tab, pe[j], po[j], d, sd, sd2);
        }
        // place the lanes' pieces: E = offset before this lane's first site, from x = 0 inclusive
        const int64_t incl = warp_incl_scan((int64_t)d);
        const int64_t E = incl - d;
        const int64_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        uint32_t w0 = 0, c = 0;
        if (lane == 0) {
            w0 = pe[0];
            c = A[(size_t)(se * 2 + 1) * plane + (size_t)y * W] & 1u;
        }
        w0 = __shfl_sync(0xFFFFFFFFu, w0, 0);
        // g(x) = h(x) - h(0) = offset(x) - s(0): the slope of site 0 is not part of h(0, y)
        const int64_t G = E - (2 * (int64_t)(w0 & 1u) - 1);
        const int64_t Ay = warp_sum(n * G + sd);
        const int64_t By = warp_sum(n * G * G + 2 * G * (int64_t)sd + sd2);
        if (lane == 0) {
            sA[y - r0] = Ay;
            if (c) atomicOr(&sbits[(y - r0) >> 5], 1u << ((y - r0) & 31));
            sB += (unsigned __int128)(uint64_t)By;
            if (total != 0) flags |= 2u;            // the row does not close around x
        }
    }
    if (lane == 0) {
        red2[warp][0] = (uint64_t)sB;
        red2[warp][1] = (uint64_t)(sB >> 64);
        if (flags) atomicOr(&red_flag, flags);
    }
    __syncthreads();
    if (warp != 0) return;
    // warp 0: the chunk's column sums; lane l takes rows [l m / 32, (l+1) m / 32) of the chunk
    const uint32_t m = r1 - r0;
    const uint32_t a0 = (uint32_t)(((uint64_t)lane * m) / 32), a1 = (uint32_t)(((uint64_t)(lane + 1) * m) / 32);
    auto slope = [&](uint32_t i) -> int64_t {       // s(y) for y = r0 + i, 0 for y = 0
        if (r0 + i == 0) return 0;
        return 2 * (int64_t)((sbits[i >> 5] >> (i & 31)) & 1u) - 1;
    };
    int64_t u = 0;
    for (uint32_t i = a0; i < a1; ++i) u += slope(i);
    const int64_t ui = warp_incl_scan(u);
    int64_t hl = ui - u;
    int64_t SA = 0, Sh = 0, Sh2 = 0, ShA = 0;
    for (uint32_t i = a0; i < a1; ++i) {
        hl += slope(i);
        const int64_t Ay = sA[i];
        SA += Ay;
        Sh += hl;
        Sh2 += hl * hl;
        ShA += hl * Ay;
    }
    SA = warp_sum(SA);
    Sh = warp_sum(Sh);
    Sh2 = warp_sum(Sh2);
    ShA = warp_sum(ShA);
    const int64_t Utot = __shfl_sync(0xFFFFFFFFu, ui, 31);
    if (lane == 0) {
        unsigned __int128 t2 = 0;
        for (int w = 0; w < kObsRowsWarps; ++w) t2 += ((unsigned __int128)red2[w][1] << 64) | red2[w][0];
        ObsChunk ch;
        ch.U = Utot;
        ch.SA = SA;
        ch.Sh = Sh;
        ch.Sh2 = Sh2;
        ch.ShA = ShA;
        ch.SB_lo = (uint64_t)t2;
        ch.SB_hi = (uint64_t)(t2 >> 64);
        ch.n = m;
        ch.flags = red_flag | ((r0 == 0 && (sbits[0] & 1u)) ? 4u : 0u);
        *chunk = ch;
    }
}

// Block b owns the contiguous rows [b Y / G, (b+1) Y / G) of the lattice (L sites per row).
template <bool VEC>
__global__ void __launch_bounds__(32 * kObsRowsWarps) k_obs_rows(const uint32_t *A, uint32_t L, uint32_t Y,
                                                                ObsChunk *chunks)
{
    const uint32_t r0 = (uint32_t)(((uint64_t)blockIdx.x * Y) / gridDim.x);
    const uint32_t r1 = (uint32_t)(((uint64_t)(blockIdx.x + 1) * Y) / gridDim.x);
    obs_rows_chunk<VEC>(A, L, Y, r0, r1, chunks + blockIdx.x);
}

// Many lattices of one size: block b takes chunk b % nch of lattice b / nch (first word at
// base + off[lattice]).
__global__ void __launch_bounds__(32 * kObsRowsWarps) k_obs_rows_batch(const uint32_t *base, const uint64_t *off,
                                                                      uint32_t L, uint32_t nch, ObsChunk *chunks)
{
    const uint32_t li = blockIdx.x / nch, c = blockIdx.x - li * nch;
    const uint32_t r0 = (uint32_t)(((uint64_t)c * L) / nch), r1 = (uint32_t)(((uint64_t)(c + 1) * L) / nch);
    obs_rows_chunk<false>(base + off[li], L, L, r0, r1, chunks + blockIdx.x);
}

// One block: thread c takes chunk c, P_c = sum of U over earlier chunks (block scan), then
// with L sites per row and Y rows (N = L Y)
//   S1 = sum_c L (n_c P_c + Sh_c) + SA_c,
//   S2 = sum_c L (n_c P_c^2 + 2 P_c Sh_c + Sh2_c) + 2 (P_c SA_c + ShA_c) + SB_c,
// num = N S2 - S1^2, all in 128-bit integers.  Flags: bit 0 column 0 does not close around y
// (h(0, Y-1) + s(0) != 0), bit 1 some row does not close around x.
constexpr int kObsFinalThreads = 1024;

__device__ __forceinline__ void block_sum_i128(__int128 &v, __int128 *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t lo = __shfl_xor_sync(0xFFFFFFFFu, (uint64_t)v, o);
        const uint64_t hi = __shfl_xor_sync(0xFFFFFFFFu, (uint64_t)((unsigned __int128)v >> 64), o);
        v += (__int128)(((unsigned __int128)hi << 64) | lo);
    }
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        __int128 t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        sh[0] = t;
    }
    __syncthreads();
    v = sh[0];
}

__global__ void __launch_bounds__(kObsFinalThreads) k_obs_final(const ObsChunk *chunks, int nchunks,
                                                                uint32_t L, uint32_t Y, uint64_t t, ObsDev *out,
                                                                const int64_t *h00)
{
    __shared__ __int128 sh[32];
    __shared__ int64_t wsum[32];
    __shared__ uint32_t fl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    ObsChunk ch{};
    if (tid < nchunks) ch = chunks[tid];
    const int64_t incl = warp_incl_scan(ch.U);
    if (tid == 0) fl = 0;
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        v = warp_incl_scan(v);
        wsum[lane] = v;
    }
    __syncthreads();
    const int64_t P = incl - ch.U + (warp > 0 ? wsum[warp - 1] : 0);
    const int64_t col_total = wsum[(blockDim.x >> 5) - 1];
    const __int128 Li = (__int128)L, Pi = (__int128)P, ni = (__int128)ch.n;
    __int128 s1 = Li * (ni * Pi + ch.Sh) + ch.SA;
    __int128 s2 = Li * (ni * Pi * Pi + 2 * Pi * ch.Sh + ch.Sh2) + 2 * (Pi * ch.SA + ch.ShA) +
                  (__int128)(((unsigned __int128)ch.SB_hi << 64) | ch.SB_lo);
    uint32_t flags = __reduce_or_sync(0xFFFFFFFFu, ch.flags);
    if (lane == 0 && flags) atomicOr(&fl, flags);
    block_sum_i128(s1, sh);
    block_sum_i128(s2, sh);
    if (tid != 0) return;
    flags = fl;
    // closure around the y cycle: h(0, Y-1) + s(0) must return to h(0, 0) = 0
    const int64_t s0 = (flags & 4u) ? 1 : -1;
    flags &= 3u;
    if (col_total + s0 != 0) flags |= 1u;
    const unsigned __int128 S2 = (unsigned __int128)s2;
    const unsigned __int128 N = (unsigned __int128)L * Y;
    const unsigned __int128 num = N * S2 - (unsigned __int128)(s1 * s1);
    out->t = t;
    out->N = (uint64_t)N;
    out->S1 = (int64_t)s1;
    out->S2_lo = (uint64_t)S2;
    out->S2_hi = (uint64_t)(S2 >> 64);
    out->num_lo = (uint64_t)num;
    out->num_hi = (uint64_t)(num >> 64);
    out->w2 = 0.0;
    out->status = flags ? -7 : 0;   // SCA_ESTATE
    out->reserved = (int32_t)flags;
    out->h00 = h00 ? *h00 : 0;
}

// Many lattices: one warp per lattice combines its nch (<= 32) chunk records as k_obs_final
// does and writes the record to out[dst[lattice] * stride].
__device__ __forceinline__ __int128 warp_sum_i128(__int128 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t lo = __shfl_xor_sync(0xFFFFFFFFu, (uint64_t)v, o);
        const uint64_t hi = __shfl_xor_sync(0xFFFFFFFFu, (uint64_t)((unsigned __int128)v >> 64), o);
        v += (__int128)(((unsigned __int128)hi << 64) | lo);
    }
    return v;
}

__global__ void k_obs_final_batch(const ObsChunk *chunks, uint32_t nch, uint32_t n_lat, uint32_t L, uint64_t t,
                                  const uint32_t *dst, uint32_t stride, ObsDev *out)
{
    const uint32_t li = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (li >= n_lat) return;                                   // whole warp
    ObsChunk ch{};
    if ((uint32_t)lane < nch) ch = chunks[(size_t)li * nch + lane];
    const int64_t incl = warp_incl_scan(ch.U);
    const int64_t P = incl - ch.U;
    const int64_t col_total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    const __int128 Li = (__int128)L, Pi = (__int128)P, ni = (__int128)ch.n;
    const __int128 s1 = warp_sum_i128(Li * (ni * Pi + ch.Sh) + ch.SA);
    const __int128 s2 = warp_sum_i128(Li * (ni * Pi * Pi + 2 * Pi * ch.Sh + ch.Sh2) + 2 * (Pi * ch.SA + ch.ShA) +
                                      (__int128)(((unsigned __int128)ch.SB_hi << 64) | ch.SB_lo));
    uint32_t flags = __reduce_or_sync(0xFFFFFFFFu, ch.flags);
    if (lane != 0) return;
    const int64_t s0 = (flags & 4u) ? 1 : -1;
    flags &= 3u;
    if (col_total + s0 != 0) flags |= 1u;
    const unsigned __int128 S2 = (unsigned __int128)s2;
    const unsigned __int128 N = (unsigned __int128)L * L;
    const unsigned __int128 num = N * S2 - (unsigned __int128)(s1 * s1);
    ObsDev o;
    o.t = t;
    o.N = (uint64_t)N;
    o.S1 = (int64_t)s1;
    o.S2_lo = (uint64_t)S2;
    o.S2_hi = (uint64_t)(S2 >> 64);
    o.num_lo = (uint64_t)num;
    o.num_hi = (uint64_t)(num >> 64);
    o.w2 = 0.0;
    o.status = flags ? -7 : 0;   // SCA_ESTATE
    o.reserved = (int32_t)flags;
    o.h00 = 0;
    out[(size_t)dst[li] * stride] = o;
}

// ---------------------------------------------------------------------- two-time correlation
// C(t, s) for two states A (the simulation's) and B (a reference) of one X x Y lattice:
// Sa = sum h_a, Sb = sum h_b, Sab = sum h_a h_b, cnum = N Sab - Sa Sb, each height from
// h(0, 0) = 0 as in the roughness.  Per row y, with g = h - h(0, y): A_a = sum_x g_a,
// A_b = sum_x g_b, AB = sum_x g_a g_b, and sum_x h_a h_b = X ha0 hb0 + ha0 A_b + hb0 A_a + AB
// (ha0 = h_a(0, y)).  Column 0 is integrated per chunk as in the roughness (ha0 = P_a + hl_a).
struct CorrChunk {
    int64_t Ua, Ub;            // column-0 slope totals over the chunk's rows y >= 1
    int64_t Sha, Shb, Shab;    // sums of hl_a, hl_b, hl_a hl_b
    int64_t Aa, Ab;            // sums of A_a, A_b
    int64_t ShaAb, ShbAa;      // sums of hl_a A_b, hl_b A_a
    int64_t AB;                // sum of AB
    uint32_t n, flags;         // rows; bit 1 a row does not close, bit 2 / 3: s_a(0) / s_b(0) = +1
    int64_t pad[5];
};
static_assert(sizeof(CorrChunk) == 4 * sizeof(ObsPartial), "a correlation chunk fills four partial slots");
constexpr int kCorrChunkCap = kObsGridCap / 4;

// One warp per row of the chunk [r0, r1); lane l walks words [l W / 32, (l+1) W / 32) of the
// row's even-x and odd-x planes of both states, site by site in x order.
__global__ void __launch_bounds__(32 * kObsRowsWarps) k_corr_rows(const uint32_t *A, const uint32_t *B, uint32_t X,
                                                                 uint32_t Y, CorrChunk *chunks)
{
    __shared__ int64_t sAa[kObsChunkRows], sAb[kObsChunkRows], sAB[kObsChunkRows];
    __shared__ uint32_t bits_a[kObsChunkRows / 32], bits_b[kObsChunkRows / 32];
    __shared__ uint32_t red_flag;
    const uint32_t r0 = (uint32_t)(((uint64_t)blockIdx.x * Y) / gridDim.x);
    const uint32_t r1 = (uint32_t)(((uint64_t)(blockIdx.x + 1) * Y) / gridDim.x);
    if (threadIdx.x < kObsChunkRows / 32) bits_a[threadIdx.x] = bits_b[threadIdx.x] = 0;
    if (threadIdx.x == 0) red_flag = 0;
    __syncthreads();
    const uint32_t W = X / 64;
    const size_t plane = (size_t)Y * W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t c0 = (uint32_t)(((uint64_t)lane * W) / 32), c1 = (uint32_t)(((uint64_t)(lane + 1) * W) / 32);
    const int64_t n = 64 * (int64_t)(c1 - c0);
    for (uint32_t y = r0 + warp; y < r1; y += kObsRowsWarps) {
        const uint32_t se = y & 1u, so = se ^ 1u;
        const size_t oe = (size_t)(se * 2) * plane + (size_t)y * W, oo = (size_t)(so * 2) * plane + (size_t)y * W;
        int32_t da = 0, db = 0;
        int64_t sda = 0, sdb = 0, sdab = 0;
        for (uint32_t j = c0; j < c1; ++j) {
            const uint32_t ea = A[oe + j], oa = A[oo + j], eb = B[oe + j], ob = B[oo + j];
#pragma unroll 8
            for (int k = 0; k < 32; ++k) {
                da += 2 * (int32_t)((ea >> k) & 1u) - 1;
                db += 2 * (int32_t)((eb >> k) & 1u) - 1;
                sda += da;
                sdb += db;
                sdab += (int64_t)da * db;
                da += 2 * (int32_t)((oa >> k) & 1u) - 1;
                db += 2 * (int32_t)((ob >> k) & 1u) - 1;
                sda += da;
                sdb += db;
                sdab += (int64_t)da * db;
            }
        }
        // place the lanes' pieces (E: offset before the lane's first site, from x = 0 inclusive;
        // g(x) = offset(x) - s(0), the slope of site 0 not being part of h(0, y))
        const int64_t ia = warp_incl_scan((int64_t)da), ib = warp_incl_scan((int64_t)db);
        const int64_t ta = __shfl_sync(0xFFFFFFFFu, ia, 31), tb = __shfl_sync(0xFFFFFFFFu, ib, 31);
        uint32_t w0a = 0, w0b = 0, ca = 0, cb = 0;
        if (lane == 0) {
            w0a = A[oe];
            w0b = B[oe];
            ca = A[(size_t)(se * 2 + 1) * plane + (size_t)y * W] & 1u;
            cb = B[(size_t)(se * 2 + 1) * plane + (size_t)y * W] & 1u;
        }
        w0a = __shfl_sync(0xFFFFFFFFu, w0a, 0);
        w0b = __shfl_sync(0xFFFFFFFFu, w0b, 0);
        const int64_t Ga = (ia - da) - (2 * (int64_t)(w0a & 1u) - 1);
        const int64_t Gb = (ib - db) - (2 * (int64_t)(w0b & 1u) - 1);
        const int64_t Aa = warp_sum(n * Ga + sda);
        const int64_t Ab = warp_sum(n * Gb + sdb);
        const int64_t AB = warp_sum(n * Ga * Gb + Ga * sdb + Gb * sda + sdab);
        if (lane == 0) {
            sAa[y - r0] = Aa;
            sAb[y - r0] = Ab;
            sAB[y - r0] = AB;
            if (ca) atomicOr(&bits_a[(y - r0) >> 5], 1u << ((y - r0) & 31));
            if (cb) atomicOr(&bits_b[(y - r0) >> 5], 1u << ((y - r0) & 31));
            if (ta != 0 || tb != 0) atomicOr(&red_flag, 2u);
        }
    }
    __syncthreads();
    if (warp != 0) return;
    const uint32_t m = r1 - r0;
    const uint32_t a0 = (uint32_t)(((uint64_t)lane * m) / 32), a1 = (uint32_t)(((uint64_t)(lane + 1) * m) / 32);
    auto slope = [&](const uint32_t *bits, uint32_t i) -> int64_t {
        if (r0 + i == 0) return 0;
        return 2 * (int64_t)((bits[i >> 5] >> (i & 31)) & 1u) - 1;
    };
    int64_t ua = 0, ub = 0;
    for (uint32_t i = a0; i < a1; ++i) {
        ua += slope(bits_a, i);
        ub += slope(bits_b, i);
    }
    const int64_t uia = warp_incl_scan(ua), uib = warp_incl_scan(ub);
    int64_t hla = uia - ua, hlb = uib - ub;
    int64_t Sha = 0, Shb = 0, Shab = 0, SAa = 0, SAb = 0, ShaAb = 0, ShbAa = 0, SAB = 0;
    for (uint32_t i = a0; i < a1; ++i) {
        hla += slope(bits_a, i);
        hlb += slope(bits_b, i);
        Sha += hla;
        Shb += hlb;
        Shab += hla * hlb;
        SAa += sAa[i];
        SAb += sAb[i];
        ShaAb += hla * sAb[i];
        ShbAa += hlb * sAa[i];
        SAB += sAB[i];
    }
    CorrChunk ch{};
    ch.Ua = __shfl_sync(0xFFFFFFFFu, uia, 31);
    ch.Ub = __shfl_sync(0xFFFFFFFFu, uib, 31);
    ch.Sha = warp_sum(Sha);
    ch.Shb = warp_sum(Shb);
    ch.Shab = warp_sum(Shab);
    ch.Aa = warp_sum(SAa);
    ch.Ab = warp_sum(SAb);
    ch.ShaAb = warp_sum(ShaAb);
    ch.ShbAa = warp_sum(ShbAa);
    ch.AB = warp_sum(SAB);
    if (lane == 0) {
        ch.n = m;
        ch.flags = red_flag | ((r0 == 0 && (bits_a[0] & 1u)) ? 4u : 0u) | ((r0 == 0 && (bits_b[0] & 1u)) ? 8u : 0u);
        chunks[blockIdx.x] = ch;
    }
}

// Result of one correlation (the layout of sca_corr).
struct CorrDev {
    uint64_t t, N;
    int64_t Sa, Sb;
    uint64_t Sab_lo;
    int64_t Sab_hi;
    uint64_t cnum_lo;
    int64_t cnum_hi;
    double c;
    int32_t status, reserved;
};

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *wsum, int64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t incl = warp_incl_scan(v);
    __syncthreads();
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t u = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        wsum[lane] = warp_incl_scan(u);
    }
    __syncthreads();
    *total = wsum[(blockDim.x >> 5) - 1];
    return incl - v + (warp > 0 ? wsum[warp - 1] : 0);
}

__global__ void __launch_bounds__(kCorrChunkCap) k_corr_final(const CorrChunk *chunks, int nchunks, uint32_t X,
                                                             uint32_t Y, uint64_t t, CorrDev *out)
{
    __shared__ __int128 sh[32];
    __shared__ int64_t wsum[32];
    __shared__ uint32_t fl;
    const int tid = threadIdx.x, lane = tid & 31;
    CorrChunk ch{};
    if (tid < nchunks) ch = chunks[tid];
    if (tid == 0) fl = 0;
    int64_t tot_a = 0, tot_b = 0;
    const int64_t Pa = block_excl_scan(ch.Ua, wsum, &tot_a);
    const int64_t Pb = block_excl_scan(ch.Ub, wsum, &tot_b);
    const __int128 Xi = (__int128)X, ni = (__int128)ch.n, pa = (__int128)Pa, pb = (__int128)Pb;
    __int128 sa = Xi * (ni * pa + ch.Sha) + ch.Aa;
    __int128 sb = Xi * (ni * pb + ch.Shb) + ch.Ab;
    __int128 sab = Xi * (ni * pa * pb + pa * ch.Shb + pb * ch.Sha + ch.Shab) + pa * ch.Ab + ch.ShaAb +
                   pb * ch.Aa + ch.ShbAa + ch.AB;
    uint32_t flags = __reduce_or_sync(0xFFFFFFFFu, ch.flags);
    if (lane == 0 && flags) atomicOr(&fl, flags);
    block_sum_i128(sa, sh);
    block_sum_i128(sb, sh);
    block_sum_i128(sab, sh);
    if (tid != 0) return;
    flags = fl;
    uint32_t bad = flags & 2u;
    if (tot_a + ((flags & 4u) ? 1 : -1) != 0) bad |= 1u;    // column 0 of A closes around y
    if (tot_b + ((flags & 8u) ? 1 : -1) != 0) bad |= 1u;    // column 0 of B closes around y
    const __int128 N = (__int128)X * Y;
    const __int128 cnum = N * sab - sa * sb;
    out->t = t;
    out->N = (uint64_t)N;
    out->Sa = (int64_t)sa;
    out->Sb = (int64_t)sb;
    out->Sab_lo = (uint64_t)sab;
    out->Sab_hi = (int64_t)(sab >> 64);
    out->cnum_lo = (uint64_t)cnum;
    out->cnum_hi = (int64_t)(cnum >> 64);
    out->c = 0.0;
    out->status = bad ? -7 : 0;     // SCA_ESTATE
    out->reserved = (int32_t)bad;
}

size_t corr_record_bytes() { return sizeof(CorrDev); }

// chunks of at most kObsChunkRows rows, at most kCorrChunkCap of them, about 4 per SM
static int corr_chunks(uint32_t rows)
{
    int g = sm_count() * 4;
    if (g > kCorrChunkCap) g = kCorrChunkCap;
    if ((uint32_t)g > rows) g = (int)rows;
    while ((rows + g - 1) / g > (uint32_t)kObsChunkRows) g *= 2;
    return g;
}

cudaError_t launch_correlate(const uint32_t *A, const uint32_t *B, uint32_t X, uint32_t Y, ObsPartial *partials,
                             void *result, uint64_t t, cudaStream_t st)
{
    const int grid = corr_chunks(Y);
    if (grid > kCorrChunkCap) return cudaErrorInvalidValue;
    CorrChunk *chunks = reinterpret_cast<CorrChunk *>(partials);
    k_corr_rows<<<grid, 32 * kObsRowsWarps, 0, st>>>(A, B, X, Y, chunks);
    k_corr_final<<<1, kCorrChunkCap, 0, st>>>(chunks, grid, X, Y, t, static_cast<CorrDev *>(result));
    count_launches(2);
    return cudaGetLastError();
}

// Chunks per lattice for the batched observation (rows per chunk at most kObsChunkRows,
// at most 32 chunks).
uint32_t obs_batch_chunks(uint32_t L)
{
    uint32_t nch = 1;
    while ((L + nch - 1) / nch > (uint32_t)kObsChunkRows && nch < 32) nch *= 2;
    if (L >= 1024 && nch < 4) nch = 4;          // keep enough blocks for small ensembles
    return nch;
}

cudaError_t launch_observe_batch(const uint32_t *base, const uint64_t *off, uint32_t n_lat, uint32_t L,
                                 void *chunk_scratch, const uint32_t *dst, uint32_t stride, ObsDev *out,
                                 uint64_t t, cudaStream_t st)
{
    const uint32_t nch = obs_batch_chunks(L);
    ObsChunk *chunks = reinterpret_cast<ObsChunk *>(chunk_scratch);
    k_obs_rows_batch<<<n_lat * nch, 32 * kObsRowsWarps, 0, st>>>(base, off, L, nch, chunks);
    k_obs_final_batch<<<(n_lat * 32 + 255) / 256, 256, 0, st>>>(chunks, nch, n_lat, L, t, dst, stride, out);
    count_launches(2);
    return cudaGetLastError();
}

size_t obs_batch_scratch_bytes(uint32_t n_lat, uint32_t L)
{
    return (size_t)n_lat * obs_batch_chunks(L) * sizeof(ObsChunk);
}

int obs_partials(uint32_t rows)
{
    // chunks of at most kObsChunkRows rows, at most kObsChunkCap of them, about 4 per SM
    int g = sm_count() * 4;
    if (g > kObsChunkCap) g = kObsChunkCap;
    if ((uint32_t)g > rows) g = (int)rows;
    while ((rows + g - 1) / g > (uint32_t)kObsChunkRows) g *= 2;
    return g;
}

// h0: unused (kept in the scratch layout); partials: the chunk records (two partial slots each).
cudaError_t launch_observe(const uint32_t *A, uint32_t L, int64_t *h0, ObsPartial *partials,
                           ObsDev *result, uint64_t t, cudaStream_t st)
{
    (void)h0;
    return launch_observe_xy(A, L, L, partials, result, t, st);
}

cudaError_t launch_observe_xy(const uint32_t *A, uint32_t X, uint32_t Y, ObsPartial *partials, ObsDev *result,
                              uint64_t t, cudaStream_t st, const int64_t *h00)
{
    const uint32_t W = X / 64;
    const int grid = obs_partials(Y);
    if (grid > kObsChunkCap) return cudaErrorInvalidValue;
    ObsChunk *chunks = reinterpret_cast<ObsChunk *>(partials);
    if (W % 128 == 0) k_obs_rows<true><<<grid, 32 * kObsRowsWarps, 0, st>>>(A, X, Y, chunks);
    else k_obs_rows<false><<<grid, 32 * kObsRowsWarps, 0, st>>>(A, X, Y, chunks);
    k_obs_final<<<1, kObsFinalThreads, 0, st>>>(chunks, grid, X, Y, t, result, h00);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace sca
