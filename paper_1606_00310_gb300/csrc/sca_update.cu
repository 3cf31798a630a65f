// Sublattice update of the octahedron-model SCA on the canonical packed words.
//
// Two-pass path (one launch per sublattice, the structure of the paper's algorithm, Fig. 3):
// a "row team" of threads spans one sublattice row, each thread owning V consecutive words
// (128 sites for V = 4, read with one 128-bit load per array).  The only couplings between
// threads are the one-bit shift of sx+ in rows where the neighbour sublattice is offset
// (Sec. II.B: rows of one parity need the rotated word) and the carry of the mask's top bit
// into the next word; both go through shared memory with a barrier, as in the paper, but
// only at team-boundary words (the rest stays in registers).  Rows of one sublattice are
// independent, so every team works on its own rows in any order.
#include <atomic>

#include "sca_internal.h"

namespace sca {

template <int V>
__device__ __forceinline__ void ld_words(const uint32_t *p, uint32_t (&r)[V])
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
__device__ __forceinline__ void st_words(uint32_t *p, const uint32_t (&r)[V])
{
    if constexpr (V == 4) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(r[0], r[1], r[2], r[3]);
    } else if constexpr (V == 2) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(r[0], r[1]);
    } else {
        *p = r[0];
    }
}

struct HalfArgs {
    uint32_t *A;
    uint32_t L, W;       // row length X (sites) and its words per sublattice row
    uint32_t Y;          // rows
    uint64_t t;          // MCS index, or its offset from *t_dev when t_dev is set
    const uint64_t *t_dev;
    int s;
    int T;       // threads owning words in a team
    int TP;      // threads per team (= T)
    Rule R;
};

// MODE 0: p, q in {0,1}; 1: dyadic draws; 2: per-site uniform draws.
template <int V, int MODE>
__global__ void __launch_bounds__(512) k_half_step(const HalfArgs a)
{
    extern __shared__ uint32_t sh[];
    const int tpb = blockDim.x / a.TP;                  // teams per block
    const int team = threadIdx.x / a.TP;
    const int lane = threadIdx.x - team * a.TP;
    const bool owner = lane < a.T;
    uint32_t *sh_first = sh + team * a.TP;              // first sx+ source word of each lane
    uint32_t *sh_carry = sh + tpb * a.TP + team * a.TP; // top mask bit of each lane
    const int s = a.s, ns = s ^ 1;
    const uint32_t L = a.L, W = a.W, Y = a.Y;
    const uint64_t t = a.t_dev ? *a.t_dev + a.t : a.t;
    const size_t plane = (size_t)Y * W;
    uint32_t *Asx = a.A + (size_t)(s * 2 + 0) * plane;
    uint32_t *Asy = a.A + (size_t)(s * 2 + 1) * plane;
    uint32_t *Anx = a.A + (size_t)(ns * 2 + 0) * plane;
    uint32_t *Any = a.A + (size_t)(ns * 2 + 1) * plane;

    for (uint32_t base = blockIdx.x * tpb; base < Y; base += gridDim.x * tpb) {
        const uint32_t y = base + team;
        const bool active = owner && y < Y;
        const uint32_t j = (uint32_t)lane * V;
        const size_t row = (size_t)y * W + j;
        const size_t rown = (size_t)(y + 1 == Y ? 0 : y + 1) * W + j;
        const bool shifted = ((s + y) & 1u) != 0;

        uint32_t xm[V], ym[V], nx[V], ny[V];
        if (active) {
            ld_words<V>(Asx + row, xm);
            ld_words<V>(Asy + row, ym);
            ld_words<V>(Anx + row, nx);
            ld_words<V>(Any + rown, ny);
            sh_first[lane] = nx[0];
        }
        __syncthreads();
        uint32_t m[V];
        if (active) {
            uint32_t xpl[V];
            if (shifted) {
                const uint32_t next = sh_first[lane + 1 == a.T ? 0 : lane + 1];
#pragma unroll
                for (int v = 0; v < V; ++v)
                    xpl[v] = (nx[v] >> 1) | ((v + 1 < V ? nx[(v + 1) % V] : next) << 31);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) xpl[v] = nx[v];
            }
            uint32_t xip[V], xiq[V];
            if constexpr (MODE == 0) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    xip[v] = a.R.Pp ? 0xFFFFFFFFu : 0u;
                    xiq[v] = a.R.Pq ? 0xFFFFFFFFu : 0u;
                }
            } else if constexpr (MODE == 1) {
                xi_dyadic<V>(a.R, a.R.rk, row, t, s, xip, xiq);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const uint32_t need = eligible(xm[v], ym[v], xpl[v], ny[v]);
                    xi_uniform_word(a.R, a.R.rk, (uint64_t)y * (L / 2) + 32u * (j + v), t, s,
                                    need, xip[v], xiq[v]);
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                m[v] = update_mask(xm[v], ym[v], xpl[v], ny[v], xip[v], xiq[v]);
                xm[v] ^= m[v];
                ym[v] ^= m[v];
                ny[v] ^= m[v];
            }
            st_words<V>(Asx + row, xm);
            st_words<V>(Asy + row, ym);
            st_words<V>(Any + rown, ny);
            if (!shifted) {
#pragma unroll
                for (int v = 0; v < V; ++v) nx[v] ^= m[v];
                st_words<V>(Anx + row, nx);
            } else {
                sh_carry[lane] = m[V - 1] >> 31;
            }
        }
        __syncthreads();
        if (active && shifted) {
            // sx- of the offset neighbour sublattice: site k's partner is site k+1, so the
            // mask moves up one bit, and word j's top bit enters word j+1 (periodic in x).
            const uint32_t cin = sh_carry[lane == 0 ? a.T - 1 : lane - 1];
#pragma unroll
            for (int v = 0; v < V; ++v)
                nx[v] ^= (m[v] << 1) | (v == 0 ? cin : (m[(v + V - 1) % V] >> 31));
            st_words<V>(Anx + row, nx);
        }
    }
}

static TeamShape team_shape_v(uint32_t W, int V, int max_block)
{
    TeamShape ts;
    ts.V = V;
    ts.T = (int)(W / ts.V);
    // teams packed back to back: the kernel couples a team's threads through shared memory
    // and block barriers only, so a warp may span two teams, and no lane idles for padding
    // (rows of W = 100 words, say, would leave 7 of every 32 lanes idle in power-of-two teams)
    ts.TP = ts.T;
    ts.teams = ts.TP >= max_block ? 1 : max_block / ts.TP;
    ts.block = ts.teams * ts.TP;
    return ts;
}

TeamShape team_shape(uint32_t W, int max_block)
{
    return team_shape_v(W, (W % 4 == 0) ? 4 : (W % 2 == 0) ? 2 : 1, max_block);
}

static uint64_t g_launches = 0;
void count_launches(uint64_t n) { __atomic_fetch_add(&g_launches, n, __ATOMIC_RELAXED); }
uint64_t launches_total() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <int V, int MODE>
static cudaError_t launch_half_v(const HalfArgs &a, const TeamShape &ts, cudaStream_t st)
{
    const int rows_per_block = ts.teams;
    int grid = (int)((a.Y + rows_per_block - 1) / rows_per_block);
    const int cap = sm_count() * (2048 / ts.block);
    if (grid > cap) grid = cap;
    const size_t smem = 2 * sizeof(uint32_t) * ts.block;
    k_half_step<V, MODE><<<grid, ts.block, smem, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

// Resident warps per SM of the per-site uniform kernel with V words per thread (asked once per
// V with 128-thread blocks; registers bound it, so the count is per warp).
static int uniform_warps_per_sm(int V)
{
    static std::atomic<int> cached[3];
    int w = cached[V].load(std::memory_order_relaxed);
    if (w == 0) {
        int n = 0;
        cudaError_t e = V == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_half_step<1, 2>, 128, 2 * 4 * 128)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_half_step<2, 2>, 128, 2 * 4 * 128);
        w = (e == cudaSuccess && n > 0) ? 4 * n : 4;
        cached[V].store(w, std::memory_order_relaxed);
    }
    return w;
}

// Team shape of a per-site uniform half-step.  Each word costs eight Philox calls, so on a
// lattice too small to fill the GPU the launch lasts about as long as one thread's chain of
// calls, and fewer words per thread shorten it.  The fewest words per thread (1, then 2) whose
// warps still fit within 1.2 resident waves is taken (blocks of about 128 threads; a row team
// of more than 512 threads, the kernel's bound, rules a count out), else the default shape.
// Measured on GB300 (two-pass kernel alone): L = 4096 8.2e11 against 6.8e11 updates/s with
// four words per thread, L = 2048 3.4e11 against 2.6e11, L = 1024 1.3e11 against 6.4e10;
// L >= 8192 keeps four words per thread.
static TeamShape uniform_shape(uint32_t W, uint32_t Y)
{
    for (int v = 1; v <= 2; ++v) {
        if (W % (uint32_t)v || W / (uint32_t)v > 512u) continue;
        const TeamShape ts = team_shape_v(W, v, 128);
        const uint64_t blocks = ((uint64_t)Y + ts.teams - 1) / ts.teams;
        const uint64_t warps = blocks * (uint64_t)((ts.block + 31) / 32);
        const uint64_t resident = (uint64_t)sm_count() * (uint64_t)uniform_warps_per_sm(v);
        if (5 * warps <= 6 * resident) return ts;
    }
    return team_shape(W, 256);
}

cudaError_t launch_half_step(uint32_t *A, uint32_t L, uint64_t t, int s, const Rule &R,
                             cudaStream_t st, const uint64_t *t_dev)
{
    return launch_half_step_xy(A, L, L, t, s, R, st, t_dev);
}

cudaError_t launch_half_step_xy(uint32_t *A, uint32_t X, uint32_t Y, uint64_t t, int s, const Rule &R,
                                cudaStream_t st, const uint64_t *t_dev)
{
    const uint32_t W = X / 64;
    const TeamShape ts = R.mode == 2 ? uniform_shape(W, Y) : team_shape(W, 256);
    HalfArgs a{A, X, W, Y, t, t_dev, s, ts.T, ts.TP, R};
    const int mode = (int)R.mode;
#define SCA_HALF(VV)                                                        \
    if (ts.V == VV) {                                                       \
        if (mode == 0) return launch_half_v<VV, 0>(a, ts, st);              \
        if (mode == 1) return launch_half_v<VV, 1>(a, ts, st);              \
        return launch_half_v<VV, 2>(a, ts, st);                             \
    }
    SCA_HALF(4)
    SCA_HALF(2)
    SCA_HALF(1)
#undef SCA_HALF
    return cudaErrorInvalidValue;
}

}  // namespace sca

namespace sca {

// Advance a device-resident MCS counter (used by replayed step graphs).
__global__ void k_add_t(uint64_t *t_dev, uint64_t n) { *t_dev += n; }
__global__ void k_set_t(uint64_t *t_dev, uint64_t v) { *t_dev = v; }

cudaError_t launch_add_t(uint64_t *t_dev, uint64_t n, cudaStream_t st)
{
    k_add_t<<<1, 1, 0, st>>>(t_dev, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_set_t(uint64_t *t_dev, uint64_t v, cudaStream_t st)
{
    k_set_t<<<1, 1, 0, st>>>(t_dev, v);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sca
