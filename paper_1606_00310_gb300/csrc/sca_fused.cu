// Fused even+odd update: one launch per MCS, state read once and written once.
//
// The paper's kernel (Fig. 3) makes one pass over all rows per sublattice, so every slope bit
// crosses the memory bus twice in each direction per MCS (Sec. III accounting).  Here one CTA
// owns a slab of rows [y0, y1) and walks it as a wavefront: the odd half-step of row r-1
// needs the even half-step of rows r-2, r-1 and r only, so after the even update of row r the
// odd update of row r-1 can run, and row r-2 is final.  The CTA reads its rows plus a halo of
// two rows above and two below from the source buffer and writes only its own rows to the
// destination buffer (ping-pong), so slabs never race.  Halo rows are updated again by the
// neighbouring slab with identical results because the random bits are a pure function of
// (seed, MCS, sublattice, word).
//
// Data movement: whole lattice rows (all four role planes) stream through a ring of shared
// memory slots.  One elected thread issues 1D TMA bulk copies (cp.async.bulk) global->shared
// with an mbarrier per slot and bulk stores shared->global once a row is final; every thread
// updates its V words per plane in shared memory.  Word-boundary couplings (the rotated sx+
// word and the mask carry, paper Sec. II.B) go through shared memory: the carry of one
// half-step is applied after the next barrier, which the pipeline needs anyway.
#include "sca_internal.h"

namespace sca {

constexpr int kMaxRing = 12;              // row slots: 3 in use, the rest prefetch/store in flight
constexpr int kHeader = 256;              // mbarriers (2 x kMaxRing x 8 bytes) before the carries
constexpr long long kWaitCycles = 1ll << 31;   // ~1 s at 2 GHz before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, uint32_t bytes,
                                          uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst_smem)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_store(void *dst, const void *src_smem, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Wait until at most N bulk-store groups still read shared memory (N is an immediate).
template <int N>
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait until the mbarrier phase with `parity` completes, giving up after limit_cycles: then set
// *abort (shared, so the rest of the CTA stops waiting at once) and bit 0 of *err (read by the
// host) and return false.  Never traps and never spins without bound.
__device__ __forceinline__ bool bounded_wait(uint64_t *bar, uint32_t parity, long long limit_cycles,
                                             volatile int *abort, uint32_t *err)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long start = clock64();
    while (!*abort) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - start > limit_cycles) {
            *abort = 1;
            atomicOr(err, 1u);
        }
    }
    return false;
}

// Self-test of the wait limit: one thread waits on an mbarrier that nothing ever completes.
__global__ void k_wait_selftest(long long limit_cycles, uint32_t *err)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ volatile int abort_flag;
    if (threadIdx.x != 0) return;
    abort_flag = 0;
    mbar_init(&bar, 1);
    fence_mbar_init();
    bounded_wait(&bar, 0u, limit_cycles, &abort_flag, err);
}

cudaError_t launch_wait_selftest(long long limit_cycles, uint32_t *err, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(limit_cycles, err);
    count_launches(1);
    return cudaGetLastError();
}

struct FusedArgs {
    const uint32_t *src;
    uint32_t *dst;
    uint32_t L, W;
    int T;              // threads per CTA = W / V
    int nslabs;
    int ring;           // row slots in shared memory (6, 8 or 12)
    uint64_t t;         // MCS index, or its offset from *t_dev when t_dev is set
    const uint64_t *t_dev;
    Rule R;
    uint32_t *err;      // bit 0: a wait gave up
};

template <int V>
__device__ __forceinline__ void lds(const uint32_t *p, uint32_t (&r)[V])
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
__device__ __forceinline__ void sts(uint32_t *p, const uint32_t (&r)[V])
{
    if constexpr (V == 4) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(r[0], r[1], r[2], r[3]);
    } else if constexpr (V == 2) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(r[0], r[1]);
    } else {
        *p = r[0];
    }
}

// One half-step on one row held in shared memory.  own_x/own_y: the updated sublattice's sx-
// and sy- words of this row; nb_x: the other sublattice's sx- words of this row (sx+ source);
// nb_yn: the other sublattice's sy- words of the next row (sy+).  In a shifted row the mask
// enters nb_x one bit up and the top bit of each thread's last word is published in carry[]
// for the owner of the next word, who applies it after the next barrier.
template <int V, int MODE, int ND>
__device__ __forceinline__ void half_row(uint32_t *own_x, uint32_t *own_y, uint32_t *nb_x,
                                         uint32_t *nb_yn, bool shifted, int lane, int T,
                                         uint32_t W, const Rule &R, uint32_t y, uint32_t L,
                                         uint64_t t, int s, uint32_t *carry)
{
    const uint32_t j = (uint32_t)lane * V;
    uint32_t xm[V], ym[V], nx[V], ny[V], xpl[V];
    lds<V>(own_x + j, xm);
    lds<V>(own_y + j, ym);
    lds<V>(nb_x + j, nx);
    lds<V>(nb_yn + j, ny);
    if (shifted) {
        const uint32_t next = nb_x[(j + V == W) ? 0 : j + V];   // only bit 0 is used
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
        xi_dyadic_any<V, ND>(R, R.rk, (uint64_t)y * W + j, t, s, xip, xiq);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const uint32_t need = eligible(xm[v], ym[v], xpl[v], ny[v]);
            xi_uniform_word(R, R.rk, (uint64_t)y * (L / 2) + 32u * (j + v), t, s, need, xip[v], xiq[v]);
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
    sts<V>(own_x + j, xm);
    sts<V>(own_y + j, ym);
    sts<V>(nb_yn + j, ny);
    if (!shifted) {
#pragma unroll
        for (int v = 0; v < V; ++v) nx[v] ^= m[v];
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) nx[v] ^= (m[v] << 1) | (v > 0 ? (m[(v + V - 1) % V] >> 31) : 0u);
        carry[lane] = m[V - 1] >> 31;
    }
    sts<V>(nb_x + j, nx);
    (void)T;
}

// Warp-specialized pipeline.  T compute threads update rows in shared memory; one extra
// producer warp (one elected thread) owns all TMA traffic.  RING row slots; full[s] completes
// when a row's four planes have landed in slot s, rel[s] when the compute threads are done with
// the row in slot s (released rows 2..n+1 are final and get stored; rows 0 and 1 are halo).
// The producer takes releases in row order: store the row (if it is one of the slab's), wait
// until the store has read the slot, load the row RING further down into it.  Row k is
// released at loop step k+2, and the row needed at step r (r+1) was released at step
// r+3-RING < r for RING >= 6, so neither side can wait on the other in a cycle.
template <int V, int MODE, int ND, int RING>
__global__ void __launch_bounds__(544) k_fused_mcs(const FusedArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ volatile int abort_wait;
    const uint32_t W = a.W, L = a.L;
    const int T = a.T;
    const int lane = threadIdx.x;
    const uint64_t tt = a.t_dev ? *a.t_dev + a.t : a.t;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *rel = full + RING;
    uint32_t *cE = reinterpret_cast<uint32_t *>(smem + kHeader);
    uint32_t *cO = cE + T;
    const size_t ring_off = (kHeader + 8 * (size_t)T + 127) & ~(size_t)127;
    uint32_t *ring = reinterpret_cast<uint32_t *>(smem + ring_off);
    const size_t plane = (size_t)L * W;
    const uint32_t row_bytes = W * 4u;

    const uint32_t b = blockIdx.x;
    const uint32_t y0 = (uint32_t)(((uint64_t)b * L) / a.nslabs);
    const uint32_t y1 = (uint32_t)(((uint64_t)(b + 1) * L) / a.nslabs);
    const int n = (int)(y1 - y0);
    const int total = n + 4;                 // rows y0-2 .. y1+1
    auto gy = [&](int r) -> uint32_t { return (uint32_t)(((int64_t)y0 - 2 + r + 2 * (int64_t)L) % L); };
    auto slot = [&](int r) -> uint32_t * { return ring + (size_t)(r % RING) * 4 * W; };
    auto wait_bar = [&](uint64_t *bar, uint32_t parity) {
        bounded_wait(bar, parity, kWaitCycles, &abort_wait, a.err);
    };

    if (lane == 0) {
        abort_wait = 0;
        for (int i = 0; i < RING; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&rel[i], 1);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (lane >= T) {
        // ------------------------------------------------------------------ producer warp
        if (lane != T) return;
        auto issue_load = [&](int r) {
            uint64_t *bar = &full[r % RING];
            mbar_expect_tx(bar, 4 * row_bytes);
            uint32_t *d = slot(r);
            const size_t row = (size_t)gy(r) * W;
#pragma unroll
            for (int pl = 0; pl < 4; ++pl)
                bulk_load(d + (size_t)pl * W, a.src + (size_t)pl * plane + row, row_bytes, bar);
        };
        for (int r = 0; r < RING && r < total; ++r) issue_load(r);
        for (int k = 0; k <= n + 1; ++k) {
            wait_bar(&rel[k % RING], (uint32_t)((k / RING) & 1));
            if (k >= 2) {
                const uint32_t *sl = slot(k);
                const size_t row = (size_t)gy(k) * W;
#pragma unroll
                for (int pl = 0; pl < 4; ++pl)
                    bulk_store(a.dst + (size_t)pl * plane + row, sl + (size_t)pl * W, row_bytes);
                bulk_commit();
            }
            if (k + RING < total) {
                bulk_wait_read<0>();         // the slot's last reader was that store
                issue_load(k + RING);
            }
        }
        bulk_wait_all();
        if (abort_wait) {
            // a wait gave up: let the loads still in flight land before shared memory goes
            // away (each slot's last load, bounded like every other wait)
            for (int k = 0; k < RING && k < total; ++k) {
                const int last = k + ((total - 1 - k) / RING) * RING;
                const long long start = clock64();
                while (!mbar_try_wait(&full[k], (uint32_t)((last / RING) & 1)) &&
                       clock64() - start < kWaitCycles) {
                }
            }
        }
        return;
    }

    // ---------------------------------------------------------------------- compute threads
    auto sync_compute = [&]() { asm volatile("bar.sync 1, %0;" ::"r"(T) : "memory"); };
    auto wait_row = [&](int r) { wait_bar(&full[r % RING], (uint32_t)((r / RING) & 1)); };
    auto release = [&](int r) {
        if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&rel[r % RING]))
                         : "memory");
    };
    // plane order in a slot: 0 = A[0][x], 1 = A[0][y], 2 = A[1][x], 3 = A[1][y]
    auto even_row = [&](int r) {      // sublattice 0 at row r, reads rows r and r+1
        const uint32_t y = gy(r);
        uint32_t *cur = slot(r), *nxt = slot(r + 1);
        half_row<V, MODE, ND>(cur, cur + W, cur + 2 * W, nxt + 3 * W, (y & 1u) != 0, lane, T, W, a.R,
                              y, L, tt, 0, cE);
    };
    auto odd_row = [&](int r) {       // sublattice 1 at row r, reads rows r and r+1
        const uint32_t y = gy(r);
        uint32_t *cur = slot(r), *nxt = slot(r + 1);
        half_row<V, MODE, ND>(cur + 2 * W, cur + 3 * W, cur, nxt + W, (y & 1u) == 0, lane, T, W, a.R,
                              y, L, tt, 1, cO);
    };
    auto prev_lane = [&]() { return lane == 0 ? T - 1 : lane - 1; };

    wait_row(0);
    wait_row(1);
    even_row(0);          // only its sy+ effect on row 1 matters
    for (int r = 1; r <= n + 2; ++r) {
        wait_row(r + 1);
        // phase E: finish the odd update of row r-2 (its carry), then the even update of row r
        if (r - 2 >= 1 && (gy(r - 2) & 1u) == 0)
            slot(r - 2)[(size_t)lane * V] ^= cO[prev_lane()];
        even_row(r);
        fence_proxy_async();
        sync_compute();
        // row r-2 is final (or, for r-2 < 2, a halo row no longer needed): hand it over
        if (r >= 2) release(r - 2);
        // phase O: finish the even update of row r, then the odd update of row r-1
        if (gy(r) & 1u) slot(r)[2 * W + (size_t)lane * V] ^= cE[prev_lane()];
        if (r >= 2) odd_row(r - 1);
        sync_compute();
    }
    // epilogue: carry of the odd update of row n+1 (= y1-1), then hand it over
    if ((gy(n + 1) & 1u) == 0) slot(n + 1)[(size_t)lane * V] ^= cO[prev_lane()];
    fence_proxy_async();
    sync_compute();
    release(n + 1);
}

// Launch shape: V words per thread per plane (T = W / V threads per CTA) and the ring depth.
// Default: V = 4 with 6 slots (two CTAs per SM at L = 65536); sca_set_fused_shape can pick
// another shape (results do not depend on it).
struct FusedShape { int V, ring; };

static bool shape_ok(uint32_t L, FusedShape sh)
{
    if (L % 2048 != 0) return false;
    const uint32_t W = L / 64;
    if (W % (uint32_t)sh.V != 0 || !(sh.ring == 6 || ((sh.ring == 8 || sh.ring == 12) && sh.V == 4)))
        return false;
    const int T = (int)(W / sh.V);
    return T >= 32 && T <= 512 && T % 32 == 0;
}

static FusedShape default_shape(uint32_t L)
{
    const uint32_t W = L / 64;
    FusedShape sh{(W % 128 == 0) ? 4 : 1, 6};
    if (!shape_ok(L, sh)) sh.V = (W % 64 == 0 && shape_ok(L, FusedShape{2, 6})) ? 2 : sh.V;
    return sh;
}

bool fused_supported(uint32_t L) { return shape_ok(L, default_shape(L)); }

bool fused_shape_ok(uint32_t L, int V, int ring) { return shape_ok(L, FusedShape{V, ring}); }

static size_t smem_for(uint32_t L, FusedShape sh)
{
    const uint32_t W = L / 64;
    const int T = (int)(W / sh.V);
    const size_t ring_off = (kHeader + 8 * (size_t)T + 127) & ~(size_t)127;
    return ring_off + (size_t)sh.ring * 4 * W * sizeof(uint32_t);
}

size_t fused_smem_bytes(uint32_t L) { return smem_for(L, default_shape(L)); }

template <int V, int MODE, int ND, int RING>
static cudaError_t launch_fused_r(FusedArgs a, size_t smem, cudaStream_t st)
{
    auto kern = k_fused_mcs<V, MODE, ND, RING>;
    // raise the shared-memory limit once, to what the largest lattice needs, so no later launch
    // (including one being captured into a graph) has to change a kernel attribute
    static int configured_smem = 0;
    if (configured_smem == 0) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        cudaError_t e0 = cudaFuncGetAttributes(&fa, kern);
        if (e0 != cudaSuccess) return e0;
        const int want = optin - (int)fa.sharedSizeBytes;   // every shape that fits is allowed
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        if (e != cudaSuccess) return e;
        configured_smem = want;
    }
    if ((int)smem > configured_smem) return cudaErrorInvalidConfiguration;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, a.T + 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = sm_count() * per_sm;
    const int max_slabs = (int)(a.L / 8);     // at least 8 rows per slab
    if (grid > max_slabs) grid = max_slabs;
    a.nslabs = grid;
    kern<<<grid, a.T + 32, smem, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int V, int MODE, int ND>
static cudaError_t launch_fused_v(FusedArgs a, size_t smem, cudaStream_t st)
{
    if (a.ring == 6) return launch_fused_r<V, MODE, ND, 6>(a, smem, st);
    if constexpr (V == 4) {            // deeper rings only with 4 words per thread
        if (a.ring == 8) return launch_fused_r<V, MODE, ND, 8>(a, smem, st);
        if (a.ring == 12) return launch_fused_r<V, MODE, ND, 12>(a, smem, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fused_mcs(const uint32_t *src, uint32_t *dst, uint32_t L, uint64_t t,
                             const Rule &R, uint32_t *err, cudaStream_t st, const uint64_t *t_dev,
                             int V_req, int ring_req)
{
    FusedShape sh = default_shape(L);
    if (V_req > 0) sh = FusedShape{V_req, ring_req};
    if (!shape_ok(L, sh)) return cudaErrorNotSupported;
    const uint32_t W = L / 64;
    const int V = sh.V;
    FusedArgs a{src, dst, L, W, (int)(W / V), 0, sh.ring, t, t_dev, R, err};
    const size_t smem = smem_for(L, sh);
    const int mode = (int)R.mode;
#define SCA_FUSED_V(VV)                                                         \
    if (V == VV) {                                                              \
        if (mode == 0) return launch_fused_v<VV, 0, 0>(a, smem, st);            \
        if (mode == 2) return launch_fused_v<VV, 2, 0>(a, smem, st);            \
        switch (R.n_draws) {                                                    \
        case 1: return launch_fused_v<VV, 1, 1>(a, smem, st);                   \
        case 2: return launch_fused_v<VV, 1, 2>(a, smem, st);                   \
        case 3: return launch_fused_v<VV, 1, 3>(a, smem, st);                   \
        case 4: return launch_fused_v<VV, 1, 4>(a, smem, st);                   \
        default: return launch_fused_v<VV, 1, 0>(a, smem, st);                  \
        }                                                                       \
    }
    SCA_FUSED_V(4)
    SCA_FUSED_V(2)
    SCA_FUSED_V(1)
#undef SCA_FUSED_V
    return cudaErrorInvalidValue;
}

}  // namespace sca
