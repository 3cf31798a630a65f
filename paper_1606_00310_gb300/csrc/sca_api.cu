// C ABI of the single-lattice simulation (declared in include/sca.h).
//
// A simulation owns two canonical-word buffers (the fused update reads one and writes the
// other; the two-pass update works in place), the observation scratch, and a stream.  The
// host side only validates, lays out memory and enqueues kernels; all dynamics and all
// observables are computed by the kernels in sca_update.cu / sca_observe.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sca.h"
#include "sca_internal.h"

static_assert(sizeof(sca_obs) == sizeof(sca::ObsDev), "sca_obs layout");

namespace sca {
uint64_t launches_total();
thread_local std::string g_last_error;

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    return fail(SCA_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// p = P / 2^n with P odd (n = 0 for p in {0, 1}); false if p is not a multiple of 2^-32.
static bool split_dyadic(double p, uint32_t &P, uint32_t &n)
{
    const double scaled = std::ldexp(p, 32);
    if (!(scaled >= 0.0 && scaled <= 4294967296.0) || scaled != std::floor(scaled)) return false;
    uint64_t v = (uint64_t)scaled;
    if (v == 0) { P = 0; n = 0; return true; }
    int tz = __builtin_ctzll(v);
    if (tz > 32) tz = 32;
    P = (uint32_t)(v >> tz);
    n = 32u - (uint32_t)tz;
    return true;
}

int make_rule(const sca_params &prm, Rule &R)
{
    if (!(prm.p >= 0.0 && prm.p <= 1.0) || !(prm.q >= 0.0 && prm.q <= 1.0))
        return fail(SCA_EINVAL, "p and q must lie in [0, 1]");
    std::memset(&R, 0, sizeof(R));
    R.k0 = (uint32_t)prm.seed;
    R.k1 = (uint32_t)(prm.seed >> 32);
    for (uint32_t r = 0; r < 10; ++r) {          // Philox key schedule, round r
        R.rk[2 * r] = R.k0 + r * 0x9E3779B9u;
        R.rk[2 * r + 1] = R.k1 + r * 0xBB67AE85u;
    }
    uint32_t Pp, np, Pq, nq;
    const bool dy = split_dyadic(prm.p, Pp, np) && split_dyadic(prm.q, Pq, nq);
    uint32_t rng = prm.rng;
    if (rng == SCA_RNG_AUTO) rng = dy ? SCA_RNG_DYADIC : SCA_RNG_UNIFORM32;
    if (rng == SCA_RNG_DYADIC) {
        if (!dy) return fail(SCA_EINVAL, "dyadic mode needs p and q to be multiples of 2^-32");
        R.Pp = Pp; R.np = np; R.Pq = Pq; R.nq = nq;
        R.n_draws = np > nq ? np : nq;
        R.mode = R.n_draws == 0 ? 0u : 1u;
    } else if (rng == SCA_RNG_UNIFORM32) {
        R.Tp = (uint64_t)std::floor(std::ldexp(prm.p, 32));
        R.Tq = (uint64_t)std::floor(std::ldexp(prm.q, 32));
        const bool trivial = (R.Tp == 0 || R.Tp == (1ull << 32)) && (R.Tq == 0 || R.Tq == (1ull << 32));
        R.mode = trivial ? 0u : 2u;
        R.Pp = R.Tp == (1ull << 32);   // used when mode == 0
        R.Pq = R.Tq == (1ull << 32);
    } else {
        return fail(SCA_EINVAL, "unknown rng mode");
    }
    return SCA_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }


// X sites per row (a multiple of 64), Y rows (even); both at most 131072.
static bool layout_for(uint32_t X, uint32_t Y, Layout &lo)
{
    if (X < 64 || X % 64 != 0 || X > 131072) return false;
    if (Y < 2 || Y % 2 != 0 || Y > 131072) return false;
    const size_t W = X / 64;
    lo.state_bytes = 4 * (size_t)Y * W * sizeof(uint32_t);
    lo.off_b = align256(lo.state_bytes);
    lo.off_h0 = lo.off_b + align256(lo.state_bytes);
    lo.off_part = lo.off_h0 + align256((size_t)Y * sizeof(int64_t));
    lo.off_res = lo.off_part + align256((size_t)(kObsGridCap + 1) * sizeof(ObsPartial));
    lo.off_err = lo.off_res + align256((size_t)kResCap * sizeof(ObsDev));
    lo.total = lo.off_err + 256;
    return true;
}

}  // namespace sca

using namespace sca;

static void finish_obs(sca_obs &o)
{
    const double num = std::ldexp((double)o.num_hi, 64) + (double)o.num_lo;
    const double N = (double)o.N;
    o.w2 = num / (N * N);
}

extern "C" {

size_t sca_workspace_bytes(uint32_t L)
{
    Layout lo;
    return layout_for(L, L, lo) ? lo.total : 0;
}

size_t sca_workspace_bytes_xy(uint32_t X, uint32_t Y)
{
    Layout lo;
    return layout_for(X, Y, lo) ? lo.total : 0;
}

int sca_init(const sca_params *params, void *stream, void *dev_buf, size_t dev_buf_bytes,
             sca_sim **out)
{
    if (!params || !out) return fail(SCA_EINVAL, "NULL argument");
    *out = nullptr;
    Layout lo;
    const uint32_t Y = params->Ly ? params->Ly : params->L;
    if (!layout_for(params->L, Y, lo))
        return fail(SCA_EINVAL, "L must be a multiple of 64 in [64, 131072] and Ly even in [2, 131072]");
    Rule R;
    int rc = make_rule(*params, R);
    if (rc) return rc;
    if (params->dynamics > SCA_DYN_RANDOM_SEQUENTIAL) return fail(SCA_EINVAL, "unknown dynamics");
    if (params->dynamics == SCA_DYN_RANDOM_SEQUENTIAL && !rs_supported(params->L, Y))
        return fail(SCA_EINVAL, "random-sequential dynamics needs Y a multiple of 8");
    if (dev_buf) {
        if (dev_buf_bytes < lo.total) return fail(SCA_EINVAL, "device buffer too small");
        if ((uintptr_t)dev_buf % 256 != 0) return fail(SCA_EINVAL, "device buffer not 256-byte aligned");
    }
    sca_sim *s = new sca_sim();
    s->R = R;
    s->L = params->L;
    s->W = params->L / 64;
    s->Ly = Y;
    s->dynamics = params->dynamics;
    s->rs_Tp = (uint64_t)std::floor(std::ldexp(params->p, 32));
    s->rs_Tq = (uint64_t)std::floor(std::ldexp(params->q, 32));
    s->lo = lo;
    s->t = 0;
    s->kernel = 0;
    s->fused_V = 0;
    s->fused_ring = 0;
    s->tb_k = 4;
    s->tb_set = false;
    s->wave_bands = 0;
    s->surface = true;
    s->chk_host = nullptr;
    s->chk_ev = nullptr;
    s->chk_pending = false;
    s->async_obs = 0;
    s->cur = 0;
    s->timing = false;
    s->timed_launches = 0;
    if (stream) {
        s->stream = (cudaStream_t)stream;
        s->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete s; return cuda_fail(e, "cudaStreamCreate"); }
        s->own_stream = true;
    }
    if (dev_buf) {
        s->base = (char *)dev_buf;
        s->own_mem = false;
    } else {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, lo.total);
        if (e != cudaSuccess) {
            if (s->own_stream) cudaStreamDestroy(s->stream);
            delete s;
            return fail(SCA_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        s->base = (char *)p;
        s->own_mem = true;
    }
    s->buf[0] = (uint32_t *)s->base;
    s->buf[1] = (uint32_t *)(s->base + lo.off_b);
    s->h0 = (int64_t *)(s->base + lo.off_h0);
    s->part = (ObsPartial *)(s->base + lo.off_part);
    s->res = (ObsDev *)(s->base + lo.off_res);
    s->err = (uint32_t *)(s->base + lo.off_err);
    s->h00 = (int64_t *)(s->base + lo.off_err + 8);
    s->track_origin = false;
    {
        cudaError_t e = cudaMemsetAsync(s->err, 0, 16, s->stream);
        if (e != cudaSuccess) {
            sca_free(s);
            return cuda_fail(e, "cudaMemsetAsync");
        }
    }
    int rc2 = sca_reset(s);
    if (rc2) {
        sca_free(s);
        return rc2;
    }
    *out = s;
    return SCA_OK;
}

int sca_reset(sca_sim *s)
{
    if (!s) return fail(SCA_EINVAL, "NULL simulation");
    // flat surface: sublattice 0 slopes all -1 (bits 0), sublattice 1 all +1 (bits 1)
    const size_t half = s->lo.state_bytes / 2;
    cudaError_t e = cudaMemsetAsync(s->buf[s->cur], 0x00, half, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync((char *)s->buf[s->cur] + half, 0xFF, half, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->h00, 0, sizeof(int64_t), s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    s->t = 0;
    s->surface = true;
    s->chk_pending = false;
    return SCA_OK;
}

int sca_set_kernel(sca_sim *s, int kernel)
{
    if (!s || kernel < 0 || kernel > 4) return fail(SCA_EINVAL, "kernel must be 0, 1, 2, 3 or 4");
    if ((kernel == 2 || kernel == 3) && s->Ly != s->L)
        return fail(SCA_EINVAL, "kernels 2 and 3 take square lattices only");
    if (kernel == 2 && !fused_supported(s->L))
        return fail(SCA_EINVAL, "fused kernel needs L to be a multiple of 2048");
    if (kernel == 3) {
        uint32_t ns;
        size_t sm;
        if (!tblock_plan(s->L, (uint32_t)s->tb_k, &ns, &sm))
            return fail(SCA_EINVAL, "temporal blocking does not fit this lattice size");
    }
    if (kernel == 4) {
        if (!wave_supported_xy(s->L, s->Ly, (uint32_t)wave_max_k((int)s->R.mode), (int)s->R.mode))
            return fail(SCA_EINVAL, "the wavefront kernel does not fit this lattice size");
    }
    s->kernel = kernel;
    return SCA_OK;
}

int sca_set_wave_bands(sca_sim *s, int bands)
{
    if (!s || bands < 0 || (uint32_t)bands > s->Ly / 2)
        return fail(SCA_EINVAL, "bands must be 0 (automatic) or 1..Y/2");
    s->wave_bands = (uint32_t)bands;
    return SCA_OK;
}

int sca_set_temporal_block(sca_sim *s, int mcs_per_launch)
{
    if (!s) return fail(SCA_EINVAL, "NULL simulation");
    const int k = mcs_per_launch > 0 ? mcs_per_launch : 4;
    if (k > 64 || (64 % k) != 0) return fail(SCA_EINVAL, "MCS per launch must divide 64");
    if (s->kernel == 4 || s->Ly != s->L) {   // launches of the largest supported power of two <= k
        s->tb_k = k;
        s->tb_set = true;
        return SCA_OK;
    }
    uint32_t ns;
    size_t sm;
    if (!tblock_plan(s->L, (uint32_t)k, &ns, &sm))
        return fail(SCA_EINVAL, "temporal blocking does not fit this lattice size");
    s->tb_k = k;
    s->tb_set = true;
    return SCA_OK;
}

}  // extern "C"

// Automatic kernel choice (measured on GB300).  For a surface state the register-wavefront
// kernel (4) wins wherever the lattice gives it enough tiles: with {0, 1} probabilities from
// L = 4096 on (8 MCS per launch up to L = 8192, 16 above); with dyadic draws from L = 32768 on
// for one or two draws per word and from L = 65536 on for three (MCS per launch: 4 for one draw
// with q = 0, 1 for three draws with q != 0 -- the Philox chains leave no registers for a deeper
// window -- and 2 otherwise); four or more draws
// run at the fused kernel's speed or below.  Otherwise the fused kernel halves HBM traffic once
// the state is far larger than L2 and the update is not arithmetic-bound; shared-memory
// temporal blocking (several MCS per launch) wins while the lattice is small enough that
// launches and L2 round trips dominate (dyadic draws up to L = 8192, per-site uniforms up to
// L = 2048); the two-pass kernel covers the rest.
// For an X x Y lattice the thresholds apply to the area (X Y >= L^2), and the MCS per launch
// are held to at most Y/8 (a band of rows is at least 8 K rows tall, so the recomputed halo
// stays at most half of what a band streams).
static bool area_at_least(const sca_sim *s, uint64_t L) { return (uint64_t)s->L * s->Ly >= L * L; }

static uint32_t wave_default_k(const sca_sim *s)
{
    const Rule &R = s->R;
    uint32_t k;
    if (R.mode == 0) {
        k = area_at_least(s, 16384) ? 16u : 8u;
    } else if (R.mode == 2) {
        k = 2u;
    } else {
        const bool q0 = R.nq == 0 && R.Pq == 0;
        if (R.n_draws == 1 && q0) k = 4u;       // p = 1/2: the lightest draws, the deepest window
        else k = R.n_draws >= 3 && !q0 ? 1u : 2u;
    }
    while (k > 1 && 8u * k > s->Ly) k /= 2;
    return k;
}

static bool wave_auto(const sca_sim *s)
{
    if (!s->surface) return false;
    const Rule &R = s->R;
    if (R.mode == 0) return area_at_least(s, 4096);
    if (R.mode != 1 || s->L % 256 != 0) return false;
    if (R.n_draws <= 2) return area_at_least(s, 32768);
    return R.n_draws == 3 && area_at_least(s, 65536);
}

// An asynchronous state load decides `surface` when its check completes; the first decision
// that needs it waits for that check (the copy and one pass over the state, on this stream).
static int resolve_surface(sca_sim *s)
{
    if (!s->chk_pending) return SCA_OK;
    cudaError_t e = cudaEventSynchronize(s->chk_ev);
    if (e != cudaSuccess) return cuda_fail(e, "surface check");
    s->surface = surface_from(s->chk_host, s->L, s->Ly);
    s->chk_pending = false;
    return SCA_OK;
}

int sca::effective_kernel(const sca_sim *s, int *tb_k)
{
    int k = s->kernel;
    int kk = s->tb_k;
    const int mode = (int)s->R.mode;
    const bool square = s->Ly == s->L;
    if (k == 4) kk = (int)wave_pick_k(s->tb_set ? (uint32_t)kk : wave_default_k(s), mode);
    if (k == 0) {
        uint32_t ns;
        size_t sm;
        const bool wave_ok = wave_auto(s) && wave_supported_xy(s->L, s->Ly, wave_default_k(s), mode);
        if (wave_ok) {
            k = 4;
            kk = (int)wave_pick_k(s->tb_set ? (uint32_t)kk : wave_default_k(s), mode);
        } else if (!square) {                   // X != Y: the two-pass kernel covers the rest
            k = 1;
        } else if (fused_supported(s->L) && s->L >= 32768 && s->R.mode != 2) {
            k = 2;
        } else if (s->R.mode != 2 && s->L <= 8192 && tblock_plan(s->L, s->tb_set ? kk : 8, &ns, &sm)) {
            k = 3;
            if (!s->tb_set) kk = 8;
        } else if (s->R.mode == 2 && s->L <= 2048 && tblock_plan(s->L, s->tb_set ? kk : 4, &ns, &sm)) {
            k = 3;
            if (!s->tb_set) kk = 4;
        } else {
            k = 1;
        }
    }
    if (tb_k) *tb_k = kk;
    return k;
}

bool sca::use_fused(const sca_sim *s) { return effective_kernel(s, nullptr) == 2; }

extern "C" {

}  // extern "C"

static cudaError_t record_event(sca_sim *s)
{
    cudaEvent_t e;
    cudaError_t rc = cudaEventCreate(&e);
    if (rc != cudaSuccess) return rc;
    s->ev.push_back(e);
    return cudaEventRecord(e, s->stream);
}

int sca_set_fused_shape(sca_sim *s, int words_per_thread, int ring)
{
    if (!s) return fail(SCA_EINVAL, "NULL simulation");
    if (words_per_thread == 0) {
        s->fused_V = 0;
        s->fused_ring = 0;
        return SCA_OK;
    }
    if (!fused_shape_ok(s->L, words_per_thread, ring))
        return fail(SCA_EINVAL, "fused shape does not fit this lattice size");
    s->fused_V = words_per_thread;
    s->fused_ring = ring;
    return SCA_OK;
}

int sca_get_kernel(const sca_sim *s)
{
    if (!s) return fail(SCA_EINVAL, "NULL simulation");
    if (s->dynamics == SCA_DYN_RANDOM_SEQUENTIAL) return 5;
    int rc = resolve_surface(const_cast<sca_sim *>(s));
    if (rc) return rc;
    return effective_kernel(s, nullptr);
}

#ifndef SCA_WAVE_SX_SKIP
#define SCA_WAVE_SX_SKIP 1
#endif

int sca::step_impl(sca_sim *s, uint64_t n)
{
    if (n == 0) return SCA_OK;
    {
        int rc = resolve_surface(s);
        if (rc) return rc;
    }
    if (s->dynamics == SCA_DYN_RANDOM_SEQUENTIAL) {  // in place, the other buffer as local words
        if (s->timing) {
            cudaError_t e = record_event(s);
            if (e != cudaSuccess) return cuda_fail(e, "timing event");
        }
        cudaError_t e = launch_rs(s->buf[s->cur], s->buf[s->cur ^ 1], s->L, s->Ly, s->t, n, s->R, s->rs_Tp,
                                  s->rs_Tq, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "random-sequential launch");
        s->t += n;
        if (s->timing) {
            s->timed_launches += 2 * n;
            e = record_event(s);
            if (e != cudaSuccess) return cuda_fail(e, "timing event");
        }
        return SCA_OK;
    }
    int tbk = 0;
    const int kern = effective_kernel(s, &tbk);
    const bool fused = kern == 2;
    if (kern == 4 && !s->surface)
        return fail(SCA_ESTATE, "the wavefront kernel needs a surface state (every plaquette closes)");
    if (s->track_origin && !s->surface)
        return fail(SCA_ESTATE, "tracking the origin's height needs a surface state");
    if (s->track_origin && tbk > origin_max_k()) tbk = origin_max_k();
    if (kern == 3 || kern == 4) {              // temporal blocking: tbk MCS per launch
        if (s->timing) {
            cudaError_t e = record_event(s);
            if (e != cudaSuccess) return cuda_fail(e, "timing event");
        }
        uint64_t done = 0, launches = 0;
        while (done < n) {
            const uint64_t k = (n - done) < (uint64_t)tbk ? (n - done) : (uint64_t)tbk;
            const uint64_t kk = kern == 3 ? k : wave_pick_k((uint32_t)k, (int)s->R.mode);
            // a wavefront launch followed by one of the same plan leaves the sx- planes to it,
            // except the rows that launch starts its bands from; the last one writes them all
            bool sx_all = true;
            if (SCA_WAVE_SX_SKIP && kern == 4 && !s->track_origin) {
                const uint64_t rest = n - done - kk;
                const uint64_t k2 = rest < (uint64_t)tbk ? rest : (uint64_t)tbk;
                sx_all = rest == 0 || wave_pick_k((uint32_t)k2, (int)s->R.mode) != kk;
            }
            if (s->track_origin) {           // the launch's MCS re-run around the origin first
                cudaError_t e = launch_origin_track(s->buf[s->cur], s->L, s->Ly, s->t + done,
                                                    (uint32_t)(kern == 3 ? k : kk), s->R, s->h00, s->stream);
                if (e != cudaSuccess) return cuda_fail(e, "origin tracker launch");
            }
            cudaError_t e = kern == 3
                ? launch_tblock(s->buf[s->cur], s->buf[s->cur ^ 1], s->L, s->t + done, (uint32_t)k,
                                s->R, s->stream)
                : launch_wave_xy(s->buf[s->cur], s->buf[s->cur ^ 1], s->L, s->Ly, s->t + done, (uint32_t)kk,
                                 s->R, s->stream, nullptr, s->wave_bands, sx_all);
            if (e != cudaSuccess) {
                s->t += done;
                return cuda_fail(e, "temporal-blocking launch");
            }
            s->cur ^= 1;
            done += kern == 3 ? k : kk;
            ++launches;
        }
        s->t += n;
        if (s->timing) {
            s->timed_launches += launches;
            cudaError_t e = record_event(s);
            if (e != cudaSuccess) return cuda_fail(e, "timing event");
        }
        return SCA_OK;
    }
    if (s->timing) {
        cudaError_t e = record_event(s);
        if (e != cudaSuccess) return cuda_fail(e, "timing event");
    }
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t t = s->t + i;
        cudaError_t e;
        if (s->track_origin) {
            e = launch_origin_track(s->buf[s->cur], s->L, s->Ly, t, 1u, s->R, s->h00, s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "origin tracker launch");
        }
        if (fused) {
            e = launch_fused_mcs(s->buf[s->cur], s->buf[s->cur ^ 1], s->L, t, s->R, s->err,
                                 s->stream, nullptr, s->fused_V, s->fused_ring);
            if (e == cudaSuccess) s->cur ^= 1;
        } else {
            e = launch_half_step_xy(s->buf[s->cur], s->L, s->Ly, t, 0, s->R, s->stream);
            if (e == cudaSuccess) e = launch_half_step_xy(s->buf[s->cur], s->L, s->Ly, t, 1, s->R, s->stream);
        }
        if (e != cudaSuccess) {
            s->t = t;
            return cuda_fail(e, "update launch");
        }
    }
    s->t += n;
    if (s->timing) {
        s->timed_launches += fused ? n : 2 * n;
        cudaError_t e = record_event(s);
        if (e != cudaSuccess) return cuda_fail(e, "timing event");
    }
    return SCA_OK;
}

extern "C" {

static void clear_events(sca_sim *s)
{
    for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
    s->ev.clear();
    s->timed_launches = 0;
}

int sca_step(sca_sim *s, uint64_t n_mcs)
{
    if (!s) return fail(SCA_EINVAL, "NULL simulation");
    return step_impl(s, n_mcs);
}

int sca_run(sca_sim *s, const uint64_t *times, uint32_t n, sca_obs *out)
{
    if (!s || (n && (!times || !out))) return fail(SCA_EINVAL, "NULL argument");
    uint64_t prev = s->t;
    for (uint32_t i = 0; i < n; ++i) {
        if (times[i] < prev) return fail(SCA_EINVAL, "observation times must be non-decreasing");
        prev = times[i];
    }
    int first_bad = SCA_OK;
    uint32_t done = 0;
    while (done < n) {
        const uint32_t chunk = (n - done) < (uint32_t)kResCap ? (n - done) : (uint32_t)kResCap;
        for (uint32_t i = 0; i < chunk; ++i) {
            int rc = step_impl(s, times[done + i] - s->t);
            if (rc) return rc;
            cudaError_t e = launch_observe_xy(s->buf[s->cur], s->L, s->Ly, s->part, s->res + i, s->t,
                                              s->stream, s->track_origin ? s->h00 : nullptr);
            if (e != cudaSuccess) return cuda_fail(e, "observe launch");
        }
        uint32_t err = 0;
        cudaError_t e = cudaMemcpyAsync(out + done, s->res, chunk * sizeof(ObsDev),
                                        cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&err, s->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "observe copy");
        if (err) {
            cudaMemsetAsync(s->err, 0, sizeof(uint32_t), s->stream);
            return fail(SCA_ETIMEOUT, "an update kernel's pipeline wait gave up; state invalid");
        }
        for (uint32_t i = 0; i < chunk; ++i) {
            finish_obs(out[done + i]);
            if (out[done + i].status && !first_bad) first_bad = out[done + i].status;
        }
        done += chunk;
    }
    if (first_bad) return fail(first_bad, "slopes do not close around the torus");
    return SCA_OK;
}

int sca_observe(sca_sim *s, sca_obs *out)
{
    if (!s || !out) return fail(SCA_EINVAL, "NULL argument");
    const uint64_t t = s->t;
    return sca_run(s, &t, 1, out);
}

int sca_track_origin(sca_sim *s, int enable)
{
    if (!s) return fail(SCA_EINVAL, "NULL simulation");
    if (enable && s->dynamics != SCA_DYN_SCA)
        return fail(SCA_EINVAL, "the origin's height is tracked for the SCA dynamics only");
    cudaError_t e = cudaMemsetAsync(s->h00, 0, sizeof(int64_t), s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sca_track_origin");
    s->track_origin = enable != 0;
    return SCA_OK;
}

int sca_correlate(sca_sim *s, const uint32_t *ref_words_dev, sca_corr *out)
{
    if (!s || !ref_words_dev || !out) return fail(SCA_EINVAL, "NULL argument");
    if (s->async_obs) return fail(SCA_EBUSY, "collect the asynchronous run's records first (sca_wait)");
    static_assert(sizeof(sca_corr) <= kResCap * sizeof(ObsDev), "the record fits the result area");
    if (corr_record_bytes() != sizeof(sca_corr)) return fail(SCA_ECUDA, "correlation record layout");
    cudaError_t e = launch_correlate(s->buf[s->cur], ref_words_dev, s->L, s->Ly, s->part, s->res, s->t,
                                     s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, s->res, sizeof(sca_corr), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sca_correlate");
    const double cn = std::ldexp((double)out->cnum_hi, 64) + (double)out->cnum_lo;
    const double N = (double)out->N;
    out->c = cn / (N * N);
    if (out->status) return fail(out->status, "slopes do not close around the torus");
    return SCA_OK;
}

int sca_get_state(sca_sim *s, uint32_t *host_words, size_t n_words)
{
    if (!s || !host_words) return fail(SCA_EINVAL, "NULL argument");
    if (n_words * sizeof(uint32_t) < s->lo.state_bytes) return fail(SCA_EINVAL, "host buffer too small");
    cudaError_t e = cudaMemcpyAsync(host_words, s->buf[s->cur], s->lo.state_bytes,
                                    cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? SCA_OK : cuda_fail(e, "sca_get_state");
}

int sca_set_state(sca_sim *s, const uint32_t *host_words, size_t n_words, uint64_t t)
{
    if (!s || !host_words) return fail(SCA_EINVAL, "NULL argument");
    if (n_words * sizeof(uint32_t) != s->lo.state_bytes) return fail(SCA_EINVAL, "wrong word count");
    cudaError_t e = cudaMemcpyAsync(s->buf[s->cur], host_words, s->lo.state_bytes,
                                    cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->h00, 0, sizeof(int64_t), s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sca_set_state");
    bool surf = false;
    e = surface_check(s->buf[s->cur], s->L, s->Ly, reinterpret_cast<uint32_t *>(s->part), s->stream, &surf);
    if (e != cudaSuccess) return cuda_fail(e, "surface check");
    s->surface = surf;
    s->chk_pending = false;
    s->t = t;
    return SCA_OK;
}

int sca_set_state_async(sca_sim *s, const uint32_t *host_words, size_t n_words, uint64_t t)
{
    if (!s || !host_words) return fail(SCA_EINVAL, "NULL argument");
    if (n_words * sizeof(uint32_t) != s->lo.state_bytes) return fail(SCA_EINVAL, "wrong word count");
    if (!s->chk_host) {
        cudaError_t e = cudaMallocHost(&s->chk_host, 4 * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->chk_ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "sca_set_state_async");
    }
    cudaError_t e = cudaMemcpyAsync(s->buf[s->cur], host_words, s->lo.state_bytes,
                                    cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->h00, 0, sizeof(int64_t), s->stream);
    if (e == cudaSuccess)
        e = surface_check_async(s->buf[s->cur], s->L, s->Ly, reinterpret_cast<uint32_t *>(s->part), s->chk_host,
                                s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->chk_ev, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sca_set_state_async");
    s->chk_pending = true;
    s->t = t;
    return SCA_OK;
}

int sca_get_state_async(sca_sim *s, uint32_t *host_words, size_t n_words)
{
    if (!s || !host_words) return fail(SCA_EINVAL, "NULL argument");
    if (n_words * sizeof(uint32_t) < s->lo.state_bytes) return fail(SCA_EINVAL, "host buffer too small");
    cudaError_t e = cudaMemcpyAsync(host_words, s->buf[s->cur], s->lo.state_bytes,
                                    cudaMemcpyDeviceToHost, s->stream);
    return e == cudaSuccess ? SCA_OK : cuda_fail(e, "sca_get_state_async");
}

int sca_run_async(sca_sim *s, const uint64_t *times, uint32_t n)
{
    if (!s || (n && !times)) return fail(SCA_EINVAL, "NULL argument");
    if (n > (uint32_t)kResCap) return fail(SCA_EINVAL, "at most 64 observation times per asynchronous run");
    uint64_t prev = s->t;
    for (uint32_t i = 0; i < n; ++i) {
        if (times[i] < prev) return fail(SCA_EINVAL, "observation times must be non-decreasing");
        prev = times[i];
    }
    s->async_obs = 0;
    for (uint32_t i = 0; i < n; ++i) {
        int rc = step_impl(s, times[i] - s->t);
        if (rc) return rc;
        cudaError_t e = launch_observe_xy(s->buf[s->cur], s->L, s->Ly, s->part, s->res + i, s->t, s->stream,
                                          s->track_origin ? s->h00 : nullptr);
        if (e != cudaSuccess) return cuda_fail(e, "observe launch");
    }
    s->async_obs = n;
    return SCA_OK;
}

int sca_wait(sca_sim *s, sca_obs *out, uint32_t n)
{
    if (!s || (n && !out)) return fail(SCA_EINVAL, "NULL argument");
    if (n > s->async_obs) return fail(SCA_EINVAL, "more records than the last asynchronous run made");
    // the records and the error word are read on the simulation's own stream, behind its work,
    // so waiting never involves another stream's copies or kernels
    uint32_t err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, s->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess && n)
        e = cudaMemcpyAsync(out, s->res, n * sizeof(ObsDev), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sca_wait");
    s->async_obs = 0;
    if (err) {
        cudaMemsetAsync(s->err, 0, sizeof(uint32_t), s->stream);
        return fail(SCA_ETIMEOUT, "an update kernel's pipeline wait gave up; state invalid");
    }
    int first_bad = SCA_OK;
    for (uint32_t i = 0; i < n; ++i) {
        finish_obs(out[i]);
        if (out[i].status && !first_bad) first_bad = out[i].status;
    }
    if (first_bad) return fail(first_bad, "slopes do not close around the torus");
    return SCA_OK;
}

int sca_state_device(sca_sim *s, uint32_t **words_dev)
{
    if (!s || !words_dev) return fail(SCA_EINVAL, "NULL argument");
    *words_dev = s->buf[s->cur];
    return SCA_OK;
}

uint64_t sca_time(const sca_sim *s) { return s ? s->t : 0; }

int sca_timing(sca_sim *s, int enable)
{
    if (!s) return fail(SCA_EINVAL, "NULL simulation");
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sca_timing");
    if (enable) clear_events(s);
    s->timing = enable != 0;
    return SCA_OK;
}

int sca_timing_read(sca_sim *s, double *update_ms, uint64_t *update_launches)
{
    if (!s || !update_ms || !update_launches) return fail(SCA_EINVAL, "NULL argument");
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sca_timing_read");
    double total = 0.0;
    for (size_t i = 0; i + 1 < s->ev.size(); i += 2) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, s->ev[i], s->ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        total += ms;
    }
    *update_ms = total;
    *update_launches = s->timed_launches;
    return SCA_OK;
}

void sca_free(sca_sim *s)
{
    if (!s) return;
    clear_events(s);
    if (s->own_stream) {
        cudaStreamSynchronize(s->stream);
        cudaStreamDestroy(s->stream);
    } else {
        cudaStreamSynchronize(s->stream);
    }
    if (s->own_mem) cudaFree(s->base);
    if (s->chk_host) cudaFreeHost(s->chk_host);
    if (s->chk_ev) cudaEventDestroy(s->chk_ev);
    delete s;
}

const char *sca_strerror(int status)
{
    switch (status) {
    case SCA_OK: return "ok";
    case SCA_EINVAL: return "invalid argument";
    case SCA_ENOMEM: return "out of device memory";
    case SCA_ECUDA: return "CUDA error";
    case SCA_EBUDGET: return "request exceeds the device-memory budget";
    case SCA_ETIMEOUT: return "timed out";
    case SCA_EBUSY: return "busy";
    case SCA_ESTATE: return "slopes do not close around the torus";
    case SCA_ENOTFOUND: return "unknown ticket";
    case SCA_ECANCELED: return "cancelled";
    default: return "unknown status";
    }
}

const char *sca_last_error(void) { return g_last_error.c_str(); }

int sca_selftest_wait_timeout(uint32_t limit_us)
{
    if (limit_us == 0 || limit_us > 2000000) return fail(SCA_EINVAL, "limit must be 1 us .. 2 s");
    int dev = 0, khz = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    const long long cycles = (long long)limit_us * (khz > 0 ? khz : 2000000) / 1000;
    uint32_t *err = nullptr;
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocAsync(&err, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = launch_wait_selftest(cycles, err, st);
    uint32_t h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (err) cudaFreeAsync(err, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    return h ? fail(SCA_ETIMEOUT, "the wait gave up as designed") : SCA_OK;
}

uint64_t sca_kernel_launches(void) { return launches_total(); }

}  // extern "C"
