// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "sca_rng.cuh"

namespace sca {

// Launch shape of a "row team": T threads own W words of one sublattice row, V words each;
// a team's threads share only the block's shared memory, so teams sit back to back.
struct TeamShape {
    int V;          // words per thread per row (1, 2 or 4)
    int T;          // threads that own words
    int TP;         // threads per team (= T; teams are packed back to back)
    int teams;      // teams per block
    int block;      // threads per block = teams * TP
};
TeamShape team_shape(uint32_t W, int max_block);

// Device-side result of one observation (the layout of sca_obs without w2 filled).
struct ObsDev {
    uint64_t t, N;
    int64_t S1;
    uint64_t S2_lo, S2_hi, num_lo, num_hi;
    double w2;
    int32_t status, reserved;
    int64_t h00;        // absolute height of the origin (0 when it is not tracked)
};

struct ObsPartial {
    int64_t s1;
    uint64_t s2_lo, s2_hi;
    uint32_t flags, pad;
};

// Update kernels.  A is the canonical word array (in place for the two-pass path); src/dst
// for the fused path.  Launch counts are added to the library's counter.
// t_dev: when set, the MCS index is *t_dev + t, read by the kernel (lets a captured graph of
// steps be replayed; launch_add_t / launch_set_t maintain the counter).
cudaError_t launch_half_step(uint32_t *A, uint32_t L, uint64_t t, int s, const Rule &R,
                             cudaStream_t st, const uint64_t *t_dev = nullptr);
// The same on an X x Y lattice (X sites per row, Y rows); launch_half_step is X = Y = L.
cudaError_t launch_half_step_xy(uint32_t *A, uint32_t X, uint32_t Y, uint64_t t, int s, const Rule &R,
                                cudaStream_t st, const uint64_t *t_dev = nullptr);
cudaError_t launch_add_t(uint64_t *t_dev, uint64_t n, cudaStream_t st);
cudaError_t launch_set_t(uint64_t *t_dev, uint64_t v, cudaStream_t st);
// err: device word; bit 0 is set if a pipeline wait gave up (the result is then invalid).
// V_req / ring_req: launch shape (words per thread, row slots); 0 = default for L.
cudaError_t launch_fused_mcs(const uint32_t *src, uint32_t *dst, uint32_t L, uint64_t t,
                             const Rule &R, uint32_t *err, cudaStream_t st,
                             const uint64_t *t_dev = nullptr, int V_req = 0, int ring_req = 0);
bool fused_supported(uint32_t L);
cudaError_t launch_wait_selftest(long long limit_cycles, uint32_t *err, cudaStream_t st);
// Temporal blocking: k MCS per launch, src -> dst (ping-pong), MCS index t0 (+ *t_dev if set).
cudaError_t launch_tblock(const uint32_t *src, uint32_t *dst, uint32_t L, uint64_t t0, uint32_t k,
                          const Rule &R, cudaStream_t st, const uint64_t *t_dev = nullptr);
bool tblock_plan(uint32_t L, uint32_t k, uint32_t *nslabs, size_t *smem);
// Register-wavefront temporal blocking on height bits: k MCS per launch (a power of two up to
// wave_max_k(mode)), src -> dst (ping-pong); bands of rows per column of tiles (0 = automatic).
// Needs a surface state (surface_check); dyadic and {0,1} probabilities only.
cudaError_t launch_wave(const uint32_t *src, uint32_t *dst, uint32_t L, uint64_t t0, uint32_t k,
                        const Rule &R, cudaStream_t st, const uint64_t *t_dev = nullptr,
                        uint32_t bands = 0);
// The same on an X x Y lattice (X sites per row, Y rows).  sx_all false: the output's sx-
// planes are written only on the rows the next launch of the same plan (same k and bands)
// integrates its first rows from; the output is then a valid state only for such a launch.
cudaError_t launch_wave_xy(const uint32_t *src, uint32_t *dst, uint32_t X, uint32_t Y, uint64_t t0, uint32_t k,
                           const Rule &R, cudaStream_t st, const uint64_t *t_dev = nullptr,
                           uint32_t bands = 0, bool sx_all = true);
bool wave_supported(uint32_t L, uint32_t k, int mode);
bool wave_supported_xy(uint32_t X, uint32_t Y, uint32_t k, int mode);
int wave_max_k(int mode);
uint32_t wave_pick_k(uint32_t want, int mode);   // largest supported power of two <= want
// Is A a surface (every plaquette closes, row 0 and column 0 close around the torus)?  Uses 3
// words of device scratch; synchronises the stream.
cudaError_t surface_check(const uint32_t *A, uint32_t X, uint32_t Y, uint32_t *scratch, cudaStream_t st,
                          bool *is_surface);
// The same check enqueued only: the three result words land in host3 (pinned) when the stream
// gets there; surface_from() reads them.  X sites per row, Y rows.
cudaError_t surface_check_async(const uint32_t *A, uint32_t X, uint32_t Y, uint32_t *scratch, uint32_t *host3,
                                cudaStream_t st);
bool surface_from(const uint32_t *host3, uint32_t X, uint32_t Y);
bool fused_shape_ok(uint32_t L, int V, int ring);
size_t fused_smem_bytes(uint32_t L);

// Streaming engine of the batch (sca_wave_batch.cu): one work item per (lattice, band).
struct WBItem {
    uint64_t off;       // first canonical word of the lattice in the batch state buffers
    uint32_t k0, k1;    // the lattice's Philox key (seed low / high)
    uint32_t y0;        // first row of the band
    uint32_t pad;
};
bool wave_batch_supported(uint32_t L, const Rule &R);
int wave_batch_max_k(const Rule &R);
cudaError_t launch_wave_batch(const uint32_t *src, uint32_t *dst, const WBItem *items, uint32_t n_items,
                              uint32_t L, uint32_t rows_per_band, uint64_t t0, uint32_t k, const Rule &R,
                              cudaStream_t st, bool sx_all = true);
cudaError_t launch_wave_batch_copy(const uint32_t *src, uint32_t *dst, const WBItem *items, uint32_t n_items,
                                   uint32_t L, cudaStream_t st);
// Batched observation of n_lat lattices of size L (first words at base + off[i]); record of
// lattice i to out[dst[i] * stride]; chunk scratch of obs_batch_scratch_bytes(n_lat, L).
cudaError_t launch_observe_batch(const uint32_t *base, const uint64_t *off, uint32_t n_lat, uint32_t L,
                                 void *chunk_scratch, const uint32_t *dst, uint32_t stride, ObsDev *out,
                                 uint64_t t, cudaStream_t st);
size_t obs_batch_scratch_bytes(uint32_t n_lat, uint32_t L);

// Observation kernels: h0 scratch of L int64; partials scratch of obs_partials(L) + 1 entries
// (never more than kObsGridCap + 1).
constexpr int kObsGridCap = 2048;
int obs_partials(uint32_t rows);
cudaError_t launch_observe(const uint32_t *A, uint32_t L, int64_t *h0, ObsPartial *partials,
                           ObsDev *result, uint64_t t, cudaStream_t st);
// The same on an X x Y lattice (X sites per row, Y rows; N = X * Y).
// h00: the origin-height counter copied into the record (nullptr: 0).
cudaError_t launch_observe_xy(const uint32_t *A, uint32_t X, uint32_t Y, ObsPartial *partials, ObsDev *result,
                              uint64_t t, cudaStream_t st, const int64_t *h00 = nullptr);
// Origin-height tracker (sca_origin.cu): re-runs K <= origin_max_k() MCS from the state A (MCS
// index t0) on a patch around the origin and adds the origin's height change to *h00.
cudaError_t launch_origin_track(const uint32_t *A, uint32_t X, uint32_t Y, uint64_t t0, uint32_t K, const Rule &R,
                                int64_t *h00, cudaStream_t st);
int origin_max_k();
// Random-sequential dynamics on the local 4 x 4 encoding (sca_rs.cu): n_mcs MCS on the
// canonical words A in place, Lw (X Y / 4 bytes) the local-encoding buffer.
cudaError_t launch_rs(uint32_t *A, uint32_t *Lw, uint32_t X, uint32_t Y, uint64_t t0, uint64_t n_mcs,
                      const Rule &R, uint64_t Tp, uint64_t Tq, cudaStream_t st);
bool rs_supported(uint32_t X, uint32_t Y);

// Two-time height correlation of the states A and B of one X x Y lattice (chunk records in
// partials, at most obs_partials scratch; result record of corr_record_bytes() bytes).
cudaError_t launch_correlate(const uint32_t *A, const uint32_t *B, uint32_t X, uint32_t Y, ObsPartial *partials,
                             void *result, uint64_t t, cudaStream_t st);
size_t corr_record_bytes();

void count_launches(uint64_t n);
int sm_count();

// Workspace layout of one simulation (all offsets 256-byte aligned).
struct Layout {
    size_t state_bytes, off_b, off_h0, off_part, off_res, off_err, total;
};
constexpr int kResCap = 64;   // observation records per simulation

}  // namespace sca

struct sca_params;

// One single-lattice simulation (opaque on the ABI).
struct sca_sim {
    sca::Rule R;
    uint32_t L, W;      // row length X (sites) and words per sublattice row
    uint32_t Ly;        // rows Y (L for a square lattice)
    sca::Layout lo;
    char *base;
    bool own_mem;
    uint32_t *buf[2];
    int cur;
    int64_t *h0;
    sca::ObsPartial *part;
    sca::ObsDev *res;
    uint32_t *err;      // device word: bit 0 = a kernel wait gave up
    int64_t *h00;       // device: absolute height of the origin site (tracked when track_origin)
    bool track_origin;
    uint32_t dynamics;  // SCA_DYN_*
    uint64_t rs_Tp, rs_Tq;   // random-sequential acceptance thresholds floor(p 2^32), floor(q 2^32)
    cudaStream_t stream;
    bool own_stream;
    uint64_t t;
    int kernel;
    int fused_V, fused_ring;          // fused launch shape (0 = default)
    int tb_k;                         // MCS per temporal-blocking launch
    bool tb_set;                      // tb_k chosen by the caller (else automatic)
    uint32_t wave_bands;              // row bands of the register-wavefront kernel (0 = auto)
    bool surface;                     // the state is known to be a surface (kernel 4 needs it)
    uint32_t *chk_host;               // pinned: result of an enqueued surface check (or null)
    cudaEvent_t chk_ev;               // recorded after that check's result copy
    bool chk_pending;                 // surface is decided by that check once it completes
    uint32_t async_obs;               // records of the last sca_run_async not yet collected
    bool timing;
    std::vector<cudaEvent_t> ev;      // start/stop pairs around update launches
    uint64_t timed_launches;
};


namespace sca {
int make_rule(const sca_params &prm, Rule &R);
bool use_fused(const sca_sim *s);
// Kernel actually used (1 two-pass, 2 fused, 3 shared-memory temporal blocking, 4 register
// wavefront) and, for 3 and 4, MCS per launch.
int effective_kernel(const sca_sim *s, int *tb_k);
int step_impl(sca_sim *s, uint64_t n);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *where);
}  // namespace sca
