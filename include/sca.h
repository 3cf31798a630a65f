/*
 * sca.h: C ABI of the GB300 octahedron-model stochastic cellular automaton (SCA) library.
 *
 * The library advances the 2+1D octahedron (KPZ) surface-growth model of Kelling, Odor and
 * Gemming, "Bit-Vectorized GPU Implementation of a Stochastic Cellular Automaton Model for
 * Surface Growth" (arXiv 1606.00310), on one GPU, and measures the surface roughness exactly.
 *
 * Conventions for every entry point:
 *   - Return 0 (SCA_OK) on success or a negative SCA_E* status; sca_strerror() names it and
 *     sca_last_error() gives the detail of the last failure on the calling thread.
 *   - Pointers named *_dev are device pointers; every other pointer is host memory.
 *   - Memory passed in by the caller stays owned by the caller and is never freed here.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the library creates and owns a
 *     non-blocking stream for the object.  Work is enqueued on that stream; calls that return
 *     host results synchronise it.
 *   - Types are plain C; no PyTorch or CUDA types appear in the signatures.
 *
 * Model (paper Sec. I.A, Eq. 1): slopes sx-, sy- in {-1,+1} per site of an X x Y periodic
 * lattice (X = L sites per row, Y rows; Y = L unless sca_params.Ly says otherwise, Sec. II.B
 * names the two lateral sizes); a local minimum (sx-, sx+, sy-, sy+) = (-1, +1, -1, +1) turns into the maximum
 * (+1, -1, +1, -1) with probability p (deposition) and back with probability q (removal).
 * One Monte-Carlo step (MCS) updates every even site ((x + y) & 1 == 0), then every odd site.
 *
 * State format (the only one that crosses this ABI): the "canonical packed words".  A slope
 * -1 is bit 0, +1 is bit 1 (paper Sec. II.A); sx-(x,y) = h(x,y) - h(x-1,y) and
 * sy-(x,y) = h(x,y) - h(x,y-1).  With W = X/64 words per sublattice row, the word at index
 *     ((s * 2 + d) * Y + y) * W + j        (s = sublattice, d = 0 for x / 1 for y, row y)
 * holds in bit b the slope of sublattice site k = 32 j + b, lattice site x = 2k + ((s + y) & 1)
 * (the paper's role-grouped "non-local" encoding, Sec. II.A, with this offset convention).
 * Total 4 * Y * W words = X*Y/4 bytes (L*L/4 for a square lattice).
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) in place of the paper's TinyMT, keyed by
 * the seed with counter (g, t, s | (draw - 1) << 1 | (t >> 32) << 6, tag | (g >> 32) << 1):
 *   - dyadic probabilities (p = P / 2^n, n <= 32; paper Sec. III): draw i = 1..n of packed
 *     word u = y * W + j uses g = u >> 2, output lane u & 3, tag 0; a site is accepted iff its
 *     n draw bits, draw 1 most significant, form R >= 2^n - P (equal to the paper's and/or
 *     construction, xi = r_n; xi = b_i ? r_i | xi : r_i & xi for i = n-1..1);
 *   - any probability (paper Sec. II.B, one random number per site): site unit
 *     u = y * (X/2) + k uses g = u >> 2, lane u & 3, draw 1, tag 1; accepted iff the 32-bit
 *     output < floor(p * 2^32);
 *   - t is the 0-based index of the MCS being executed; deposition and removal share draws.
 *
 * Roughness (paper Sec. I.A names the roughness; its definition here): heights from h(0,0) = 0
 * down column 0 (sy-) then along each row (sx-); S1 = sum h, S2 = sum h^2 (128-bit),
 * num = N * S2 - S1^2 (128-bit), W^2 = num / N^2 with N = X*Y.
 */
#ifndef SCA_H
#define SCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------ */
#define SCA_OK 0
#define SCA_EINVAL (-1)    /* bad argument: L not a positive multiple of 64, p/q outside [0,1],
                              dyadic mode with a probability that needs more than 32 bits,
                              decreasing observation times, NULL pointer, short buffer */
#define SCA_ENOMEM (-2)    /* a library allocation failed */
#define SCA_ECUDA (-3)     /* a CUDA call or kernel launch failed (detail in sca_last_error) */
#define SCA_EBUDGET (-4)   /* a request does not fit the server's device-memory budget */
#define SCA_ETIMEOUT (-5)  /* a wait gave up before the work finished */
#define SCA_EBUSY (-6)     /* the object is in use (server queue full) */
#define SCA_ESTATE (-7)    /* the slope state does not close around the torus (heights would
                              not be single-valued), e.g. after sca_set_state with bad words */
#define SCA_ENOTFOUND (-8) /* unknown ticket */
#define SCA_ECANCELED (-9) /* the request was cancelled */

/* ---- random-number modes ------------------------------------------------------------------ */
#define SCA_RNG_AUTO 0       /* dyadic if p and q are multiples of 2^-32, else per-site */
#define SCA_RNG_DYADIC 1     /* packed-word draws with the and/or construction (Sec. III)  */
#define SCA_RNG_UNIFORM32 2  /* one 32-bit uniform per site (Sec. II.B, arbitrary p)       */

typedef struct sca_params {
    uint32_t L;      /* lateral size X (sites per row): a multiple of 64, 64 <= L <= 131072 */
    uint32_t rng;    /* SCA_RNG_* */
    uint64_t seed;   /* Philox key */
    double p;        /* deposition probability at local minima, 0 <= p <= 1 */
    double q;        /* removal probability at local maxima, 0 <= q <= 1 */
    uint32_t Ly;     /* lateral size Y (rows): 0 for a square lattice (Y = L), else even,
                        2 <= Ly <= 131072.  X != Y runs on the two-pass kernel (1) and the
                        wavefront kernel (4) of sca_set_kernel; batches, servers and
                        sca_observe_noalloc take square lattices only */
    uint32_t dynamics;  /* SCA_DYN_SCA (0): the stochastic cellular automaton of the paper;
                           SCA_DYN_RANDOM_SEQUENTIAL (1): its non-vectorized comparison (see
                           there); single lattices only (batches and servers refuse it) */
} sca_params;

/* ---- dynamics ------------------------------------------------------------------------------- */
#define SCA_DYN_SCA 0   /* sublattice-parallel updates, even sites then odd (Sec. I.A) */
/* Random-sequential updates on the local encoding (Sec. II.A: 4 x 4 sites per 32-bit word, the
 * encoding of choice when sites are selected at random; Sec. III benchmarks it against the
 * bit-vectorized SCA).  The paper gives no schedule; this library's: the words hold the
 * 4 x 4 tiles 4 wx <= x < 4 wx + 4, 4 wy <= y < 4 wy + 4; each MCS is two phases over the
 * checkerboard of words ((wx + wy) & 1 == phase; active words share no bond), and an active
 * word w = wy * (X/4) + wx takes 16 attempts in sequence: attempt a of MCS t, phase ph, uses the
 * Philox4x32-10 call with counter (w, t, ph | a << 1 | (t >> 32) << 6, 2), picks site
 * out[0] >> 28 (column & 3, row >> 2 of the tile) and flips it if it is a local minimum and
 * out[1] < floor(p 2^32) or a local maximum and out[1] < floor(q 2^32).  On a 4 x 4 torus this
 * is plain random-sequential dynamics.  Needs Y a multiple of 8 (X is a multiple of 64).  The
 * state on this ABI stays the canonical words; sca_track_origin is not available. */
#define SCA_DYN_RANDOM_SEQUENTIAL 1

/* One exact roughness observation. */
typedef struct sca_obs {
    uint64_t t;        /* MCS completed when observed */
    uint64_t N;        /* X * Y sites */
    int64_t S1;        /* sum of heights */
    uint64_t S2_lo;    /* sum of squared heights, low 64 bits */
    uint64_t S2_hi;    /*                        high 64 bits */
    uint64_t num_lo;   /* N * S2 - S1^2, low 64 bits (W^2 = num / N^2) */
    uint64_t num_hi;   /*                high 64 bits */
    double w2;         /* num / N^2 rounded to double, for convenience */
    int32_t status;    /* SCA_OK, or SCA_ESTATE if the slopes did not close */
    int32_t reserved;
    int64_t h00;       /* absolute height of the origin site while sca_track_origin is on (see
                          there): <h> = h00 + S1 / N is the absolute mean height; 0 otherwise */
} sca_obs;

/* One exact two-time height correlation (see sca_correlate).  Signed 128-bit values are split
 * into an unsigned low and a signed high 64-bit word. */
typedef struct sca_corr {
    uint64_t t;        /* MCS of the simulation's current state (state a) */
    uint64_t N;        /* X * Y sites */
    int64_t Sa;        /* sum of the heights of state a (h(0,0) = 0) */
    int64_t Sb;        /* sum of the heights of the reference state b */
    uint64_t Sab_lo;   /* sum of h_a h_b over the sites, low 64 bits */
    int64_t Sab_hi;    /*                                high 64 bits (signed) */
    uint64_t cnum_lo;  /* N * Sab - Sa * Sb, low 64 bits (C = cnum / N^2) */
    int64_t cnum_hi;   /*                    high 64 bits (signed) */
    double c;          /* cnum / N^2 rounded to double */
    int32_t status;    /* SCA_OK, or SCA_ESTATE if either state does not close */
    int32_t reserved;
} sca_corr;

typedef struct sca_sim sca_sim;   /* one simulation: state, stream, scratch; opaque */

/* ---- single lattice ------------------------------------------------------------------------ */

/* Device bytes one simulation of lateral size L needs when the caller supplies the memory
 * (two state buffers for the ping-pong update, plus observation scratch).  0 if L is invalid. */
size_t sca_workspace_bytes(uint32_t L);

/* The same for an X x Y lattice (X = sca_params.L, Y = sca_params.Ly); 0 if invalid. */
size_t sca_workspace_bytes_xy(uint32_t X, uint32_t Y);

/* Create a simulation at MCS 0 in the flat state h(x,y) = (x + y) & 1 (sublattice-0 words all
 * zero, sublattice-1 words all ones).  dev_buf: caller-owned device memory of at least
 * sca_workspace_bytes_xy(L, Ly) bytes (sca_workspace_bytes(L) when square), 256-byte aligned,
 * or NULL to let the library allocate.
 * Errors: SCA_EINVAL (bad params or short buffer), SCA_ENOMEM, SCA_ECUDA. */
int sca_init(const sca_params *params, void *stream, void *dev_buf, size_t dev_buf_bytes,
             sca_sim **out);

/* Return to the flat state at MCS 0 (device-side fill, asynchronous on the stream). */
int sca_reset(sca_sim *sim);

/* Enqueue n_mcs Monte-Carlo steps (Sec. I.A: even sublattice, then odd, per step) on the
 * simulation's stream.  Asynchronous.  Errors: SCA_EINVAL, SCA_ECUDA. */
int sca_step(sca_sim *sim, uint64_t n_mcs);

/* Exact roughness of the current state; synchronises the stream.  Errors: SCA_ECUDA; a state
 * that does not close is reported in out->status = SCA_ESTATE and returned as SCA_ESTATE. */
int sca_observe(sca_sim *sim, sca_obs *out);

/* Advance to each of the absolute MCS counts times[0..n-1] (non-decreasing, >= the current
 * count) and observe there; one synchronisation at the end.  out[i] receives observation i.
 * Errors: SCA_EINVAL, SCA_ECUDA, SCA_ESTATE (first failing observation's status). */
int sca_run(sca_sim *sim, const uint64_t *times, uint32_t n, sca_obs *out);

/* Track the absolute height of the origin site (x, y) = (0, 0) through the updates (enable != 0)
 * or stop (0).  Slopes fix heights only up to a constant; the origin's height, changed by +2
 * at each deposition there and -2 at each removal (Eq. 1), fixes it, so that every observation
 * then reports h00 and the absolute mean height <h> = h00 + S1 / N, whose rate of change is the
 * growth velocity.  Enabling sets the counter to 0: the true absolute height after sca_init or
 * sca_reset (flat start, h(0,0) = 0), the height relative to the moment of enabling otherwise;
 * sca_reset and sca_set_state also set it to 0.  Cost: one small launch before each update
 * launch (it re-runs that launch's MCS on a patch around the origin), and launches of at most
 * 16 MCS.  Needs a surface state.  Errors: SCA_EINVAL; SCA_ESTATE when the state is not a
 * surface (the next sca_step reports it). */
int sca_track_origin(sca_sim *sim, int enable);

/* Two-time height correlation of the current state a (MCS t) with a reference state b of the
 * same lattice, typically a copy of an earlier state (MCS s < t): the paper's aging studies
 * (Sec. I, Sec. IV) measure two-time functions; the one computed here is the covariance of the
 * two height fields over the sites,
 *     C(t, s) = (1/N) sum_x (h(x,t) - <h(t)>)(h(x,s) - <h(s)>) = cnum / N^2,
 * exact in integers (cnum = N sum h_a h_b - sum h_a sum h_b), unchanged by the unknown absolute
 * height of either state; C(t, t) equals the roughness W^2(t).
 *   ref_words_dev: caller-owned device memory with the reference state's canonical words
 *                  (4 * Y * X/64 words, the layout of sca_get_state), read only; e.g. a copy of
 *                  the words sca_state_device pointed to at MCS s.
 * Synchronises the stream.  Errors: SCA_EINVAL, SCA_EBUSY (an asynchronous run's records are
 * still pending), SCA_ECUDA; SCA_ESTATE (in out->status too) if either state does not close. */
int sca_correlate(sca_sim *sim, const uint32_t *ref_words_dev, sca_corr *out);

/* Copy the current canonical words to host memory (n_words >= 4 * Y * X/64); synchronises. */
int sca_get_state(sca_sim *sim, uint32_t *host_words, size_t n_words);

/* Replace the state by n_words = 4 * Y * X/64 canonical words from host memory and set the
 * MCS count to t (the next step uses MCS index t); synchronises.  The words are accepted as
 * they are; one device pass records whether they form a surface (every plaquette closes and
 * the slopes sum to zero around the torus), which kernel 4 of sca_set_kernel requires, and
 * sca_observe reports a state that does not close. */
int sca_set_state(sca_sim *sim, const uint32_t *host_words, size_t n_words, uint64_t t);

/* Asynchronous host I/O and runs, for pipelining: with two simulations on two streams, one
 * simulation's state copies overlap the other's updates.  Each call only enqueues work on the
 * simulation's stream and returns; host buffers must stay untouched until sca_wait returns
 * (pinned memory makes the copies asynchronous; pageable memory works but copies in place).
 *
 * sca_set_state_async: as sca_set_state (same words, same t), including the surface check,
 * whose result the next call that chooses a kernel collects (it waits for the copy and the
 * check to finish).  Errors: SCA_EINVAL, SCA_ECUDA.
 * sca_get_state_async: as sca_get_state, without the synchronisation.  Errors: SCA_EINVAL,
 * SCA_ECUDA.
 * sca_run_async: as sca_run with at most 64 times, without the synchronisation; the n
 * observation records stay on the device until sca_wait (or the next run or observation).
 * Errors: SCA_EINVAL, SCA_ECUDA, SCA_ESTATE (kernel 4 chosen for a state that is not a surface).
 * sca_wait: synchronises the simulation's stream and copies the first n (<= the last
 * sca_run_async's count) observation records to out.  Errors: SCA_EINVAL, SCA_ECUDA,
 * SCA_ETIMEOUT, SCA_ESTATE (as sca_run). */
int sca_set_state_async(sca_sim *sim, const uint32_t *host_words, size_t n_words, uint64_t t);
int sca_get_state_async(sca_sim *sim, uint32_t *host_words, size_t n_words);
int sca_run_async(sca_sim *sim, const uint64_t *times, uint32_t n);
int sca_wait(sca_sim *sim, sca_obs *out, uint32_t n);

/* Device pointer to the current canonical words (valid until the next call on sim).  Read
 * only: write a new state with sca_set_state. */
int sca_state_device(sca_sim *sim, uint32_t **words_dev);

/* MCS completed so far. */
uint64_t sca_time(const sca_sim *sim);

/* Update kernel choice: 0 = automatic (fused when L is a multiple of 2048, L >= 32768 and the
 * draws are not per-site uniforms; temporal blocking for dyadic draws up to L = 8192 and for
 * per-site uniforms up to L = 2048; else two-pass), 1 = two-pass (one launch per sublattice, the
 * paper's Fig. 3 structure), 2 = fused even+odd wavefront (one launch per MCS; needs L a
 * multiple of 2048), 3 = temporal blocking (several MCS per launch in shared memory, see
 * sca_set_temporal_block), 4 = register-wavefront temporal blocking (each warp streams a band
 * of rows through registers as one height bit per site and advances it up to 16 MCS per launch
 * with {0, 1} probabilities, 4 with dyadic draws, 2 with per-site uniforms; sca_step returns
 * SCA_ESTATE if the state is not a surface, see sca_set_state).
 * Results are identical for every choice; only speed differs.
 * Errors: SCA_EINVAL (unknown kernel, or one that does not support this lattice or rule). */
int sca_set_kernel(sca_sim *sim, int kernel);

/* Temporal blocking (kernels 3 and 4 of sca_set_kernel): each launch advances mcs_per_launch
 * MCS (a divisor of 64) with a halo of 2 rows per MCS above and below every block of rows; 0 =
 * default: 4 for kernel 3; for kernel 4 the measured best for the rule (with {0, 1}
 * probabilities 16 from L = 16384 on and 8 below; with dyadic draws 4 for one draw and q = 0,
 * 1 for three draws and q != 0, 2 otherwise; 2 with per-site uniforms).  Kernel 4 caps a launch
 * at 16 MCS ({0, 1} probabilities), 4 (dyadic draws) or 2 (per-site uniforms).  Errors:
 * SCA_EINVAL if mcs_per_launch does not divide 64 or, for kernel 3, the block with its halo does
 * not fit for this L. */
int sca_set_temporal_block(sca_sim *sim, int mcs_per_launch);

/* Row bands of the register-wavefront kernel (kernel 4): the lattice is cut into `bands` bands
 * of rows times columns of 30 packed words, one warp per tile; 0 = automatic (enough tiles for
 * one full wave of resident warps).  Results do not depend on it.  Errors: SCA_EINVAL unless
 * 0 <= bands <= Y/2. */
int sca_set_wave_bands(sca_sim *sim, int bands);

/* Launch shape of the fused kernel: words_per_thread (1, 2 or 4; the CTA has L/64 /
 * words_per_thread threads, 32..512) and ring = lattice rows held in shared memory (6; or 8 or
 * 12 with 4 words per thread: deeper rings prefetch further and leave stores more time).  0 restores the default (4 words,
 * 6 rows).  Results do not depend
 * on the shape.  Errors: SCA_EINVAL if the shape does not fit L. */
int sca_set_fused_shape(sca_sim *sim, int words_per_thread, int ring);

/* Update kernel the simulation uses now (1 = two-pass, 2 = fused, 3 = temporal blocking in
 * shared memory, 4 = register-wavefront temporal blocking), after automatic choice; 5 for the
 * random-sequential dynamics (sca_params.dynamics = 1, which ignores the kernel choice). */
int sca_get_kernel(const sca_sim *sim);

/* Kernel timing: while enabled, the library records a CUDA event pair on the simulation's
 * stream around every run of consecutive update launches (no observation kernels inside).
 * Enabling clears earlier records.  Errors: SCA_EINVAL, SCA_ECUDA. */
int sca_timing(sca_sim *sim, int enable);

/* Sum of the recorded update-kernel time in milliseconds and the number of update launches
 * it covers; synchronises the stream.  Errors: SCA_EINVAL, SCA_ECUDA. */
int sca_timing_read(sca_sim *sim, double *update_ms, uint64_t *update_launches);

/* Release library-owned memory and stream.  Caller-owned memory is left alone. */
void sca_free(sca_sim *sim);

/* ---- batched ensemble ------------------------------------------------------------------------
 * Many independent lattices (each its own L, seed, p, q, rng mode) advanced together by one
 * persistent kernel launch, captured in a CUDA graph and replayed while the observation times
 * repeat.  Each lattice stays in on-chip shared memory for the whole run; lattices too large
 * for one CTA are split by rows over up to 8 CTAs of a thread-block cluster that exchange the
 * boundary sy+ row through distributed shared memory.  Every lattice follows exactly the
 * single-lattice dynamics (same canonical words, same Philox counters), so its result equals
 * a sca_sim run with the same parameters, alone or in any mix. */
typedef struct sca_batch sca_batch;   /* opaque */

/* Create `count` lattices, all flat at MCS 0.  params[i].L must be a multiple of 64 in
 * [128, 2048].  The library allocates the states (sum of L*L/4 bytes) and result buffers.
 * Errors: SCA_EINVAL, SCA_ENOMEM, SCA_ECUDA. */
int sca_batch_init(const sca_params *params, uint32_t count, void *stream, sca_batch **out);

/* Launch shape: cluster size (1..8 or 16 CTAs; a lattice may be split over any number of them,
 * in parts that differ by at most one row) and threads per CTA (128..512).  Every shape gives
 * identical results; sca_batch_tune picks the fastest.  Errors: SCA_EINVAL when a lattice does
 * not fit the cluster's shared memory. */
int sca_batch_set_shape(sca_batch *b, int cluster, int threads);

/* Engine of the batch: 1 = clusters (every lattice in shared memory for the whole run, as height
 * bits, split by rows over the CTAs of a thread-block cluster; any lattice of the batch limits),
 * 2 = streaming (lattices grouped by size and rule; each group of lanes of a warp holds whole
 * rows of one lattice and streams a band of its rows through registers for up to 8 MCS per
 * launch; needs L a power-of-two multiple of 64 up to 2048 and dyadic or {0, 1} probabilities
 * for every lattice), 0 = automatic (streaming when every lattice fits it, else clusters;
 * sca_batch_tune picks the faster).  Results do not depend on the engine.  Errors: SCA_EINVAL
 * (unknown engine, or streaming requested for a batch it does not fit). */
int sca_batch_set_engine(sca_batch *b, int engine);
/* Engine the next run uses (1 or 2). */
int sca_batch_get_engine(const sca_batch *b);
int sca_batch_get_shape(const sca_batch *b, int *cluster, int *threads, int *clusters_launched,
                        int *units);

/* Autotuner: times a probe_mcs-MCS run for each launch shape that fits (cluster sizes 4, 5, 6,
 * 8, 16; 256, 384, 512 threads), keeps the fastest, and leaves every lattice flat at MCS 0.  The
 * chosen shape is returned through best_cluster / best_threads (either may be NULL).  Only
 * speed depends on the shape.  Errors: SCA_EINVAL, SCA_ECUDA. */
int sca_batch_tune(sca_batch *b, uint32_t probe_mcs, int *best_cluster, int *best_threads);

/* Advance every lattice to each time in times[0..n-1] (increasing, after the current MCS,
 * n <= 64) in one graph launch and observe there.  out (may be NULL) receives count * n records,
 * lattice-major (out[i * n + k] = lattice i at times[k]); ensemble_w2 (may be NULL) receives n
 * ensemble means of W^2, summed in lattice order.  Synchronises.  Errors: SCA_EINVAL, SCA_ECUDA,
 * SCA_ESTATE. */
int sca_batch_run(sca_batch *b, const uint64_t *times, uint32_t n, sca_obs *out,
                  double *ensemble_w2);

/* Diagnostics of the last run: for each work unit (units are ordered by decreasing estimated
 * cost), the device clock (ns) when its cluster started and finished it, and the index of its
 * first lattice.  n must be at least the unit count (sca_batch_get_shape).  Synchronises. */
int sca_batch_unit_times(sca_batch *b, uint64_t *start_ns, uint64_t *end_ns,
                         int32_t *first_lattice, uint32_t n);

/* Canonical words of lattice `index` (4 * L * L/64 words) to host memory; synchronises. */
int sca_batch_get_state(sca_batch *b, uint32_t index, uint32_t *host_words, size_t n_words);

/* Canonical words of lattice `index` (4 * L * L/64 words, the layout of sca_set_state) from host
 * memory; the batch time is unchanged, so the lattice continues from MCS sca_batch_time(b).  The
 * state must be a surface (every plaquette closes, row 0 and column 0 close around the torus):
 * both engines update height bits.  Synchronises.  Errors: SCA_EINVAL (bad index or short
 * buffer), SCA_ESTATE (not a surface: the lattice is reset to flat), SCA_ECUDA. */
int sca_batch_set_state(sca_batch *b, uint32_t index, const uint32_t *host_words, size_t n_words);

/* All lattices back to flat at MCS 0 (asynchronous). */
int sca_batch_reset(sca_batch *b);
uint64_t sca_batch_time(const sca_batch *b);
void sca_batch_free(sca_batch *b);

/* ---- serving: continuous batching of independent simulations -------------------------------
 * A server owns a scheduler thread and up to max_active slots (two streams each, one at the
 * device's highest priority).  Requests queue in arrival order and are admitted while a slot is
 * free and the sum of admitted requests' state (sca_workspace_bytes(L) + 256 each) stays within
 * budget_bytes; their memory comes from the device's stream-ordered pool.  Admitted requests
 * run concurrently, each on its own stream, advancing in replayed CUDA graphs of 64 MCS;
 * requests of at most 2^33 site updates (L * L * n_mcs) take the high-priority stream, so the
 * GPU starts their blocks first, and per-site uniform requests run the two-pass kernel (the
 * kernel that shares the GPU best).  A request's results equal those of a sca_sim with the same
 * parameters run alone, whatever the kernel.  Times are seconds since sca_server_create. */
typedef struct sca_server sca_server;   /* opaque */

typedef struct sca_request_info {
    uint64_t ticket;
    uint64_t n_mcs;
    uint32_t n_obs;      /* observations the request returns */
    int32_t status;      /* SCA_EBUSY while pending or running, then the final status */
    uint32_t L;
    uint32_t reserved;
    double submit_s;     /* when submitted */
    double admit_s;      /* when admitted to a slot (0: not yet) */
    double done_s;       /* when finished (0: not yet) */
} sca_request_info;

typedef struct sca_server_stats {
    uint64_t submitted, admitted, completed, cancelled, failed;
    uint32_t active;        /* requests holding a slot now */
    uint32_t pending;       /* requests waiting for a slot or memory */
    uint64_t bytes_in_use;  /* state memory of admitted requests */
    uint64_t budget_bytes;
    uint64_t updates_done;  /* site updates of completed requests */
} sca_server_stats;

/* Create a server on the current device.  max_L bounds the lattice size of requests.  Errors:
 * SCA_EINVAL, SCA_ECUDA. */
int sca_server_create(size_t budget_bytes, uint32_t max_active, uint32_t max_L, sca_server **out);

/* Queue one simulation: params (L, seed, p, q, rng), n_mcs steps from the flat state, observed
 * at times[0..n_times-1] (increasing, within 1..n_mcs; n_mcs is appended if missing) or, if
 * times is NULL, at 1, 2, 4, ... and n_mcs; at most 64 observations.  Returns at once with a
 * ticket.  Errors: SCA_EINVAL (bad parameters, L above max_L), SCA_EBUDGET (the state alone
 * exceeds the budget). */
int sca_server_submit(sca_server *srv, const sca_params *params, uint64_t n_mcs,
                      const uint64_t *times, uint32_t n_times, uint64_t *ticket);

/* As sca_server_submit, and the request's final state comes back too: when it finishes, its
 * canonical words (4 * L * L/64 of them, the layout of sca_get_state) are copied into
 * final_words, caller-owned host memory of n_words >= 4 * L * L/64 words that must stay valid
 * until the request has finished (pinned memory keeps the copy asynchronous; pageable memory
 * makes the scheduler thread wait for it).  The words are the result once the request's status
 * is SCA_OK; after a cancellation or an error they are unspecified.  Errors: as
 * sca_server_submit, and SCA_EINVAL for a NULL or short buffer. */
int sca_server_submit_state(sca_server *srv, const sca_params *params, uint64_t n_mcs,
                            const uint64_t *times, uint32_t n_times, uint32_t *final_words,
                            size_t n_words, uint64_t *ticket);

/* Result of a request without blocking: SCA_EBUSY while pending or running; otherwise its
 * final status, with up to n_out observations copied to out (may be NULL) and info filled (may
 * be NULL).  Errors: SCA_ENOTFOUND. */
int sca_server_poll(sca_server *srv, uint64_t ticket, sca_obs *out, uint32_t n_out,
                    sca_request_info *info);

/* As sca_server_poll, but blocks until the request finishes or timeout_ms passes (negative:
 * no limit); SCA_ETIMEOUT if it did not finish in time. */
int sca_server_wait(sca_server *srv, uint64_t ticket, int timeout_ms, sca_obs *out,
                    uint32_t n_out, sca_request_info *info);

/* Cancel a pending or running request (its status becomes SCA_ECANCELED).  Finished requests
 * are left as they are. */
int sca_server_cancel(sca_server *srv, uint64_t ticket);

/* Forget a finished request.  Errors: SCA_EBUSY (not finished), SCA_ENOTFOUND. */
int sca_server_release(sca_server *srv, uint64_t ticket);

int sca_server_get_stats(sca_server *srv, sca_server_stats *out);

/* Stop the scheduler (running requests are cancelled) and free everything. */
void sca_server_destroy(sca_server *srv);

/* ---- observation without allocation ---------------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot let the
 * library allocate device memory (a host application that owns all GPU memory through its own
 * pool, a plug-in barred from the CUDA allocator, a loop that must not pay for cudaMalloc or
 * its implicit device synchronisation).  It computes the same exact roughness as sca_observe
 * for canonical words the caller already holds, using a fixed file-scope device array of
 * 66,048 bytes as scratch (held by every GPU that loads this library until the process exits):
 * room for the row kernel's chunk records (at most 1024 chunks of at most 256 rows) and the
 * result record.
 *   words_dev: caller-owned device memory with 4 * L * L/64 canonical words (read only).
 *   L:         multiple of 64, 64 <= L <= 131072 (the library's largest lattice); larger L is
 *              rejected with SCA_EINVAL before any device work.
 *   t:         copied into out->t.
 *   stream:    cudaStream_t as void*, NULL for the legacy default stream; synchronised.
 *   out:       host result, as from sca_observe (SCA_ESTATE if the slopes do not close).
 * The first call on each device looks up the array's device address with that device current;
 * make that first call before any stream capture.  All calls share the array: calls that
 * overlap on the GPU race and must be serialised by the caller.  Each call overwrites all the
 * scratch it reads, so nothing carries over between calls.  No allocation or free is made. */
int sca_observe_noalloc(const uint32_t *words_dev, uint32_t L, uint64_t t, void *stream,
                        sca_obs *out);

/* ---- diagnostics --------------------------------------------------------------------------- */
const char *sca_strerror(int status);
const char *sca_last_error(void);   /* detail of the last failure on this thread */

/* Failure-detection self-test: runs the bounded wait that every pipeline wait in the update
 * kernels uses, on a barrier that nothing ever completes, with a limit of limit_us (1 us..2 s).
 * Returns SCA_ETIMEOUT when the wait gave up and reported it, leaving the CUDA context usable;
 * any other result means the timeout path is broken.  No trap, no fault, no unbounded spin. */
int sca_selftest_wait_timeout(uint32_t limit_us);

/* Measured issue rate of 32-bit three-input logic instructions on the current GPU, in
 * instructions per second over the whole device: one launch of independent LOP3 chains that
 * fills every SM, timed with CUDA events on a private stream (about 20 ms).  The denominator of
 * the height-bit update's ALU roofline.  Errors: SCA_EINVAL, SCA_ECUDA. */
int sca_measure_logic_rate(double *ops_per_s);

/* Measured rates of the multiply pipe on the current GPU, over the whole device, each from one
 * launch that fills every SM, timed with CUDA events on a private stream (about 30 ms):
 * wide_mul_per_s, 32 x 32 -> 64-bit multiply-adds per second (eight independent chains per
 * thread); philox_calls_per_s, Philox4x32-10 calls per second as the update kernels compute
 * them (ten rounds of two such products each, four independent counters per thread).  The
 * denominators of the rooflines of the paths that draw random numbers (Sec. II.B, Sec. III).
 * Errors: SCA_EINVAL, SCA_ECUDA. */
int sca_measure_mul_rate(double *wide_mul_per_s, double *philox_calls_per_s);

/* Number of kernels this library has launched in this process (all objects, all streams). */
uint64_t sca_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* SCA_H */
