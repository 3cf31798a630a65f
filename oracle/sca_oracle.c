/*
 * Reference oracle for the octahedron-model stochastic cellular automaton (SCA).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct CPU statement of what
 * the GPU library computes.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Model (Kelling, Odor, Gemming, arXiv 1606.00310):
 *   - Sec. I.A, Eq. (1) "generalized Kawasaki rules": a site whose slopes read
 *     (sx-, sx+; sy-, sy+) = (-1,+1; -1,+1) (a local minimum) becomes (+1,-1; +1,-1) with
 *     probability p (deposition, h += 2); the reverse (a local maximum) with probability q
 *     (removal, h -= 2).  Periodic boundary conditions.
 *   - Sec. I.A: one Monte-Carlo step (MCS) attempts one update per site: first every even
 *     site ((x xor y) and 1 == 0), then every odd site.
 *   - Sec. II.A: a slope maps to a bit (-1 -> 0, +1 -> 1); only sx- and sy- are stored per
 *     site, since sx+(x,y) = sx-(x+1,y) and sy+(x,y) = sy-(x,y+1).
 *   - Sec. II.B, Eqs. (2)-(4): the update masks m_p, m_q, m = m_p xor m_q.  The oracle applies
 *     the same rule one site at a time; same-parity sites share no slope, so the order within
 *     a sublattice does not matter.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - bit convention: sx-(x,y) = h(x,y) - h(x-1,y), bit = (slope + 1) / 2;
 *   - flat start h(x,y) = (x + y) & 1;
 *   - random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with the counter
 *     layout below instead of the paper's TinyMT (Sec. II.B);
 *   - dyadic probabilities p = P / 2^n take n random words per packed word and accept a site
 *     iff its n bits, read as an integer R with draw 1 as the most significant bit, satisfy
 *     R >= 2^n - P (the and/or construction of Sec. III, written as one comparison);
 *   - non-dyadic probabilities take one 32-bit uniform u per site and accept iff
 *     u < floor(p * 2^32) (Sec. II.B: one random number per site);
 *   - deposition and removal share the same draws (a site is never both a minimum and a
 *     maximum, so each site's acceptance law is unchanged);
 *   - heights: h(0,0) = 0, h(0,y) sums sy- down column 0, h(x,y) sums sx- along row y;
 *     roughness W^2 = (1/N) sum h^2 - ((1/N) sum h)^2, kept exact as num = N*S2 - S1^2.
 *
 * Lattice: X sites per row (x = 0..X-1) and Y rows (y = 0..Y-1), both even, periodic in both
 * directions (Sec. II.B names the lateral sizes X and Y; its benchmarks use X = Y = L, and its
 * wide-system variant X >= 2^17).  The functions without the _rect suffix are the square case
 * X = Y = L.  Everything that depends on the row length (the packed layout, the random-number
 * unit of a site) takes X; rows only enter through y and its periodic successor.
 *
 * Canonical packed layout (the only state format exchanged with the library):
 *   W = ceil(X/64) 32-bit words per sublattice row; word index ((s*2 + d)*Y + y)*W + j for
 *   sublattice s, direction d (0 = x, 1 = y), row y; bit b of word j is sublattice site
 *   k = 32*j + b, which is lattice site x = 2k + ((s + y) & 1).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------------------------
 * Philox4x32-10.  Salmon et al., SC'11, Sec. 4 (Philox): each round multiplies counter words
 * 0 and 2 by the round multipliers, xors the high halves with the other two counter words and
 * the key, and bumps the key by the Weyl constants.  Constants as published there.
 * ---------------------------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        uint64_t prod0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)prod1;
        uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)prod0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter of one Philox call (the layout both sides implement independently):
 *   key = (seed low 32, seed high 32)
 *   ctr = (g low 32, t low 32, s | (draw-1) << 1 | (t >> 32) << 6, tag | (g >> 32) << 1)
 * g = group index (unit index >> 2), t = 0-based index of the MCS being executed,
 * s = sublattice, draw = 1-based draw number, tag 0 = packed-word draws, 1 = per-site draws.
 * The unit index selects lane (unit & 3) of the output. */
static uint32_t philox_lane(uint64_t seed, uint64_t unit, uint64_t t, int s, int draw, int tag)
{
    uint64_t g = unit >> 2;
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4];
    ctr[0] = (uint32_t)g;
    ctr[1] = (uint32_t)t;
    ctr[2] = (uint32_t)s | ((uint32_t)(draw - 1) << 1) | ((uint32_t)(t >> 32) << 6);
    ctr[3] = (uint32_t)tag | ((uint32_t)(g >> 32) << 1);
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[unit & 3];
}

/* Words per sublattice row in the packed layout (X sites per row). */
static uint64_t words_per_row(int64_t X) { return (uint64_t)((X / 2 + 31) / 32); }

/* Draw `draw` of the packed-word stream, bit of site (x,y) in sublattice s at MCS t, for rows
 * of X sites (unit = y * W + word of the site). */
uint32_t oracle_word_draw_bit(int64_t X, uint64_t seed, uint64_t t, int s, int draw,
                              int64_t x, int64_t y)
{
    uint64_t k = (uint64_t)(x >> 1);
    uint64_t unit = (uint64_t)y * words_per_row(X) + (k >> 5);
    return (philox_lane(seed, unit, t, s, draw, 0) >> (k & 31)) & 1u;
}

/* Per-site 32-bit uniform of site (x,y) in sublattice s at MCS t, for rows of X sites
 * (unit = y * X/2 + sublattice index of the site). */
uint32_t oracle_site_uniform(int64_t X, uint64_t seed, uint64_t t, int s, int64_t x, int64_t y)
{
    uint64_t k = (uint64_t)(x >> 1);
    uint64_t unit = (uint64_t)y * (uint64_t)(X / 2) + k;
    return philox_lane(seed, unit, t, s, 1, 1);
}

/* p = P / 2^n with P odd and n minimal (n = 0 for p = 0 or 1).  Returns 0 if p is not a
 * multiple of 2^-32 in [0,1]. */
int oracle_dyadic_split(double p, uint64_t *P, int *n)
{
    if (!(p >= 0.0 && p <= 1.0)) return 0;
    double scaled = ldexp(p, 32);
    if (scaled != floor(scaled)) return 0;
    uint64_t num = (uint64_t)scaled;          /* p = num / 2^32 */
    int bits = 32;
    if (num == 0) { *P = 0; *n = 0; return 1; }
    while (bits > 0 && (num & 1u) == 0) { num >>= 1; bits--; }
    *P = num; *n = bits;
    return 1;
}

/* Acceptance of one site under the dyadic construction: the first n_r draws' bits, draw 1 the
 * most significant, form R; accept iff R >= 2^n_r - P_r. */
static int dyadic_accept(uint64_t P, int n, const uint32_t *draw_bits)
{
    if (n == 0) return P == 1;                /* p = 1: always; p = 0: never */
    uint64_t R = 0;
    for (int i = 1; i <= n; i++) R = (R << 1) | draw_bits[i - 1];
    return R >= ((uint64_t)1 << n) - P;
}

typedef struct {
    int64_t L;           /* row length X (the random-number unit of a site depends on it) */
    uint64_t seed;
    int mode;            /* 1 = dyadic (packed-word draws), 2 = per-site 32-bit uniform */
    uint64_t Pp, Pq;     /* dyadic numerators */
    int np, nq;          /* dyadic exponents */
    uint64_t Tp, Tq;     /* per-site thresholds floor(p * 2^32) */
} rule_t;

static int rule_make(rule_t *r, int64_t L, uint64_t seed, double p, double q, int mode)
{
    if (!(p >= 0.0 && p <= 1.0 && q >= 0.0 && q <= 1.0)) return -1;
    r->L = L; r->seed = seed; r->mode = mode;
    if (mode == 1) {
        if (!oracle_dyadic_split(p, &r->Pp, &r->np)) return -1;
        if (!oracle_dyadic_split(q, &r->Pq, &r->nq)) return -1;
    } else if (mode == 2) {
        r->Tp = (uint64_t)floor(ldexp(p, 32));
        r->Tq = (uint64_t)floor(ldexp(q, 32));
    } else {
        return -1;
    }
    return 0;
}

/* Is the update at site (x,y) of sublattice s, MCS t, accepted for the given process
 * (0 = deposition with p, 1 = removal with q)? */
static int accepted(const rule_t *r, uint64_t t, int s, int64_t x, int64_t y, int removal)
{
    if (r->mode == 1) {
        uint64_t P = removal ? r->Pq : r->Pp;
        int n = removal ? r->nq : r->np;
        uint32_t bits[32];
        for (int i = 1; i <= n; i++)
            bits[i - 1] = oracle_word_draw_bit(r->L, r->seed, t, s, i, x, y);
        return dyadic_accept(P, n, bits);
    } else {
        uint64_t T = removal ? r->Tq : r->Tp;
        return (uint64_t)oracle_site_uniform(r->L, r->seed, t, s, x, y) < T;
    }
}

/* One attempted update of site (x,y) per Eq. (1); bx/by hold sx- / sy- bits row-major with X
 * sites per row.  Rows are addressed through `row` so that the band variant below can reuse
 * the rule.  Returns the site's height change: +2 (deposition), -2 (removal) or 0. */
static int update_site(const rule_t *r, uint8_t *bx, uint8_t *by, int64_t X,
                       int64_t row, int64_t row_next, int64_t x, int64_t y, uint64_t t, int s)
{
    int64_t xr = (x + 1) % X;
    uint8_t *a = &bx[row * X + x];        /* sx-(x,y)            */
    uint8_t *b = &by[row * X + x];        /* sy-(x,y)            */
    uint8_t *c = &bx[row * X + xr];       /* sx+(x,y)=sx-(x+1,y) */
    uint8_t *d = &by[row_next * X + x];   /* sy+(x,y)=sy-(x,y+1) */
    int is_min = (*a == 0 && *b == 0 && *c == 1 && *d == 1);
    int is_max = (*a == 1 && *b == 1 && *c == 0 && *d == 0);
    if ((is_min && accepted(r, t, s, x, y, 0)) || (is_max && accepted(r, t, s, x, y, 1))) {
        *a ^= 1; *b ^= 1; *c ^= 1; *d ^= 1;
        return is_min ? 2 : -2;
    }
    return 0;
}

/* Flat initial surface h(x,y) = (x + y) & 1: sx-(x,y) = h(x,y) - h(x-1,y) is -1 on even
 * sites and +1 on odd sites (X, Y even), likewise sy-. */
void oracle_init_flat_rect(int64_t X, int64_t Y, uint8_t *bx, uint8_t *by)
{
    for (int64_t y = 0; y < Y; y++)
        for (int64_t x = 0; x < X; x++) {
            uint8_t v = (uint8_t)((x + y) & 1);
            bx[y * X + x] = v;
            by[y * X + x] = v;
        }
}

void oracle_init_flat(int64_t L, uint8_t *bx, uint8_t *by) { oracle_init_flat_rect(L, L, bx, by); }

/* Run n_mcs Monte-Carlo steps starting at MCS index t0 (Sec. I.A schedule) on the X x Y
 * lattice, adding to *origin_dh the height changes of site (0, 0) (+2 per deposition, -2 per
 * removal there: with the absolute height of the origin known at the start, it stays known,
 * and with it the absolute mean height, whose rate of change is the growth velocity) and to
 * *total_dh those of every site (either pointer may be NULL).  Returns 0, or -1 on bad
 * parameters. */
int oracle_run_rect_counted(int64_t X, int64_t Y, uint8_t *bx, uint8_t *by, uint64_t seed, double p,
                            double q, int mode, uint64_t t0, uint64_t n_mcs, int64_t *origin_dh,
                            int64_t *total_dh)
{
    rule_t r;
    if (X < 2 || (X & 1) || Y < 2 || (Y & 1)) return -1;
    if (rule_make(&r, X, seed, p, q, mode)) return -1;
    int64_t org = 0, tot = 0;
    for (uint64_t t = t0; t < t0 + n_mcs; t++) {
        for (int s = 0; s <= 1; s++) {
            #pragma omp parallel for schedule(static) reduction(+:org, tot)
            for (int64_t y = 0; y < Y; y++)
                for (int64_t x = 0; x < X; x++)
                    if (((x + y) & 1) == s) {
                        int dh = update_site(&r, bx, by, X, y, (y + 1) % Y, x, y, t, s);
                        tot += dh;
                        if (x == 0 && y == 0) org += dh;
                    }
        }
    }
    if (origin_dh) *origin_dh += org;
    if (total_dh) *total_dh += tot;
    return 0;
}

int oracle_run_rect(int64_t X, int64_t Y, uint8_t *bx, uint8_t *by, uint64_t seed, double p,
                    double q, int mode, uint64_t t0, uint64_t n_mcs)
{
    return oracle_run_rect_counted(X, Y, bx, by, seed, p, q, mode, t0, n_mcs, NULL, NULL);
}

int oracle_run(int64_t L, uint8_t *bx, uint8_t *by, uint64_t seed, double p, double q,
               int mode, uint64_t t0, uint64_t n_mcs)
{
    return oracle_run_rect(L, L, bx, by, seed, p, q, mode, t0, n_mcs);
}

/* The same dynamics on a band of `nrows` consecutive lattice rows starting at global row
 * y_first (taken mod Y), full width X.  Only rows whose successor is inside the band are
 * updated, so after n MCS the band rows [2n, nrows - 2n) hold exactly the full lattice's rows
 * (an update at row y reads rows y and y+1 and writes them, so each half-step widens the
 * dependence by one row either way).  Used to check samples of lattices too large to hold. */
int oracle_run_band_rect(int64_t X, int64_t Y, int64_t y_first, int64_t nrows, uint8_t *bx,
                         uint8_t *by, uint64_t seed, double p, double q, int mode, uint64_t t0,
                         uint64_t n_mcs)
{
    rule_t r;
    if (X < 2 || (X & 1) || Y < 2 || (Y & 1) || nrows < 2) return -1;
    if (rule_make(&r, X, seed, p, q, mode)) return -1;
    for (uint64_t t = t0; t < t0 + n_mcs; t++) {
        for (int s = 0; s <= 1; s++) {
            #pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < nrows - 1; i++) {
                int64_t y = (y_first + i) % Y;
                for (int64_t x = 0; x < X; x++)
                    if (((x + y) & 1) == s)
                        update_site(&r, bx, by, X, i, i + 1, x, y, t, s);
            }
        }
    }
    return 0;
}

int oracle_run_band(int64_t L, int64_t y_first, int64_t nrows, uint8_t *bx, uint8_t *by,
                    uint64_t seed, double p, double q, int mode, uint64_t t0, uint64_t n_mcs)
{
    return oracle_run_band_rect(L, L, y_first, nrows, bx, by, seed, p, q, mode, t0, n_mcs);
}

/* Flat start for a band (global row coordinates). */
void oracle_init_flat_band_rect(int64_t X, int64_t Y, int64_t y_first, int64_t nrows, uint8_t *bx,
                                uint8_t *by)
{
    for (int64_t i = 0; i < nrows; i++) {
        int64_t y = (y_first + i) % Y;
        for (int64_t x = 0; x < X; x++) {
            uint8_t v = (uint8_t)((x + y) & 1);
            bx[i * X + x] = v;
            by[i * X + x] = v;
        }
    }
}

void oracle_init_flat_band(int64_t L, int64_t y_first, int64_t nrows, uint8_t *bx, uint8_t *by)
{
    oracle_init_flat_band_rect(L, L, y_first, nrows, bx, by);
}

/* Heights of the whole lattice (small sizes): h(0,0) = 0, down column 0 with sy-, then along
 * each row with sx-.  Returns 0, or -1 if the slopes do not close around a torus cycle
 * (heights would not be single-valued). */
int oracle_heights_rect(int64_t X, int64_t Y, const uint8_t *bx, const uint8_t *by, int64_t *h)
{
    int64_t h0 = 0;
    for (int64_t y = 0; y < Y; y++) {
        if (y > 0) h0 += 2 * (int64_t)by[y * X + 0] - 1;
        int64_t hx = h0;
        h[y * X + 0] = hx;
        for (int64_t x = 1; x < X; x++) {
            hx += 2 * (int64_t)bx[y * X + x] - 1;
            h[y * X + x] = hx;
        }
        if (hx + 2 * (int64_t)bx[y * X + 0] - 1 != h0) return -1;
    }
    if (h0 + 2 * (int64_t)by[0] - 1 != 0) return -1;
    return 0;
}

int oracle_heights(int64_t L, const uint8_t *bx, const uint8_t *by, int64_t *h)
{
    return oracle_heights_rect(L, L, bx, by, h);
}

/* Exact roughness sums.  S1 = sum h, S2 = sum h^2 (128-bit), num = N*S2 - S1^2 (128-bit,
 * never negative) with N = X*Y.  Heights are built one row at a time as in
 * oracle_heights_rect.  Returns 0, or -1 if a row or column 0 does not close. */
int oracle_observe_rect(int64_t X, int64_t Y, const uint8_t *bx, const uint8_t *by,
                        int64_t *S1_out, uint64_t S2_out[2], uint64_t num_out[2])
{
    __int128 S1 = 0;
    unsigned __int128 S2 = 0;
    int bad = 0;
    int64_t h0 = 0;
    int64_t *col0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)Y);
    if (!col0) return -1;
    for (int64_t y = 0; y < Y; y++) {
        if (y > 0) h0 += 2 * (int64_t)by[y * X + 0] - 1;
        col0[y] = h0;
    }
    if (h0 + 2 * (int64_t)by[0] - 1 != 0) bad = 1;
    #pragma omp parallel
    {
        __int128 s1 = 0;
        unsigned __int128 s2 = 0;
        int rowbad = 0;
        #pragma omp for schedule(static)
        for (int64_t y = 0; y < Y; y++) {
            int64_t hx = col0[y];
            s1 += hx;
            s2 += (unsigned __int128)((__int128)hx * hx);
            for (int64_t x = 1; x < X; x++) {
                hx += 2 * (int64_t)bx[y * X + x] - 1;
                s1 += hx;
                s2 += (unsigned __int128)((__int128)hx * hx);
            }
            if (hx + 2 * (int64_t)bx[y * X + 0] - 1 != col0[y]) rowbad = 1;
        }
        #pragma omp critical
        {
            S1 += s1;
            S2 += s2;
            if (rowbad) bad = 1;
        }
    }
    free(col0);
    unsigned __int128 N = (unsigned __int128)((uint64_t)X * (uint64_t)Y);
    unsigned __int128 num = N * S2 - (unsigned __int128)(S1 * S1);
    *S1_out = (int64_t)S1;
    S2_out[0] = (uint64_t)S2; S2_out[1] = (uint64_t)(S2 >> 64);
    num_out[0] = (uint64_t)num; num_out[1] = (uint64_t)(num >> 64);
    return bad ? -1 : 0;
}

int oracle_observe(int64_t L, const uint8_t *bx, const uint8_t *by,
                   int64_t *S1_out, uint64_t S2_out[2], uint64_t num_out[2])
{
    return oracle_observe_rect(L, L, bx, by, S1_out, S2_out, num_out);
}

/* ------------------------------------------------------------------------------------------
 * Random-sequential (RS) dynamics on the local encoding (Sec. II.A: 4 x 4 sites per 32-bit
 * word, the encoding of choice when sites are selected at random; the paper's non-vectorized
 * comparison).  Reading (the paper gives no schedule for it): random-sequential updates
 * decomposed over the 4 x 4 words.  Word (wx, wy) holds the sites 4 wx <= x < 4 wx + 4,
 * 4 wy <= y < 4 wy + 4 (X, Y multiples of 8).  One MCS is two phases; in phase ph the words with
 * (wx + wy) & 1 == ph are active (no two active sites are neighbours, so the active words
 * evolve independently and in any order); an active word receives 16 attempts in sequence
 * a = 0..15 (on average one per site and MCS).  Attempt a of word w = wy * (X/4) + wx in
 * phase ph of MCS t takes the Philox4x32-10 call with counter
 *     (w low 32, t low 32, ph | a << 1 | (t >> 32) << 6, 2 | (w >> 32) << 2)
 * and key (seed low, seed high): the site is i = out[0] >> 28, (x, y) = (4 wx + (i & 3),
 * 4 wy + (i >> 2)); a local minimum deposits iff out[1] < floor(p 2^32), a local maximum is
 * removed iff out[1] < floor(q 2^32) (Eq. 1).  On a 4 x 4 torus (one word) this is plain
 * random-sequential dynamics, 16 uniform site choices per MCS.
 * ---------------------------------------------------------------------------------------- */
int oracle_rs_run_rect(int64_t X, int64_t Y, uint8_t *bx, uint8_t *by, uint64_t seed, double p, double q,
                       uint64_t t0, uint64_t n_mcs)
{
    if (X < 4 || Y < 4 || (X % 4) || (Y % 4)) return -1;
    if ((X > 4 && X % 8) || (Y > 4 && Y % 8)) return -1;
    if (!(p >= 0.0 && p <= 1.0 && q >= 0.0 && q <= 1.0)) return -1;
    const uint64_t Tp = (uint64_t)floor(ldexp(p, 32)), Tq = (uint64_t)floor(ldexp(q, 32));
    const int64_t WX = X / 4, WY = Y / 4;
    const uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (uint64_t t = t0; t < t0 + n_mcs; t++) {
        for (int ph = 0; ph <= 1; ph++) {
            #pragma omp parallel for schedule(static)
            for (int64_t wy = 0; wy < WY; wy++)
                for (int64_t wx = 0; wx < WX; wx++) {
                    if (((wx + wy) & 1) != ph) continue;
                    const uint64_t w = (uint64_t)(wy * WX + wx);
                    for (int a = 0; a < 16; a++) {
                        uint32_t ctr[4] = { (uint32_t)w, (uint32_t)t,
                                            (uint32_t)ph | ((uint32_t)a << 1) | ((uint32_t)(t >> 32) << 6),
                                            2u | ((uint32_t)(w >> 32) << 2) };
                        uint32_t out[4];
                        oracle_philox4x32_10(ctr, key, out);
                        const int i = (int)(out[0] >> 28);
                        const int64_t x = 4 * wx + (i & 3), y = 4 * wy + (i >> 2);
                        const int64_t xr = (x + 1) % X, yu = (y + 1) % Y;
                        uint8_t *sa = &bx[y * X + x], *sb = &by[y * X + x];
                        uint8_t *sc = &bx[y * X + xr], *sd = &by[yu * X + x];
                        const int is_min = (*sa == 0 && *sb == 0 && *sc == 1 && *sd == 1);
                        const int is_max = (*sa == 1 && *sb == 1 && *sc == 0 && *sd == 0);
                        if ((is_min && (uint64_t)out[1] < Tp) || (is_max && (uint64_t)out[1] < Tq)) {
                            *sa ^= 1; *sb ^= 1; *sc ^= 1; *sd ^= 1;
                        }
                    }
                }
        }
    }
    return 0;
}

/* Two-time height correlation of two states of the same X x Y lattice (the paper's two-time
 * functions and aging studies, Sec. I and Sec. IV; definition here): with heights h_a, h_b of
 * the two states (each from h(0,0) = 0, as in oracle_heights_rect),
 *   Sa = sum h_a, Sb = sum h_b, Sab = sum h_a h_b (128-bit),
 *   cnum = N * Sab - Sa * Sb (signed 128-bit), C = cnum / N^2,
 * the covariance of the two height fields over the sites, unchanged by a constant shift of
 * either field (so the unknown absolute heights do not enter).  C(t, t) = W^2(t).
 * Returns 0, or -1 if either state does not close. */
int oracle_corr_rect(int64_t X, int64_t Y, const uint8_t *ax, const uint8_t *ay, const uint8_t *bx,
                     const uint8_t *by, int64_t *Sa_out, int64_t *Sb_out, int64_t Sab_out[2],
                     int64_t cnum_out[2])
{
    size_t n = (size_t)X * (size_t)Y;
    int64_t *ha = (int64_t *)malloc(sizeof(int64_t) * n);
    int64_t *hb = (int64_t *)malloc(sizeof(int64_t) * n);
    if (!ha || !hb) { free(ha); free(hb); return -1; }
    int bad = oracle_heights_rect(X, Y, ax, ay, ha) != 0 || oracle_heights_rect(X, Y, bx, by, hb) != 0;
    __int128 Sa = 0, Sb = 0, Sab = 0;
    for (size_t i = 0; i < n; i++) {
        Sa += ha[i];
        Sb += hb[i];
        Sab += (__int128)ha[i] * hb[i];
    }
    free(ha);
    free(hb);
    __int128 cnum = (__int128)n * Sab - Sa * Sb;
    *Sa_out = (int64_t)Sa;
    *Sb_out = (int64_t)Sb;
    Sab_out[0] = (int64_t)(uint64_t)Sab; Sab_out[1] = (int64_t)(Sab >> 64);
    cnum_out[0] = (int64_t)(uint64_t)cnum; cnum_out[1] = (int64_t)(cnum >> 64);
    return bad ? -1 : 0;
}

/* Byte arrays -> canonical packed words (4 * Y * W words, zero padding bits). */
void oracle_pack_rect(int64_t X, int64_t Y, const uint8_t *bx, const uint8_t *by, uint32_t *words)
{
    uint64_t W = words_per_row(X);
    memset(words, 0, sizeof(uint32_t) * 4 * (size_t)Y * W);
    for (int64_t y = 0; y < Y; y++)
        for (int64_t x = 0; x < X; x++) {
            int s = (int)((x + y) & 1);
            uint64_t k = (uint64_t)(x >> 1);
            for (int d = 0; d < 2; d++) {
                uint8_t v = d == 0 ? bx[y * X + x] : by[y * X + x];
                uint64_t idx = ((uint64_t)(s * 2 + d) * (uint64_t)Y + (uint64_t)y) * W + (k >> 5);
                words[idx] |= (uint32_t)v << (k & 31);
            }
        }
}

void oracle_pack(int64_t L, const uint8_t *bx, const uint8_t *by, uint32_t *words)
{
    oracle_pack_rect(L, L, bx, by, words);
}

/* Canonical packed words -> byte arrays. */
void oracle_unpack_rect(int64_t X, int64_t Y, const uint32_t *words, uint8_t *bx, uint8_t *by)
{
    uint64_t W = words_per_row(X);
    for (int64_t y = 0; y < Y; y++)
        for (int64_t x = 0; x < X; x++) {
            int s = (int)((x + y) & 1);
            uint64_t k = (uint64_t)(x >> 1);
            uint64_t ix = ((uint64_t)(s * 2 + 0) * (uint64_t)Y + (uint64_t)y) * W + (k >> 5);
            uint64_t iy = ((uint64_t)(s * 2 + 1) * (uint64_t)Y + (uint64_t)y) * W + (k >> 5);
            bx[y * X + x] = (uint8_t)((words[ix] >> (k & 31)) & 1u);
            by[y * X + x] = (uint8_t)((words[iy] >> (k & 31)) & 1u);
        }
}

void oracle_unpack(int64_t L, const uint32_t *words, uint8_t *bx, uint8_t *by)
{
    oracle_unpack_rect(L, L, words, bx, by);
}

#ifdef _OPENMP
#include <omp.h>
#endif

/* Thread count for the parallel loops (results do not depend on it).  n <= 0 queries only. */
int oracle_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
