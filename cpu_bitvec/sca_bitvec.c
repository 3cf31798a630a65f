/*
 * Bit-vectorized CPU implementation of the octahedron-model SCA with 64-bit words: the paper's
 * CPU counterpart of its GPU kernel (Sec. II.B, last paragraph: the same update on 64-bit
 * words, rows of a sublattice split over OpenMP threads), kept as the like-for-like CPU
 * baseline of the GPU numbers (Sec. III compares the two).
 *
 * BASELINE ONLY.  The GPU library neither uses nor loads this file; it shares no code with the
 * CUDA library or with the oracle (its Philox and its update are written here again), and the
 * tests check it bit for bit against the oracle.
 *
 * State: the canonical packed words of the library (X sites per row, Y rows; 32-bit word
 * ((s*2 + d)*Y + y)*W + j holds sublattice sites k = 32 j .. 32 j + 31 of row y), read as 64-bit
 * words: on a little-endian host 32-bit words 2m and 2m + 1 form 64-bit word m, whose bit b is
 * sublattice site 64 m + b.  Needs X a multiple of 128 (whole 64-bit words per row).
 *
 * Update (Eqs. 2-4) for the words of sublattice s in row y: xm = sx-, ym = sy- (own), xpl = sx+
 * (the other sublattice's sx- words of the same row, shifted down by one site where (s + y) is
 * odd), ypl = sy+ (the other sublattice's sy- words of row y + 1); m_p = xi_p & ~(xm | ym) &
 * xpl & ypl, m_q = xi_q & ~(xpl | ypl) & xm & ym, m = m_p ^ m_q; m is XORed into the four slope
 * words (into sx+ shifted back up, with the top bit carried into the next word).  Rows of one
 * sublattice touch disjoint words, so threads take rows in any order.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) with the library's counter layout, so
 * that results equal the oracle's: for 32-bit packed-word unit u = y * (X/64) + j the draw i
 * of sublattice s at MCS t is lane u & 3 of the call with counter (u >> 2, t, s | (i-1) << 1 |
 * (t >> 32) << 6, (u >> 2) >> 32 << 1) and key (seed low, seed high); one call gives 128 bits,
 * two 64-bit words.  Dyadic p = P / 2^n: xi = r_n; xi = b_i ? r_i | xi : r_i & xi for
 * i = n-1 .. 1 (Sec. III).  Other p: site k of row y uses lane (y * X/2 + k) & 3 of the call
 * with counter ((y * X/2 + k) >> 2, t, s | (t >> 32) << 6, 1 | ... << 1), accepted iff below
 * floor(p * 2^32).  Deposition and removal share the draws.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static void philox(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; r++) {
        uint64_t a = (uint64_t)0xD2511F53u * c[0];
        uint64_t b = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t n0 = (uint32_t)(b >> 32) ^ c[1] ^ k0;
        uint32_t n2 = (uint32_t)(a >> 32) ^ c[3] ^ k1;
        c[1] = (uint32_t)b;
        c[3] = (uint32_t)a;
        c[0] = n0;
        c[2] = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

typedef struct {
    uint32_t k0, k1;
    int mode;                 /* 0: p, q in {0, 1}; 1: dyadic; 2: per-site uniform */
    int n, np, nq;            /* dyadic: draws, exponents */
    uint64_t Pp, Pq;          /* dyadic numerators; mode 0: 1 for probability 1 */
    uint64_t Tp, Tq;          /* per-site thresholds floor(p 2^32) */
} rule_t;

static int dyadic(double p, uint64_t *P, int *n)
{
    if (!(p >= 0.0 && p <= 1.0)) return 0;
    double v = ldexp(p, 32);
    if (v != floor(v)) return 0;
    uint64_t num = (uint64_t)v;
    int e = 32;
    if (num == 0) { *P = 0; *n = 0; return 1; }
    while (e > 0 && !(num & 1u)) { num >>= 1; e--; }
    *P = num;
    *n = e;
    return 1;
}

static int make_rule(rule_t *R, uint64_t seed, double p, double q, int mode)
{
    memset(R, 0, sizeof(*R));
    if (!(p >= 0.0 && p <= 1.0 && q >= 0.0 && q <= 1.0)) return -1;
    R->k0 = (uint32_t)seed;
    R->k1 = (uint32_t)(seed >> 32);
    if (mode == 1) {
        if (!dyadic(p, &R->Pp, &R->np) || !dyadic(q, &R->Pq, &R->nq)) return -1;
        R->n = R->np > R->nq ? R->np : R->nq;
        R->mode = R->n == 0 ? 0 : 1;
    } else if (mode == 2) {
        R->Tp = (uint64_t)floor(ldexp(p, 32));
        R->Tq = (uint64_t)floor(ldexp(q, 32));
        R->mode = 2;
        R->Pp = R->Tp == (1ull << 32);
        R->Pq = R->Tq == (1ull << 32);
        if ((R->Tp == 0 || R->Pp) && (R->Tq == 0 || R->Pq)) R->mode = 0;
    } else {
        return -1;
    }
    return 0;
}

/* Draw i of the two 32-bit units u, u + 1 (u even) as one 64-bit word. */
static uint64_t draw64(const rule_t *R, uint64_t u, uint64_t t, int s, int i)
{
    uint64_t g = u >> 2;
    uint32_t c[4] = {(uint32_t)g, (uint32_t)t, (uint32_t)s | ((uint32_t)(i - 1) << 1) | ((uint32_t)(t >> 32) << 6),
                     (uint32_t)(g >> 32) << 1};
    philox(c, R->k0, R->k1);
    int l = (int)(u & 3);      /* 0 or 2 */
    return (uint64_t)c[l] | ((uint64_t)c[l + 1] << 32);
}

/* xi_p, xi_q of 64-bit word m of row y (units 2m, 2m + 1 of the 32-bit layout). */
static void xi64(const rule_t *R, uint64_t W32, uint64_t y, uint64_t m, uint64_t t, int s, uint64_t X,
                 uint64_t *xp, uint64_t *xq)
{
    if (R->mode == 0) {
        *xp = R->Pp ? ~0ull : 0;
        *xq = R->Pq ? ~0ull : 0;
        return;
    }
    if (R->mode == 1) {
        uint64_t p = (R->np == 0 && R->Pp) ? ~0ull : 0, q = (R->nq == 0 && R->Pq) ? ~0ull : 0;
        for (int i = R->n; i >= 1; i--) {
            uint64_t r = draw64(R, y * W32 + 2 * m, t, s, i);
            if (i <= R->np) p = i == R->np ? r : (((R->Pp >> (R->np - i)) & 1) ? (r | p) : (r & p));
            if (i <= R->nq) q = i == R->nq ? r : (((R->Pq >> (R->nq - i)) & 1) ? (r | q) : (r & q));
        }
        *xp = p;
        *xq = q;
        return;
    }
    uint64_t p = 0, q = 0;
    const uint64_t base = y * (X / 2) + 64 * m;        /* site unit of bit 0; a multiple of 4 */
    for (int c4 = 0; c4 < 16; c4++) {
        uint64_t g = (base >> 2) + (uint64_t)c4;
        uint32_t c[4] = {(uint32_t)g, (uint32_t)t, (uint32_t)s | ((uint32_t)(t >> 32) << 6),
                         1u | ((uint32_t)(g >> 32) << 1)};
        philox(c, R->k0, R->k1);
        for (int l = 0; l < 4; l++) {
            p |= (uint64_t)((uint64_t)c[l] < R->Tp) << (4 * c4 + l);
            q |= (uint64_t)((uint64_t)c[l] < R->Tq) << (4 * c4 + l);
        }
    }
    *xp = p;
    *xq = q;
}

#define BITVEC_MAX_W 1024   /* 64-bit words per row at X = 131072 */

/* n_mcs MCS from MCS index t0 on the canonical words A (X sites per row, Y rows). */
int bitvec_run(uint32_t *A, uint64_t X, uint64_t Y, uint64_t seed, double p, double q, int mode, uint64_t t0,
               uint64_t n_mcs)
{
    rule_t R;
    if (X < 128 || X % 128 || X / 128 > BITVEC_MAX_W || Y < 2 || (Y & 1)) return -1;
    if (make_rule(&R, seed, p, q, mode)) return -1;
    const uint64_t W32 = X / 64, W = X / 128, plane = Y * W;
    uint64_t *B = (uint64_t *)(void *)A;
    for (uint64_t t = t0; t < t0 + n_mcs; t++) {
        for (int s = 0; s <= 1; s++) {
            uint64_t *SX = B + (uint64_t)(2 * s) * plane, *SY = B + (uint64_t)(2 * s + 1) * plane;
            uint64_t *NX = B + (uint64_t)(2 * (s ^ 1)) * plane, *NY = B + (uint64_t)(2 * (s ^ 1) + 1) * plane;
            #pragma omp parallel for schedule(static)
            for (int64_t yy = 0; yy < (int64_t)Y; yy++) {
                const uint64_t y = (uint64_t)yy, yn = y + 1 == Y ? 0 : y + 1;
                uint64_t *xm = SX + y * W, *ym = SY + y * W, *nx = NX + y * W, *ny = NY + yn * W;
                const int shifted = (int)((s + y) & 1);
                uint64_t mk[BITVEC_MAX_W];
                /* pass 1: masks from the words as they were (sx+ of a shifted row reads the next
                 * word of the other sublattice, periodic in x); the own words and sy+ change now */
                for (uint64_t m = 0; m < W; m++) {
                    uint64_t xpl = nx[m];
                    if (shifted) xpl = (xpl >> 1) | (nx[m + 1 < W ? m + 1 : 0] << 63);
                    uint64_t xip, xiq;
                    xi64(&R, W32, y, m, t, s, X, &xip, &xiq);
                    const uint64_t a = xm[m], b = ym[m], d = ny[m];
                    mk[m] = (xip & ~(a | b) & xpl & d) ^ (xiq & ~(xpl | d) & a & b);
                    xm[m] = a ^ mk[m];
                    ym[m] = b ^ mk[m];
                    ny[m] = d ^ mk[m];
                }
                /* pass 2: sx+ is the other sublattice's sx- of site k (aligned) or of site k + 1
                 * (shifted: the mask moves up one bit, the top bit into the next word) */
                for (uint64_t m = 0; m < W; m++)
                    nx[m] ^= shifted ? (mk[m] << 1) | (mk[m ? m - 1 : W - 1] >> 63) : mk[m];
            }
        }
    }
    return 0;
}

int bitvec_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
