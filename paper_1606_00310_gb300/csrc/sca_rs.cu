// Random-sequential dynamics on the local 4 x 4 encoding (the paper's non-vectorized comparison
// path, Sec. II.A and Sec. III).
//
// Local encoding: 32-bit word w = wy * (X/4) + wx holds the 16 sites 4 wx <= x < 4 wx + 4,
// 4 wy <= y < 4 wy + 4; bit 2 (4 ly + lx) is sx-(x, y) and bit 2 (4 ly + lx) + 1 is sy-(x, y)
// with (lx, ly) = (x - 4 wx, y - 4 wy).  A site's four slopes are its own two bits, sx- of its
// right neighbour (same word, or column 0 of the word to the right) and sy- of its upper
// neighbour (same word, or row 0 of the word above).
//
// Dynamics (the same process as the oracle's): each MCS is two phases over the checkerboard of
// words, (wx + wy) & 1 == phase; an active word takes 16 attempts in sequence, attempt a with
// the Philox call (w, t, ph | a << 1 | (t >> 32) << 6, 2 | (w >> 32) << 2): site out.x >> 28,
// flipped if it is a local minimum and out.y < floor(p 2^32), or a local maximum and
// out.y < floor(q 2^32) (Eq. 1).  One thread per active word keeps its word and the two
// neighbour words it touches in registers.  No two active sites are neighbours, so a bond is
// touched by at most one thread per phase: the own word is stored, and the bonds that live in
// the (inactive) right and upper words are flipped there with one atomic XOR of the changes,
// since other active words flip other bits of those words.
#include "sca_internal.h"

namespace sca {

constexpr int kRsThreads = 256;
// Draws made ahead of the attempts they decide: all 16 of a word (2.51e11 attempts/s at
// L = 16384, against 2.31e11 for groups of 8, 2.28e11 of 4 and 2.21e11 one at a time).
constexpr int kRsDraws = 16;

// canonical -> local: one thread per local word
__global__ void k_rs_to_local(const uint32_t *A, uint32_t *Lw, uint32_t X, uint32_t Y)
{
    const uint32_t WX = X / 4, nw = WX * (Y / 4), W = X / 64;
    const size_t plane = (size_t)Y * W;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
        const uint32_t wx = w % WX, wy = w / WX;
        uint32_t v = 0;
#pragma unroll
        for (int ly = 0; ly < 4; ++ly) {
            const uint32_t y = 4 * wy + ly;
#pragma unroll
            for (int lx = 0; lx < 4; ++lx) {
                const uint32_t x = 4 * wx + lx, s = (x + y) & 1u, k = x >> 1;
                const size_t o = (size_t)y * W + (k >> 5);
                const uint32_t bx = (A[(size_t)(2 * s) * plane + o] >> (k & 31)) & 1u;
                const uint32_t by = (A[(size_t)(2 * s + 1) * plane + o] >> (k & 31)) & 1u;
                v |= (bx | (by << 1)) << (2 * (4 * ly + lx));
            }
        }
        Lw[w] = v;
    }
}

// local -> canonical: one thread per canonical word (32 sites of sublattice s in row y)
__global__ void k_rs_to_canonical(const uint32_t *Lw, uint32_t *A, uint32_t X, uint32_t Y)
{
    const uint32_t W = X / 64, WX = X / 4;
    const size_t plane = (size_t)Y * W, n = 2 * plane;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t s = (uint32_t)(i / plane);
        const size_t r = i - (size_t)s * plane;
        const uint32_t y = (uint32_t)(r / W), j = (uint32_t)(r - (size_t)y * W);
        uint32_t vx = 0, vy = 0;
        for (int b = 0; b < 32; ++b) {
            const uint32_t k = 32 * j + b, x = 2 * k + ((s + y) & 1u);
            const uint32_t v = Lw[(y / 4) * WX + x / 4] >> (2 * (4 * (y & 3) + (x & 3)));
            vx |= (v & 1u) << b;
            vy |= ((v >> 1) & 1u) << b;
        }
        A[(size_t)(2 * s) * plane + r] = vx;
        A[(size_t)(2 * s + 1) * plane + r] = vy;
    }
}

struct RsArgs {
    uint32_t *Lw;
    uint32_t X, Y;
    uint64_t t;
    int ph;
    uint32_t k0, k1;
    uint64_t Tp, Tq;      // floor(p 2^32), floor(q 2^32); 2^32 means always
    uint32_t rk[20];
};

__global__ void __launch_bounds__(kRsThreads) k_rs_phase(const RsArgs a)
{
    const uint32_t WX = a.X / 4, WY = a.Y / 4, half = WX / 2;
    const uint32_t nact = half * WY;                // WX even: half the words of each row
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nact; c += gridDim.x * blockDim.x) {
        const uint32_t wy = c / half, i = c - wy * half;
        const uint32_t wx = 2 * i + ((wy + (uint32_t)a.ph) & 1u);
        const uint32_t w = wy * WX + wx;
        const uint32_t wr = wy * WX + (wx + 1 == WX ? 0 : wx + 1);
        const uint32_t wu = (wy + 1 == WY ? 0 : wy + 1) * WX + wx;
        uint32_t own = a.Lw[w];
        const uint32_t r0 = a.Lw[wr], u0 = a.Lw[wu];
        uint32_t rgt = r0, up = u0;
        // the draws do not depend on the state: they are made ahead as independent Philox
        // chains, then applied in attempt order
#pragma unroll 1
        for (uint32_t a0 = 0; a0 < 16; a0 += kRsDraws) {
            uint32_t ox[kRsDraws], oy[kRsDraws];
#pragma unroll
            for (int j = 0; j < kRsDraws; ++j) {
                const uint32_t at = a0 + (uint32_t)j;
                const Ctr4 o = philox4x32_10_rk(
                    Ctr4{w, (uint32_t)a.t, (uint32_t)a.ph | (at << 1) | ((uint32_t)(a.t >> 32) << 6), 2u}, a.rk);
                ox[j] = o.x;
                oy[j] = o.y;
            }
#pragma unroll
            for (int j = 0; j < kRsDraws; ++j) {
                const Ctr4 o{ox[j], oy[j], 0u, 0u};
                const uint32_t si = o.x >> 28, lx = si & 3u, ly = si >> 2;
                const uint32_t pa = 2 * (4 * ly + lx);                         // sx-, sy- of the site
                const uint32_t pc = lx < 3 ? pa + 2 : 2 * (4 * ly);            // sx- of the right site
                const uint32_t pd = ly < 3 ? pa + 8 + 1 : 2 * lx + 1;          // sy- of the upper site
                const uint32_t &cw = lx < 3 ? own : rgt;
                const uint32_t &dw = ly < 3 ? own : up;
                const uint32_t sa = (own >> pa) & 1u, sb = (own >> (pa + 1)) & 1u;
                const uint32_t sc = (cw >> pc) & 1u, sd = (dw >> pd) & 1u;
                const bool mn = !sa && !sb && sc && sd, mx = sa && sb && !sc && !sd;
                if ((mn && (uint64_t)o.y < a.Tp) || (mx && (uint64_t)o.y < a.Tq)) {
                    own ^= 3u << pa;
                    if (lx < 3) own ^= 1u << pc; else rgt ^= 1u << pc;
                    if (ly < 3) own ^= 1u << pd; else up ^= 1u << pd;
                }
            }
        }
        a.Lw[w] = own;
        if (rgt != r0) atomicXor(a.Lw + wr, rgt ^ r0);
        if (up != u0) atomicXor(a.Lw + wu, up ^ u0);
    }
}

bool rs_supported(uint32_t X, uint32_t Y) { return X % 64 == 0 && X >= 64 && Y % 8 == 0 && Y >= 8; }

static int rs_grid(size_t n)
{
    size_t g = (n + kRsThreads - 1) / kRsThreads;
    const size_t cap = (size_t)sm_count() * 16;
    return (int)(g < cap ? (g ? g : 1) : cap);
}

// n_mcs MCS of random-sequential dynamics on the canonical words A, with Lw (X Y / 4 bytes) as
// the local-encoding buffer: A -> Lw, the phases, Lw -> A.
cudaError_t launch_rs(uint32_t *A, uint32_t *Lw, uint32_t X, uint32_t Y, uint64_t t0, uint64_t n_mcs,
                      const Rule &R, uint64_t Tp, uint64_t Tq, cudaStream_t st)
{
    if (!rs_supported(X, Y)) return cudaErrorInvalidValue;
    const size_t nw = (size_t)(X / 4) * (Y / 4);
    k_rs_to_local<<<rs_grid(nw), kRsThreads, 0, st>>>(A, Lw, X, Y);
    count_launches(1);
    RsArgs a{};
    a.Lw = Lw;
    a.X = X;
    a.Y = Y;
    a.k0 = R.k0;
    a.k1 = R.k1;
    a.Tp = Tp;
    a.Tq = Tq;
    for (int r = 0; r < 20; ++r) a.rk[r] = R.rk[r];
    for (uint64_t m = 0; m < n_mcs; ++m) {
        a.t = t0 + m;
        for (int ph = 0; ph < 2; ++ph) {
            a.ph = ph;
            k_rs_phase<<<rs_grid(nw / 2), kRsThreads, 0, st>>>(a);
            count_launches(1);
        }
    }
    k_rs_to_canonical<<<rs_grid(2 * (size_t)Y * (X / 64)), kRsThreads, 0, st>>>(Lw, A, X, Y);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sca
