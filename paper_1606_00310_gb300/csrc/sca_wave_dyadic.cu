// Register-wavefront temporal blocking with dyadic draws (Sec. III): instantiations of the
// height-bit kernel in sca_wave.cuh for MODE 1, kept in their own translation unit so they
// compile in parallel with the rest of the library.  Four words per lane (one Philox call per
// draw covers them) with the draw count fixed at compile time for 1..3 draws and q = 0 or not;
// everything else takes the run-time draw loop.
#include "sca_wave.cuh"

namespace sca {

template <int K, int V, bool DQ, int ND, int MINB = -1>
static cudaError_t launch_one(const WaveArgs &a, int grid, cudaStream_t st, int *blocks)
{
    auto kern = k_wave<K, V, kWaveU1, 1, true, DQ, ND, MINB>;
    if (blocks) {
        static int n = 0;
        if (n == 0) {
            int b = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 32 * kWaveWarps, 0) != cudaSuccess || b <= 0)
                b = 1;
            n = b;
        }
        *blocks = n;
        return cudaSuccess;
    }
    kern<<<grid, 32 * kWaveWarps, 0, st>>>(a);
    return cudaGetLastError();
}

// The one-draw, q = 0 kernel at 4 MCS per launch is held to 128 registers (16 warps per SM
// instead of 12) on lattices of 2^32 sites or more: +1.3 % at L = 65536 and +2.6 % at 131072,
// but -2.5 % at 32768, where the plan then cuts more, shorter bands.
template <int K>
static cudaError_t dispatch_k(const WaveArgs &a, int V, int grid, cudaStream_t st, int *blocks)
{
    const Rule &R = a.R;
    const bool dp = !(R.np == 0 && R.Pp == 0), dq = !(R.nq == 0 && R.Pq == 0);
    if (V == 4 && dp && R.n_draws >= 1 && R.n_draws <= 3) {
        const bool large = (uint64_t)a.L * a.Y >= (1ull << 32);
        switch (R.n_draws * 2 + (dq ? 1 : 0)) {
        case 2:
            if constexpr (K == 4) {
                if (large) return launch_one<4, 4, false, 1, 16>(a, grid, st, blocks);
            }
            return launch_one<K, 4, false, 1>(a, grid, st, blocks);
        case 3: return launch_one<K, 4, true, 1>(a, grid, st, blocks);
        case 4: return launch_one<K, 4, false, 2>(a, grid, st, blocks);
        case 5: return launch_one<K, 4, true, 2>(a, grid, st, blocks);
        case 6: return launch_one<K, 4, false, 3>(a, grid, st, blocks);
        default: return launch_one<K, 4, true, 3>(a, grid, st, blocks);
        }
    }
    if (V == 4) return launch_one<K, 4, true, 0>(a, grid, st, blocks);
    return launch_one<K, 1, true, 0>(a, grid, st, blocks);
}

static cudaError_t dispatch(const WaveArgs &a, int K, int V, int grid, cudaStream_t st, int *blocks)
{
    switch (K) {
    case 1: return dispatch_k<1>(a, V, grid, st, blocks);
    case 2: return dispatch_k<2>(a, V, grid, st, blocks);
    case 4: return dispatch_k<4>(a, V, grid, st, blocks);
    default: return cudaErrorInvalidValue;
    }
}

int wave_dyadic_blocks_per_sm(const Rule &R, int K, int V, uint32_t X, uint32_t Y)
{
    WaveArgs a{};
    a.R = R;
    a.L = X;
    a.Y = Y;
    int b = 1;
    if (dispatch(a, K, V, 0, nullptr, &b) != cudaSuccess) return 1;
    return b;
}

cudaError_t launch_wave_dyadic(const WaveArgs &a, int K, int V, int grid, cudaStream_t st)
{
    return dispatch(a, K, V, grid, st, nullptr);
}

}  // namespace sca
