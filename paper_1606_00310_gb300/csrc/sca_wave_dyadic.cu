// Register-wavefront temporal blocking with dyadic draws (Sec. III): instantiations of the
// height-bit kernel in sca_wave.cuh for MODE 1, kept in their own translation unit so they
// compile in parallel with the rest of the library.
#include "sca_wave.cuh"

namespace sca {

template <int K, int V>
static int blocks_dyadic()
{
    static int n = 0;
    if (n == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_wave<K, V, kWaveU1, 1, true, true>, 32 * kWaveWarps, 0) !=
                cudaSuccess || b <= 0)
            b = 1;
        n = b;
    }
    return n;
}

int wave_dyadic_blocks_per_sm(int K, int V)
{
    if (V == 4) return K == 1 ? blocks_dyadic<1, 4>() : K == 2 ? blocks_dyadic<2, 4>() : blocks_dyadic<4, 4>();
    return K == 1 ? blocks_dyadic<1, 1>() : K == 2 ? blocks_dyadic<2, 1>() : blocks_dyadic<4, 1>();
}

template <int V>
static cudaError_t launch_v(const WaveArgs &a, int K, int grid, cudaStream_t st)
{
    switch (K) {
    case 1: k_wave<1, V, kWaveU1, 1, true, true><<<grid, 32 * kWaveWarps, 0, st>>>(a); break;
    case 2: k_wave<2, V, kWaveU1, 1, true, true><<<grid, 32 * kWaveWarps, 0, st>>>(a); break;
    case 4: k_wave<4, V, kWaveU1, 1, true, true><<<grid, 32 * kWaveWarps, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_wave_dyadic(const WaveArgs &a, int K, int V, int grid, cudaStream_t st)
{
    return V == 4 ? launch_v<4>(a, K, grid, st) : launch_v<1>(a, K, grid, st);
}

}  // namespace sca
