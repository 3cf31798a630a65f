// Register-wavefront temporal blocking with per-site uniform draws (Sec. II.B: one 32-bit
// random number per site, four sites per Philox call, accept below floor(p 2^32)): the
// instantiations of the height-bit kernel in sca_wave.cuh for MODE 2, one word per lane.
#include "sca_wave.cuh"

namespace sca {

template <int K>
static int blocks_uniform()
{
    static int n = 0;
    if (n == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_wave<K, 1, kWaveU1, 2, true, true, 0>,
                                                          32 * kWaveWarps, 0) != cudaSuccess || b <= 0)
            b = 1;
        n = b;
    }
    return n;
}

int wave_uniform_blocks_per_sm(int K) { return K == 1 ? blocks_uniform<1>() : blocks_uniform<2>(); }

cudaError_t launch_wave_uniform(const WaveArgs &a, int K, int grid, cudaStream_t st)
{
    switch (K) {
    case 1: k_wave<1, 1, kWaveU1, 2, true, true, 0><<<grid, 32 * kWaveWarps, 0, st>>>(a); break;
    case 2: k_wave<2, 1, kWaveU1, 2, true, true, 0><<<grid, 32 * kWaveWarps, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sca
