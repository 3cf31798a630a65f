// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "sca_rng.cuh"

namespace sca {

// Launch shape of a "row team": T threads own W words of one sublattice row, V words each,
// padded to TP threads so teams never straddle a warp in a way the scans cannot handle.
struct TeamShape {
    int V;          // words per thread per row (1, 2 or 4)
    int T;          // threads that own words
    int TP;         // padded team size (power of two <= 32, or a multiple of 32)
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
};

struct ObsPartial {
    int64_t s1;
    uint64_t s2_lo, s2_hi;
    uint32_t flags, pad;
};

// Update kernels.  A is the canonical word array (in place for the two-pass path); src/dst
// for the fused path.  Launch counts are added to the library's counter.
cudaError_t launch_half_step(uint32_t *A, uint32_t L, uint64_t t, int s, const Rule &R,
                             cudaStream_t st);
// err: device word; bit 0 is set if a pipeline wait gave up (the result is then invalid).
cudaError_t launch_fused_mcs(const uint32_t *src, uint32_t *dst, uint32_t L, uint64_t t,
                             const Rule &R, uint32_t *err, cudaStream_t st);
bool fused_supported(uint32_t L);
size_t fused_smem_bytes(uint32_t L);

// Observation kernels: h0 scratch of L int64; partials scratch of obs_partials(L) + 1 entries
// (never more than kObsGridCap + 1).
constexpr int kObsGridCap = 2048;
int obs_partials(uint32_t L);
cudaError_t launch_observe(const uint32_t *A, uint32_t L, int64_t *h0, ObsPartial *partials,
                           ObsDev *result, uint64_t t, cudaStream_t st);

void count_launches(uint64_t n);
int sm_count();

}  // namespace sca
