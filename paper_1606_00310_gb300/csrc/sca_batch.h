// Batched ensemble, cluster engine: the device structures shared by the persistent cluster
// kernel (sca_batch.cu) and the batch's host side (sca_batch_api.cu).
#pragma once

#include "sca_internal.h"

namespace sca {

struct BatchLattice {
    uint64_t state_off;  // word offset of its canonical words in the batch buffer
    uint32_t L, W, G, V; // size, words per sublattice row, CTAs sharing it, words per item
    uint32_t part_off;   // first partial: part_off + obs * G + part
    uint32_t pad;
    Rule R;
};

struct BatchSlot {
    int32_t lattice;     // -1: this CTA idles in the unit
    int16_t part;
    int16_t unit_G;      // parts per lattice in this unit (same for every slot of the unit)
};

struct BatchArgs {
    uint32_t *state;
    const BatchLattice *lat;
    const BatchSlot *slots;    // n_units x C
    int n_units, C;
    uint32_t *unit_counter;
    const uint64_t *times;
    int n_times;
    uint64_t t0;
    ObsPartial *partials;
    uint64_t *unit_ns;         // per unit: start and end time (globaltimer, ns)
};

// Shared memory of one part (two planes of height bits and the observation's column-0 heights
// of the largest of G parts of an L x L lattice).
size_t batch_part_smem(uint32_t L, uint32_t G);
// Kernel attributes for a launch shape (cluster size C, dynamic shared memory per CTA).
cudaError_t batch_prepare(int C, size_t smem);
// One persistent launch of n_clusters clusters of a.C CTAs.
cudaError_t launch_batch(const BatchArgs &a, int n_clusters, int threads, size_t smem, cudaStream_t st);
// Clusters of the launch shape resident at once on the device.
cudaError_t batch_max_clusters(int C, int threads, size_t smem, int *out);
// Exact roughness records of n_lat lattices at n_times times from the per-part partials.
cudaError_t launch_batch_finalize(const BatchLattice *lat, int n_lat, const ObsPartial *part,
                                  const uint64_t *times, int n_times, ObsDev *out, cudaStream_t st);

}  // namespace sca
