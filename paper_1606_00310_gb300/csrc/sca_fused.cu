// Fused even+odd update (one launch per MCS); filled in below the two-pass path.
#include "sca_internal.h"

namespace sca {

bool fused_supported(uint32_t) { return false; }
size_t fused_smem_bytes(uint32_t) { return 0; }
cudaError_t launch_fused_mcs(const uint32_t *, uint32_t *, uint32_t, uint64_t, const Rule &,
                             cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace sca
