// Roughness observation that allocates nothing (sca_observe_noalloc in include/sca.h).
//
// Some callers cannot let a library allocate device memory: a host application that owns all
// GPU memory through its own pool and budgets every byte, a plug-in that is not allowed to
// call the CUDA allocator, or a latency-sensitive loop that must not pay for (or fail in)
// cudaMalloc, which can also synchronise the device.  Such callers already hold the lattice's
// canonical words in memory they allocated themselves.  For them this entry point runs the
// same observation kernels as sca_observe, with their scratch (the per-chunk records of the row
// kernel and the result record) in one file-scope device array instead of an allocation.
//
// The array is static: every GPU that loads this library holds kScratchBytes of it until the
// process exits.  All calls on a device share it, so calls that overlap on the GPU (two
// streams, or two host threads) race on it and must be serialised by the caller.  Each call
// writes every scratch byte it later reads, so leftovers of an earlier call never matter and
// nothing needs clearing.
#include <cmath>
#include <mutex>
#include <string>

#include "sca.h"
#include "sca_internal.h"

namespace sca {
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *where);

// The library's largest lattice.  The row kernel reduces at most kObsChunkCap chunks of at most
// 256 rows each (obs_partials), which covers it; the chunk records take two partial slots each.
constexpr uint32_t kNoAllocMaxL = 131072;
// layout: the partial slots (kObsGridCap + 1 of them, the chunk records), then the result record
constexpr size_t kPartBytes = ((size_t)(kObsGridCap + 1) * sizeof(ObsPartial) + 255) & ~(size_t)255;
constexpr size_t kResOff = kPartBytes;
constexpr size_t kScratchBytes = kResOff + 256;
static_assert(sizeof(ObsDev) <= 256, "result record fits");
static_assert(kScratchBytes == 66048, "the size the header states");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the array on each device, looked up once per device with that device
// current (host code cannot use the symbol itself as a device address).
constexpr int kMaxDevices = 64;
static void *g_scratch_addr[kMaxDevices];
static std::once_flag g_scratch_once[kMaxDevices];
static cudaError_t g_scratch_err[kMaxDevices];

static cudaError_t scratch_for_current_device(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(g_scratch_once[dev], [dev]() {
        void *p = nullptr;
        g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        g_scratch_addr[dev] = p;
    });
    if (g_scratch_err[dev] != cudaSuccess) return g_scratch_err[dev];
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace sca

using namespace sca;

extern "C" int sca_observe_noalloc(const uint32_t *words_dev, uint32_t L, uint64_t t, void *stream,
                                   sca_obs *out)
{
    if (!words_dev || !out) return fail(SCA_EINVAL, "NULL argument");
    if (L < 64 || L % 64 != 0)
        return fail(SCA_EINVAL, "L must be a positive multiple of 64");
    if (L > kNoAllocMaxL)
        return fail(SCA_EINVAL, "L exceeds the library's largest lattice, 131072");
    if (obs_partials(L) > kObsGridCap / 2)
        return fail(SCA_EINVAL, "L needs more chunk records than the scratch array holds");
    void *base = nullptr;
    cudaError_t e = scratch_for_current_device(&base);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    unsigned char *b = static_cast<unsigned char *>(base);
    ObsPartial *part = reinterpret_cast<ObsPartial *>(b);
    ObsDev *res = reinterpret_cast<ObsDev *>(b + kResOff);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = launch_observe(words_dev, L, nullptr, part, res, t, st);
    if (e != cudaSuccess) return cuda_fail(e, "observe launch");
    e = cudaMemcpyAsync(out, res, sizeof(ObsDev), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "observe copy");
    const double num = std::ldexp((double)out->num_hi, 64) + (double)out->num_lo;
    const double N = (double)out->N;
    out->w2 = num / (N * N);
    if (out->status) return fail(out->status, "slopes do not close around the torus");
    return SCA_OK;
}
