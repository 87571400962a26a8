// Per-term Taylor propagation for callers that cannot allocate device memory.
//
// ctqw_propagate_taylor's per-term path needs three state-sized scratch
// buffers that the caller passes in.  Some callers have no way to obtain
// them: real-time loops that must never call cudaMalloc because it can
// synchronize the whole device, and plugins embedded in a host program that
// owns the device memory budget.  This entry point takes
// its scratch from one statically sized device array instead, so it never
// allocates, frees or calls an allocating library routine.
#include <mutex>

#include "ctqw_internal.cuh"

// Scratch of the no-allocation entry point: three states of the per-term
// path (running sum and two Taylor terms).  48 MiB, i.e. 2 Mi complex-float
// or 1 Mi complex-double amplitudes per state, summed over realizations.
// Every GPU that loads this library holds the array until the process exits.
static constexpr size_t kNoAllocScratchBytes = size_t(48) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
int noalloc_scratch_address(void **out) {
    int dev = 0;
    CTQW_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        ctqw_set_error("no-allocation path: device ordinal %d above %d", dev, kMaxDevices - 1);
        return CTQW_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return ctqw_cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return CTQW_OK;
}

}  // namespace

extern "C" int ctqw_propagate_taylor_noalloc(const ctqw_hamiltonian *h, int32_t dtype,
                                             void *psi_dev, double dt, int32_t K, int64_t n_steps,
                                             int32_t obs_every, double *P_mean_dev,
                                             double *norm_dev, double *energy_dev, void *stream) {
    if (!h) {
        ctqw_set_error("null handle");
        return CTQW_EINVAL;
    }
    if (dtype != CTQW_C64 && dtype != CTQW_C128) {
        ctqw_set_error("dtype %d", dtype);
        return CTQW_EINVAL;
    }
    const size_t elem = dtype == CTQW_C64 ? sizeof(float2) : sizeof(double2);
    const size_t need = 3 * (size_t)h->total_amp * elem;
    if (need > kNoAllocScratchBytes) {
        ctqw_set_error("no-allocation path: %lld amplitudes need %zu bytes of scratch, above its "
                       "fixed %zu bytes; use ctqw_propagate_taylor with a workspace",
                       (long long)h->total_amp, need, kNoAllocScratchBytes);
        return CTQW_EINVAL;
    }
    // the scratch address is per device: the handle's device must be current
    int dev = -1;
    CTQW_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != h->device) {
        ctqw_set_error("no-allocation path: device %d is current but the handle lives on device %d",
                       dev, h->device);
        return CTQW_EINVAL;
    }
    void *scratch = nullptr;
    const int st = noalloc_scratch_address(&scratch);
    if (st != CTQW_OK) return st;
    // Nothing left in the array by an earlier call is read.  CTQW_C128: the
    // first Taylor term of every step writes the running sum and the term
    // buffer in full before they are read.  CTQW_C64: every Horner stage
    // writes its iterate in full before the next stage reads it, and the
    // carried error word is cleared by a memset at the start of the call.
    return ctqw_propagate_taylor(h, dtype, psi_dev, dt, K, n_steps, obs_every, P_mean_dev,
                                 norm_dev, energy_dev, CTQW_FLAG_PLAIN, scratch,
                                 kNoAllocScratchBytes, stream);
}
