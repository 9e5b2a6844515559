// noalloc.cu -- pwa_eval_device_noalloc: the fused pass with its reduction
// scratch in a fixed, statically allocated device array.
//
// Who needs it: callers that must not call cudaMalloc while they evaluate --
// for example code running under an external memory manager that has already
// reserved the device's memory, or a real-time loop that may not take the
// device-wide synchronisation an allocation can imply.  They create the handle
// once (that allocates), then evaluate through this entry point, which
// allocates nothing: the per-block and per-group partial sums and the
// completion counters of the last-block-done reduction live in the array
// below, not in the handle's buffers.
//
// The array is a file-scope __device__ object: every GPU that loads libpwa
// holds it (kNoAllocScratchBytes) until the process exits.  Host code cannot
// use its name as a device address; its address is looked up once per device
// with cudaGetSymbolAddress (on the first call made on that device, with that
// device current) and passed to the kernel.  All calls share the array and it
// keeps the last call's contents, so the counters are cleared at every call
// and calls whose kernels overlap on the GPU race on it.  The looked-up
// address is kept for the life of the process; after a cudaDeviceReset it
// belongs to a destroyed context, so the entry point must not be used then.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "pwa_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(2) << 20;  // 2 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
pwa_status scratch_address(pwa_handle* h, unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return pwa::cuda_error(h, e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return pwa::set_error(h, PWA_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "cudaGetSymbolAddress(scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return PWA_OK;
}

}  // namespace

extern "C" pwa_status pwa_eval_device_noalloc(pwa_handle* h, const double* d_theta, const double* d_v,
                                              double* d_out, int want_grad, int want_hv)
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    if (h->broken) return pwa::set_error(h, PWA_ETIMEOUT, "handle is unusable after a device-side timeout");
    if (!d_theta || !d_out || (want_hv && !d_v))
        return pwa::set_error(h, PWA_EINVAL, "d_theta, d_out (and d_v for hv) must not be NULL");
    const pwa::Tiling& t = h->tiling;
    const int mode = want_hv ? pwa::MODE_HVP : (want_grad ? pwa::MODE_GRAD : pwa::MODE_NLL);

    // scratch layout: block partials | group partials | counters (ngroups + 1)
    const size_t rec = (size_t)h->rec_len;
    const size_t block_bytes = sizeof(double) * rec * (size_t)t.grid;
    const size_t group_bytes = sizeof(double) * rec * (size_t)h->ngroups;
    const size_t count_bytes = sizeof(unsigned) * (size_t)(h->ngroups + 1);
    const size_t need = block_bytes + group_bytes + count_bytes;
    if (need > kNoAllocScratchBytes)
        return pwa::set_error(h, PWA_EINVAL, "this handle needs " + std::to_string(need) +
                                                 " bytes of reduction scratch; the allocation-free entry "
                                                 "point has " + std::to_string(kNoAllocScratchBytes));
    unsigned char* base = nullptr;
    pwa_status st = scratch_address(h, &base);
    if (st != PWA_OK) return st;
    unsigned* counts = reinterpret_cast<unsigned*>(base + block_bytes + group_bytes);
    // the counters must start at zero (an earlier call may have been cut short)
    cudaError_t e = cudaMemsetAsync(counts, 0, count_bytes, h->stream);
    if (e != cudaSuccess) return pwa::cuda_error(h, e, "clearing the scratch counters");

    // the handle's pass arguments with the reduction scratch moved into the array
    pwa::PassArgs a = pwa::pass_args(h, d_theta, want_hv ? d_v : nullptr, d_out);
    a.block_rec = reinterpret_cast<double*>(base);
    a.group_rec = reinterpret_cast<double*>(base + block_bytes);
    a.group_count = counts;
    a.top_count = counts + h->ngroups;
    return pwa::launch_pass_args(h, a, mode);
}
