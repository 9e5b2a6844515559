// multi.cu -- one launch of the fused pass over several likelihood handles.
//
// Toy fits (the paper's multi-start and toy experiments, Sec. 3) evaluate many
// small likelihoods of different sizes, resonance counts K and projections S
// at once.  One launch serves all of them: its work list is every (handle,
// parameter vector, block) of the handles' batched passes, the blocks of
// handle i taking entries first[i] .. first[i + 1] - 1.  The CTAs are
// persistent: grid = the CTAs that fit on the GPU, each walking the work list
// with a stride of the grid.  Every entry runs the same per-block pass as
// pass_kernel (pass_body: its tiles, FP32 sums folded into compensated
// FP32, FP64 records, the last-block-done reduction and the Eq. 4-7 combine
// into the handle's own scratch and output rows), compiled once per S for
// eight warps with four resonances per warp in the second sweep, so any
// K <= 32 runs with K a runtime value; the handles' tile records are read
// with their own layout rotation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "pwa_internal.h"

namespace {

constexpr int kMW = 8;    // warps per CTA: 8 lanes per event in the first sweep
constexpr int kMKPW = 4;  // resonances per warp in the second sweep (K <= 32)

struct MultiArgs {
    const pwa::PassArgs* args;  // [n] batched-pass arguments of each handle
    const int* first;           // [n + 1] first work-list entry of each handle
    int n, total;
};

template <int MODE>
__global__ void __launch_bounds__(32 * kMW, 2) multi_pass_kernel(const MultiArgs m)
{
    extern __shared__ __align__(128) unsigned char smem[];
    for (int j = blockIdx.x; j < m.total; j += gridDim.x) {
        int hi = 0;
        while (hi + 1 < m.n && j >= m.first[hi + 1]) ++hi;
        const pwa::PassArgs a = m.args[hi];
        const int jj = j - m.first[hi];
        const int bt = jj % a.B, gb = jj / a.B;
        switch (a.S) {
            case 1: pwa::pass_body<MODE, 1, kMW, kMKPW>(a, bt, gb, smem); break;
            case 2: pwa::pass_body<MODE, 2, kMW, kMKPW>(a, bt, gb, smem); break;
            case 3: pwa::pass_body<MODE, 3, kMW, kMKPW>(a, bt, gb, smem); break;
            case 4: pwa::pass_body<MODE, 4, kMW, kMKPW>(a, bt, gb, smem); break;
            default: break;
        }
        // The next entry lays its shared memory out for another handle: its
        // TMA copies and stores may land where this entry kept mbarriers,
        // constants and sums.  So every thread has finished this entry, the
        // mbarriers are invalidated before their bytes are reused, and this
        // entry's generic-proxy writes are ordered before the next entry's
        // async-proxy (TMA) writes.
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t* bar = pwa::pass_mbarriers(smem, a, kMW);
            for (int s = 0; s < a.NST; ++s) pwa::mbar_inval(&bar[s]);
        }
        pwa::fence_proxy_async();
        __syncthreads();
    }
}

using MultiFn = void (*)(const MultiArgs);

MultiFn pick_multi(int mode)
{
    switch (mode) {
        case pwa::MODE_GRAD: return multi_pass_kernel<pwa::MODE_GRAD>;
        case pwa::MODE_HVP: return multi_pass_kernel<pwa::MODE_HVP>;
        default: return nullptr;
    }
}

}  // namespace

namespace pwa {

MultiScratch::~MultiScratch()
{
    if (d_args) cudaFree(d_args);
    if (d_first) cudaFree(d_first);
    if (h_stage) cudaFreeHost(h_stage);
    cudaGetLastError();
}

pwa_status launch_multi_reserve(pwa_handle* h0, int n, MultiScratch& ms)
{
    cudaError_t e = cudaSuccess;
    if (n > ms.cap) {
        if (ms.d_args) cudaFree(ms.d_args);
        if (ms.d_first) cudaFree(ms.d_first);
        if (ms.h_stage) cudaFreeHost(ms.h_stage);
        ms.d_args = nullptr;
        ms.d_first = nullptr;
        ms.h_stage = nullptr;
        ms.cap = 0;
        const int cap = std::max(n, 64);
        e = cudaMalloc(&ms.d_args, sizeof(PassArgs) * cap);
        if (e == cudaSuccess) e = cudaMalloc(&ms.d_first, sizeof(int) * (cap + 1));
        if (e == cudaSuccess)
            e = cudaMallocHost(&ms.h_stage, sizeof(PassArgs) * cap + sizeof(int) * (cap + 1));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(h0, PWA_ENOMEM, "allocation of the multi-handle launch arguments failed");
        }
        ms.cap = cap;
    }
    return PWA_OK;
}

pwa_status launch_multi(int n, pwa_handle* const* hs, const int* B, const double* const* d_theta,
                        const double* const* d_v, double* const* d_out, int mode, bool err_vec, cudaStream_t stream,
                        MultiScratch& ms)
{
    pwa_handle* h0 = hs[0];
    MultiFn fn = pick_multi(mode);
    if (!fn) return set_error(h0, PWA_EINVAL, "the multi-handle pass runs the gradient and H v modes");
    pwa_status rs = launch_multi_reserve(h0, n, ms);
    if (rs != PWA_OK) return rs;
    cudaError_t e = cudaSuccess;
    PassArgs* args = reinterpret_cast<PassArgs*>(ms.h_stage);
    int* first = reinterpret_cast<int*>(ms.h_stage + sizeof(PassArgs) * ms.cap);
    size_t smem = 0;
    long long total = 0;
    for (int i = 0; i < n; ++i) {
        pwa_handle* h = hs[i];
        if (h->K > kMW * kMKPW)
            return set_error(h, PWA_EINVAL, "the multi-handle pass supports K <= " + std::to_string(kMW * kMKPW));
        const Tiling& t = h->tiling;
        for (int s = 0; s < 2; ++s)
            if (h->tile_bytes[s] > t.stage_bytes || (long long)h->ntiles[s] * t.E < h->n[s] ||
                h->tile_bytes[s] % 16 != 0)
                return set_error(h, PWA_EINVAL, "inconsistent tile geometry");
        pwa_status st = prepare_batch(h, B[i], d_theta[i], mode == MODE_HVP ? d_v[i] : nullptr, d_out[i], err_vec,
                                      stream, args[i]);
        if (st != PWA_OK) return st;
        first[i] = (int)total;
        total += (long long)B[i] * args[i].Gb;
        smem = std::max(smem, pass_smem_bytes(h, kMW));
    }
    first[n] = (int)total;
    if (total > 0x7fffffffLL) return set_error(h0, PWA_EINVAL, "work list too long for one launch");
    int dev = 0, max_optin = 0, sms = 0, occ = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(fn));
    if (e != cudaSuccess) return cuda_error(h0, e, "multi-handle launch set-up");
    const int dyn_max = max_optin - (int)fa.sharedSizeBytes;
    if ((int)smem > dyn_max) return set_error(h0, PWA_EINVAL, "multi-handle pass: a handle's tiles need too much shared memory");
    e = cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<const void*>(fn), 32 * kMW, smem);
    if (e != cudaSuccess) return cuda_error(h0, e, "multi-handle occupancy");
    if (occ < 1) return set_error(h0, PWA_EINVAL, "multi-handle pass does not fit on an SM");
    const int grid = (int)std::max(1LL, std::min((long long)sms * occ, total));
    e = cudaMemcpyAsync(ms.d_args, args, sizeof(PassArgs) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ms.d_first, first, sizeof(int) * (n + 1), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_error(h0, e, "multi-handle arguments");
    MultiArgs m{ms.d_args, ms.d_first, n, (int)total};
    fn<<<grid, 32 * kMW, smem, stream>>>(m);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(h0, e, "multi-handle pass launch");
    return PWA_OK;
}

}  // namespace pwa

extern "C" pwa_status pwa_eval_multi_device(int n, pwa_handle* const* hs, const int* B, const double* const* d_theta,
                                            const double* const* d_v, double* const* d_out, int want_grad,
                                            int want_hv, void* stream)
{
    if (n < 1 || !hs || !B || !d_theta || !d_out) return PWA_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) return PWA_EINVAL;
        hs[i]->err.clear();
        if (!d_theta[i] || !d_out[i] || B[i] < 1 || (want_hv && (!d_v || !d_v[i])))
            return pwa::set_error(hs[i], PWA_EINVAL, "every handle needs d_theta, d_out (and d_v for hv) and B >= 1");
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return pwa::set_error(hs[i], PWA_EINVAL, "a handle appears twice");
    }
    if (!want_grad && !want_hv) return pwa::set_error(hs[0], PWA_EINVAL, "the multi-handle pass computes gradients");
    // the arguments' pinned staging of this thread; the previous call's copies
    // from it are done once its stream has drained
    static thread_local pwa::MultiScratch ms;
    static thread_local cudaStream_t last = nullptr;
    static thread_local bool used = false;
    if (used) {
        cudaError_t e = cudaStreamSynchronize(last);
        if (e != cudaSuccess) return pwa::cuda_error(hs[0], e, "multi-handle launch");
    }
    last = static_cast<cudaStream_t>(stream);
    used = true;
    return pwa::launch_multi(n, hs, B, d_theta, d_v, d_out, want_hv ? pwa::MODE_HVP : pwa::MODE_GRAD, true, last, ms);
}
