// pwa_api.cu -- the libpwa C ABI (handle, layout, fused pass dispatch).
//
// pwa_create copies the caller's events to the device, validates them, and
// re-lays F out in contiguous event tiles (see pass_kernel.cuh).  Every
// evaluation is one launch of the fused pass: TMA-staged sweeps over the
// tiles, FP32 per event, FP64 partial sums, FP64 combination of paper
// Eqs. 4, 6, 7 in the last block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pwa_internal.h"

using pwa::ResParam;
using pwa::Tiling;

namespace {

thread_local std::string g_create_error;

__global__ void validate_kernel(const float* __restrict__ x, long long count, long long per_event,
                                int nonneg, unsigned long long* first_bad)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float v = x[i];
        const bool ok = isfinite(v) && (!nonneg || v >= 0.f);
        if (!ok) atomicMin(first_bad, (unsigned long long)(i / per_event));
    }
}

// m2 is [3][n]: the event of element i is i % n
__global__ void validate_m2_kernel(const float* __restrict__ x, long long n, unsigned long long* first_bad)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * n;
         i += (long long)gridDim.x * blockDim.x) {
        if (!isfinite(x[i])) atomicMin(first_bad, (unsigned long long)(i % n));
    }
}

// Build the tile records of one sample: F rows [K][S][E] (rotated event
// positions), then m2 [3][E], then w [E] (data only).  Events past n are zero.
__global__ void layout_kernel(const float2* __restrict__ F, const float* __restrict__ m2,
                              const float* __restrict__ w, long long n, int K, int S, int E, int ev,
                              long long ntiles, unsigned char* __restrict__ tiles, uint32_t tile_bytes,
                              int with_w)
{
    const long long per_tile_F = (long long)K * S * E;
    const int extra = (3 + with_w) * E;
    const long long per_tile = per_tile_F + extra;  // in 8-byte F slots + 4-byte scalars: handled apart
    const long long total_F = ntiles * per_tile_F;
    const long long total_x = ntiles * (long long)extra;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total_F + total_x;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < total_F) {
            // i enumerates (tile, k, s, p); the destination follows f_re
            const long long t = i / per_tile_F;
            const long long r = i % per_tile_F;
            const int k = (int)(r / ((long long)S * E));
            const int s = (int)((r / E) % S);
            const int p = (int)(r % E);
            const int el = (p - pwa::tile_shift(k, ev) + E) % E;
            const long long e = t * E + el;
            float2 val = make_float2(0.f, 0.f);
            if (e < n) val = F[(e * K + k) * S + s];
            float* Ft = reinterpret_cast<float*>(tiles + (size_t)t * tile_bytes);
            const int o = pwa::f_re(k, s, p, S, E);
            Ft[o] = val.x;
            Ft[o + pwa::f_im_off(S)] = val.y;
        } else {
            const long long j = i - total_F;
            const long long t = j / extra;
            const int r = (int)(j % extra);
            const int el = r % E;
            const int which = r / E;  // 0..2: m2 channel, 3: w
            const long long e = t * E + el;
            float val = 0.f;
            if (e < n) val = which < 3 ? m2[(size_t)which * n + e] : (w ? w[e] : 1.f);
            float* dst = reinterpret_cast<float*>(tiles + (size_t)t * tile_bytes + (size_t)per_tile_F * 8);
            dst[r] = val;
        }
    }
    (void)per_tile;
}

// I(e) for every event of one sample, read from the tile layout.
__global__ void intensity_kernel(pwa::PassArgs a, int smp, int S, float* __restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem_i[];
    pwa::KConst* kc = reinterpret_cast<pwa::KConst*>(smem_i);
    const int K = a.K, E = a.E;
    const int ev = 32 / a.W;
    for (int k = threadIdx.x; k < K; k += blockDim.x) kc[k] = pwa::make_kconst(a, a.theta, nullptr, k, false, ev);
    __syncthreads();
    const long long n = a.nev[smp];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long t = e / E;
        const int el = (int)(e % E);
        const unsigned char* rec = a.tiles[smp] + (size_t)t * a.tile_bytes[smp];
        const float2* Fs = reinterpret_cast<const float2*>(rec);
        const float* m2s = reinterpret_cast<const float*>(Fs + (size_t)K * S * E);
        float I = 0.f;
        for (int s = 0; s < S; ++s) {
            float Ar = 0.f, Ai = 0.f;
            for (int k = 0; k < K; ++k) {
                const pwa::KConst c = kc[k];
                float br, bi;
                pwa::breit_wigner(c, m2s[c.ch * E + el], br, bi);
                const float cr = c.gre * br - c.gim * bi, ci = c.gre * bi + c.gim * br;
                int p = el + c.shift;
                p = p >= E ? p - E : p;
                const int o = pwa::f_re(k, s, p, S, E);
                const float2 f = make_float2(reinterpret_cast<const float*>(Fs)[o],
                                             reinterpret_cast<const float*>(Fs)[o + pwa::f_im_off(S)]);
                Ar = fmaf(cr, f.x, fmaf(-ci, f.y, Ar));
                Ai = fmaf(cr, f.y, fmaf(ci, f.x, Ai));
            }
            I = fmaf(Ar, Ar, fmaf(Ai, Ai, I));
        }
        out[e] = I;
    }
}

// One block waits on an mbarrier that nothing completes, with the bounded
// wait of the streaming kernel; records whether the wait ran out.
__global__ void bounded_wait_kernel(long long budget, int* out)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        pwa::mbar_init(&bar, 1);
        pwa::fence_mbar_init();
    }
    __syncthreads();
    const bool done = pwa::mbar_wait(&bar, 0, budget);
    if (threadIdx.x == 0) *out = done ? 1 : 2;
}

// ---------------------------------------------------------------------------
// dispatch over the compile-time shapes (instances live in pass_*.cu)
// ---------------------------------------------------------------------------

using pwa::KernelFn;

KernelFn pick_kernel(int mode, int S, int W, int kpw)
{
#define PWA_PICK(m)                                       \
    switch (S) {                                          \
        case 1: return pwa::pick_pass_##m##_s1(W, kpw);   \
        case 2: return pwa::pick_pass_##m##_s2(W, kpw);   \
        case 3: return pwa::pick_pass_##m##_s3(W, kpw);   \
        case 4: return pwa::pick_pass_##m##_s4(W, kpw);   \
        default: return nullptr;                          \
    }
    switch (mode) {
        case pwa::MODE_NLL: PWA_PICK(nll)
        case pwa::MODE_GRAD: PWA_PICK(grad)
        case pwa::MODE_HVP: PWA_PICK(hvp)
        case pwa::MODE_HVP_REUSE: PWA_PICK(hvpr)
        default: return nullptr;
    }
#undef PWA_PICK
}

size_t smem_bytes(const Tiling& t, int K, int S)
{
    // stages | KConst[K] | per-warp (hi, lo) FP32 sums [W][10 K + 2] | stage counters[4] | issued[4] | mbarriers[NST]
    (void)S;
    return (size_t)t.NST * t.stage_bytes + (size_t)K * sizeof(pwa::KConst) +
           (size_t)t.W * (K * pwa::kNV + 2) * 8 + 16 + 32 + (size_t)t.NST * 8;
}

pwa_status alloc(pwa_handle* h, void** p, size_t bytes, const char* what)
{
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return pwa::set_error(h, PWA_ENOMEM, std::string("cudaMalloc failed for ") + what + ": " +
                                                 cudaGetErrorString(e));
    }
    return PWA_OK;
}

#define PWA_CUDA(h, call)                                              \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return pwa::cuda_error((h), e_, #call); \
    } while (0)

#define PWA_TRY(call)                  \
    do {                               \
        pwa_status s_ = (call);        \
        if (s_ != PWA_OK) return s_;   \
    } while (0)

// Fill t.E, t.H, t.KPW, stage bytes, smem and occupancy for (W, NST, bps).
pwa_status finish_tiling(pwa_handle* h, Tiling& t)
{
    const int K = h->K, S = h->S;
    if (!(t.W == 1 || t.W == 2 || t.W == 4 || t.W == 8))
        return pwa::set_error(h, PWA_EINVAL, "warps must be 1, 2, 4 or 8");
    if (t.NST < 2 || t.NST > 4) return pwa::set_error(h, PWA_EINVAL, "stages must be 2..4");
    t.E = pwa::kTileE;
    t.H = t.W;
    t.KPW = (K + t.W - 1) / t.W;
    if (t.KPW > 8) return pwa::set_error(h, PWA_EINVAL, "too many resonances per warp (K > 8 * warps)");
    const size_t rec_data = (size_t)t.E * (8ull * K * S + 16);
    t.stage_bytes = (uint32_t)((rec_data + 127) / 128 * 128);
    if (rec_data >= (1u << 20)) return pwa::set_error(h, PWA_EINVAL, "tile record too large");
    t.smem = smem_bytes(t, K, S);
    int dev = 0;
    PWA_CUDA(h, cudaGetDevice(&dev));
    int max_optin = 0;
    PWA_CUDA(h, cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    int occ = 1 << 30;
    for (int mode = 0; mode < 4; ++mode) {
        KernelFn f = pick_kernel(mode, S, t.W, t.KPW);
        if (!f) return pwa::set_error(h, PWA_EINVAL, "no compiled kernel for this S / warps / K combination");
        cudaFuncAttributes fa;
        PWA_CUDA(h, cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(f)));
        const int dyn_max = max_optin - (int)fa.sharedSizeBytes;
        if ((int)t.smem > dyn_max)
            return pwa::set_error(h, PWA_EINVAL, "tiling needs " + std::to_string(t.smem) +
                                                     " bytes of shared memory per block (max " +
                                                     std::to_string(dyn_max) + ")");
        // permit the largest size (another handle may launch the same instance
        // with a larger tiling); occupancy below uses this handle's size
        PWA_CUDA(h, cudaFuncSetAttribute(reinterpret_cast<const void*>(f),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
        int o = 0;
        PWA_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, reinterpret_cast<const void*>(f),
                                                                  32 * t.W, t.smem));
        occ = std::min(occ, o);
    }
    if (occ < 1) return pwa::set_error(h, PWA_EINVAL, "tiling does not fit on an SM");
    t.blocks_per_sm = t.bps > 0 ? std::min(t.bps, occ) : occ;
    return PWA_OK;
}

Tiling default_tiling(int K, int S)
{
    // The fewest warps per block whose second sweep leaves few resonance slots
    // idle (K close to W * KPW, KPW <= 8): small K runs one warp per event
    // (no cross-lane reduction in the first sweep), larger K splits each
    // event over W lanes.  Two stages; three when tile records are small.
    Tiling t;
    const int Ws[] = {1, 2, 4, 8};
    for (int W : Ws) {
        const int kpw = (K + W - 1) / W;
        if (kpw > 8) continue;
        t.W = W;
        if ((double)K / (W * kpw) >= 0.8) break;
    }
    const double rec = (double)pwa::kTileE * (8.0 * K * S + 16);
    t.NST = rec < 8 * 1024 ? 3 : 2;
    return t;
}

pwa_status build_tiles(pwa_handle* h)
{
    if (h->released)
        return pwa::set_error(h, PWA_EINVAL, "the events' caller-layout copies were released: the tiling is fixed");
    Tiling& t = h->tiling;
    PWA_TRY(finish_tiling(h, t));  // sets t.E first: everything below depends on it
    const int ev = 32 / t.W;
    for (int smp = 0; smp < 2; ++smp) {
        const int with_w = smp == 0;
        const size_t rec = (size_t)t.E * (8ull * h->K * h->S + 12 + 4 * with_w);
        h->tile_bytes[smp] = (uint32_t)rec;
        h->ntiles[smp] = (int)((h->n[smp] + t.E - 1) / t.E);
    }
    const long long T = (long long)h->ntiles[0] + h->ntiles[1];
    t.grid = (int)std::max(1LL, std::min((long long)h->num_sms * t.blocks_per_sm, T));
    for (int smp = 0; smp < 2; ++smp) {
        if (h->d_tiles[smp]) cudaFree(h->d_tiles[smp]);
        h->d_tiles[smp] = nullptr;
        PWA_TRY(alloc(h, reinterpret_cast<void**>(&h->d_tiles[smp]), (size_t)h->ntiles[smp] * h->tile_bytes[smp],
                      "event tiles"));
        const long long total = (long long)h->ntiles[smp] * t.E * (1ll * h->K * h->S + 3 + (smp == 0));
        const int blocks = (int)std::min<long long>((total + 255) / 256, 65535LL * 8);
        layout_kernel<<<blocks, 256, 0, h->stream>>>(reinterpret_cast<const float2*>(h->d_F[smp]), h->d_m2[smp],
                                                     smp == 0 ? h->d_w : nullptr, h->n[smp], h->K, h->S, t.E, ev,
                                                     h->ntiles[smp], h->d_tiles[smp], h->tile_bytes[smp],
                                                     smp == 0);
        PWA_CUDA(h, cudaGetLastError());
    }
    // reduction scratch sized for the grid
    if (h->d_block_rec) cudaFree(h->d_block_rec);
    if (h->d_group_rec) cudaFree(h->d_group_rec);
    if (h->d_counts) cudaFree(h->d_counts);
    h->d_block_rec = h->d_group_rec = nullptr;
    h->d_counts = nullptr;
    h->rec_len = 2 * (h->K * pwa::kNV + pwa::kNScal);
    h->ngroups = (t.grid + h->group_size - 1) / h->group_size;
    PWA_TRY(alloc(h, reinterpret_cast<void**>(&h->d_block_rec), sizeof(double) * (size_t)t.grid * h->rec_len,
                  "block partials"));
    PWA_TRY(alloc(h, reinterpret_cast<void**>(&h->d_group_rec), sizeof(double) * (size_t)h->ngroups * h->rec_len,
                  "group partials"));
    if (!h->d_cache) {
        // the reused totals; theta NaN until the first full HVP pass (no reuse can match it)
        PWA_TRY(alloc(h, reinterpret_cast<void**>(&h->d_cache), sizeof(double) * ((size_t)h->rec_len + h->P),
                      "H v reuse cache"));
        PWA_CUDA(h, cudaMemsetAsync(h->d_cache, 0xFF, sizeof(double) * ((size_t)h->rec_len + h->P), h->stream));
    }
    PWA_TRY(alloc(h, reinterpret_cast<void**>(&h->d_counts), sizeof(unsigned) * (h->ngroups + 1), "counters"));
    PWA_CUDA(h, cudaMemsetAsync(h->d_counts, 0, sizeof(unsigned) * (h->ngroups + 1), h->stream));
    PWA_CUDA(h, cudaStreamSynchronize(h->stream));
    return PWA_OK;
}

pwa::PassArgs make_args(pwa_handle* h, const double* d_theta, const double* d_v, double* d_out)
{
    const Tiling& t = h->tiling;
    pwa::PassArgs a;
    for (int s = 0; s < 2; ++s) {
        a.tiles[s] = h->d_tiles[s];
        a.tile_bytes[s] = h->tile_bytes[s];
        a.ntiles[s] = h->ntiles[s];
        a.nev[s] = h->n[s];
    }
    a.K = h->K;
    a.E = t.E;
    a.H = t.H;
    a.W = t.W;
    a.NST = t.NST;
    a.stage_bytes = t.stage_bytes;
    a.ev = 32 / t.W;
    a.S = h->S;
    a.P = h->P;
    a.res = h->d_res;
    a.theta = d_theta;
    a.v = d_v;
    a.Nd = h->Nd;
    a.Nmc = h->Nmc;
    a.B = 1;
    a.Gb = t.grid;
    a.block_rec = h->d_block_rec;
    a.group_rec = h->d_group_rec;
    a.group_count = h->d_counts;
    a.top_count = h->d_counts + h->ngroups;
    a.group_size = h->group_size;
    a.ngroups = h->ngroups;
    a.rec_len = h->rec_len;
    a.out = d_out;
    a.bad = h->d_bad;
    a.err = h->d_err;
    a.timeout_cycles = h->timeout_cycles;
    return a;
}

// Copy an ABI event array to the device (from host or device memory).
pwa_status upload(pwa_handle* h, float** dst, const float* src, size_t count, int on_device, const char* what)
{
    PWA_TRY(alloc(h, reinterpret_cast<void**>(dst), count * sizeof(float), what));
    PWA_CUDA(h, cudaMemcpyAsync(*dst, src, count * sizeof(float),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    return PWA_OK;
}

pwa_status validate_sample(pwa_handle* h, int smp, const char* name)
{
    const long long n = h->n[smp];
    const int per_ev = h->K * h->S * 2;
    unsigned long long* d_first = h->d_bad;
    unsigned long long first = ~0ull;
    const char* what[3] = {"F", "m2", "w"};
    for (int which = 0; which < 3; ++which) {
        if (which == 2 && (smp != 0 || !h->d_w)) continue;
        PWA_CUDA(h, cudaMemsetAsync(d_first, 0xFF, sizeof(unsigned long long), h->stream));
        if (which == 0)
            validate_kernel<<<1024, 256, 0, h->stream>>>(h->d_F[smp], n * per_ev, per_ev, 0, d_first);
        else if (which == 1)
            validate_m2_kernel<<<1024, 256, 0, h->stream>>>(h->d_m2[smp], n, d_first);
        else
            validate_kernel<<<1024, 256, 0, h->stream>>>(h->d_w, n, 1, 1, d_first);
        PWA_CUDA(h, cudaGetLastError());
        PWA_CUDA(h, cudaMemcpyAsync(&first, d_first, sizeof(first), cudaMemcpyDeviceToHost, h->stream));
        PWA_CUDA(h, cudaStreamSynchronize(h->stream));
        if (first != ~0ull)
            return pwa::set_error(h, PWA_EINVAL, std::string(name) + " event " + std::to_string(first) +
                                                     " has a non-finite " + what[which] +
                                                     (which == 2 ? " or negative weight" : ""));
    }
    return PWA_OK;
}

pwa_status create_impl(pwa_handle* h, const pwa_events* data, const pwa_events* mc, const pwa_resonance* table,
                       int K, int S)
{
    if (!data || !mc || !table) return pwa::set_error(h, PWA_EINVAL, "data, mc and table must not be NULL");
    if (K < 1 || K > 128) return pwa::set_error(h, PWA_EINVAL, "K must be in 1..128");
    if (S < 1 || S > 4) return pwa::set_error(h, PWA_EINVAL, "S must be in 1..4");
    if (data->n < 1 || mc->n < 1) return pwa::set_error(h, PWA_EINVAL, "both samples need at least one event");
    if (!data->m2 || !data->F || !mc->m2 || !mc->F) return pwa::set_error(h, PWA_EINVAL, "NULL event array");
    if (mc->w) return pwa::set_error(h, PWA_EINVAL, "the MC sample takes no weights (w must be NULL)");
    h->K = K;
    h->S = S;
    h->n[0] = data->n;
    h->n[1] = mc->n;
    // parameter map
    int P = 0;
    h->res.assign(K, ResParam{});
    for (int k = 0; k < K; ++k) {
        const pwa_resonance& r = table[k];
        if (r.channel < 0 || r.channel > 2) return pwa::set_error(h, PWA_EINVAL, "channel must be 0, 1 or 2");
        if (!(std::isfinite(r.mass) && r.mass > 0 && std::isfinite(r.width) && r.width > 0 &&
              std::isfinite(r.mag) && std::isfinite(r.phase)))
            return pwa::set_error(h, PWA_EINVAL, "resonance " + std::to_string(k) +
                                                     ": mass and width must be finite and positive, mag and "
                                                     "phase finite");
        ResParam& p = h->res[k];
        p.channel = r.channel;
        p.fixed[0] = r.mag;
        p.fixed[1] = r.phase;
        p.fixed[2] = r.mass;
        p.fixed[3] = r.width;
        for (int j = 0; j < 4; ++j) p.idx[j] = -1;
    }
    for (int k = 0; k < K; ++k)
        if (!table[k].fix_coupling) h->res[k].idx[0] = P++;
    for (int k = 0; k < K; ++k)
        if (!table[k].fix_coupling) h->res[k].idx[1] = P++;
    for (int k = 0; k < K; ++k)
        if (!table[k].fix_mass) h->res[k].idx[2] = P++;
    for (int k = 0; k < K; ++k)
        if (!table[k].fix_width) h->res[k].idx[3] = P++;
    h->P = P;

    int dev = 0;
    PWA_CUDA(h, cudaGetDevice(&dev));
    PWA_CUDA(h, cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
    int clock_khz = 0;
    if (cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev) != cudaSuccess || clock_khz <= 0) {
        cudaGetLastError();
        clock_khz = 2000000;
    }
    h->timeout_cycles = (long long)clock_khz * 1000LL * 2;  // about two seconds of SM clock

    PWA_TRY(alloc(h, reinterpret_cast<void**>(&h->d_res), sizeof(ResParam) * K, "parameter map"));
    PWA_CUDA(h, cudaMemcpyAsync(h->d_res, h->res.data(), sizeof(ResParam) * K, cudaMemcpyHostToDevice, h->stream));
    // one device block for a call's inputs and results, so that a host call
    // needs one copy each way: theta[P] | v[P] | err (8 B) | bad (8 B) | out[1 + 2P]
    PWA_TRY(alloc(h, reinterpret_cast<void**>(&h->d_theta), sizeof(double) * (2 * (size_t)P + 3 + 2 * P),
                  "call buffers"));
    h->d_v = h->d_theta + P;
    h->d_err = reinterpret_cast<int*>(h->d_theta + 2 * P);
    h->d_bad = reinterpret_cast<unsigned long long*>(h->d_theta + 2 * P + 1);
    h->d_out = h->d_theta + 2 * P + 2;
    PWA_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(double), h->stream));
    if (cudaMallocHost(reinterpret_cast<void**>(&h->h_pin), sizeof(double) * (8 + 4 * P)) != cudaSuccess) {
        cudaGetLastError();
        return pwa::set_error(h, PWA_ENOMEM, "pinned host allocation failed");
    }

    const pwa_events* ev[2] = {data, mc};
    for (int smp = 0; smp < 2; ++smp) {
        const long long n = h->n[smp];
        PWA_TRY(upload(h, &h->d_F[smp], ev[smp]->F, (size_t)n * K * S * 2, ev[smp]->on_device, "F"));
        PWA_TRY(upload(h, &h->d_m2[smp], ev[smp]->m2, (size_t)n * 3, ev[smp]->on_device, "m2"));
    }
    if (data->w) PWA_TRY(upload(h, &h->d_w, data->w, (size_t)data->n, data->on_device, "w"));
    PWA_TRY(validate_sample(h, 0, "data"));
    PWA_TRY(validate_sample(h, 1, "MC"));
    PWA_CUDA(h, cudaMemsetAsync(h->d_bad, 0xFF, sizeof(unsigned long long), h->stream));

    // N_d = sum of the data weights (Eq. 3), in FP64 on the host
    if (h->d_w) {
        std::vector<float> w((size_t)data->n);
        PWA_CUDA(h, cudaMemcpyAsync(w.data(), h->d_w, sizeof(float) * w.size(), cudaMemcpyDeviceToHost, h->stream));
        PWA_CUDA(h, cudaStreamSynchronize(h->stream));
        double s = 0.0;
        for (float x : w) s += (double)x;
        h->Nd = s;
        if (!(s > 0)) return pwa::set_error(h, PWA_EINVAL, "the data weights sum to zero");
    } else {
        h->Nd = (double)data->n;
    }
    h->Nmc = (double)mc->n;

    h->tiling = default_tiling(K, S);
    PWA_TRY(build_tiles(h));
    return PWA_OK;
}

}  // namespace

namespace pwa {

pwa_status set_error(pwa_handle* h, pwa_status st, const std::string& msg)
{
    if (h) h->err = msg;
    return st;
}

pwa_status cuda_error(pwa_handle* h, cudaError_t e, const char* what)
{
    cudaGetLastError();
    return set_error(h, PWA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

PassArgs pass_args(pwa_handle* h, const double* d_theta, const double* d_v, double* d_out)
{
    return make_args(h, d_theta, d_v, d_out);
}

pwa_status launch_pass_args(pwa_handle* h, const PassArgs& a, int mode)
{
    if (h->broken) return set_error(h, PWA_ETIMEOUT, "handle is unusable after a device-side timeout");
    KernelFn fn = pick_kernel(mode, h->S, h->tiling.W, h->tiling.KPW);
    if (!fn) return set_error(h, PWA_EINVAL, "no kernel for this shape");
    // the geometry the kernel relies on: every tile record fits a stage and
    // the tiles cover every event
    const Tiling& t = h->tiling;
    for (int s = 0; s < 2; ++s)
        if (h->tile_bytes[s] > t.stage_bytes || (long long)h->ntiles[s] * t.E < h->n[s] ||
            h->tile_bytes[s] % 16 != 0)
            return set_error(h, PWA_EINVAL, "inconsistent tile geometry");
    fn<<<h->tiling.grid, 32 * h->tiling.W, h->tiling.smem, h->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(h, e, "pass kernel launch");
    return PWA_OK;
}

pwa_status launch_pass(pwa_handle* h, const double* d_theta, const double* d_v, double* d_out, int mode,
                       const int* skip)
{
    PassArgs a = make_args(h, d_theta, d_v, d_out);
    a.skip = skip;
    if (mode == MODE_HVP || mode == MODE_HVP_REUSE) a.cache = h->d_cache;
    return launch_pass_args(h, a, mode);
}

// ---- batched evaluation: B parameter vectors share one launch ----
//
// Block i of the launch works for vector i % B and is block i / B of the Gb
// blocks that split the events for that vector, so neighbouring blocks stream
// the same tiles (the second and later reads hit L2).  Each vector has its own
// block records, groups and counters; its totals and results are those of a
// single-vector pass over a grid of Gb blocks.

namespace {

void batch_geometry(const pwa_handle* h, int B, int& Gb, int& ngroups)
{
    const long long T = (long long)h->ntiles[0] + h->ntiles[1];
    const long long want = ((long long)h->tiling.grid + B - 1) / B;
    Gb = (int)std::max(1LL, std::min(want, T));
    ngroups = (Gb + h->group_size - 1) / h->group_size;
}

}  // namespace

pwa_status batch_io(pwa_handle* h, int B)
{
    BatchState& bs = h->batch;
    if (B <= bs.cap_B) return PWA_OK;
    if (bs.d_io) cudaFree(bs.d_io);
    if (bs.h_io) cudaFreeHost(bs.h_io);
    bs.d_io = nullptr;
    bs.h_io = nullptr;
    bs.cap_B = 0;
    const size_t words = (size_t)B * (4 * (size_t)h->P + 1);
    PWA_TRY(alloc(h, reinterpret_cast<void**>(&bs.d_io), sizeof(double) * words, "batch vectors"));
    // pinned staging: the same layout, then B + 1 error words (B + 2 doubles of room)
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&bs.h_io), sizeof(double) * (words + B + 2));
    if (e != cudaSuccess) {
        bs.h_io = nullptr;
        return cuda_error(h, e, "cudaMallocHost(batch staging)");
    }
    bs.cap_B = B;
    return PWA_OK;
}

size_t pass_smem_bytes(const pwa_handle* h, int W)
{
    Tiling t = h->tiling;
    t.W = W;
    return smem_bytes(t, h->K, h->S);
}

pwa_status prepare_batch(pwa_handle* h, int B, const double* d_theta, const double* d_v, double* d_out,
                         bool err_vec, cudaStream_t stream, PassArgs& a)
{
    if (h->broken) return set_error(h, PWA_ETIMEOUT, "handle is unusable after a device-side timeout");
    if (B < 1) return set_error(h, PWA_EINVAL, "the batch needs at least one parameter vector");
    int Gb = 0, ngroups = 0;
    batch_geometry(h, B, Gb, ngroups);
    if ((long long)B * Gb > 0x7fffffffLL) return set_error(h, PWA_EINVAL, "batch too large for one launch");
    BatchState& bs = h->batch;
    const size_t blocks = (size_t)B * Gb, groups = (size_t)B * ngroups;
    if (blocks > bs.cap_blocks || groups > bs.cap_groups || (size_t)B > bs.cap_top) {
        // grow the scratch (block records, group records, counters); the
        // counters start at zero and every completed pass leaves them at zero
        PWA_CUDA(h, cudaStreamSynchronize(h->stream));
        PWA_CUDA(h, cudaStreamSynchronize(stream));
        if (bs.d_block_rec) cudaFree(bs.d_block_rec);
        if (bs.d_group_rec) cudaFree(bs.d_group_rec);
        if (bs.d_counts) cudaFree(bs.d_counts);
        bs.d_block_rec = bs.d_group_rec = nullptr;
        bs.d_counts = nullptr;
        bs.cap_blocks = bs.cap_groups = bs.cap_top = 0;
        const size_t cb = std::max(blocks, (size_t)h->tiling.grid), cg = std::max(groups, (size_t)h->ngroups);
        const size_t ct = std::max<size_t>(B, 64);
        PWA_TRY(alloc(h, reinterpret_cast<void**>(&bs.d_block_rec), sizeof(double) * cb * h->rec_len,
                      "batch block partials"));
        PWA_TRY(alloc(h, reinterpret_cast<void**>(&bs.d_group_rec), sizeof(double) * cg * h->rec_len,
                      "batch group partials"));
        PWA_TRY(alloc(h, reinterpret_cast<void**>(&bs.d_counts), sizeof(unsigned) * (cg + 2 * ct), "batch counters"));
        PWA_CUDA(h, cudaMemsetAsync(bs.d_counts, 0, sizeof(unsigned) * (cg + 2 * ct), stream));
        bs.d_err_vec = reinterpret_cast<int*>(bs.d_counts + cg + ct);
        bs.cap_blocks = cb;
        bs.cap_groups = cg;
        bs.cap_top = ct;
    }
    a = make_args(h, d_theta, d_v, d_out);
    a.B = B;
    a.Gb = Gb;
    a.block_rec = bs.d_block_rec;
    a.group_rec = bs.d_group_rec;
    a.group_count = bs.d_counts;
    a.top_count = bs.d_counts + bs.cap_groups;
    a.ngroups = ngroups;
    if (err_vec) {
        PWA_CUDA(h, cudaMemsetAsync(bs.d_err_vec, 0, sizeof(int) * B, stream));
        a.err_vec = bs.d_err_vec;
    }
    return PWA_OK;
}

pwa_status launch_batch(pwa_handle* h, int B, const double* d_theta, const double* d_v, double* d_out, int mode,
                        bool err_vec)
{
    KernelFn fn = pick_kernel(mode, h->S, h->tiling.W, h->tiling.KPW);
    if (!fn) return set_error(h, PWA_EINVAL, "no kernel for this shape");
    PassArgs a;
    PWA_TRY(prepare_batch(h, B, d_theta, d_v, d_out, err_vec, h->stream, a));
    const size_t blocks = (size_t)B * a.Gb;
    fn<<<(unsigned)blocks, 32 * h->tiling.W, h->tiling.smem, h->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(h, e, "batched pass kernel launch");
    return PWA_OK;
}

void free_batch(pwa_handle* h)
{
    BatchState& bs = h->batch;
    void* ptrs[] = {bs.d_block_rec, bs.d_group_rec, bs.d_counts, bs.d_io};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (bs.h_io) cudaFreeHost(bs.h_io);
    bs = BatchState();
}

pwa_status check_device_errors(pwa_handle* h)
{
    int err = 0;
    unsigned long long bad = 0;
    PWA_CUDA(h, cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    PWA_CUDA(h, cudaMemcpyAsync(&bad, h->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
    PWA_CUDA(h, cudaStreamSynchronize(h->stream));
    if (!err) return PWA_OK;
    PWA_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
    PWA_CUDA(h, cudaMemsetAsync(h->d_bad, 0xFF, sizeof(unsigned long long), h->stream));
    PWA_CUDA(h, cudaStreamSynchronize(h->stream));
    if (err & ERR_TIMEOUT) {
        h->broken = true;
        return set_error(h, PWA_ETIMEOUT, "a tile copy did not arrive within the wait limit");
    }
    if (err & ERR_STALE)
        return set_error(h, PWA_EINVAL, "H v reuse: the last full H v pass was not at this theta");
    return set_error(h, PWA_ENONFINITE, "event " + std::to_string(bad) +
                                            " has a non-finite intensity (or a non-positive one for data)");
}

}  // namespace pwa

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

pwa_status pwa_create(pwa_handle** out, const pwa_events* data, const pwa_events* mc, const pwa_resonance* table,
                      int K, int S, void* cuda_stream)
{
    g_create_error.clear();
    if (!out) {
        g_create_error = "out must not be NULL";
        return PWA_EINVAL;
    }
    *out = nullptr;
    pwa_handle* h = new (std::nothrow) pwa_handle();
    if (!h) {
        g_create_error = "host allocation failed";
        return PWA_ENOMEM;
    }
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    pwa_status st;
    try {
        st = create_impl(h, data, mc, table, K, S);
    } catch (...) {
        st = pwa::set_error(h, PWA_ENOMEM, "host exception during create");
    }
    if (st != PWA_OK) {
        g_create_error = h->err;
        pwa_destroy(h);
        return st;
    }
    *out = h;
    return PWA_OK;
}

const char* pwa_last_create_error(void) { return g_create_error.c_str(); }

pwa_status pwa_release_event_copies(pwa_handle* h)
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    if (h->released) return PWA_OK;
    PWA_CUDA(h, h->stream ? cudaStreamSynchronize(h->stream) : cudaDeviceSynchronize());
    float* ptrs[] = {h->d_F[0], h->d_F[1], h->d_m2[0], h->d_m2[1], h->d_w};
    for (float* p : ptrs)
        if (p) cudaFree(p);
    h->d_F[0] = h->d_F[1] = h->d_m2[0] = h->d_m2[1] = h->d_w = nullptr;
    h->released = true;
    PWA_CUDA(h, cudaGetLastError());
    return PWA_OK;
}

pwa_status pwa_device_bytes(const pwa_handle* h, long long* out)
{
    if (!h || !out) return PWA_EINVAL;
    long long b = 0;
    const long long n0 = h->n[0], n1 = h->n[1], KS = (long long)h->K * h->S;
    if (!h->released) b += (n0 + n1) * (8 * KS + 12) + (h->d_w ? 4 * n0 : 0);
    b += (long long)h->ntiles[0] * h->tile_bytes[0] + (long long)h->ntiles[1] * h->tile_bytes[1];
    b += 8LL * ((long long)h->tiling.grid + h->ngroups) * h->rec_len + 4LL * (h->ngroups + 1);
    b += 8LL * (4 * (long long)h->P + 3) + (long long)sizeof(pwa::ResParam) * h->K;
    b += (long long)h->hess.cap_bytes;
    const pwa::BatchState& bs = h->batch;
    b += 8LL * (long long)(bs.cap_blocks + bs.cap_groups) * h->rec_len + 4LL * (long long)(bs.cap_groups + 2 * bs.cap_top);
    b += 8LL * (long long)bs.cap_B * (2 * (long long)h->P + 1 + 2 * (long long)h->P);
    *out = b;
    return PWA_OK;
}

int pwa_num_params(const pwa_handle* h) { return h ? h->P : -1; }

namespace {
pwa_status eval_impl(pwa_handle* h, const double* theta, const double* v, double* nll, double* grad, double* hv,
                     bool reuse)
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    if (!theta || !nll) return pwa::set_error(h, PWA_EINVAL, "theta and nll must not be NULL");
    if (hv && !v) return pwa::set_error(h, PWA_EINVAL, "v is required for hv");
    const int P = h->P;
    for (int i = 0; i < P; ++i)
        if (!std::isfinite(theta[i]) || (hv && !std::isfinite(v[i])))
            return pwa::set_error(h, PWA_EINVAL, "theta and v must be finite");
    const int mode = hv ? (reuse ? pwa::MODE_HVP_REUSE : pwa::MODE_HVP) : (grad ? pwa::MODE_GRAD : pwa::MODE_NLL);
    double* pin = h->h_pin;
    std::memcpy(pin, theta, sizeof(double) * P);
    if (hv) std::memcpy(pin + P, v, sizeof(double) * P);
    PWA_CUDA(h, cudaMemcpyAsync(h->d_theta, pin, sizeof(double) * (hv ? 2 * P : P), cudaMemcpyHostToDevice,
                                h->stream));
    PWA_TRY(pwa::launch_pass(h, h->d_theta, hv ? h->d_v : nullptr, h->d_out, mode));
    // error word, first bad event and the results in one copy
    double* st = pin + 2 * P;
    PWA_CUDA(h, cudaMemcpyAsync(st, h->d_err, sizeof(double) * (3 + 2 * P), cudaMemcpyDeviceToHost, h->stream));
    PWA_CUDA(h, cudaStreamSynchronize(h->stream));
    int err_word = 0;
    std::memcpy(&err_word, st, sizeof(int));
    if (err_word) PWA_TRY(pwa::check_device_errors(h));
    const double* res = st + 2;
    *nll = res[0];
    if (grad) std::memcpy(grad, res + 1, sizeof(double) * P);
    if (hv) std::memcpy(hv, res + 1 + P, sizeof(double) * P);
    return PWA_OK;
}
}  // namespace

pwa_status pwa_eval(pwa_handle* h, const double* theta, const double* v, double* nll, double* grad, double* hv)
{
    return eval_impl(h, theta, v, nll, grad, hv, false);
}

pwa_status pwa_hvp_reuse(pwa_handle* h, const double* theta, const double* v, double* hv)
{
    if (!hv) return h ? pwa::set_error(h, PWA_EINVAL, "hv must not be NULL") : PWA_EINVAL;
    double nll = 0.0;
    return eval_impl(h, theta, v, &nll, nullptr, hv, true);
}

pwa_status pwa_hvp_reuse_device(pwa_handle* h, const double* d_theta, const double* d_v, double* d_out)
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    if (!d_theta || !d_v || !d_out) return pwa::set_error(h, PWA_EINVAL, "d_theta, d_v and d_out must not be NULL");
    return pwa::launch_pass(h, d_theta, d_v, d_out, pwa::MODE_HVP_REUSE);
}

pwa_status pwa_nll(pwa_handle* h, const double* theta, double* nll)
{
    return pwa_eval(h, theta, nullptr, nll, nullptr, nullptr);
}

pwa_status pwa_grad(pwa_handle* h, const double* theta, double* nll_or_null, double* grad)
{
    if (!h) return PWA_EINVAL;
    if (!grad) return pwa::set_error(h, PWA_EINVAL, "grad must not be NULL");
    double f = 0.0;
    pwa_status st = pwa_eval(h, theta, nullptr, &f, grad, nullptr);
    if (st == PWA_OK && nll_or_null) *nll_or_null = f;
    return st;
}

pwa_status pwa_hvp(pwa_handle* h, const double* theta, const double* v, double* hv)
{
    if (!h) return PWA_EINVAL;
    if (!hv || !v) return pwa::set_error(h, PWA_EINVAL, "v and hv must not be NULL");
    double f = 0.0;
    std::vector<double> g(h->P);
    return pwa_eval(h, theta, v, &f, g.data(), hv);
}

pwa_status pwa_eval_device(pwa_handle* h, const double* d_theta, const double* d_v, double* d_out, int want_grad,
                           int want_hv)
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    if (!d_theta || !d_out || (want_hv && !d_v))
        return pwa::set_error(h, PWA_EINVAL, "d_theta, d_out (and d_v for hv) must not be NULL");
    const int mode = want_hv ? pwa::MODE_HVP : (want_grad ? pwa::MODE_GRAD : pwa::MODE_NLL);
    return pwa::launch_pass(h, d_theta, want_hv ? d_v : nullptr, d_out, mode);
}

pwa_status pwa_eval_batch_device(pwa_handle* h, int B, const double* d_theta, const double* d_v, double* d_out,
                                 int want_grad, int want_hv)
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    if (B < 1) return pwa::set_error(h, PWA_EINVAL, "B must be at least 1");
    if (!d_theta || !d_out || (want_hv && !d_v))
        return pwa::set_error(h, PWA_EINVAL, "d_theta, d_out (and d_v for hv) must not be NULL");
    const int mode = want_hv ? pwa::MODE_HVP : (want_grad ? pwa::MODE_GRAD : pwa::MODE_NLL);
    return pwa::launch_batch(h, B, d_theta, want_hv ? d_v : nullptr, d_out, mode);
}

pwa_status pwa_eval_batch(pwa_handle* h, int B, const double* theta, const double* v, double* nll, double* grad,
                          double* hv)
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    if (B < 1) return pwa::set_error(h, PWA_EINVAL, "B must be at least 1");
    if (!theta || !nll) return pwa::set_error(h, PWA_EINVAL, "theta and nll must not be NULL");
    if (hv && !v) return pwa::set_error(h, PWA_EINVAL, "v is required for hv");
    const int P = h->P;
    const size_t BP = (size_t)B * P;
    for (size_t i = 0; i < BP; ++i)
        if (!std::isfinite(theta[i]) || (hv && !std::isfinite(v[i])))
            return pwa::set_error(h, PWA_EINVAL, "theta and v must be finite");
    PWA_TRY(pwa::batch_io(h, B));
    pwa::BatchState& bs = h->batch;
    // staging: theta [B][P] then v [B][P]; results [B][1 + 2P]; then the error word
    double* pin = bs.h_io;
    std::memcpy(pin, theta, sizeof(double) * BP);
    if (hv) std::memcpy(pin + BP, v, sizeof(double) * BP);
    double* d_th = bs.d_io;
    double* d_v = bs.d_io + BP;
    double* d_out = bs.d_io + 2 * BP;
    PWA_CUDA(h, cudaMemcpyAsync(d_th, pin, sizeof(double) * (hv ? 2 * BP : BP), cudaMemcpyHostToDevice, h->stream));
    const int mode = hv ? pwa::MODE_HVP : (grad ? pwa::MODE_GRAD : pwa::MODE_NLL);
    PWA_TRY(pwa::launch_batch(h, B, d_th, hv ? d_v : nullptr, d_out, mode));
    const size_t ow = (size_t)B * (1 + 2 * (size_t)P);
    double* res = pin + 2 * BP;
    double* st = pin + 2 * BP + ow;
    PWA_CUDA(h, cudaMemcpyAsync(res, d_out, sizeof(double) * ow, cudaMemcpyDeviceToHost, h->stream));
    PWA_CUDA(h, cudaMemcpyAsync(st, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    PWA_CUDA(h, cudaStreamSynchronize(h->stream));
    int err_word = 0;
    std::memcpy(&err_word, st, sizeof(int));
    if (err_word) PWA_TRY(pwa::check_device_errors(h));
    for (int b = 0; b < B; ++b) {
        const double* r = res + (size_t)b * (1 + 2 * P);
        nll[b] = r[0];
        if (grad) std::memcpy(grad + (size_t)b * P, r + 1, sizeof(double) * P);
        if (hv) std::memcpy(hv + (size_t)b * P, r + 1 + P, sizeof(double) * P);
    }
    return PWA_OK;
}

pwa_status pwa_sync(pwa_handle* h)
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    return pwa::check_device_errors(h);
}

pwa_status pwa_event_intensity(pwa_handle* h, int sample, const double* theta, float* out, int out_on_device)
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    if (sample != 0 && sample != 1) return pwa::set_error(h, PWA_EINVAL, "sample must be 0 (data) or 1 (MC)");
    if (!theta || !out) return pwa::set_error(h, PWA_EINVAL, "theta and out must not be NULL");
    const int P = h->P;
    std::memcpy(h->h_pin, theta, sizeof(double) * P);
    PWA_CUDA(h, cudaMemcpyAsync(h->d_theta, h->h_pin, sizeof(double) * P, cudaMemcpyHostToDevice, h->stream));
    const long long n = h->n[sample];
    float* dst = out;
    float* tmp = nullptr;
    if (!out_on_device) {
        PWA_TRY(alloc(h, reinterpret_cast<void**>(&tmp), sizeof(float) * n, "intensity output"));
        dst = tmp;
    }
    pwa::PassArgs a = make_args(h, h->d_theta, nullptr, h->d_out);
    const int blocks = (int)std::min<long long>((n + 255) / 256, (long long)h->num_sms * 8);
    intensity_kernel<<<blocks, 256, sizeof(pwa::KConst) * h->K, h->stream>>>(a, sample, h->S, dst);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && tmp)
        e = cudaMemcpyAsync(out, tmp, sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return pwa::cuda_error(h, e, "event intensity");
    return PWA_OK;
}

pwa_status pwa_set_stream(pwa_handle* h, void* cuda_stream)
{
    if (!h) return PWA_EINVAL;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    return PWA_OK;
}

pwa_status pwa_set_tiling(pwa_handle* h, int warps, int stages, int blocks_per_sm)
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    if (h->released)  // the tiling stays (re-tiling needs the released copies)
        return pwa::set_error(h, PWA_EINVAL, "the events' caller-layout copies were released: the tiling is fixed");
    Tiling t;
    t.W = warps;
    t.NST = stages;
    t.bps = blocks_per_sm;
    const Tiling old = h->tiling;
    h->tiling = t;
    pwa_status st = build_tiles(h);
    if (st != PWA_OK) {
        std::string msg = h->err;
        h->tiling = old;
        if (build_tiles(h) != PWA_OK) h->broken = true;
        h->err = msg;
    }
    return st;
}

pwa_status pwa_autotune(pwa_handle* h, const double* theta, int B, int out3[3])
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    if (!theta || B < 1) return pwa::set_error(h, PWA_EINVAL, "theta must not be NULL and B >= 1");
    if (h->released)
        return pwa::set_error(h, PWA_EINVAL, "the events' caller-layout copies were released: the tiling is fixed");
    const int P = h->P;
    for (int i = 0; i < P; ++i)
        if (!std::isfinite(theta[i])) return pwa::set_error(h, PWA_EINVAL, "theta must be finite");
    // B copies of theta and a fixed direction as the timed batch
    PWA_TRY(pwa::batch_io(h, B));
    pwa::BatchState& bs = h->batch;
    const size_t BP = (size_t)B * P;
    for (int b = 0; b < B; ++b) {
        std::memcpy(bs.h_io + (size_t)b * P, theta, sizeof(double) * P);
        for (int i = 0; i < P; ++i) bs.h_io[BP + (size_t)b * P + i] = 1.0 / std::sqrt((double)P);
    }
    PWA_CUDA(h, cudaMemcpyAsync(bs.d_io, bs.h_io, sizeof(double) * 2 * BP, cudaMemcpyHostToDevice, h->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PWA_CUDA(h, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return pwa::cuda_error(h, cudaGetLastError(), "cudaEventCreate");
    }
    struct Events {
        cudaEvent_t a, b;
        ~Events()
        {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } ev{e0, e1};
    const Tiling start = h->tiling;
    Tiling best = start;
    float best_ms = INFINITY;
    const int Ws[] = {1, 2, 4, 8};
    for (int W : Ws) {
        if ((h->K + W - 1) / W > 8) continue;
        for (int NST = 2; NST <= 3; ++NST) {
            for (int half = 0; half < 2; ++half) {
                // all blocks per SM the tiling allows, then half as many
                if (pwa_set_tiling(h, W, NST, 0) != PWA_OK) {
                    h->err.clear();
                    continue;
                }
                if (half) {
                    const int bps = std::max(1, h->tiling.blocks_per_sm / 2);
                    if (bps == h->tiling.blocks_per_sm || pwa_set_tiling(h, W, NST, bps) != PWA_OK) {
                        h->err.clear();
                        continue;
                    }
                }
                double* d_th = bs.d_io;
                double* d_v = bs.d_io + BP;
                double* d_out = bs.d_io + 2 * BP;
                pwa_status st = PWA_OK;
                for (int r = 0; r < 2 && st == PWA_OK; ++r)
                    st = pwa::launch_batch(h, B, d_th, d_v, d_out, pwa::MODE_HVP);
                PWA_CUDA(h, cudaEventRecord(e0, h->stream));
                constexpr int kReps = 5;
                for (int r = 0; r < kReps && st == PWA_OK; ++r)
                    st = pwa::launch_batch(h, B, d_th, d_v, d_out, pwa::MODE_HVP);
                PWA_CUDA(h, cudaEventRecord(e1, h->stream));
                PWA_CUDA(h, cudaEventSynchronize(e1));
                if (st != PWA_OK) return st;
                PWA_TRY(pwa::check_device_errors(h));
                float ms = 0.f;
                PWA_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best_ms) {
                    best_ms = ms;
                    best = h->tiling;
                }
            }
        }
    }
    PWA_TRY(pwa_set_tiling(h, best.W, best.NST, best.blocks_per_sm));
    if (out3) {
        out3[0] = h->tiling.W;
        out3[1] = h->tiling.NST;
        out3[2] = h->tiling.blocks_per_sm;
    }
    return PWA_OK;
}

pwa_status pwa_get_tiling(const pwa_handle* h, int out6[6])
{
    if (!h || !out6) return PWA_EINVAL;
    out6[0] = h->tiling.W;
    out6[1] = h->tiling.NST;
    out6[2] = h->tiling.blocks_per_sm;
    out6[3] = h->tiling.E;
    out6[4] = h->tiling.grid;
    out6[5] = (int)h->tiling.smem;
    return PWA_OK;
}

pwa_status pwa_selftest_bounded_wait(double seconds)
{
    if (!(seconds > 0 && seconds <= 10)) return PWA_EINVAL;
    int dev = 0, clock_khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev) != cudaSuccess || clock_khz <= 0) {
        cudaGetLastError();
        return PWA_ECUDA;
    }
    int* d_out = nullptr;
    if (cudaMalloc(&d_out, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return PWA_ENOMEM;
    }
    int h_out = 0;
    cudaError_t e = cudaMemset(d_out, 0, sizeof(int));
    if (e == cudaSuccess) {
        bounded_wait_kernel<<<1, 32>>>((long long)(seconds * clock_khz * 1000.0), d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h_out, d_out, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d_out);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PWA_ECUDA;
    }
    return h_out == 2 ? PWA_ETIMEOUT : (h_out == 1 ? PWA_OK : PWA_ECUDA);
}

const char* pwa_last_error(const pwa_handle* h) { return h ? h->err.c_str() : "NULL handle"; }

void pwa_destroy(pwa_handle* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    // d_v, d_err, d_bad and d_out live inside the d_theta block
    void* ptrs[] = {h->d_res,      h->d_F[0],     h->d_F[1],      h->d_m2[0],     h->d_m2[1], h->d_w,
                    h->d_tiles[0], h->d_tiles[1], h->d_block_rec, h->d_group_rec, h->d_counts, h->d_theta,
                    h->d_cache};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->h_pin) cudaFreeHost(h->h_pin);
    pwa::free_batch(h);
    pwa::free_hessian(h);
    cudaGetLastError();
    delete h;
}

}  // extern "C"
