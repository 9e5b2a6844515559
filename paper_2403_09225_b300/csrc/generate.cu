// generate.cu -- pseudo-experiment generation on the device: accept-reject
// selection of events from a pool by their model intensity (paper Sec. 3 makes
// its test samples from the PWA model itself), the binned Dalitz histogram of
// a selection, and the gather of the selected events into a data sample.
//
// The uniform numbers of the accept-reject step are a counter-based stream:
// event j of the pool draws u_j from output j + 1 of splitmix64 started at
// `seed` (Steele, Lea and Flood, OOPSLA 2014), u_j = (z >> 11) 2^-53, so the
// selection depends only on (seed, start, n_target, I) and not on the launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "pwa_internal.h"

namespace {

constexpr int kSelThreads = 1024;  // events per selection block (one per thread)

thread_local std::string g_gen_error;

__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t j)
{
    uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ bool accepted(const float* __restrict__ I, long long n, long long start, long long i,
                                         uint64_t seed, double C)
{
    long long j = start + i;
    if (j >= n) j -= n;
    const double u = (double)(splitmix64_at(seed, (uint64_t)j) >> 11) * 0x1.0p-53;
    return u * C < (double)I[j];
}

// largest I (as ordered bits: all values are >= 0) and a flag for a negative or non-finite I
__global__ void max_kernel(const float* __restrict__ I, long long n, unsigned int* __restrict__ max_bits,
                           int* __restrict__ bad)
{
    unsigned int m = 0;
    int b = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = I[i];
        if (!(v >= 0.f) || !isfinite(v)) b = 1;
        else m = max(m, __float_as_uint(v));
    }
    for (int o = 16; o; o >>= 1) {
        m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        b |= __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(max_bits, m);
        if (b) atomicOr(bad, 1);
    }
}

// accepted events per block of kSelThreads sequence positions
__global__ void count_kernel(const float* __restrict__ I, long long n, long long start, uint64_t seed, double C,
                             int* __restrict__ block_count)
{
    const long long i = blockIdx.x * (long long)kSelThreads + threadIdx.x;
    const bool a = i < n && accepted(I, n, start, i, seed, C);
    const int c = __syncthreads_count(a);
    if (threadIdx.x == 0) block_count[blockIdx.x] = c;
}

// exclusive prefix sum of the block counts (one block; serial over chunks of 1024)
__global__ void scan_kernel(const int* __restrict__ count, int nb, long long* __restrict__ offset,
                            long long* __restrict__ total)
{
    __shared__ long long part[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        const long long v = b < nb ? count[b] : 0;
        long long x = v;  // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) part[warp] = x;
        __syncthreads();
        if (warp == 0) {
            long long p = part[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, p, o);
                if (lane >= o) p += y;
            }
            part[lane] = p;  // inclusive over warps
        }
        __syncthreads();
        const long long excl = carry + (warp ? part[warp - 1] : 0) + x - v;
        if (b < nb) offset[b] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// pool index of every accepted event whose rank in the sequence is < n_target
__global__ void scatter_kernel(const float* __restrict__ I, long long n, long long start, uint64_t seed, double C,
                               const long long* __restrict__ offset, int n_target, int* __restrict__ idx)
{
    __shared__ int wsum[32];
    const long long i = blockIdx.x * (long long)kSelThreads + threadIdx.x;
    const bool a = i < n && accepted(I, n, start, i, seed, C);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, a);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    const long long rank = offset[blockIdx.x] + before + __popc(bal & ((1u << lane) - 1u));
    if (a && rank < n_target) {
        long long j = start + i;
        if (j >= n) j -= n;
        idx[rank] = (int)j;
    }
}

// bin counts of (m12^2, m23^2) for the selected events; bin index bx * nb + by
__global__ void histogram_kernel(const float* __restrict__ m2, long long ld, const int* __restrict__ idx, int n, int nb,
                                 double x0, double x1, double y0, double y1, float* __restrict__ h)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const long long e = idx[i];
        const double x = (double)m2[e], y = (double)m2[2 * ld + e];
        int bx = (int)floor((x - x0) * nb / (x1 - x0)), by = (int)floor((y - y0) * nb / (y1 - y0));
        bx = min(max(bx, 0), nb - 1);
        by = min(max(by, 0), nb - 1);
        atomicAdd(&h[bx * nb + by], 1.f);  // integer-valued sums below 2^24: exact in any order
    }
}

__global__ void log_scale_kernel(float* __restrict__ h, int nbins, float scale)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nbins) h[i] = log1pf(h[i] * scale);
}

__global__ void gather_kernel(const float* __restrict__ m2, long long ld, const float2* __restrict__ F, int KS,
                              const int* __restrict__ idx, int n, float* __restrict__ m2_out,
                              float2* __restrict__ F_out)
{
    // one warp per event: F rows are KS complex values, contiguous in both layouts
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const long long e = idx[i];
        const int lane = threadIdx.x & 31;
        if (lane < 3) m2_out[(long long)lane * n + i] = m2[(long long)lane * ld + e];
        for (int q = lane; q < KS; q += 32) F_out[(long long)i * KS + q] = F[e * KS + q];
    }
}

pwa_status gen_fail(pwa_status st, const std::string& msg)
{
    g_gen_error = msg;
    return st;
}

pwa_status gen_cuda(cudaError_t e, const char* what)
{
    cudaGetLastError();
    return gen_fail(PWA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define GEN_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return gen_cuda(e_, #call); \
    } while (0)

int grid_for(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    return (int)std::max(1LL, std::min(b, 148LL * 16));
}

}  // namespace

extern "C" {

pwa_status pwa_accept_reject(const float* d_I, long long n, double C, unsigned long long seed, long long start,
                             int n_target, int* d_idx, int* n_out, double* C_used, void* cuda_stream)
{
    g_gen_error.clear();
    if (!d_I || !d_idx || !n_out || n <= 0 || n > (1LL << 31) - 1 || start < 0 || start >= n || n_target < 0 ||
        !(C >= 0.0) || !std::isfinite(C))
        return gen_fail(PWA_EINVAL, "accept-reject: need 0 < n < 2^31, 0 <= start < n, n_target >= 0, finite C >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int nb = (int)((n + kSelThreads - 1) / kSelThreads);
    // scratch: [max bits, bad flag] ints, block counts, block offsets, total
    void* scratch = nullptr;
    const size_t bytes = 16 + sizeof(int) * (size_t)nb + sizeof(long long) * ((size_t)nb + 1) + 16;
    GEN_CUDA(cudaMallocAsync(&scratch, bytes, s));
    unsigned char* p = static_cast<unsigned char*>(scratch);
    unsigned int* d_max = reinterpret_cast<unsigned int*>(p);
    int* d_bad = reinterpret_cast<int*>(p + 4);
    long long* d_total = reinterpret_cast<long long*>(p + 8);
    long long* d_off = reinterpret_cast<long long*>(p + 16);
    int* d_cnt = reinterpret_cast<int*>(p + 16 + sizeof(long long) * (size_t)nb + 8);
    pwa_status st = PWA_OK;
    cudaError_t e = cudaMemsetAsync(p, 0, 16, s);
    unsigned int hmax[2] = {0, 0};
    if (e == cudaSuccess) {
        max_kernel<<<grid_for(n, 256), 256, 0, s>>>(d_I, n, d_max, d_bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hmax, p, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && hmax[1]) st = gen_fail(PWA_ENONFINITE, "accept-reject: an intensity is negative or not finite");
    double Cu = C;
    if (e == cudaSuccess && st == PWA_OK && Cu <= 0.0) {
        float m;
        std::memcpy(&m, &hmax[0], 4);
        Cu = (double)m;
    }
    long long total = 0;
    if (e == cudaSuccess && st == PWA_OK) {
        count_kernel<<<nb, kSelThreads, 0, s>>>(d_I, n, start, seed, Cu, d_cnt);
        scan_kernel<<<1, 1024, 0, s>>>(d_cnt, nb, d_off, d_total);
        scatter_kernel<<<nb, kSelThreads, 0, s>>>(d_I, n, start, seed, Cu, d_off, n_target, d_idx);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&total, d_total, sizeof(long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaError_t ef = cudaFreeAsync(scratch, s);
    if (e == cudaSuccess) e = ef;
    if (e != cudaSuccess) return gen_cuda(e, "accept-reject");
    if (st != PWA_OK) return st;
    *n_out = (int)std::min<long long>(total, n_target);
    if (C_used) *C_used = Cu;
    return PWA_OK;
}

pwa_status pwa_dalitz_histogram(const float* d_m2, long long ld, const int* d_idx, int n, int nb, double x0,
                                double x1, double y0, double y1, int log_scale, float* d_out, void* cuda_stream)
{
    g_gen_error.clear();
    if (!d_m2 || !d_out || (n > 0 && !d_idx) || n < 0 || ld <= 0 || nb <= 0 || nb > 1024 || !(x1 > x0) ||
        !(y1 > y0))
        return gen_fail(PWA_EINVAL, "histogram: need n >= 0, ld > 0, 0 < nb <= 1024, x1 > x0, y1 > y0");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int nbins = nb * nb;
    GEN_CUDA(cudaMemsetAsync(d_out, 0, sizeof(float) * (size_t)nbins, s));
    if (n > 0) {
        histogram_kernel<<<grid_for(n, 256), 256, 0, s>>>(d_m2, ld, d_idx, n, nb, x0, x1, y0, y1, d_out);
        GEN_CUDA(cudaGetLastError());
    }
    if (log_scale) {
        const float scale = n > 0 ? (float)nbins / (float)n : 0.f;
        log_scale_kernel<<<(nbins + 255) / 256, 256, 0, s>>>(d_out, nbins, scale);
        GEN_CUDA(cudaGetLastError());
    }
    GEN_CUDA(cudaStreamSynchronize(s));
    return PWA_OK;
}

pwa_status pwa_gather_events(const float* d_m2, long long ld, const float* d_F, int KS, const int* d_idx, int n,
                             float* d_m2_out, float* d_F_out, void* cuda_stream)
{
    g_gen_error.clear();
    if (!d_m2 || !d_F || !d_m2_out || !d_F_out || (n > 0 && !d_idx) || n < 0 || ld <= 0 || KS <= 0)
        return gen_fail(PWA_EINVAL, "gather: need n >= 0, ld > 0, KS > 0 and non-NULL arrays");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (n > 0) {
        gather_kernel<<<grid_for((long long)n * 32, 256), 256, 0, s>>>(
            d_m2, ld, reinterpret_cast<const float2*>(d_F), KS, d_idx, n, d_m2_out, reinterpret_cast<float2*>(d_F_out));
        GEN_CUDA(cudaGetLastError());
    }
    GEN_CUDA(cudaStreamSynchronize(s));
    return PWA_OK;
}

const char* pwa_last_generate_error(void) { return g_gen_error.c_str(); }

}  // extern "C"
