// mlp.cu -- the learned starting-point proposal: a small MLP with BF16 weights
// and FP32 accumulation, trained and run by this library's own kernels.
//
// Network: x (a log-scaled 64 x 64 Dalitz histogram, 4096 inputs) -> three
// hidden layers of 512 with GELU -> P outputs (a starting theta, standardised).
// Every matrix product runs on the tensor cores (tcgen05.mma kind::f16, BF16
// operands, FP32 accumulation in tensor memory) in one kernel,
// C[M x N] = A[M x K] B[N x K]^T with both operands K-major BF16 in global
// memory (row-major, K contiguous).  The backward pass forms the transposed
// operands it needs with explicit transpose kernels.  Loss: squared error on
// the standardised outputs, 1 - cos(difference) on outputs flagged periodic
// (phases); Adam on FP32 master weights, whose BF16 copies the products read.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pwa_internal.h"
#include "tcgen05.cuh"

namespace {

// ---------------------------------------------------------------------------
// GEMM: 128 x 64 output tile per CTA, K in chunks of 64 staged in shared memory
// by TMA tensor copies, kGStages chunks in flight
// ---------------------------------------------------------------------------

constexpr int kGM = 128, kGN = 64, kGK = 64;  // tile; K chunk (four MMAs of K = 16)
constexpr int kGThreads = 128;                // 4 warps: one per TMEM lane quarter
constexpr int kGStages = 4;                   // K chunks in flight

using pwa::tc::mma_bf16;
using pwa::tc::mma_commit;
using pwa::tc::sa;
using pwa::tc::sdesc;

// C = A B^T: A [M][K], B [N][K] BF16 row-major with leading dimensions lda, ldb
// (elements), read through tensor maps (tmA, tmB: 2D, K innermost, boxes of
// 8 K x 128 rows and 8 K x 64 rows); C [M][N] FP32 with ldc.  M % 128 == 0,
// N % 64 == 0, K % 64 == 0, leading dimensions multiples of 8.  Split K: CTA z
// of gridDim.z takes the K chunks [z n / Z, (z + 1) n / Z) of the n = K / 64
// and writes its partial product to C + z split_stride (a workspace the
// caller reduces in fixed order).
//
// Shared memory per stage: the A chunk as eight 8-K slices of 128 rows x 16
// bytes (slice j at j 2048: element (r, k) at (k >> 3) 2048 + r 16 + (k & 7) 2),
// then the B chunk likewise with 64 rows (slice stride 1024).  That is the
// canonical K-major layout without swizzle, core matrices of 8 rows x 16
// bytes: LBO (between core matrices along K) = rows x 16, SBO (between 8-row
// groups) = 128.  Each slice is one TMA tensor copy (16 per chunk, issued by
// one thread with the stage's transaction count).
constexpr int kGABytes = kGM * kGK * 2, kGBBytes = kGN * kGK * 2;
constexpr int kGStageBytes = kGABytes + kGBBytes;         // 24 KB
constexpr int kGSmem = kGStages * kGStageBytes + 1024;     // stages + alignment slack

// Bounded wait for phase `parity` of an mbarrier; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long timeout)
{
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
    if (done) return true;
    const long long t0 = clock64();
    while (true) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > timeout) return false;
    }
}

// one 2D tensor-map box (x = K element, y = row) into shared memory, counted on bar
__device__ __forceinline__ void tma_box(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__global__ void __launch_bounds__(kGThreads, 1) gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ CUtensorMap tmB,
                                                                float* __restrict__ C, int ldc,
                                                                long long split_stride, int K,
                                                                long long timeout, int* err)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[kGStages], empty[kGStages];  // chunk landed / its MMAs done
    __shared__ uint32_t tslot;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kGM, n0 = blockIdx.x * kGN;
    const int nchunk = K / kGK, z = blockIdx.z, Z = gridDim.z;
    const int cbeg = (int)((long long)z * nchunk / Z), cend = (int)((long long)(z + 1) * nchunk / Z);
    const int n = cend - cbeg;
    C += (long long)z * split_stride;
    if (tid == 0) {
        for (int s = 0; s < kGStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&empty[s])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(sa(&tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tm = tslot;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kGN >> 3) << 17) | ((uint32_t)(kGM >> 4) << 24);
    const uint32_t s0 = sa(smem);

    if (tid == 0) {
        // chunk i (of this CTA's n) goes to stage i mod kGStages, its (i / kGStages)-th use
        auto issue = [&](int i) {
            const int st = i % kGStages, k0 = (cbeg + i) * kGK;
            const uint32_t dA = s0 + st * kGStageBytes, dB = dA + kGABytes, fb = sa(&full[st]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kGStageBytes)
                         : "memory");
#pragma unroll
            for (int j = 0; j < kGK / 8; ++j) {
                tma_box(dA + j * (kGM * 16), &tmA, k0 + 8 * j, m0, fb);
                tma_box(dB + j * (kGN * 16), &tmB, k0 + 8 * j, n0, fb);
            }
        };
        // chunks whose copies were issued / whose MMAs were committed
        int issued = 0, committed = 0;
        bool ok = true;
        for (; issued < n && issued < kGStages; ++issued) issue(issued);
        while (committed < n) {
            const int c = committed, st = c % kGStages;
            ok = mbar_wait_bounded(sa(&full[st]), (uint32_t)((c / kGStages) & 1), timeout);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dA = s0 + st * kGStageBytes, dB = dA + kGABytes;
#pragma unroll
            for (int ks = 0; ks < kGK / 16; ++ks) {
                const uint64_t ad = sdesc(dA + ks * 2 * (kGM * 16), kGM * 16, 128);
                const uint64_t bd = sdesc(dB + ks * 2 * (kGN * 16), kGN * 16, 128);
                mma_bf16(tm, ad, bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(&empty[st]);
            ++committed;
            // refill the stage of chunk c - 1 (issued = c - 1 + kGStages) once its MMAs have read
            // it; chunk c's MMAs are queued meanwhile, so the tensor cores keep working
            if (c >= 1 && issued < n) {
                const int sp = (c - 1) % kGStages;
                ok = mbar_wait_bounded(sa(&empty[sp]), (uint32_t)(((c - 1) / kGStages) & 1), timeout);
                if (!ok) break;
                issue(issued++);
            }
        }
        // the last chunk's MMAs (and with them every earlier one) before the accumulator is read
        if (ok && n > 0) ok = mbar_wait_bounded(sa(&empty[(n - 1) % kGStages]), (uint32_t)(((n - 1) / kGStages) & 1), timeout);
        if (!ok) {
            // wait (bounded) for the copies and MMAs still in flight: each stage's last armed phase
            for (int s = 0; s < kGStages; ++s) {
                if (issued > s) {
                    const int last = issued - 1 - (issued - 1 - s) % kGStages;  // last chunk copied into stage s
                    (void)mbar_wait_bounded(sa(&full[s]), (uint32_t)((last / kGStages) & 1), timeout);
                }
                if (committed > s) {
                    const int last = committed - 1 - (committed - 1 - s) % kGStages;  // last chunk computed from s
                    (void)mbar_wait_bounded(sa(&empty[s]), (uint32_t)((last / kGStages) & 1), timeout);
                }
            }
            s_ok = 0;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool ok = s_ok != 0;
    if (ok && n > 0) {
        // row m0 + 32 warp + lane of C from TMEM lane 32 warp + lane
        const int m = m0 + 32 * warp + lane;
        for (int c0 = 0; c0 < kGN; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(tm + ((uint32_t)(32 * warp) << 16) + c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float4* crow = reinterpret_cast<float4*>(C + (size_t)m * ldc + n0 + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                crow[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                      __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
        }
    } else if (!ok && tid == 0) {
        atomicOr(err, pwa::ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tm));
}

// C [M][N] (ldc) = sum over z = 0 .. Z - 1 of W [z][M][N] (ldw, stride), in that order
__global__ void split_reduce_kernel(const float* __restrict__ W, int ldw, long long stride, int Z, int M, int N,
                                    float* __restrict__ C, int ldc)
{
    const long long n = (long long)M * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / N), c = (int)(i % N);
        float s = 0.f;
        for (int z = 0; z < Z; ++z) s += W[z * stride + (long long)r * ldw + c];
        C[(size_t)r * ldc + c] = s;
    }
}

// ---------------------------------------------------------------------------
// elementwise parts
// ---------------------------------------------------------------------------

__device__ __forceinline__ float gelu(float z)  // tanh form
{
    const float u = 0.7978845608028654f * (z + 0.044715f * z * z * z);
    return 0.5f * z * (1.f + tanhf(u));
}

__device__ __forceinline__ float gelu_grad(float z)
{
    const float u = 0.7978845608028654f * (z + 0.044715f * z * z * z);
    const float t = tanhf(u);
    const float du = 0.7978845608028654f * (1.f + 3.f * 0.044715f * z * z);
    return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * du;
}

// z = acc + bias (pre-activation, kept for the backward pass); h = GELU(z) (or z
// for the output layer) in BF16 for the next product.  [rows][cols], leading dims.
__global__ void bias_act_kernel(const float* __restrict__ acc, int lda, const float* __restrict__ bias, int rows,
                                int cols, int act, float* __restrict__ z, int ldz, __nv_bfloat16* __restrict__ h, int ldh)
{
    const long long n = (long long)rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        const float v = acc[(size_t)r * lda + c] + bias[c];
        z[(size_t)r * ldz + c] = v;
        if (h) h[(size_t)r * ldh + c] = __float2bfloat16_rn(act ? gelu(v) : v);
    }
}

// Loss over the output rows and its gradient with respect to the outputs:
// squared error, or 1 - cos(y - t) where periodic[c]; weights per output.
// dy[r][c] = d loss / d y / rows; loss_part[r] = the row's loss.
__global__ void loss_kernel(const float* __restrict__ y, int ldy, const float* __restrict__ t, int rows, int cols,
                            const float* __restrict__ wgt, const int* __restrict__ periodic, float* __restrict__ dy,
                            int lddy, float* __restrict__ loss_row)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float l = 0.f;
    for (int c = 0; c < cols; ++c) {
        const float d = y[(size_t)r * ldy + c] - t[(size_t)r * cols + c];
        float lc, g;
        if (periodic[c]) {
            lc = 1.f - cosf(d);
            g = sinf(d);
        } else {
            lc = 0.5f * d * d;
            g = d;
        }
        l += wgt[c] * lc;
        dy[(size_t)r * lddy + c] = wgt[c] * g / rows;
    }
    loss_row[r] = l / rows;
}

// dz = dh * GELU'(z) (hidden layers) as BF16 for the next products
__global__ void act_back_kernel(const float* __restrict__ dh, int lddh, const float* __restrict__ z, int ldz, int rows,
                                int cols, __nv_bfloat16* __restrict__ dz, int lddz, float* __restrict__ dz32)
{
    const long long n = (long long)rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        const float v = dh[(size_t)r * lddh + c] * gelu_grad(z[(size_t)r * ldz + c]);
        dz[(size_t)r * lddz + c] = __float2bfloat16_rn(v);
        if (dz32) dz32[(size_t)r * cols + c] = v;
    }
}

// out[c][r] = in[r][c] (BF16), zero in the padding of out
__global__ void transpose_bf16_kernel(const __nv_bfloat16* __restrict__ in, int ldin, int rows, int cols,
                                      __nv_bfloat16* __restrict__ out, int ldout, int out_rows, int out_cols)
{
    const long long n = (long long)out_rows * out_cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / out_cols), r = (int)(i % out_cols);
        out[(size_t)c * ldout + r] = (c < cols && r < rows) ? in[(size_t)r * ldin + c] : __float2bfloat16_rn(0.f);
    }
}

// FP32 [rows][cols] -> BF16 with leading dimension ld (zero in the padding)
__global__ void to_bf16_kernel(const float* __restrict__ in, int rows, int cols, __nv_bfloat16* __restrict__ out,
                               int ld, int out_rows)
{
    const long long n = (long long)out_rows * ld;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / ld), c = (int)(i % ld);
        out[i] = __float2bfloat16_rn((r < rows && c < cols) ? in[(size_t)r * cols + c] : 0.f);
    }
}

// bias gradient: db[c] = sum_r dz[r][c] (fixed order)
__global__ void bias_grad_kernel(const float* __restrict__ dz, int ld, int rows, int cols, float* __restrict__ db)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dz[(size_t)r * ld + c];
    db[c] = s;
}

// Adam on FP32 masters; the BF16 copy (leading dimension ldb, rows x cols) follows
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, int ldg, float* __restrict__ m1,
                            float* __restrict__ m2, int rows, int cols, float lr, float b1, float b2, float eps,
                            float c1, float c2, __nv_bfloat16* __restrict__ wb, int ldb)
{
    const long long n = (long long)rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        const float gi = g[(size_t)r * ldg + c];
        const float a = b1 * m1[i] + (1.f - b1) * gi, b = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = b;
        const float v = w[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
        w[i] = v;
        if (wb) wb[(size_t)r * ldb + c] = __float2bfloat16_rn(v);
    }
}

int blocks_for(long long n) { return (int)std::max(1LL, std::min((n + 255) / 256, 65535LL * 4)); }

int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

// ---------------------------------------------------------------------------
// the network object
// ---------------------------------------------------------------------------

struct pwa_mlp {
    int in = 0, hid = 0, out = 0, layers = 0;  // layers: hidden layers (3)
    int outp = 0;                             // out padded to 128 (rows of the last W in dW products)
    int maxB = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int* d_err = nullptr;
    long long timeout = 0;
    // per layer l = 0 .. layers (the last is the output layer): W [fan_out][fan_in] FP32 master,
    // BF16 copy [fan_out_p][fan_in], bias, Adam moments, gradients
    std::vector<int> fin, fout, foutp;
    std::vector<float*> W, b, mW1, mW2, mb1, mb2, gW, gb;
    std::vector<__nv_bfloat16*> Wb;
    // activations for up to maxB rows: H_l (BF16 input of layer l) [maxB][fin], Z_l [maxB][fout_p]
    std::vector<__nv_bfloat16*> H;
    std::vector<float*> Z;
    float* acc = nullptr;     // GEMM output scratch [maxB x max(fout_p, fin)] or [fout_p x fin]
    float* dY = nullptr;      // [maxB][outp]
    __nv_bfloat16* dZb = nullptr;   // BF16 dz [maxB][max fout_p]
    float* dZ32 = nullptr;    // FP32 dz [maxB][max fout]
    __nv_bfloat16* T1 = nullptr;    // transposes
    __nv_bfloat16* T2 = nullptr;
    float* loss_rows = nullptr;
    float* ws = nullptr;      // split-K partial products
    size_t ws_floats = 0;
    float* T = nullptr;       // targets of the current batch [maxB][out] (copied in, read by the loss)
    cudaStream_t own_stream = nullptr;  // created when the caller passes none (graphs need a real stream)
    // the gradient pass of a batch size (layers' products, loss, backward) as a CUDA
    // graph, captured on the third call with that size; index B / 128
    std::vector<cudaGraphExec_t> graph;
    std::vector<int> graph_uses;
    int* d_periodic = nullptr;
    float* d_wgt = nullptr;
    int step = 0;
};

namespace {

pwa_status mlp_fail(pwa_mlp* m, pwa_status st, const std::string& msg)
{
    m->err = msg;
    return st;
}

pwa_status mlp_cuda(pwa_mlp* m, cudaError_t e, const char* what)
{
    cudaGetLastError();
    return mlp_fail(m, PWA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MLP_CUDA(m, call)                                        \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return mlp_cuda((m), e_, #call);  \
    } while (0)

// K splits for an M x N x K product: enough CTAs for two waves over the SMs,
// at least two K chunks per split
int k_splits(int M, int N, int K)
{
    const int tiles = (M / kGM) * (N / kGN), chunks = K / kGK;
    int z = std::max(1, (2 * 148 + tiles - 1) / tiles);
    return std::max(1, std::min(z, chunks / 2));
}

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point query
// (no link against the driver library); null when the driver does not offer it
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled()
{
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiledFn) nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// 2D map of a row-major BF16 matrix [rows][K] (leading dimension ld elements):
// K innermost, boxes of 8 K x box_rows rows, no swizzle
bool bf16_map(CUtensorMap* map, const __nv_bfloat16* base, int rows, int K, int ld, int box_rows)
{
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {8, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C[M][N] = A[M][K] B[N][K]^T on the tensor cores (split K through the workspace when it pays)
pwa_status gemm(pwa_mlp* m, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, float* C, int ldc, int M,
                int N, int K)
{
    if (M % kGM || N % kGN || K % kGK || lda % 8 || ldb % 8 || lda < K || ldb < K)
        return mlp_fail(m, PWA_EINVAL, "internal: GEMM shape not tile-aligned");
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) % 16)
        return mlp_fail(m, PWA_EINVAL, "internal: GEMM operands not 16-byte aligned");
    CUtensorMap tmA, tmB;
    if (!bf16_map(&tmA, A, M, K, lda, kGM) || !bf16_map(&tmB, B, N, K, ldb, kGN))
        return mlp_fail(m, PWA_ECUDA, "tensor map encoding failed for a GEMM operand");
    const int Z = k_splits(M, N, K);
    if (Z > 1 && (size_t)Z * M * N > m->ws_floats) return mlp_fail(m, PWA_EINVAL, "internal: split-K workspace too small");
    dim3 grid(N / kGN, M / kGM, Z);
    if (Z == 1) {
        gemm_bf16_kernel<<<grid, kGThreads, kGSmem, m->stream>>>(tmA, tmB, C, ldc, 0, K, m->timeout, m->d_err);
        MLP_CUDA(m, cudaGetLastError());
        return PWA_OK;
    }
    const long long stride = (long long)M * N;
    gemm_bf16_kernel<<<grid, kGThreads, kGSmem, m->stream>>>(tmA, tmB, m->ws, N, stride, K, m->timeout, m->d_err);
    MLP_CUDA(m, cudaGetLastError());
    split_reduce_kernel<<<blocks_for(stride), 256, 0, m->stream>>>(m->ws, N, stride, Z, M, N, C, ldc);
    MLP_CUDA(m, cudaGetLastError());
    return PWA_OK;
}

#define MLP_TRY(call)                 \
    do {                              \
        pwa_status s_ = (call);       \
        if (s_ != PWA_OK) return s_;  \
    } while (0)

// forward over B rows (B % 128 == 0) from X (FP32 [B][in]); outputs in Z[layers] (FP32)
// the network's input in BF16 (H[0]) from the caller's FP32 rows
pwa_status forward_input(pwa_mlp* m, int B, const float* d_x)
{
    to_bf16_kernel<<<blocks_for((long long)B * m->in), 256, 0, m->stream>>>(d_x, B, m->in, m->H[0], m->in, B);
    MLP_CUDA(m, cudaGetLastError());
    return PWA_OK;
}

// the layers from H[0]; outputs in Z[layers] (FP32)
pwa_status forward_layers(pwa_mlp* m, int B)
{
    const int L = m->layers + 1;
    for (int l = 0; l < L; ++l) {
        const bool last = l == L - 1;
        MLP_TRY(gemm(m, m->H[l], m->fin[l], m->Wb[l], m->fin[l], m->acc, m->foutp[l], B, m->foutp[l], m->fin[l]));
        bias_act_kernel<<<blocks_for((long long)B * m->fout[l]), 256, 0, m->stream>>>(
            m->acc, m->foutp[l], m->b[l], B, m->fout[l], last ? 0 : 1, m->Z[l], m->foutp[l], last ? nullptr : m->H[l + 1],
            m->fin[l + 1 < L ? l + 1 : l]);
        MLP_CUDA(m, cudaGetLastError());
    }
    return PWA_OK;
}

// forward over B rows (B % 128 == 0) from X (FP32 [B][in]); outputs in Z[layers] (FP32)
pwa_status forward(pwa_mlp* m, int B, const float* d_x)
{
    MLP_TRY(forward_input(m, B, d_x));
    return forward_layers(m, B);
}

// backward after forward, with the targets in m->T: gradients into gW, gb; loss rows in loss_rows
pwa_status backward(pwa_mlp* m, int B)
{
    const int L = m->layers + 1;
    const float* d_t = m->T;
    loss_kernel<<<(B + 127) / 128, 128, 0, m->stream>>>(m->Z[L - 1], m->foutp[L - 1], d_t, B, m->out, m->d_wgt,
                                                       m->d_periodic, m->dY, m->outp, m->loss_rows);
    MLP_CUDA(m, cudaGetLastError());
    // dZ of the output layer (no activation): BF16 copy of dY with the padding zero
    to_bf16_kernel<<<blocks_for((long long)B * m->outp), 256, 0, m->stream>>>(m->dY, B, m->outp, m->dZb, m->outp, B);
    MLP_CUDA(m, cudaGetLastError());
    const float* dz32 = m->dY;
    int dz_ld32 = m->outp;
    for (int l = L - 1; l >= 0; --l) {
        const int fo = m->fout[l], fop = m->foutp[l], fi = m->fin[l];
        // bias gradient
        bias_grad_kernel<<<(fo + 127) / 128, 128, 0, m->stream>>>(dz32, dz_ld32, B, fo, m->gb[l]);
        MLP_CUDA(m, cudaGetLastError());
        // dW [fop][fi] = dZ^T [fop][B] x H^T [fi][B]^T
        transpose_bf16_kernel<<<blocks_for((long long)fop * B), 256, 0, m->stream>>>(m->dZb, fop, B, fop, m->T1, B, fop, B);
        MLP_CUDA(m, cudaGetLastError());
        transpose_bf16_kernel<<<blocks_for((long long)fi * B), 256, 0, m->stream>>>(m->H[l], fi, B, fi, m->T2, B, fi, B);
        MLP_CUDA(m, cudaGetLastError());
        MLP_TRY(gemm(m, m->T1, B, m->T2, B, m->gW[l], fi, fop, fi, B));
        if (l == 0) break;
        // dH_l [B][fi] = dZ [B][fop] x W [fop][fi]: second operand W^T [fi][fop]
        transpose_bf16_kernel<<<blocks_for((long long)fi * fop), 256, 0, m->stream>>>(m->Wb[l], fi, fop, fi, m->T1, fop, fi,
                                                                                     fop);
        MLP_CUDA(m, cudaGetLastError());
        MLP_TRY(gemm(m, m->dZb, fop, m->T1, fop, m->acc, fi, B, fi, fop));
        act_back_kernel<<<blocks_for((long long)B * fi), 256, 0, m->stream>>>(m->acc, fi, m->Z[l - 1], m->foutp[l - 1], B,
                                                                             fi, m->dZb, m->foutp[l - 1], m->dZ32);
        MLP_CUDA(m, cudaGetLastError());
        dz32 = m->dZ32;
        dz_ld32 = fi;
    }
    return PWA_OK;
}

pwa_status alloc_f(pwa_mlp* m, float** p, size_t n)
{
    MLP_CUDA(m, cudaMalloc(p, std::max<size_t>(n, 1) * sizeof(float)));
    MLP_CUDA(m, cudaMemsetAsync(*p, 0, std::max<size_t>(n, 1) * sizeof(float), m->stream));
    return PWA_OK;
}

pwa_status alloc_b(pwa_mlp* m, __nv_bfloat16** p, size_t n)
{
    MLP_CUDA(m, cudaMalloc(p, std::max<size_t>(n, 1) * sizeof(__nv_bfloat16)));
    MLP_CUDA(m, cudaMemsetAsync(*p, 0, std::max<size_t>(n, 1) * sizeof(__nv_bfloat16), m->stream));
    return PWA_OK;
}

pwa_status create_impl(pwa_mlp* m, int in, int hid, int layers, int out, int maxB, unsigned long long seed,
                       const int* periodic, const float* wgt)
{
    m->in = in;
    m->hid = hid;
    m->layers = layers;
    m->out = out;
    m->outp = round_up(out, kGM);
    m->maxB = maxB;
    int dev = 0, clock_khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev);
    m->timeout = (long long)std::max(clock_khz, 1000000) * 2000LL;  // about 2 s of SM cycles
    const int L = layers + 1;
    for (int l = 0; l < L; ++l) {
        m->fin.push_back(l == 0 ? in : hid);
        m->fout.push_back(l == L - 1 ? out : hid);
        m->foutp.push_back(l == L - 1 ? m->outp : hid);
    }
    MLP_CUDA(m, cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem));
    MLP_CUDA(m, cudaMalloc(&m->d_err, sizeof(int)));
    MLP_CUDA(m, cudaMemsetAsync(m->d_err, 0, sizeof(int), m->stream));
    size_t max_f = 0;
    for (int l = 0; l < L; ++l) {
        const size_t nW = (size_t)m->fout[l] * m->fin[l];
        float *W, *b, *a1, *a2, *c1, *c2, *gW, *gb;
        __nv_bfloat16* Wb;
        MLP_TRY(alloc_f(m, &W, nW));
        MLP_TRY(alloc_f(m, &b, m->fout[l]));
        MLP_TRY(alloc_f(m, &a1, nW));
        MLP_TRY(alloc_f(m, &a2, nW));
        MLP_TRY(alloc_f(m, &c1, m->fout[l]));
        MLP_TRY(alloc_f(m, &c2, m->fout[l]));
        MLP_TRY(alloc_f(m, &gW, (size_t)m->foutp[l] * m->fin[l]));
        MLP_TRY(alloc_f(m, &gb, m->fout[l]));
        MLP_TRY(alloc_b(m, &Wb, (size_t)m->foutp[l] * m->fin[l]));
        m->W.push_back(W);
        m->b.push_back(b);
        m->mW1.push_back(a1);
        m->mW2.push_back(a2);
        m->mb1.push_back(c1);
        m->mb2.push_back(c2);
        m->gW.push_back(gW);
        m->gb.push_back(gb);
        m->Wb.push_back(Wb);
        __nv_bfloat16* H;
        float* Z;
        MLP_TRY(alloc_b(m, &H, (size_t)maxB * m->fin[l]));
        MLP_TRY(alloc_f(m, &Z, (size_t)maxB * m->foutp[l]));
        m->H.push_back(H);
        m->Z.push_back(Z);
        max_f = std::max(max_f, (size_t)std::max(m->foutp[l], m->fin[l]));
    }
    MLP_TRY(alloc_f(m, &m->acc, (size_t)maxB * max_f));
    MLP_TRY(alloc_f(m, &m->dY, (size_t)maxB * m->outp));
    MLP_TRY(alloc_b(m, &m->dZb, (size_t)maxB * std::max(m->outp, hid)));
    MLP_TRY(alloc_f(m, &m->dZ32, (size_t)maxB * hid));
    MLP_TRY(alloc_b(m, &m->T1, std::max((size_t)max_f * maxB, (size_t)hid * std::max(hid, m->outp))));
    MLP_TRY(alloc_b(m, &m->T2, (size_t)max_f * maxB));
    MLP_TRY(alloc_f(m, &m->loss_rows, maxB));
    MLP_TRY(alloc_f(m, &m->T, (size_t)maxB * out));
    m->graph.assign(maxB / kGM + 1, nullptr);
    m->graph_uses.assign(maxB / kGM + 1, 0);
    // split-K workspace: the largest Z M N over the network's products at batches up to maxB
    for (int B = kGM; B <= maxB; B += kGM)
        for (int l = 0; l < L; ++l) {
            const int fi = m->fin[l], fop = m->foutp[l];
            const int shapes[3][3] = {{B, fop, fi}, {fop, fi, B}, {B, fi, fop}};
            for (const auto& sh : shapes) {
                const int Z = k_splits(sh[0], sh[1], sh[2]);
                if (Z > 1) m->ws_floats = std::max(m->ws_floats, (size_t)Z * sh[0] * sh[1]);
            }
        }
    if (m->ws_floats) MLP_TRY(alloc_f(m, &m->ws, m->ws_floats));
    MLP_CUDA(m, cudaMalloc(&m->d_periodic, sizeof(int) * out));
    MLP_CUDA(m, cudaMalloc(&m->d_wgt, sizeof(float) * out));
    std::vector<int> per(out, 0);
    std::vector<float> wg(out, 1.f);
    for (int c = 0; c < out; ++c) {
        if (periodic) per[c] = periodic[c] != 0;
        if (wgt) wg[c] = wgt[c];
    }
    MLP_CUDA(m, cudaMemcpyAsync(m->d_periodic, per.data(), sizeof(int) * out, cudaMemcpyHostToDevice, m->stream));
    MLP_CUDA(m, cudaMemcpyAsync(m->d_wgt, wg.data(), sizeof(float) * out, cudaMemcpyHostToDevice, m->stream));
    // initial weights: uniform in +-sqrt(6 / (fan_in + fan_out)) from a splitmix64 stream (host), biases 0
    unsigned long long st = seed;
    auto next = [&st]() {
        st += 0x9E3779B97F4A7C15ull;
        unsigned long long z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    for (int l = 0; l < L; ++l) {
        const size_t nW = (size_t)m->fout[l] * m->fin[l];
        std::vector<float> w(nW);
        const double lim = std::sqrt(6.0 / (m->fin[l] + m->fout[l]));
        for (size_t i = 0; i < nW; ++i) w[i] = (float)(lim * (2.0 * ((next() >> 11) * (1.0 / 9007199254740992.0)) - 1.0));
        MLP_CUDA(m, cudaMemcpy(m->W[l], w.data(), nW * sizeof(float), cudaMemcpyHostToDevice));
        to_bf16_kernel<<<blocks_for((long long)m->foutp[l] * m->fin[l]), 256, 0, m->stream>>>(
            m->W[l], m->fout[l], m->fin[l], m->Wb[l], m->fin[l], m->foutp[l]);
        MLP_CUDA(m, cudaGetLastError());
    }
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    return PWA_OK;
}

// forward layers + loss + backward from H[0] and T: eager for the first two calls
// with a batch size, then captured into a CUDA graph and replayed
pwa_status gradient_pass(pwa_mlp* m, int B)
{
    const int gi = B / kGM;
    if (m->graph[gi]) {
        MLP_CUDA(m, cudaGraphLaunch(m->graph[gi], m->stream));
        return PWA_OK;
    }
    if (++m->graph_uses[gi] < 3) {
        MLP_TRY(forward_layers(m, B));
        return backward(m, B);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGetLastError();
        m->graph_uses[gi] = -1000000;  // this size stays eager
        MLP_TRY(forward_layers(m, B));
        return backward(m, B);
    }
    pwa_status st = forward_layers(m, B);
    if (st == PWA_OK) st = backward(m, B);
    e = cudaStreamEndCapture(m->stream, &g);
    if (st != PWA_OK || e != cudaSuccess || !g || cudaGraphInstantiate(&m->graph[gi], g, 0) != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        m->graph[gi] = nullptr;
        m->graph_uses[gi] = -1000000;
        m->err.clear();
        MLP_TRY(forward_layers(m, B));
        return backward(m, B);
    }
    cudaGraphDestroy(g);
    MLP_CUDA(m, cudaGraphLaunch(m->graph[gi], m->stream));
    return PWA_OK;
}

pwa_status check_err(pwa_mlp* m)
{
    int e = 0;
    MLP_CUDA(m, cudaMemcpyAsync(&e, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    if (e) return mlp_fail(m, PWA_ETIMEOUT, "a tensor-core product did not complete within the wait limit");
    return PWA_OK;
}

}  // namespace

extern "C" {

thread_local std::string g_mlp_create_error;

pwa_status pwa_mlp_create(int in, int hidden, int layers, int out, int max_batch, unsigned long long seed,
                          const int* periodic, const float* loss_weight, void* cuda_stream, pwa_mlp** out_m)
{
    if (!out_m) return PWA_EINVAL;
    *out_m = nullptr;
    g_mlp_create_error.clear();
    if (in <= 0 || hidden <= 0 || layers < 1 || out <= 0 || max_batch <= 0 || in % kGK || hidden % kGM ||
        max_batch % kGM) {
        g_mlp_create_error = "sizes: in % 64 == 0, hidden % 128 == 0, max_batch % 128 == 0, layers >= 1";
        return PWA_EINVAL;
    }
    auto* m = new (std::nothrow) pwa_mlp();
    if (!m) return PWA_ENOMEM;
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    if (!m->stream) {
        // a stream of our own (ordered with the legacy default stream) so that the
        // gradient pass can be captured into a graph
        if (cudaStreamCreate(&m->own_stream) != cudaSuccess) {
            cudaGetLastError();
            g_mlp_create_error = "cannot create the network's stream";
            delete m;
            return PWA_ECUDA;
        }
        m->stream = m->own_stream;
    }
    pwa_status st = create_impl(m, in, hidden, layers, out, max_batch, seed, periodic, loss_weight);
    if (st != PWA_OK) {
        g_mlp_create_error = m->err;
        pwa_mlp_destroy(m);
        return st;
    }
    *out_m = m;
    return PWA_OK;
}

pwa_status pwa_mlp_forward(pwa_mlp* m, int B, const float* d_x, float* d_y)
{
    if (!m || !d_x || !d_y) return PWA_EINVAL;
    m->err.clear();
    if (B <= 0 || B > m->maxB || B % kGM) return mlp_fail(m, PWA_EINVAL, "B must be a multiple of 128 up to max_batch");
    MLP_TRY(forward(m, B, d_x));
    const int L = m->layers + 1;
    MLP_CUDA(m, cudaMemcpy2DAsync(d_y, sizeof(float) * m->out, m->Z[L - 1], sizeof(float) * m->foutp[L - 1],
                                  sizeof(float) * m->out, B, cudaMemcpyDeviceToDevice, m->stream));
    return check_err(m);
}

pwa_status pwa_mlp_gradients(pwa_mlp* m, int B, const float* d_x, const float* d_t, double* loss)
{
    if (!m || !d_x || !d_t) return PWA_EINVAL;
    m->err.clear();
    if (B <= 0 || B > m->maxB || B % kGM) return mlp_fail(m, PWA_EINVAL, "B must be a multiple of 128 up to max_batch");
    MLP_TRY(forward_input(m, B, d_x));
    MLP_CUDA(m, cudaMemcpyAsync(m->T, d_t, sizeof(float) * (size_t)B * m->out, cudaMemcpyDeviceToDevice, m->stream));
    MLP_TRY(gradient_pass(m, B));
    if (loss) {
        std::vector<float> lr(B);
        MLP_CUDA(m, cudaMemcpyAsync(lr.data(), m->loss_rows, sizeof(float) * B, cudaMemcpyDeviceToHost, m->stream));
        MLP_TRY(check_err(m));
        double s = 0.0;
        for (float v : lr) s += v;
        *loss = s;
    }
    return check_err(m);
}

pwa_status pwa_mlp_train_step(pwa_mlp* m, int B, const float* d_x, const float* d_t, float lr, double* loss)
{
    MLP_TRY(pwa_mlp_gradients(m, B, d_x, d_t, loss));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    m->step += 1;
    const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
    for (int l = 0; l <= m->layers; ++l) {
        adam_kernel<<<blocks_for((long long)m->fout[l] * m->fin[l]), 256, 0, m->stream>>>(
            m->W[l], m->gW[l], m->fin[l], m->mW1[l], m->mW2[l], m->fout[l], m->fin[l], lr, b1, b2, eps, c1, c2, m->Wb[l],
            m->fin[l]);
        MLP_CUDA(m, cudaGetLastError());
        adam_kernel<<<blocks_for(m->fout[l]), 256, 0, m->stream>>>(m->b[l], m->gb[l], 0, m->mb1[l], m->mb2[l], 1,
                                                                   m->fout[l], lr, b1, b2, eps, c1, c2, nullptr, 0);
        MLP_CUDA(m, cudaGetLastError());
    }
    return PWA_OK;
}

pwa_status pwa_mlp_params(pwa_mlp* m, int layer, int which, float* host, int to_device)
{
    // which: 0 W [fout][fin], 1 b [fout], 2 dW [fout][fin] (last gradients), 3 db [fout]
    if (!m || !host || layer < 0 || layer > m->layers || which < 0 || which > 3) return PWA_EINVAL;
    const int fo = m->fout[layer], fi = m->fin[layer];
    if (which == 2) {
        if (to_device) return PWA_EINVAL;
        MLP_CUDA(m, cudaMemcpy2DAsync(host, sizeof(float) * fi, m->gW[layer], sizeof(float) * fi, sizeof(float) * fi, fo,
                                      cudaMemcpyDeviceToHost, m->stream));
        MLP_CUDA(m, cudaStreamSynchronize(m->stream));
        return PWA_OK;
    }
    float* d = which == 0 ? m->W[layer] : which == 1 ? m->b[layer] : m->gb[layer];
    const size_t n = which == 0 ? (size_t)fo * fi : (size_t)fo;
    if (to_device) {
        if (which == 3) return PWA_EINVAL;
        MLP_CUDA(m, cudaMemcpyAsync(d, host, n * sizeof(float), cudaMemcpyHostToDevice, m->stream));
        if (which == 0) {
            to_bf16_kernel<<<blocks_for((long long)m->foutp[layer] * fi), 256, 0, m->stream>>>(
                m->W[layer], fo, fi, m->Wb[layer], fi, m->foutp[layer]);
            MLP_CUDA(m, cudaGetLastError());
        }
    } else {
        MLP_CUDA(m, cudaMemcpyAsync(host, d, n * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    }
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    return PWA_OK;
}

pwa_status pwa_mlp_gemm_check(pwa_mlp* m, int M, int N, int K, const float* hA, const float* hB, float* hC)
{
    // the tensor-core product alone, on BF16-rounded copies of host FP32 A [M][K], B [N][K]
    if (!m || !hA || !hB || !hC) return PWA_EINVAL;
    if (M % kGM || N % kGN || K % kGK) return mlp_fail(m, PWA_EINVAL, "M % 128, N % 64, K % 64 must be 0");
    float *dA = nullptr, *dB = nullptr, *dC = nullptr;
    __nv_bfloat16 *bA = nullptr, *bB = nullptr;
    pwa_status st = PWA_OK;
    cudaError_t e = cudaMalloc(&dA, sizeof(float) * (size_t)M * K);
    if (e == cudaSuccess) e = cudaMalloc(&dB, sizeof(float) * (size_t)N * K);
    if (e == cudaSuccess) e = cudaMalloc(&dC, sizeof(float) * (size_t)M * N);
    if (e == cudaSuccess) e = cudaMalloc(&bA, sizeof(__nv_bfloat16) * (size_t)M * K);
    if (e == cudaSuccess) e = cudaMalloc(&bB, sizeof(__nv_bfloat16) * (size_t)N * K);
    if (e == cudaSuccess) e = cudaMemcpy(dA, hA, sizeof(float) * (size_t)M * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, hB, sizeof(float) * (size_t)N * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        to_bf16_kernel<<<blocks_for((long long)M * K), 256, 0, m->stream>>>(dA, M, K, bA, K, M);
        to_bf16_kernel<<<blocks_for((long long)N * K), 256, 0, m->stream>>>(dB, N, K, bB, K, N);
        e = cudaGetLastError();
    }
    // a product larger than the network's own may need a larger split-K workspace for the call
    float* ws_saved = m->ws;
    const size_t ws_saved_n = m->ws_floats;
    float* ws_tmp = nullptr;
    const int Z = k_splits(M, N, K);
    if (e == cudaSuccess && Z > 1 && (size_t)Z * M * N > m->ws_floats) {
        e = cudaMalloc(&ws_tmp, sizeof(float) * (size_t)Z * M * N);
        if (e == cudaSuccess) {
            m->ws = ws_tmp;
            m->ws_floats = (size_t)Z * M * N;
        }
    }
    if (e == cudaSuccess) st = gemm(m, bA, K, bB, K, dC, N, M, N, K);
    if (e == cudaSuccess && st == PWA_OK) st = check_err(m);
    if (e == cudaSuccess && st == PWA_OK) e = cudaMemcpy(hC, dC, sizeof(float) * (size_t)M * N, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess && st == PWA_OK) st = mlp_cuda(m, e, "gemm check");
    if (ws_tmp) {
        cudaStreamSynchronize(m->stream);
        m->ws = ws_saved;
        m->ws_floats = ws_saved_n;
    }
    void* ps[] = {dA, dB, dC, bA, bB, ws_tmp};
    for (void* p : ps)
        if (p) cudaFree(p);
    return st;
}

const char* pwa_mlp_last_error(const pwa_mlp* m) { return m ? m->err.c_str() : g_mlp_create_error.c_str(); }

void pwa_mlp_destroy(pwa_mlp* m)
{
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    else cudaDeviceSynchronize();
    auto fr = [](void* p) {
        if (p) cudaFree(p);
    };
    for (size_t l = 0; l < m->W.size(); ++l) {
        fr(m->W[l]);
        fr(m->b[l]);
        fr(m->mW1[l]);
        fr(m->mW2[l]);
        fr(m->mb1[l]);
        fr(m->mb2[l]);
        fr(m->gW[l]);
        fr(m->gb[l]);
        fr(m->Wb[l]);
    }
    for (auto* p : m->H) fr(p);
    for (auto* p : m->Z) fr(p);
    void* ps[] = {m->acc, m->dY, m->dZb, m->dZ32, m->T1, m->T2, m->loss_rows, m->ws, m->T, m->d_periodic, m->d_wgt,
                  m->d_err};
    for (void* p : ps) fr(p);
    for (auto g : m->graph)
        if (g) cudaGraphExecDestroy(g);
    if (m->own_stream) cudaStreamDestroy(m->own_stream);
    cudaGetLastError();
    delete m;
}

}  // extern "C"
