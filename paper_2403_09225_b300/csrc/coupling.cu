// coupling.cu -- the fixed-mass coupling sub-problem on the tensor cores.
//
// With every mass and width (and the fixed couplings) held at given values,
// U_{k,s}(e) = BW_k(e) F_{k,s}(e) no longer changes and the coherent sum of
// Eq. 1 is linear in the couplings: A_s(e) = sum_k g_k U_{k,s}(e).  Two things
// follow (the paper's Eq. 1 written with the couplings outside the sum):
//  * the MC normalisation collapses to a K x K Hermitian integral matrix,
//    sum_mc I = g^H Phi g with Phi_{kk'} = sum_mc sum_s conj(U_ks) U_k's,
//    computed once, so the MC events are never read again;
//  * the data term for C coupling vectors at once is two GEMMs per tile of
//    128 (event, projection) rows: A = U G (GEMM1, the coherent sums and
//    their directional derivatives) and, after the per-event weights
//    a = w/I, b = w Idot/I^2, Q = W^T U (GEMM2, the adjoint sums of Eqs. 6-7
//    contracted over the events).
// Both GEMMs run on tcgen05 in kind::tf32 with the three-term split
// (x = hi + lo, both rounded to TF32; a b ~ ahi bhi + ahi blo + alo bhi),
// which keeps FP32-level accuracy; accumulators live in
// tensor memory, the per-event epilogue in registers, cross-tile sums in
// FP64.  Operands use the canonical K-major layout without swizzle: 8-row x
// 16-byte core matrices, LBO = stride between cores along K, SBO = stride
// between 8-row groups.  Operands written column-wise by the epilogue use a
// 144-byte core stride along K (16 bytes of padding per core) so that the 32
// threads of a warp hit 32 different banks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pwa_internal.h"

namespace {

constexpr int kCT = 256;        // threads per CTA: threads r and r + 128 share row r of a tile
                                // (each takes half of the row's K-cores and of the vectors)
constexpr int kRows = 128;      // (event, projection) rows per tile
constexpr int kCV = 16;         // coupling vectors per launch
constexpr int kN1 = 4 * kCV;    // GEMM1 columns: Re A, Im A, Re Adot, Im Adot of every vector
constexpr uint32_t kLboT = 144; // core stride along K of the column-written operands
constexpr uint32_t kSboT = 32 * kLboT;  // 8-row-group stride of those (32 cores of 4 rows)
constexpr int kMaxK2p = 48;     // 2K rounded up to 8; bounded by shared memory (K <= 24)
constexpr int kTmemCols = 256;  // D1 at column 0 (kN1 columns); GEMM2: hi x hi at column 64, the
                                // correction terms at column 64 + K2p (K2p columns each)

struct CpArgs {
    const float* U;       // [ntiles] tile records: kRows x K2p U values in the K-major core
                          // layout, then Et data weights (0 past the last event), padded to 16 bytes
    long long n;          // data events
    int ntiles, K, S, K2p, EW, Et;
    uint32_t tile_bytes;
    int nst;              // U tiles in flight (2, or 1 when two do not fit in shared memory)
    const float* gc;      // [kCV][K][4]: Re g, Im g, Re gdot, Im gdot
    int nv;               // vectors in use (the others are zero and skipped)
    double* rec;          // [grid][kN1 * K2p + kCV] FP64 partial sums per CTA (zeroed by the host)
    int* err;             // [1 + kCV]: shared word, per-vector words
    long long timeout;    // SM cycles per wait
};

__device__ __forceinline__ uint32_t sa(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor: start, LBO, SBO (bytes), no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive 32-bit columns of this thread's TMEM lane; the values are
// valid after tmem_wait() (several loads may be in flight before one wait)
__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// x rounded to the nearest TF32 value (10 mantissa bits; the low 13 bits cleared).
// Both parts of a split x = hi + lo are rounded this way, so the tensor cores
// read them exactly and the dropped remainder has no systematic sign.
__device__ __forceinline__ float tf32_rn(float x)
{
    // adding half a unit of the 10th mantissa bit carries into the exponent
    // when needed, which is round-half-away-from-zero on the magnitude
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// byte offset of element (row, col) in a K-major operand with 16-byte cores
__device__ __forceinline__ uint32_t kmaj(int row, int col, uint32_t lbo, uint32_t sbo)
{
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(col >> 2) * lbo + (uint32_t)(row & 7) * 16 + (uint32_t)(col & 3) * 4;
}

__global__ void __launch_bounds__(kCT, 1) coupling_kernel(const CpArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & (kRows - 1), half = tid >> 7, wq = warp & 3;  // wq: TMEM lane quarter
    const int K = a.K, S = a.S, K2p = a.K2p;
    const uint32_t TB = a.tile_bytes;
    const uint32_t sbo_u = (uint32_t)(K2p / 4) * 128;       // U and B1: 8-row-group stride
    const uint32_t B1B = (uint32_t)kN1 * K2p * 4;
    const uint32_t UTB = (uint32_t)(K2p / 8) * kSboT;
    const uint32_t WTB = (uint32_t)(kN1 / 8) * kSboT;
    const int NST = a.nst;
    unsigned char* uraw[2] = {sm, sm + (NST - 1) * TB};
    unsigned char* ulo = sm + NST * TB;
    unsigned char* b1hi = ulo + TB;
    unsigned char* b1lo = b1hi + B1B;
    unsigned char* uthi = b1lo + B1B;
    unsigned char* utlo = uthi + UTB;
    unsigned char* wthi = utlo + UTB;
    unsigned char* wtlo = wthi + WTB;
    // per-CTA sums of the GEMM2 results as (hi, lo) FP32 pairs (TwoSum): rows n, stride K2p + 1 pairs
    float2* acc = reinterpret_cast<float2*>(wtlo + WTB);
    const int acc_stride = K2p + 1;
    uint64_t* bars = reinterpret_cast<uint64_t*>(acc + (size_t)kN1 * acc_stride);  // tma[2], mma1, mma2
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
    __shared__ int s_abort;
    __shared__ double s_red[kCT / 32][kCV / 2];

    const int G = gridDim.x;
    // ---- GEMM1 B operand from the coupling vectors: row n, column kk of (2K | padding)
    for (int i = tid; i < kN1 * K2p; i += kCT) {
        const int n = i / K2p, kk = i % K2p;
        const int blk = n / kCV, c = n % kCV;
        float v = 0.f;
        if (kk < 2 * K) {
            const int k = kk < K ? kk : kk - K;
            const float* g = a.gc + ((size_t)c * K + k) * 4 + (blk >= 2 ? 2 : 0);  // g or gdot
            const float gr = g[0], gi = g[1];
            // Re part: Ur gr - Ui gi;  Im part: Ur gi + Ui gr
            v = (blk & 1) == 0 ? (kk < K ? gr : -gi) : (kk < K ? gi : gr);
        }
        const float hi = tf32_rn(v);
        const uint32_t off = kmaj(n, kk, 128, sbo_u);
        *reinterpret_cast<float*>(b1hi + off) = hi;
        *reinterpret_cast<float*>(b1lo + off) = tf32_rn(v - hi);
    }
    for (int i = tid; i < kN1 * acc_stride; i += kCT) acc[i] = make_float2(0.f, 0.f);
    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < 4; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&bars[i])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int i = 0; i < NST; ++i) {
            const long long t = blockIdx.x + (long long)i * G;
            if (t < a.ntiles) {
                pwa::tma_load_tile(uraw[i], reinterpret_cast<const unsigned char*>(a.U) + (size_t)t * TB, TB,
                                   &bars[i]);
            }
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tslot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = *tslot;
    const uint32_t tm_lane = (uint32_t)(32 * wq) << 16;
    // instruction descriptors: D f32, A/B tf32, both K-major, N >> 3, M >> 4
    const uint32_t idesc1 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN1 >> 3) << 17) | ((128u >> 4) << 24);
    const uint32_t idesc2 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(K2p >> 3) << 17) |
                            ((uint32_t)(kN1 >> 4) << 24);

    // this thread's row: lane quarter wq, slot j of the quarter's EW events, projection s
    const int j = lane / S, s = lane % S;
    const bool row_used = j < a.EW;
    constexpr int kCH = kCV / 2;  // vectors of this thread: c = kCH half + cc
    float2 slnI[kCH];             // per-thread sums of w ln I as (hi, lo) pairs (TwoSum)
#pragma unroll
    for (int c = 0; c < kCH; ++c) slnI[c] = make_float2(0.f, 0.f);

    int mma1_waits = 0, mma2_commits = 0, mma2_waits = 0;
    auto wait_bar = [&](uint64_t* bar, uint32_t parity) -> bool {
        const long long t0 = clock64();
        while (true) {
            uint32_t done;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(sa(bar)), "r"(parity)
                : "memory");
            if (done) return true;
            if (clock64() - t0 > a.timeout) return false;
        }
    };
    auto wait_mma2 = [&]() -> bool {
        if (mma2_waits == mma2_commits) return true;
        const bool ok = wait_bar(&bars[3], (uint32_t)(mma2_waits & 1));
        ++mma2_waits;
        return ok;
    };
    // Add one tile's GEMM2 results (rows n = 16 warp + lane for lane < 16; both
    // accumulators) into the CTA's (hi, lo) sums.  Each tile is flushed: the
    // tensor cores' FP32 accumulation then spans 16 steps at most.
    auto two_sum = [](float2& p, float x) {
        const float sum = __fadd_rn(p.x, x);
        const float bp = __fsub_rn(sum, p.x);
        const float err = __fadd_rn(__fsub_rn(p.x, __fsub_rn(sum, bp)), __fsub_rn(x, bp));
        p = make_float2(sum, __fadd_rn(p.y, err));
    };
    // The two warps of a lane quarter split the 8-column chunks.
    const int nchunk = K2p / 8, chunk0 = half ? (nchunk + 1) / 2 : 0, chunk1 = half ? nchunk : (nchunk + 1) / 2;
    auto flush_d2 = [&]() {
        tc_fence_after();
        float2* arow = acc + (size_t)(16 * wq + (lane & 15)) * acc_stride;
        for (int ch = chunk0; ch < chunk1; ch += 2) {
            // up to 16 columns of both accumulators in flight, one wait
            uint32_t vh[2][8], vl[2][8];
            const bool two = ch + 1 < chunk1;
            tmem_ld8(tm + tm_lane + 64 + 8 * ch, vh[0]);
            tmem_ld8(tm + tm_lane + 64 + K2p + 8 * ch, vl[0]);
            if (two) {
                tmem_ld8(tm + tm_lane + 64 + 8 * ch + 8, vh[1]);
                tmem_ld8(tm + tm_lane + 64 + K2p + 8 * ch + 8, vl[1]);
            }
            tmem_wait();
            if (lane < 16)
                for (int hh = 0; hh < (two ? 2 : 1); ++hh)
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        two_sum(arow[8 * ch + 8 * hh + q], __uint_as_float(vh[hh][q]));
                        two_sum(arow[8 * ch + 8 * hh + q], __uint_as_float(vl[hh][q]));
                    }
        }
    };

    long long i = 0;
    for (long long t = blockIdx.x; t < a.ntiles; t += G, ++i) {
        const int st = NST == 2 ? (int)(i & 1) : 0;
        bool ok = wait_bar(&bars[st], (uint32_t)((NST == 2 ? i >> 1 : i) & 1));
        ok = wait_mma2() && ok;  // the previous GEMM2 has read UT and Wt
        if (!ok) s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        if (i > 0) flush_d2();   // the previous tile's GEMM2 results
        // ---- split this thread's half of its U row: hi in place, lo beside it, both
        //      transposed for GEMM2; the event weight is read before the stage is refilled
        unsigned char* ub = uraw[st];
        const float wgt_tile = reinterpret_cast<const float*>(ub + (size_t)kRows * K2p * 4)[wq * a.EW + min(j, a.EW - 1)];
        const int nq = K2p / 4, q0 = half ? nq / 2 : 0, q1 = half ? nq : nq / 2;
        for (int q = q0; q < q1; ++q) {
            const uint32_t off = kmaj(row, 4 * q, 128, sbo_u);
            const float4 x = *reinterpret_cast<const float4*>(ub + off);
            const float4 h = make_float4(tf32_rn(x.x), tf32_rn(x.y), tf32_rn(x.z), tf32_rn(x.w));
            const float4 l = make_float4(tf32_rn(x.x - h.x), tf32_rn(x.y - h.y), tf32_rn(x.z - h.z), tf32_rn(x.w - h.w));
            *reinterpret_cast<float4*>(ub + off) = h;
            *reinterpret_cast<float4*>(ulo + off) = l;
            const float hv[4] = {h.x, h.y, h.z, h.w}, lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t o2 = kmaj(4 * q + e, row, kLboT, kSboT);
                *reinterpret_cast<float*>(uthi + o2) = hv[e];
                *reinterpret_cast<float*>(utlo + o2) = lv[e];
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- GEMM1: D1[r][n] = sum_kk U[r][kk] B1[n][kk]  (three-term TF32 split)
        if (tid == 0) {
            for (int ks = 0; ks < K2p / 8; ++ks) {
                const uint64_t ah = sdesc(sa(ub) + ks * 256, 128, sbo_u), al = sdesc(sa(ulo) + ks * 256, 128, sbo_u);
                const uint64_t bh = sdesc(sa(b1hi) + ks * 256, 128, sbo_u), bl = sdesc(sa(b1lo) + ks * 256, 128, sbo_u);
                mma_tf32(tm, ah, bh, idesc1, ks > 0);
                mma_tf32(tm, ah, bl, idesc1, 1);
                mma_tf32(tm, al, bh, idesc1, 1);
            }
            mma_commit(&bars[2]);
        }
        ok = wait_bar(&bars[2], (uint32_t)(mma1_waits & 1));
        ++mma1_waits;
        if (!ok) s_abort = 1;
        tc_fence_after();
        // the stage is free: thread 0 refills it with the tile two steps ahead
        if (tid == 0 && ok) {
            const long long tn = t + (long long)NST * G;
            if (tn < a.ntiles) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                pwa::tma_load_tile(ub, reinterpret_cast<const unsigned char*>(a.U) + (size_t)tn * TB, TB, &bars[st]);
            }
        }
        // ---- epilogue: this row's coherent sums for this thread's vectors
        //      (columns Re A, Im A, Re Adot, Im Adot of c = kCH half + cc)
        float d1[4][kCH];
        {
            uint32_t v[4][8];
#pragma unroll
            for (int q = 0; q < 4; ++q) tmem_ld8(tm + tm_lane + q * kCV + kCH * half, v[q]);
            tmem_wait();
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int cc = 0; cc < kCH; ++cc) d1[q][cc] = __uint_as_float(v[q][cc]);
        }
        const long long ev = t * a.Et + (long long)wq * a.EW + j;
        const bool valid = row_used && ev < a.n;
        const float wgt = valid ? wgt_tile : 0.f;
        const int base = S * j;  // first lane of this row's event
#pragma unroll
        for (int cc = 0; cc < kCH; ++cc) {
            const int c = kCH * half + cc;
            const float Ar = d1[0][cc], Ai = d1[1][cc], Dr = d1[2][cc], Di = d1[3][cc];
            const float ip = fmaf(Ar, Ar, Ai * Ai), dp = 2.f * fmaf(Ar, Dr, Ai * Di);
            float I = 0.f, Id = 0.f;
            for (int q = 0; q < S; ++q) {
                I += __shfl_sync(0xffffffffu, ip, base + q);
                Id += __shfl_sync(0xffffffffu, dp, base + q);
            }
            float wa = 0.f, wb = 0.f;
            if (valid && c < a.nv) {
                if (I > 0.f && I < INFINITY) {
                    const float rI = __frcp_rn(I);
                    wa = wgt * rI;
                    wb = wa * Id * rI;
                    if (s == 0) two_sum(slnI[cc], wgt * logf(I));
                } else if (s == 0) {
                    atomicOr(a.err, pwa::ERR_NONFINITE);
                    atomicOr(a.err + 1 + c, pwa::ERR_NONFINITE);
                }
            }
            const float wv[4] = {wa * Ar, wa * Ai, fmaf(wa, Dr, -wb * Ar), fmaf(wa, Di, -wb * Ai)};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float hi = tf32_rn(wv[q]);
                const uint32_t off = kmaj(q * kCV + c, row, kLboT, kSboT);
                *reinterpret_cast<float*>(wthi + off) = hi;
                *reinterpret_cast<float*>(wtlo + off) = tf32_rn(wv[q] - hi);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (s_abort) break;
        // ---- GEMM2: D2[n][kk] += sum_r Wt[n][r] UT[kk][r]
        if (tid == 0) {
            for (int ks = 0; ks < kRows / 8; ++ks) {
                const uint64_t ah = sdesc(sa(wthi) + ks * 2 * kLboT, kLboT, kSboT),
                               al = sdesc(sa(wtlo) + ks * 2 * kLboT, kLboT, kSboT);
                const uint64_t bh = sdesc(sa(uthi) + ks * 2 * kLboT, kLboT, kSboT),
                               bl = sdesc(sa(utlo) + ks * 2 * kLboT, kLboT, kSboT);
                mma_tf32(tm + 64, ah, bh, idesc2, ks > 0);
                mma_tf32(tm + 64 + K2p, ah, bl, idesc2, ks > 0);
                mma_tf32(tm + 64 + K2p, al, bh, idesc2, 1);
            }
            mma_commit(&bars[3]);
        }
        ++mma2_commits;
    }
    // ---- finish: the last GEMM2, its flush, the CTA's sums of w ln I
    __syncthreads();
    if (!s_abort) {
        // every thread waits; the flush (warp-collective TMEM loads) is decided together
        if (__syncthreads_or(!wait_mma2())) s_abort = 1;
        if (!s_abort && mma2_commits > 0) flush_d2();
    }
    if (s_abort) {
        if (tid == 0) atomicOr(a.err, pwa::ERR_TIMEOUT);
    } else {
        __syncthreads();
        double* rq = a.rec + (size_t)blockIdx.x * (kN1 * K2p + kCV);
        for (int q = tid; q < kN1 * K2p; q += kCT) {
            const float2 p = acc[(size_t)(q / K2p) * acc_stride + q % K2p];
            rq[q] = (double)p.x + (double)p.y;
        }
        double* rec = rq + (size_t)kN1 * K2p;
#pragma unroll
        for (int cc = 0; cc < kCH; ++cc) {
            double v = (double)slnI[cc].x + (double)slnI[cc].y;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) s_red[warp][cc] = v;
        }
        __syncthreads();
        if (tid < kCV) {
            const int h = tid / kCH, cc = tid % kCH;  // vector tid: warps 4 h .. 4 h + 3
            rec[tid] = ((s_red[4 * h][cc] + s_red[4 * h + 1][cc]) + s_red[4 * h + 2][cc]) + s_red[4 * h + 3][cc];
        }
    }
    // drain: a timed-out CTA waits (bounded) for its own copies and MMAs before freeing TMEM
    if (s_abort && tid == 0) {
        (void)wait_mma2();
        (void)wait_bar(&bars[2], (uint32_t)(mma1_waits & 1));
        for (int q = 0; q < NST; ++q) (void)wait_bar(&bars[q], (uint32_t)(((i + q) / NST) & 1));
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kTmemCols));
}

// ---------------------------------------------------------------------------
// preparation: U tiles of the data events, the MC integral matrix
// ---------------------------------------------------------------------------

struct CpRes {
    float m2hi, m2lo, mg, mg2;
    int ch;
};

__device__ __forceinline__ float2 bw_f32(const CpRes& r, float m2)
{
    const float d = (r.m2hi - m2) + r.m2lo;
    const float q = 1.0f / fmaf(d, d, r.mg2);
    return make_float2(d * q, r.mg * q);
}

// U tiles: row (warp w, slot j, projection s) of tile t is event t Et + w EW + j
__global__ void coupling_u_kernel(const float2* __restrict__ F, const float* __restrict__ m2,
                                  const float* __restrict__ w, long long n, int K, int S, int K2p, int EW, int Et,
                                  int ntiles, long long tile_floats, const CpRes* __restrict__ res,
                                  float* __restrict__ U)
{
    const uint32_t sbo = (uint32_t)(K2p / 4) * 128;
    const long long per_tile = (long long)kRows * K2p;
    const long long total = (long long)ntiles * per_tile;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long t = i / per_tile;
        const int rr = (int)(i % per_tile);
        const int r = rr / K2p, kk = rr % K2p;
        const int wv = r >> 5, ln = r & 31, j = ln / S, s = ln % S;
        const long long e = t * Et + (long long)wv * EW + j;
        float v = 0.f;
        if (j < EW && e < n && kk < 2 * K) {
            const int k = kk < K ? kk : kk - K;
            const CpRes rp = res[k];
            const float2 b = bw_f32(rp, m2[(size_t)rp.ch * n + e]);
            const float2 f = F[((size_t)e * K + k) * S + s];
            v = kk < K ? b.x * f.x - b.y * f.y : b.x * f.y + b.y * f.x;
        }
        const uint32_t off = (uint32_t)(r >> 3) * sbo + (uint32_t)(kk >> 2) * 128 + (uint32_t)(r & 7) * 16 +
                             (uint32_t)(kk & 3) * 4;
        U[t * tile_floats + off / 4] = v;
    }
    // the weights after the U block of each record (zero past the last event and in the padding)
    const int wpad = (int)(tile_floats - per_tile);
    const long long nw = (long long)ntiles * wpad;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nw;
         i += (long long)gridDim.x * blockDim.x) {
        const long long t = i / wpad;
        const int el = (int)(i % wpad);
        const long long e = t * Et + el;
        U[t * tile_floats + per_tile + el] = (el < Et && e < n) ? (w ? w[e] : 1.f) : 0.f;
    }
}

// Phi partial sums over event chunks: block b sums its events; thread p owns
// pairs (k, k') = p, p + blockDim, ...; per-thread FP32 sums over 64 events are
// added into FP64 block totals
constexpr int kPhiThreads = 256;
constexpr int kPhiChunk = 2048;

__global__ void __launch_bounds__(kPhiThreads) coupling_phi_kernel(const float2* __restrict__ F,
                                                                   const float* __restrict__ m2, long long n, int K,
                                                                   int S, const CpRes* __restrict__ res,
                                                                   double* __restrict__ part)
{
    extern __shared__ float2 u_s[];  // [K][S] of the current event
    const int KK = K * K;
    const int npair = (KK + kPhiThreads - 1) / kPhiThreads;
    double acc[2 * 8];  // up to 8 pairs per thread (K <= 45)
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    float fa[16];
    for (int q = 0; q < 16; ++q) fa[q] = 0.f;
    const long long e0 = (long long)blockIdx.x * kPhiChunk, e1 = min(n, e0 + kPhiChunk);
    int cnt = 0;
    for (long long e = e0; e < e1; ++e) {
        __syncthreads();
        for (int i = threadIdx.x; i < K * S; i += kPhiThreads) {
            const int k = i / S, s = i % S;
            const CpRes rp = res[k];
            const float2 b = bw_f32(rp, m2[(size_t)rp.ch * n + e]);
            const float2 f = F[((size_t)e * K + k) * S + s];
            u_s[i] = make_float2(b.x * f.x - b.y * f.y, b.x * f.y + b.y * f.x);
        }
        __syncthreads();
        for (int q = 0; q < npair; ++q) {
            const int p = threadIdx.x + q * kPhiThreads;
            if (p >= KK) break;
            const int k = p / K, kp = p % K;
            float re = 0.f, im = 0.f;
            for (int s = 0; s < S; ++s) {
                const float2 x = u_s[k * S + s], y = u_s[kp * S + s];
                // conj(x) y
                re = fmaf(x.x, y.x, fmaf(x.y, y.y, re));
                im = fmaf(x.x, y.y, fmaf(-x.y, y.x, im));
            }
            fa[2 * q] += re;
            fa[2 * q + 1] += im;
        }
        if (++cnt == 64) {
            for (int q = 0; q < 16; ++q) {
                acc[q] += (double)fa[q];
                fa[q] = 0.f;
            }
            cnt = 0;
        }
    }
    for (int q = 0; q < npair; ++q) {
        const int p = threadIdx.x + q * kPhiThreads;
        if (p >= KK) break;
        part[((size_t)blockIdx.x * KK + p) * 2] = acc[2 * q] + (double)fa[2 * q];
        part[((size_t)blockIdx.x * KK + p) * 2 + 1] = acc[2 * q + 1] + (double)fa[2 * q + 1];
    }
}

__global__ void coupling_phi_reduce(const double* __restrict__ part, int nblocks, int KK, double* __restrict__ phi)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * KK; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * 2 * KK + i];
        phi[i] = s;
    }
}

// ---------------------------------------------------------------------------
// combine (FP64): CTA partials + integral matrix -> NLL, gradient and H v in
// the coupling parameters (Eqs. 3, 6, 7 with the mass and width terms absent)
// ---------------------------------------------------------------------------

struct CpVec {  // per vector and resonance: rho, phi, Re g, Im g, Re gdot, Im gdot, v_rho, v_phi
    double v[8];
};

__global__ void coupling_combine_kernel(const double* __restrict__ rec, int nrec, int K, int K2p,
                                        const double* __restrict__ phi, const CpVec* __restrict__ vec,
                                        const pwa::ResParam* __restrict__ res, int Pc, double Nd, double Nmc,
                                        int nvec, double* __restrict__ out)
{
    const int c = blockIdx.x;
    if (c >= nvec) return;
    extern __shared__ double sh[];  // [K][8] partials, then 4 scalars
    const int reclen = kN1 * K2p + kCV;
    double* part = sh;
    double* scal = sh + 8 * K;
    const int k = threadIdx.x;
    double2 Q1d = make_double2(0, 0), P1d = make_double2(0, 0), Pg = make_double2(0, 0), Pd = make_double2(0, 0);
    if (k < K) {
        // data sums over the CTAs in fixed order
        double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int b = 0; b < nrec; ++b) {
            const double* r = rec + (size_t)b * reclen;
            q[0] += r[(size_t)c * K2p + k];
            q[1] += r[(size_t)c * K2p + K + k];
            q[2] += r[(size_t)(kCV + c) * K2p + k];
            q[3] += r[(size_t)(kCV + c) * K2p + K + k];
            q[4] += r[(size_t)(2 * kCV + c) * K2p + k];
            q[5] += r[(size_t)(2 * kCV + c) * K2p + K + k];
            q[6] += r[(size_t)(3 * kCV + c) * K2p + k];
            q[7] += r[(size_t)(3 * kCV + c) * K2p + K + k];
        }
        // sum_r (a Ar + i ... ) U: Q1 = sum a conj(A) U, P1 = sum (a conj(Adot) - b conj(A)) U
        Q1d = make_double2(q[0] + q[3], q[1] - q[2]);
        P1d = make_double2(q[4] + q[7], q[5] - q[6]);
        // MC via the integral matrix: (Phi g)_k, (Phi gdot)_k
        const CpVec* vv = vec + (size_t)c * K;
        for (int kp = 0; kp < K; ++kp) {
            const double pr = phi[2 * (k * K + kp)], pi = phi[2 * (k * K + kp) + 1];
            const double gr = vv[kp].v[2], gi = vv[kp].v[3], dr = vv[kp].v[4], di = vv[kp].v[5];
            Pg.x += pr * gr - pi * gi;
            Pg.y += pr * gi + pi * gr;
            Pd.x += pr * dr - pi * di;
            Pd.y += pr * di + pi * dr;
        }
        const double gr = vv[k].v[2], gi = vv[k].v[3];
        part[8 * k + 0] = gr * Pg.x + gi * Pg.y;        // Re conj(g_k) (Phi g)_k
        part[8 * k + 1] = 2.0 * (gr * Pd.x + gi * Pd.y);  // 2 Re conj(g_k) (Phi gdot)_k
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double Gm = 0.0, Gd = 0.0, sln = 0.0;
        for (int kk = 0; kk < K; ++kk) {
            Gm += part[8 * kk + 0];
            Gd += part[8 * kk + 1];
        }
        for (int b = 0; b < nrec; ++b) sln += rec[(size_t)b * reclen + (size_t)kN1 * K2p + c];
        scal[0] = Gm;
        scal[1] = Gd;
        out[(size_t)c * (1 + 2 * Pc)] = -sln + Nd * log(Gm / Nmc);
    }
    __syncthreads();
    if (k >= K) return;
    const double Gm = scal[0], Gd = scal[1];
    const CpVec v = vec[(size_t)c * K + k];
    const double cs = cos(v.v[1]), sn = sin(v.v[1]);
    const double2 E1 = make_double2(cs, sn), g1 = make_double2(v.v[2], v.v[3]);
    auto mul = [](double2 x, double2 y) { return make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x); };
    auto ii = [](double2 x) { return make_double2(-x.y, x.x); };
    // MC sums as the adjoint sums of the data: sum_mc D_k = conj((Phi g)_k), sum_mc Ddot_k = conj((Phi gdot)_k)
    const double2 Q1m = make_double2(Pg.x, -Pg.y), P1m = make_double2(Pd.x, -Pd.y);
    const double vr = v.v[6], vp = v.v[7];
    const double2 kap[2] = {E1, ii(g1)};
    const double2 lam[2] = {make_double2(vp * -E1.y, vp * E1.x),
                            make_double2(vr * -E1.y - vp * g1.x, vr * E1.x - vp * g1.y)};
    double* o = out + (size_t)c * (1 + 2 * Pc);
    for (int jj = 0; jj < 2; ++jj) {
        const int idx = res[k].idx[jj];
        if (idx < 0) continue;
        const double gD = 2.0 * mul(kap[jj], Q1d).x, gM = 2.0 * mul(kap[jj], Q1m).x;
        o[1 + idx] = -gD + Nd * gM / Gm;
        const double hD = 2.0 * (mul(kap[jj], P1d).x + mul(lam[jj], Q1d).x);
        const double hM = 2.0 * (mul(kap[jj], P1m).x + mul(lam[jj], Q1m).x);
        o[1 + Pc + idx] = -hD + Nd * (hM / Gm - gM * Gd / (Gm * Gm));
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// the coupling object
// ---------------------------------------------------------------------------

struct pwa_coupling {
    pwa_handle* h = nullptr;
    int K = 0, S = 0, Pc = 0, K2p = 0, EW = 0, Et = 0, ntiles = 0, grid = 0;
    uint32_t tile_bytes = 0;
    int nst = 2;
    size_t smem = 0;
    std::vector<double> par;   // rho, phi, M, Gamma per resonance (the fixed values)
    std::vector<int> ridx;     // theta index of rho_k, phi_k (-1 when fixed)
    float* d_U = nullptr;       // tile records: U block, then the weights
    double* d_phi = nullptr;   // [K][K] complex
    std::vector<double> phi;   // host copy
    // per launch
    float* d_gc = nullptr;     // [kCV][K][4]
    CpVec* d_vec = nullptr;    // [kCV][K]
    double* d_rec = nullptr;   // [grid][kN1 K2p + kCV]
    double* d_out = nullptr;   // [kCV][1 + 2 Pc]
    int* d_err = nullptr;      // [1 + kCV]
    double* h_pin = nullptr;   // pinned: outputs, error words
};

namespace {

pwa_status cp_cuda(pwa_coupling* cp, cudaError_t e, const char* what)
{
    return pwa::cuda_error(cp->h, e, what);
}

// Launch the tensor-core pass for nv (<= kCV) vectors and the FP64 combine.
pwa_status cp_launch(pwa_coupling* cp, int nv, const double* theta_c, const double* v_c)
{
    pwa_handle* h = cp->h;
    const int K = cp->K, Pc = cp->Pc;
    std::vector<float> gc((size_t)kCV * K * 4, 0.f);
    std::vector<CpVec> vec((size_t)kCV * K);
    for (int c = 0; c < kCV; ++c)
        for (int k = 0; k < K; ++k) {
            CpVec& q = vec[(size_t)c * K + k];
            std::memset(&q, 0, sizeof(q));
            if (c >= nv) continue;
            const int ir = cp->ridx[2 * k], ip = cp->ridx[2 * k + 1];
            const double rho = ir >= 0 ? theta_c[(size_t)c * Pc + ir] : cp->par[k];
            const double ph = ip >= 0 ? theta_c[(size_t)c * Pc + ip] : cp->par[K + k];
            const double vr = (v_c && ir >= 0) ? v_c[(size_t)c * Pc + ir] : 0.0;
            const double vp = (v_c && ip >= 0) ? v_c[(size_t)c * Pc + ip] : 0.0;
            const double cs = std::cos(ph), sn = std::sin(ph);
            const double gr = rho * cs, gi = rho * sn;
            // gdot = v_rho e^{i phi} + v_phi i g
            const double dr = vr * cs - vp * gi, di = vr * sn + vp * gr;
            q.v[0] = rho;
            q.v[1] = ph;
            q.v[2] = gr;
            q.v[3] = gi;
            q.v[4] = dr;
            q.v[5] = di;
            q.v[6] = vr;
            q.v[7] = vp;
            float* g = &gc[((size_t)c * K + k) * 4];
            g[0] = (float)gr;
            g[1] = (float)gi;
            g[2] = (float)dr;
            g[3] = (float)di;
        }
    cudaStream_t s = h->stream;
    cudaError_t e = cudaMemcpyAsync(cp->d_gc, gc.data(), gc.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cp->d_vec, vec.data(), vec.size() * sizeof(CpVec), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(cp->d_rec, 0, sizeof(double) * (size_t)cp->grid * (kN1 * cp->K2p + kCV), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cp->d_err, 0, sizeof(int) * (1 + kCV), s);
    if (e != cudaSuccess) return cp_cuda(cp, e, "coupling upload");
    CpArgs a;
    a.U = cp->d_U;
    a.n = h->n[0];
    a.ntiles = cp->ntiles;
    a.K = K;
    a.S = cp->S;
    a.K2p = cp->K2p;
    a.EW = cp->EW;
    a.Et = cp->Et;
    a.tile_bytes = cp->tile_bytes;
    a.nst = cp->nst;
    a.gc = cp->d_gc;
    a.nv = nv;
    a.rec = cp->d_rec;
    a.err = cp->d_err;
    a.timeout = h->timeout_cycles;
    coupling_kernel<<<cp->grid, kCT, cp->smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cp_cuda(cp, e, "coupling kernel launch");
    coupling_combine_kernel<<<nv, std::max(32, (K + 31) / 32 * 32), sizeof(double) * (8 * K + 4), s>>>(
        cp->d_rec, cp->grid, K, cp->K2p, cp->d_phi, cp->d_vec, h->d_res, Pc, h->Nd, h->Nmc, nv, cp->d_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cp_cuda(cp, e, "coupling combine launch");
    return PWA_OK;
}

}  // namespace

extern "C" {

pwa_status pwa_coupling_create(pwa_handle* h, const double* theta, pwa_coupling** out)
{
    if (!h || !out) return PWA_EINVAL;
    *out = nullptr;
    h->err.clear();
    if (!theta) return pwa::set_error(h, PWA_EINVAL, "theta must not be NULL");
    if (h->broken) return pwa::set_error(h, PWA_ETIMEOUT, "handle is unusable after a device-side timeout");
    const int K = h->K, S = h->S, P = h->P;
    for (int i = 0; i < P; ++i)
        if (!std::isfinite(theta[i])) return pwa::set_error(h, PWA_EINVAL, "theta must be finite");
    const int K2p = (2 * K + 7) / 8 * 8;
    if (K2p > kMaxK2p)
        return pwa::set_error(h, PWA_EINVAL, "the coupling sub-problem supports K <= " + std::to_string(kMaxK2p / 2) +
                                                 " (shared memory of one tile)");
    auto* cp = new (std::nothrow) pwa_coupling();
    if (!cp) return pwa::set_error(h, PWA_ENOMEM, "host allocation failed");
    cp->h = h;
    cp->K = K;
    cp->S = S;
    cp->K2p = K2p;
    cp->EW = 32 / S;
    cp->Et = 4 * cp->EW;
    const int Etp = (cp->Et + 3) / 4 * 4;  // weights padded to 16 bytes
    cp->tile_bytes = (uint32_t)(kRows * K2p + Etp) * 4;
    cp->ntiles = (int)((h->n[0] + cp->Et - 1) / cp->Et);
    // parameter values: theta where free, the table where fixed
    cp->par.assign(4 * K, 0.0);
    cp->ridx.assign(2 * K, -1);
    int Pc = 0;
    for (int k = 0; k < K; ++k) {
        const pwa::ResParam& r = h->res[k];
        for (int q = 0; q < 4; ++q) cp->par[q * K + k] = r.idx[q] >= 0 ? theta[r.idx[q]] : r.fixed[q];
        cp->ridx[2 * k] = r.idx[0];
        cp->ridx[2 * k + 1] = r.idx[1];
        for (int q = 0; q < 2; ++q)
            if (r.idx[q] >= 0) Pc = std::max(Pc, r.idx[q] + 1);
    }
    cp->Pc = Pc;
    // Breit-Wigner constants in FP32 (M^2 as a hi/lo pair), as the fused pass forms them
    std::vector<CpRes> rs(K);
    for (int k = 0; k < K; ++k) {
        const double M = cp->par[2 * K + k], Gw = cp->par[3 * K + k];
        const double M2 = M * M, MG = M * Gw;
        rs[k].m2hi = (float)M2;
        rs[k].m2lo = (float)(M2 - (double)rs[k].m2hi);
        rs[k].mg = (float)MG;
        rs[k].mg2 = (float)(MG * MG);
        rs[k].ch = h->res[k].channel;
    }
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    auto smem_for = [&](int nst) {
        return (size_t)(nst + 1) * cp->tile_bytes + 2 * (size_t)kN1 * K2p * 4 + 2 * (size_t)(K2p / 8) * kSboT +
               2 * (size_t)(kN1 / 8) * kSboT + (size_t)kN1 * (K2p + 1) * 8 + 64;
    };
    cp->nst = smem_for(2) + 2048 <= (size_t)optin ? 2 : 1;
    cp->smem = smem_for(cp->nst);
    pwa_status st = PWA_OK;
    cudaError_t e = cudaSuccess;
    CpRes* d_rs = nullptr;
    double* d_part = nullptr;
    const long long nmc = h->n[1];
    const int phi_blocks = (int)((nmc + kPhiChunk - 1) / kPhiChunk);
    do {
        if (cp->smem + 2048 > (size_t)optin) {
            st = pwa::set_error(h, PWA_EINVAL, "the coupling kernel does not fit in shared memory");
            break;
        }
        e = cudaFuncSetAttribute(coupling_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cp->smem);
        if (e != cudaSuccess) break;
        cp->grid = std::max(1, std::min(sms, cp->ntiles));
        const size_t ufloats = (size_t)cp->ntiles * (cp->tile_bytes / 4);
        if ((e = cudaMalloc(&cp->d_U, ufloats * sizeof(float))) != cudaSuccess) break;
        if ((e = cudaMalloc(&cp->d_phi, sizeof(double) * 2 * K * K)) != cudaSuccess) break;
        if ((e = cudaMalloc(&cp->d_gc, sizeof(float) * kCV * K * 4)) != cudaSuccess) break;
        if ((e = cudaMalloc(&cp->d_vec, sizeof(CpVec) * kCV * K)) != cudaSuccess) break;
        if ((e = cudaMalloc(&cp->d_rec, sizeof(double) * (size_t)cp->grid * (kN1 * K2p + kCV))) != cudaSuccess) break;
        if ((e = cudaMalloc(&cp->d_out, sizeof(double) * kCV * (1 + 2 * Pc))) != cudaSuccess) break;
        if ((e = cudaMalloc(&cp->d_err, sizeof(int) * (1 + kCV))) != cudaSuccess) break;
        if ((e = cudaMallocHost(&cp->h_pin, sizeof(double) * (kCV * (1 + 2 * Pc) + kCV + 2))) != cudaSuccess) break;
        if ((e = cudaMalloc(&d_rs, sizeof(CpRes) * K)) != cudaSuccess) break;
        if ((e = cudaMalloc(&d_part, sizeof(double) * 2 * K * K * (size_t)std::max(phi_blocks, 1))) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(d_rs, rs.data(), sizeof(CpRes) * K, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess)
            break;
        const long long uthreads = (long long)ufloats;
        const int ublocks = (int)std::min<long long>((uthreads + 255) / 256, 65535LL * 8);
        coupling_u_kernel<<<std::max(ublocks, 1), 256, 0, h->stream>>>(
            reinterpret_cast<const float2*>(h->d_F[0]), h->d_m2[0], h->d_w, h->n[0], K, S, K2p, cp->EW, cp->Et,
            cp->ntiles, (long long)(cp->tile_bytes / 4), d_rs, cp->d_U);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if (K * K > 8 * kPhiThreads) {
            st = pwa::set_error(h, PWA_EINVAL, "K too large for the integral-matrix kernel");
            break;
        }
        coupling_phi_kernel<<<std::max(phi_blocks, 1), kPhiThreads, sizeof(float2) * K * S, h->stream>>>(
            reinterpret_cast<const float2*>(h->d_F[1]), h->d_m2[1], nmc, K, S, d_rs, d_part);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        coupling_phi_reduce<<<(2 * K * K + 255) / 256, 256, 0, h->stream>>>(d_part, phi_blocks, K * K, cp->d_phi);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        cp->phi.resize(2 * K * K);
        if ((e = cudaMemcpyAsync(cp->phi.data(), cp->d_phi, sizeof(double) * 2 * K * K, cudaMemcpyDeviceToHost,
                                 h->stream)) != cudaSuccess)
            break;
        e = cudaStreamSynchronize(h->stream);
    } while (false);
    if (d_rs) cudaFree(d_rs);
    if (d_part) cudaFree(d_part);
    if (e != cudaSuccess && st == PWA_OK) st = pwa::cuda_error(h, e, "coupling preparation");
    if (st != PWA_OK) {
        pwa_coupling_destroy(cp);
        return st;
    }
    *out = cp;
    return PWA_OK;
}

int pwa_coupling_num_params(const pwa_coupling* cp) { return cp ? cp->Pc : -1; }

pwa_status pwa_coupling_integral_matrix(const pwa_coupling* cp, double* phi)
{
    if (!cp || !phi) return PWA_EINVAL;
    std::memcpy(phi, cp->phi.data(), sizeof(double) * cp->phi.size());
    return PWA_OK;
}

pwa_status pwa_coupling_eval(pwa_coupling* cp, int C, const double* theta_c, const double* v_c, double* nll,
                             double* grad, double* hv)
{
    if (!cp) return PWA_EINVAL;
    pwa_handle* h = cp->h;
    h->err.clear();
    if (C < 1 || !theta_c || !nll) return pwa::set_error(h, PWA_EINVAL, "C >= 1, theta_c and nll are required");
    if (hv && !v_c) return pwa::set_error(h, PWA_EINVAL, "v is required for hv");
    const int Pc = cp->Pc;
    for (size_t i = 0; i < (size_t)C * Pc; ++i)
        if (!std::isfinite(theta_c[i]) || (v_c && !std::isfinite(v_c[i])))
            return pwa::set_error(h, PWA_EINVAL, "theta_c and v must be finite");
    std::vector<double> res((size_t)C * (1 + 2 * Pc));
    std::vector<int> errw(C);
    pwa_status st = pwa::coupling_eval_rows(cp, C, theta_c, v_c, res.data(), errw.data());
    if (st != PWA_OK) return st;
    for (int c = 0; c < C; ++c)
        if (errw[c])
            return pwa::set_error(h, PWA_ENONFINITE, "coupling vector " + std::to_string(c) +
                                                         ": non-finite or non-positive data intensity");
    for (int c = 0; c < C; ++c) {
        const double* r = res.data() + (size_t)c * (1 + 2 * Pc);
        nll[c] = r[0];
        if (grad) std::memcpy(grad + (size_t)c * Pc, r + 1, sizeof(double) * Pc);
        if (hv) std::memcpy(hv + (size_t)c * Pc, r + 1 + Pc, sizeof(double) * Pc);
    }
    return PWA_OK;
}

void pwa_coupling_destroy(pwa_coupling* cp)
{
    if (!cp) return;
    if (cp->h && cp->h->stream) cudaStreamSynchronize(cp->h->stream);
    void* ptrs[] = {cp->d_U, cp->d_phi, cp->d_gc, cp->d_vec, cp->d_rec, cp->d_out, cp->d_err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (cp->h_pin) cudaFreeHost(cp->h_pin);
    cudaGetLastError();
    delete cp;
}

}  // extern "C"

namespace pwa {

pwa_handle* coupling_handle(const pwa_coupling* cp) { return cp->h; }

pwa_status coupling_eval_rows(pwa_coupling* cp, int nb, const double* theta, const double* v, double* out, int* errw)
{
    pwa_handle* h = cp->h;
    if (h->broken) return set_error(h, PWA_ETIMEOUT, "handle is unusable after a device-side timeout");
    const int Pc = cp->Pc;
    for (int c0 = 0; c0 < nb; c0 += kCV) {
        const int nv = std::min(kCV, nb - c0);
        pwa_status st = cp_launch(cp, nv, theta + (size_t)c0 * Pc, v ? v + (size_t)c0 * Pc : nullptr);
        if (st != PWA_OK) return st;
        const size_t ow = (size_t)nv * (1 + 2 * Pc);
        int* ew = reinterpret_cast<int*>(cp->h_pin + (size_t)kCV * (1 + 2 * Pc));
        cudaError_t e = cudaMemcpyAsync(cp->h_pin, cp->d_out, sizeof(double) * ow, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ew, cp->d_err, sizeof(int) * (1 + kCV), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_error(h, e, "coupling results");
        if (ew[0] & ERR_TIMEOUT) {
            h->broken = true;
            return set_error(h, PWA_ETIMEOUT, "a coupling tile or MMA did not complete within the wait limit");
        }
        std::memcpy(out + (size_t)c0 * (1 + 2 * Pc), cp->h_pin, sizeof(double) * ow);
        for (int c = 0; c < nv; ++c) errw[c0 + c] = ew[1 + c];
    }
    return PWA_OK;
}

}  // namespace pwa
