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
// Both GEMMs run on tcgen05 (kind::f16, BF16 operands, FP32 accumulation) with
// every FP32 operand split into three BF16 parts, x = x0 + x1 + x2 (each the
// nearest BF16 of what the previous parts leave), which represents it
// exactly; a b is taken as the six products with i + j <= 2 (the others are
// below FP32 resolution).  The x0 y0 products and the five correction products
// go to separate accumulators in tensor memory (the tensor cores' FP32
// accumulation of terms of very different size loses the small ones), and
// GEMM2's are flushed every tile into compensated FP32 sums (TwoSum).  U is stored split, twice: once as GEMM1's A operand and once
// transposed as GEMM2's B operand, so that a tile needs no conversion work.
// Operands use the canonical K-major layout without swizzle: 8-row x 16-byte
// core matrices (8 BF16 along K), LBO = stride between cores along K, SBO =
// stride between 8-row groups.  The W operand, written column-wise by the
// epilogue, uses a 144-byte core stride so that a warp's stores spread over
// 32 banks.
//
// Pipeline of one CTA (8 warps, one per SM): GEMM1 of tile i + 1 runs while
// the threads work on tile i (two GEMM1 accumulators); GEMM2 of tile i runs
// while the next GEMM1 is waited for; U tiles and their transposed copies are
// double-buffered and fetched by TMA bulk copies two tiles ahead.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pwa_internal.h"
#include "tcgen05.cuh"

namespace {

constexpr int kCT = 256;        // epilogue threads per CTA: threads r and r + 128 share row r of a
                                // tile; one more warp issues the copies and the MMAs
constexpr int kRows = 128;      // (event, projection) rows per tile
constexpr int kCV = 16;         // coupling vectors per launch
constexpr int kCH = kCV / 2;    // vectors per thread
constexpr int kN1 = 4 * kCV;    // GEMM1 columns: Re A, Im A, Re Adot, Im Adot of every vector
constexpr int kParts = 3;       // BF16 parts per FP32 operand
constexpr uint32_t kLboW = 144; // core stride along K of the W operand (16 bytes of padding per core)
constexpr uint32_t kSboW = (kRows / 8) * kLboW;  // its 8-row-group stride
constexpr int kMaxK2p = 48;     // 2K rounded up to 16; bounded by shared memory (K <= 24)
constexpr int kTmemCols = 512;  // GEMM1 x0 y0 (x 2 tiles) at 0 and 64, its corrections at 128 and 192;
                                // GEMM2 x0 y0 in four accumulators (K steps ks mod 4) at 256 + 48 j,
                                // its corrections at 448
constexpr int kNBars = 8;       // tmaA[2], tmaB[2], g1[2], g2, wready

struct CpArgs {
    const unsigned char* U;  // [ntiles] tile records (layout below)
    long long n;             // data events
    int ntiles, K, S, K2p, EW, Et;
    uint32_t rec_bytes;      // bytes of one tile record
    uint32_t a_bytes;        // split U (GEMM1 operand) + weights: the first TMA copy
    uint32_t b_bytes;        // split transposed U (GEMM2 operand): the second TMA copy
    const float* gc;         // [kCV][K][4]: Re g, Im g, Re gdot, Im gdot
    int nv;                  // vectors in use (the others are zero and skipped)
    double* rec;             // [grid][kN1 * K2p + kCV] FP64 partial sums per CTA
    int* err;                // [1 + kCV]: shared word, per-vector words
    long long timeout;       // SM cycles per wait
};

// Tile record: U parts [3][128 x K2p] (GEMM1 A: K-major, SBO = K2p / 8 * 128),
// then the Et weights (padded to 16 bytes), then transposed U parts
// [3][K2p x 128] (GEMM2 B: K-major, SBO = 128 / 8 * 128 = 2048).
__host__ __device__ inline uint32_t part_bytes(int K2p) { return (uint32_t)kRows * K2p * 2; }
__host__ __device__ inline uint32_t w_bytes(int Et) { return (uint32_t)((Et + 3) / 4) * 16; }

using pwa::tc::mma_bf16;
using pwa::tc::mma_commit;
using pwa::tc::sa;
using pwa::tc::sdesc;
using pwa::tc::tmem_ld8;
using pwa::tc::tmem_wait;
__device__ __forceinline__ void tc_fence_before() { pwa::tc::fence_before(); }
__device__ __forceinline__ void tc_fence_after() { pwa::tc::fence_after(); }

// x = x0 + x1 + x2 in BF16, each part the nearest BF16 of the remainder
__host__ __device__ inline void split3(float x, __nv_bfloat16& b0, __nv_bfloat16& b1, __nv_bfloat16& b2)
{
    b0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(b0);
    b1 = __float2bfloat16_rn(r1);
    b2 = __float2bfloat16_rn(r1 - __bfloat162float(b1));
}

// The same split by truncation (each part the leading 8 significant bits of
// what is left; also exact, since 8 + 8 + 8 bits hold an FP32 significand),
// returned as raw BF16 bit patterns: a few integer operations per value.
__device__ __forceinline__ void split3_bits(float x, unsigned short& b0, unsigned short& b1, unsigned short& b2)
{
    const uint32_t u0 = __float_as_uint(x);
    const float r1 = x - __uint_as_float(u0 & 0xFFFF0000u);
    const uint32_t u1 = __float_as_uint(r1);
    const float r2 = r1 - __uint_as_float(u1 & 0xFFFF0000u);
    b0 = (unsigned short)(u0 >> 16);
    b1 = (unsigned short)(u1 >> 16);
    b2 = (unsigned short)(__float_as_uint(r2) >> 16);
}

// byte offset of element (row, col) of a K-major 16-bit operand
__host__ __device__ inline uint32_t kmaj16(int row, int col, uint32_t lbo, uint32_t sbo)
{
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(col >> 3) * lbo + (uint32_t)(row & 7) * 16 + (uint32_t)(col & 7) * 2;
}

__device__ __forceinline__ void two_sum(float2& p, float x)
{
    const float sum = __fadd_rn(p.x, x);
    const float bp = __fsub_rn(sum, p.x);
    const float err = __fadd_rn(__fsub_rn(p.x, __fsub_rn(sum, bp)), __fsub_rn(x, bp));
    p = make_float2(sum, __fadd_rn(p.y, err));
}

__global__ void __launch_bounds__(kCT + 32, 1) coupling_kernel(const CpArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool producer = warp == kCT / 32;  // warp 8: TMA copies and MMA issue; warps 0-7: epilogue
    const int row = tid & (kRows - 1), half = (tid >> 7) & 1, wq = warp & 3;  // wq: TMEM lane quarter
    const int K = a.K, S = a.S, K2p = a.K2p;
    const uint32_t PB = part_bytes(K2p);
    const uint32_t sbo_a = (uint32_t)(K2p / 8) * 128;  // U parts and B1 parts: 8-row-group stride
    const uint32_t sbo_t = (uint32_t)(kRows / 8) * 128; // transposed U parts
    const uint32_t B1P = (uint32_t)kN1 * K2p * 2;       // one part of B1
    const uint32_t WTP = (uint32_t)(kN1 / 8) * kSboW;   // one part of W
    // shared memory: A stages [2] | B stages [2] | B1 parts | W parts | barriers
    unsigned char* sA[2] = {sm, sm + a.a_bytes};
    unsigned char* sB[2] = {sm + 2 * a.a_bytes, sm + 2 * a.a_bytes + a.b_bytes};
    unsigned char* b1 = sm + 2 * a.a_bytes + 2 * a.b_bytes;
    unsigned char* wt = b1 + kParts * B1P;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wt + kParts * WTP);
    // tmaA[2], tmaB[2]: tile halves arrived; g1[2]: GEMM1 of a tile done; g2: GEMM2 done;
    // wready: the 8 epilogue warps have written W and are done with the tile's D1 and weights
    uint64_t *tmaA = bars, *tmaB = bars + 2, *g1 = bars + 4, *g2 = bars + 6, *wready = bars + 7;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + kNBars);
    __shared__ volatile int s_abort;
    __shared__ double s_red[kCT / 32][kCH];

    const int G = gridDim.x;
    const int T = a.ntiles;
    const int nmine = blockIdx.x < T ? (T - 1 - (int)blockIdx.x) / G + 1 : 0;  // tiles of this CTA
    auto tile_of = [&](int i) { return (long long)blockIdx.x + (long long)i * G; };

    // ---- GEMM1 B operand from the coupling vectors: row n, column kk of (2K | padding), 3 parts
    for (int i = tid; i < kN1 * K2p; i += kCT + 32) {
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
        __nv_bfloat16 p0, p1, p2;
        split3(v, p0, p1, p2);
        const uint32_t off = kmaj16(n, kk, 128, sbo_a);
        *reinterpret_cast<__nv_bfloat16*>(b1 + off) = p0;
        *reinterpret_cast<__nv_bfloat16*>(b1 + B1P + off) = p1;
        *reinterpret_cast<__nv_bfloat16*>(b1 + 2 * B1P + off) = p2;
    }
    auto issue_A = [&](int i, int st) {
        pwa::tma_load_tile(sA[st], a.U + (size_t)tile_of(i) * a.rec_bytes, a.a_bytes, &tmaA[st]);
    };
    auto issue_B = [&](int i, int st) {
        pwa::tma_load_tile(sB[st], a.U + (size_t)tile_of(i) * a.rec_bytes + a.a_bytes, a.b_bytes, &tmaB[st]);
    };
    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < kNBars; ++i) {
            const uint32_t count = (bars + i == wready) ? kCT / 32 : 1;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(&bars[i])), "r"(count));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (producer) {
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
    const uint32_t tD2 = tm + 256, tD2c = tm + 256 + 4 * kMaxK2p;
    // instruction descriptors: D f32, A/B bf16, both K-major, N >> 3, M >> 4
    const uint32_t idesc1 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN1 >> 3) << 17) | ((128u >> 4) << 24);
    const uint32_t idesc2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(K2p >> 3) << 17) |
                            ((uint32_t)(kN1 >> 4) << 24);

    // bounded wait on a barrier phase; gives up at once when another thread has
    // already given up (the whole CTA then winds down)
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
            if (s_abort || clock64() - t0 > a.timeout) {
                s_abort = 1;
                return false;
            }
        }
    };

    // phases armed on each asynchronous barrier by the producer lane (TMA copies,
    // MMA commits): a CTA that gives up drains exactly the last phase of each
    int nA[2] = {0, 0}, nB[2] = {0, 0}, nG1[2] = {0, 0}, nG2 = 0;
    if (producer) {
        // ======== producer: one lane issues everything ========
        if (lane == 0) {
            for (int i = 0; i < 2 && i < nmine; ++i) {
                issue_A(i, i);
                issue_B(i, i);
                ++nA[i];
                ++nB[i];
            }
            for (int i = 0; i <= nmine && !s_abort; ++i) {
                if (i < nmine) {
                    // GEMM1(i) into accumulator pair i % 2 (read by the epilogue of tile i - 2, done)
                    const int st = i & 1;
                    if (!wait_bar(&tmaA[st], (uint32_t)((i >> 1) & 1))) break;
                    tc_fence_after();
                    const uint32_t ab = sa(sA[st]), bb = sa(b1);
                    const uint32_t d = tm + 64 * st, dc = tm + 128 + 64 * st;
                    for (int ks = 0; ks < K2p / 16; ++ks) {
                        uint64_t ad[kParts], bd[kParts];
                        for (int q = 0; q < kParts; ++q) {
                            ad[q] = sdesc(ab + q * PB + ks * 256, 128, sbo_a);
                            bd[q] = sdesc(bb + q * B1P + ks * 256, 128, sbo_a);
                        }
                        mma_bf16(d, ad[0], bd[0], idesc1, ks > 0);
                        mma_bf16(dc, ad[0], bd[1], idesc1, ks > 0);
                        mma_bf16(dc, ad[1], bd[0], idesc1, 1);
                        mma_bf16(dc, ad[0], bd[2], idesc1, 1);
                        mma_bf16(dc, ad[1], bd[1], idesc1, 1);
                        mma_bf16(dc, ad[2], bd[0], idesc1, 1);
                    }
                    mma_commit(&g1[st]);
                    ++nG1[st];
                }
                if (i >= 1) {
                    const int p = i - 1, sp = p & 1;
                    // W(p) written, D2 of tile p - 1 flushed, tile p's D1 and weights read
                    if (!wait_bar(wready, (uint32_t)(p & 1))) break;
                    tc_fence_after();
                    if (p + 2 < nmine) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue_A(p + 2, sp);
                        ++nA[sp];
                    }
                    if (!wait_bar(&tmaB[sp], (uint32_t)((p >> 1) & 1))) break;
                    const uint32_t ab = sa(wt), bb = sa(sB[sp]);
                    for (int ks = 0; ks < kRows / 16; ++ks) {
                        uint64_t ad[kParts], bd[kParts];
                        for (int q = 0; q < kParts; ++q) {
                            ad[q] = sdesc(ab + q * WTP + ks * 2 * kLboW, kLboW, kSboW);
                            bd[q] = sdesc(bb + q * PB + ks * 256, 128, sbo_t);
                        }
                        mma_bf16(tD2 + kMaxK2p * (ks & 3), ad[0], bd[0], idesc2, ks >= 4);
                        mma_bf16(tD2c, ad[0], bd[1], idesc2, ks > 0);
                        mma_bf16(tD2c, ad[1], bd[0], idesc2, 1);
                        mma_bf16(tD2c, ad[0], bd[2], idesc2, 1);
                        mma_bf16(tD2c, ad[1], bd[1], idesc2, 1);
                        mma_bf16(tD2c, ad[2], bd[0], idesc2, 1);
                    }
                    mma_commit(g2);
                    ++nG2;
                    // its transposed-U stage is refilled once GEMM2(p) has read it
                    if (p + 2 < nmine) {
                        if (!wait_bar(g2, (uint32_t)(p & 1))) break;
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue_B(p + 2, sp);
                        ++nB[sp];
                    }
                }
            }
        }
    } else {
        // ======== epilogue warps ========
        const int j = lane / S, s = lane % S;  // slot j of the quarter's EW events, projection s
        const bool row_used = j < a.EW;
        float2 slnI[kCH];  // per-thread sums of w ln I as (hi, lo) pairs
#pragma unroll
        for (int c = 0; c < kCH; ++c) slnI[c] = make_float2(0.f, 0.f);
        // the GEMM2 results of the CTA, rows n = 16 wq + lane (lane < 16), this warp's
        // half of the 8-column chunks, as (hi, lo) pairs
        const int nch = K2p / 16;  // chunks per half (1..3)
        float2 acc[3][8];
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[q][e] = make_float2(0.f, 0.f);
        auto flush_d2 = [&]() {
            tc_fence_after();
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (q < nch) {
                    const int col = 8 * (nch * half + q);
                    uint32_t v[5][8];
#pragma unroll
                    for (int m = 0; m < 4; ++m) tmem_ld8(tD2 + kMaxK2p * m + tm_lane + col, v[m]);
                    tmem_ld8(tD2c + tm_lane + col, v[4]);
                    tmem_wait();
                    // the tile's five partials in FP32 (rounded to nearest: no systematic
                    // error), then one compensated addition into the running sums
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float x = ((__uint_as_float(v[0][e]) + __uint_as_float(v[1][e])) +
                                         (__uint_as_float(v[2][e]) + __uint_as_float(v[3][e]))) +
                                        __uint_as_float(v[4][e]);
                        two_sum(acc[q][e], x);
                    }
                }
        };
        // a warp-uniform wait: lane 0 waits, the warp follows its verdict
        auto warp_wait = [&](uint64_t* bar, uint32_t parity) -> bool {
            int ok = 1;
            if (lane == 0) ok = wait_bar(bar, parity) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            tc_fence_after();
            return ok != 0;
        };
        for (int i = 0; i < nmine; ++i) {
            const int st = i & 1;
            const uint32_t ph = (uint32_t)((i >> 1) & 1);
            if (!warp_wait(&g1[st], ph) || !warp_wait(&tmaA[st], ph)) break;
            const float wgt_tile =
                reinterpret_cast<const float*>(sA[st] + kParts * PB)[wq * a.EW + min(j, a.EW - 1)];
            // this row's coherent sums for this thread's vectors (main + correction accumulators)
            float d1[4][kCH];
            {
                uint32_t v[4][8], vc[4][8];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    tmem_ld8(tm + 64 * st + tm_lane + q * kCV + kCH * half, v[q]);
                    tmem_ld8(tm + 128 + 64 * st + tm_lane + q * kCV + kCH * half, vc[q]);
                }
                tmem_wait();
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int cc = 0; cc < kCH; ++cc)
                        d1[q][cc] = __uint_as_float(v[q][cc]) + __uint_as_float(vc[q][cc]);
            }
            const long long t = tile_of(i);
            const long long ev = t * a.Et + (long long)wq * a.EW + j;
            const bool valid = row_used && ev < a.n;
            const float wgt = valid ? wgt_tile : 0.f;
            const int base = S * j;  // first lane of this row's event
            float wv[4][kCH];
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
                wv[0][cc] = wa * Ar;
                wv[1][cc] = wa * Ai;
                wv[2][cc] = fmaf(wa, Dr, -wb * Ar);
                wv[3][cc] = fmaf(wa, Di, -wb * Ai);
            }
            // GEMM2(i - 1) done: take its results; then W of this tile may be written
            if (i >= 1) {
                if (!warp_wait(g2, (uint32_t)((i - 1) & 1))) break;
                flush_d2();
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int cc = 0; cc < kCH; ++cc) {
                    unsigned short p0, p1, p2;
                    split3_bits(wv[q][cc], p0, p1, p2);
                    const uint32_t off = kmaj16(q * kCV + kCH * half + cc, row, kLboW, kSboW);
                    *reinterpret_cast<unsigned short*>(wt + off) = p0;
                    *reinterpret_cast<unsigned short*>(wt + WTP + off) = p1;
                    *reinterpret_cast<unsigned short*>(wt + 2 * WTP + off) = p2;
                }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(wready)) : "memory");
        }
        // the last GEMM2
        if (nmine > 0 && !s_abort && warp_wait(g2, (uint32_t)((nmine - 1) & 1))) flush_d2();
        if (!s_abort) {
            double* rq = a.rec + (size_t)blockIdx.x * (kN1 * K2p + kCV);
            if (lane < 16) {
                const int n = 16 * wq + lane;
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    if (q < nch)
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            rq[(size_t)n * K2p + 8 * (nch * half + q) + e] =
                                (double)acc[q][e].x + (double)acc[q][e].y;
            }
#pragma unroll
            for (int cc = 0; cc < kCH; ++cc) {
                double v = (double)slnI[cc].x + (double)slnI[cc].y;
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) s_red[warp][cc] = v;
            }
        }
    }
    __syncthreads();
    if (s_abort) {
        if (tid == 0) atomicOr(a.err, pwa::ERR_TIMEOUT);
    } else if (tid < kCV) {
        double* rs = a.rec + (size_t)blockIdx.x * (kN1 * K2p + kCV) + (size_t)kN1 * K2p;
        const int h = tid / kCH, cc = tid % kCH;  // vector tid: warps 4 h .. 4 h + 3
        rs[tid] = ((s_red[4 * h][cc] + s_red[4 * h + 1][cc]) + s_red[4 * h + 2][cc]) + s_red[4 * h + 3][cc];
    }
    // A CTA that gave up waits (bounded) for the last phase it armed on each
    // barrier -- every earlier phase of a barrier completed before the
    // producer armed the next one -- so that no TMA copy or MMA still writes
    // shared memory or TMEM when TMEM is freed and the CTA exits.  Barriers
    // never armed are skipped.
    if (s_abort && producer && lane == 0) {
        s_abort = 0;  // let the drain waits run their course
        for (int q = 0; q < 2; ++q) {
            if (nG1[q] > 0) (void)wait_bar(&g1[q], (uint32_t)((nG1[q] - 1) & 1));
            s_abort = 0;
            if (nA[q] > 0) (void)wait_bar(&tmaA[q], (uint32_t)((nA[q] - 1) & 1));
            s_abort = 0;
            if (nB[q] > 0) (void)wait_bar(&tmaB[q], (uint32_t)((nB[q] - 1) & 1));
            s_abort = 0;
        }
        if (nG2 > 0) (void)wait_bar(g2, (uint32_t)((nG2 - 1) & 1));
        s_abort = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (producer) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kTmemCols));
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

// Tile records: row r = (lane quarter w, slot j, projection s) of tile t is
// event t Et + w EW + j; U (split in three BF16 parts) as GEMM1's operand and,
// transposed, as GEMM2's, and the event weights.
__global__ void coupling_u_kernel(const float2* __restrict__ F, const float* __restrict__ m2,
                                  const float* __restrict__ w, long long n, int K, int S, int K2p, int EW, int Et,
                                  int ntiles, uint32_t rec_bytes, uint32_t a_bytes, const CpRes* __restrict__ res,
                                  unsigned char* __restrict__ U)
{
    const uint32_t PB = part_bytes(K2p);
    const uint32_t sbo_a = (uint32_t)(K2p / 8) * 128, sbo_t = (uint32_t)(kRows / 8) * 128;
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
        __nv_bfloat16 p[3];
        split3(v, p[0], p[1], p[2]);
        unsigned char* rec = U + (size_t)t * rec_bytes;
        const uint32_t oa = kmaj16(r, kk, 128, sbo_a), ot = kmaj16(kk, r, 128, sbo_t);
        for (int q = 0; q < 3; ++q) {
            *reinterpret_cast<__nv_bfloat16*>(rec + q * PB + oa) = p[q];
            *reinterpret_cast<__nv_bfloat16*>(rec + a_bytes + q * PB + ot) = p[q];
        }
    }
    // the weights after the U parts (zero past the last event and in the padding)
    const int nw_tile = (int)(w_bytes(Et) / 4);
    const long long nw = (long long)ntiles * nw_tile;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nw;
         i += (long long)gridDim.x * blockDim.x) {
        const long long t = i / nw_tile;
        const int el = (int)(i % nw_tile);
        const long long e = t * Et + el;
        reinterpret_cast<float*>(U + (size_t)t * rec_bytes + 3 * PB)[el] = (el < Et && e < n) ? (w ? w[e] : 1.f) : 0.f;
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

constexpr int kCombRows = 8;  // thread rows of the combine kernel (CTA records split between them)

__global__ void coupling_combine_kernel(const double* __restrict__ rec, int nrec, int K, int K2p,
                                        const double* __restrict__ phi, const CpVec* __restrict__ vec,
                                        const pwa::ResParam* __restrict__ res, int Pc, double Nd, double Nmc,
                                        int nvec, double* __restrict__ out)
{
    const int c = blockIdx.x;
    if (c >= nvec) return;
    // blockDim (32, kCombRows): thread (k, y) adds the CTA records y, y + kCombRows, ...;
    // the rows are then added in row order (fixed order, independent of the launch)
    extern __shared__ double sh[];  // [K][8] partials, then 4 scalars, then [kCombRows][32][8] row sums, [kCombRows * 32] ln-terms
    const int reclen = kN1 * K2p + kCV;
    double* part = sh;
    double* scal = sh + 8 * K;
    double* rows = scal + 4;
    double* lns = rows + kCombRows * 32 * 8;
    const int k = threadIdx.x, y = threadIdx.y;
    {
        double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (k < K)
            for (int b = y; b < nrec; b += kCombRows) {
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
#pragma unroll
        for (int i = 0; i < 8; ++i) rows[(y * 32 + k) * 8 + i] = q[i];
        // the data's sum w ln I of this vector, one record per thread
        const int t = y * 32 + k;
        double l = 0.0;
        for (int b = t; b < nrec; b += 32 * kCombRows) l += rec[(size_t)b * reclen + (size_t)kN1 * K2p + c];
        lns[t] = l;
    }
    __syncthreads();
    if (y > 0) return;
    double2 Q1d = make_double2(0, 0), P1d = make_double2(0, 0), Pg = make_double2(0, 0), Pd = make_double2(0, 0);
    if (k < K) {
        double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int yy = 0; yy < kCombRows; ++yy)
#pragma unroll
            for (int i = 0; i < 8; ++i) q[i] += rows[(yy * 32 + k) * 8 + i];
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
    __syncwarp();
    if (threadIdx.x == 0) {
        double Gm = 0.0, Gd = 0.0, sln = 0.0;
        for (int kk = 0; kk < K; ++kk) {
            Gm += part[8 * kk + 0];
            Gd += part[8 * kk + 1];
        }
        for (int t = 0; t < 32 * kCombRows; ++t) sln += lns[t];
        scal[0] = Gm;
        scal[1] = Gd;
        out[(size_t)c * (1 + 2 * Pc)] = -sln + Nd * log(Gm / Nmc);
    }
    __syncwarp();
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
    uint32_t rec_bytes = 0, a_bytes = 0, b_bytes = 0;  // tile record and its two TMA copies
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
    a.U = reinterpret_cast<const unsigned char*>(cp->d_U);
    a.n = h->n[0];
    a.ntiles = cp->ntiles;
    a.K = K;
    a.S = cp->S;
    a.K2p = cp->K2p;
    a.EW = cp->EW;
    a.Et = cp->Et;
    a.rec_bytes = cp->rec_bytes;
    a.a_bytes = cp->a_bytes;
    a.b_bytes = cp->b_bytes;
    a.gc = cp->d_gc;
    a.nv = nv;
    a.rec = cp->d_rec;
    a.err = cp->d_err;
    a.timeout = h->timeout_cycles;
    coupling_kernel<<<cp->grid, kCT + 32, cp->smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cp_cuda(cp, e, "coupling kernel launch");
    coupling_combine_kernel<<<nv, dim3(32, kCombRows),
                              sizeof(double) * (8 * K + 4 + kCombRows * 32 * 8 + kCombRows * 32), s>>>(
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
    if (h->released)
        return pwa::set_error(h, PWA_EINVAL, "the events' caller-layout copies were released; the coupling "
                                             "object is built from them");
    if (h->broken) return pwa::set_error(h, PWA_ETIMEOUT, "handle is unusable after a device-side timeout");
    const int K = h->K, S = h->S, P = h->P;
    for (int i = 0; i < P; ++i)
        if (!std::isfinite(theta[i])) return pwa::set_error(h, PWA_EINVAL, "theta must be finite");
    const int K2p = (2 * K + 15) / 16 * 16;
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
    cp->b_bytes = kParts * part_bytes(K2p);
    cp->a_bytes = cp->b_bytes + w_bytes(cp->Et);
    cp->rec_bytes = cp->a_bytes + cp->b_bytes;
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
    // A stages x 2 | B stages x 2 | B1 parts | W parts | barriers and the TMEM address
    cp->smem = 2 * (size_t)cp->a_bytes + 2 * (size_t)cp->b_bytes + kParts * (size_t)kN1 * K2p * 2 +
               kParts * (size_t)(kN1 / 8) * kSboW + kNBars * 8 + 16;
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
        if ((e = cudaMalloc(&cp->d_U, (size_t)cp->ntiles * cp->rec_bytes)) != cudaSuccess) break;
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
        const long long uthreads = (long long)cp->ntiles * kRows * K2p;
        const int ublocks = (int)std::min<long long>((uthreads + 255) / 256, 65535LL * 8);
        coupling_u_kernel<<<std::max(ublocks, 1), 256, 0, h->stream>>>(
            reinterpret_cast<const float2*>(h->d_F[0]), h->d_m2[0], h->d_w, h->n[0], K, S, K2p, cp->EW, cp->Et,
            cp->ntiles, cp->rec_bytes, cp->a_bytes, d_rs, reinterpret_cast<unsigned char*>(cp->d_U));
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
