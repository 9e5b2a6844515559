// hessian.cu -- pwa_hessian: the full P x P Hessian of the NLL, with the NLL
// and its gradient, from one pass over F.
//
// Eq. 7 of the paper contracts the Hessian of ln L with a direction; written
// out without the contraction, every entry is a sum over events of products
// of first derivatives plus a resonance-diagonal second-derivative term.  For
// resonance k with parameters theta_k = (rho, phi, M, Gamma),
//   dc_k/dtheta_kj = kappa1_j B_k + kappa2_j B_k^2,
//   d2c_k/dtheta_kj dtheta_kj' = mu1 B_k + mu2 B_k^2 + mu3 B_k^3,
// with theta-dependent complex coefficients (B_k = BW_k(e), c_k = g_k B_k).
// With V_{(k,p),s}(e) = B_k^p F_{k,s}(e) (p = 1, 2) and D_k = sum_s conj(A_s) F_ks,
//   sum_e a d2I/dtheta_i dtheta_j
//       = 2 Re sum_{p,p'} conj(kappa_p,i) kappa_p',j C[(k_i,p), (k_j,p')]
//         + delta_{k_i k_j} 2 Re (mu1 Q1 + mu2 Q2 + mu3 Q3)_k,
//   C = sum_e a sum_s conj(V_s) V_s^T   (2K x 2K Hermitian Gram matrix),
//   Qp_k = sum_e a B_k^p D_k,
// and dI/dtheta_i = 2 Re (kappa1 Z1 + kappa2 Z2)_k with Zp_k = B_k^p D_k, so
//   sum_data (w/I^2) dI/dtheta_i dI/dtheta_j = c_i^T Zg c_j,
//   Zg = sum_data (w/I^2) z z^T  (z = Re, Im of Z: 4K reals per event).
// The kernel therefore accumulates, per sample set, the real Gram matrix
// X^T X of the rows (e, s) of X = sqrt(a) (Re V, Im V) (4K columns; its
// entries give C), for data also Zg, and the sums Q1..Q3, sum w ln I and
// G = sum_mc I.  The host combines them in FP64 with the coefficients into
// H = -(sum_data (w/I) d2I - Zg) + N_d (sum_mc d2I / G - dG dG^T / G^2)
// (Eqs. 4-7 with the data weight a = w/I, a = 1 for MC).
//
// Work split (one CTA of NT threads streams tiles of 32 events, the records
// pwa_create lays out, by TMA bulk copies into two shared stages):
//   event phase: a lane per event, each warp owning every NW-th resonance: B,
//            the warp's partial coherent sums, summed over the warps through
//            shared memory, I, the weights; the lane writes its resonances'
//            columns of X and z into shared memory and accumulates their Q
//            sums;
//   Gram phase: CUDA cores (hess_kernel): every thread owns NB 4 x 4 blocks of
//            the upper triangle of the 4K x 4K Gram matrices and accumulates
//            them over the tile's rows in FP32 registers; tensor cores
//            (hess_tc_kernel, K <= 32): MMAs on BF16 splits of X and z into
//            TMEM, read back into FP32 registers (described below).
// FP32 sums are folded into per-CTA FP64 records every few tiles; a second
// kernel adds the records in a fixed order (run-to-run bit-identical).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "pwa_internal.h"
#include "tcgen05.cuh"

namespace {

using pwa::KConst;
constexpr int kE = pwa::kTileE;  // events per tile
constexpr int kFold = 16;        // tiles between FP32 -> FP64 folds
constexpr int kFoldG = 32;       // the same for the tensor-core kernel's Gram sums (FP32 adds of per-tile sums)
constexpr int kMaxKHess = pwa::kMaxKHessian;  // K (K + 1) / 2 Gram blocks fit 2 per thread of 512
constexpr int kMaxKTensor = 32;                // 4K columns fit the M = 128 tensor-core tile

struct HessArgs {
    const unsigned char* tiles[2];  // data, MC tile records (the handle's layout)
    uint32_t tile_bytes[2];
    int ntiles[2];
    long long nev[2];
    int K;
    int ev;                // events per warp of the tiling the records were laid out for
    uint32_t stage_bytes;  // shared bytes per stage (16-byte multiple >= both tile records)
    const pwa::ResParam* res;
    const double* theta;   // device [B][P]
    int P;
    // B parameter vectors per launch: CTA c works for vector c mod B and is CTA
    // c / B of the Gb that share that vector's tiles (tiles gb, gb + Gb, ...)
    int B, Gb;
    int nblk;              // 4 x 4 blocks in the upper triangle of the 4K x 4K Gram: K (K + 1) / 2
    double* rec;           // [B Gb][rec_len] per-CTA FP64 sums (zeroed before the launch)
    int rec_len;
    unsigned long long* bad;
    int* err;
    int* err_vec;          // [B] per-vector error words (zeroed before the launch)
    long long timeout_cycles;
};

// Record layout of one CTA (FP64):
//   [0, 16 nblk)           data Gram of X, block b's 16 entries row-major
//   [16 nblk, 32 nblk)     data Gram of z
//   [32 nblk, 48 nblk)     MC Gram of X
//   then Q [2 sets][K][6] (Re, Im of Q1, Q2, Q3), then the scalars [NW][2]
//   (sum w ln I of the data, G = sum I of the MC) per warp
__host__ __device__ inline int hess_rec_len(int K, int nblk, int NW) { return 48 * nblk + 12 * K + 2 * NW; }

// block index -> (bi, bj), bi <= bj, enumerating the upper triangle row by
// row.  Block (bi, bj) covers the Gram entries of columns bi + u K and
// bj + v K (u, v = 0..3): the four columns of a block are K apart, so that
// the threads of a warp (consecutive bj) read consecutive columns.
__host__ __device__ inline void block_of(int b, int nb, int& bi, int& bj)
{
    int i = 0, rem = b;
    while (rem >= nb - i) {
        rem -= nb - i;
        ++i;
    }
    bi = i;
    bj = i + rem;
}

constexpr int kKW = 3;  // resonances per warp in phase 1 (K <= 3 x warps)

// Shared-memory row strides (floats): X and z are stored column-major, a
// column's rows contiguous, so that phase 1 (a lane per event) writes 32
// consecutive floats and phase 2 reads 16-byte groups of rows; the strides
// are 4 (mod 8) floats... times an odd number of 16-byte groups, so the
// columns a warp reads start in different bank groups.
__host__ __device__ inline int x_stride(int S) { return 32 * S + 4; }
constexpr int kZStride = 36;

template <int S, int NT, int NB>
__global__ void __launch_bounds__(NT, 1) hess_kernel(const HessArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int NW = NT / 32;
    constexpr int RS = 32 * S + 4;  // x_stride(S)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = a.K, C = 4 * K;

    // shared memory: stages[2] | KConst[K] | X [C][RS] | z [C][36] | partial A [NW][2S][32] | mbarriers[2]
    unsigned char* stages = smem;
    KConst* kc = reinterpret_cast<KConst*>(smem + 2 * (size_t)a.stage_bytes);
    float* X = reinterpret_cast<float*>(kc + K);
    float* Zs = X + (size_t)C * RS;
    float* PA = Zs + (size_t)C * kZStride;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(PA + NW * 2 * S * 32);
    __shared__ long long issued[2];
    __shared__ int s_abort;

    const int bt = (int)(blockIdx.x % (unsigned)a.B), gb = (int)(blockIdx.x / (unsigned)a.B), G = a.Gb;
    const long long T = (long long)a.ntiles[0] + a.ntiles[1];
    auto tile_src = [&](long long t, int& smp, long long& lt) {
        smp = t < a.ntiles[0] ? 0 : 1;
        lt = smp ? t - a.ntiles[0] : t;
    };
    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < 2; ++s) {
            pwa::mbar_init(&mbar[s], 1);
            issued[s] = -1;
        }
        pwa::fence_mbar_init();
        for (int i = 0; i < 2; ++i) {
            const long long t = gb + (long long)i * G;
            if (t < T) {
                int smp;
                long long lt;
                tile_src(t, smp, lt);
                pwa::tma_load_tile(stages + (size_t)i * a.stage_bytes, a.tiles[smp] + (size_t)lt * a.tile_bytes[smp],
                                   a.tile_bytes[smp], &mbar[i]);
                issued[i] = i;
            }
        }
    }
    {
        pwa::PassArgs pa;
        pa.res = a.res;
        for (int k = tid; k < K; k += NT) kc[k] = pwa::make_kconst(pa, a.theta + (size_t)bt * a.P, nullptr, k, false, a.ev);
    }
    __syncthreads();

    // this thread's Gram blocks
    int bi[NB], bj[NB];
#pragma unroll
    for (int m = 0; m < NB; ++m) {
        const int b = tid + m * NT;
        if (b < a.nblk) block_of(b, K, bi[m], bj[m]);
        else bi[m] = bj[m] = -1;
    }
    float R[NB][16], Zg[NB][16];
#pragma unroll
    for (int m = 0; m < NB; ++m)
#pragma unroll
        for (int u = 0; u < 16; ++u) R[m][u] = Zg[m][u] = 0.f;
    // the warp's resonances k = warp + j NW; this lane's event's share of their Q sums
    float q[kKW][6];
#pragma unroll
    for (int j = 0; j < kKW; ++j)
#pragma unroll
        for (int u = 0; u < 6; ++u) q[j][u] = 0.f;
    float sc = 0.f;

    double* rec = a.rec + (size_t)blockIdx.x * a.rec_len;
    const int offQ = 48 * a.nblk, offS = offQ + 12 * K;
    // add the FP32 sums of the current window to the FP64 record of sample set smp
    auto fold = [&](int smp) {
        const int offR = smp == 0 ? 0 : 32 * a.nblk;
#pragma unroll
        for (int m = 0; m < NB; ++m) {
            if (bi[m] < 0) continue;
            const int b = tid + m * NT;
            double* rr = rec + offR + 16 * b;
            double* rz = rec + 16 * a.nblk + 16 * b;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                rr[u] += (double)R[m][u];
                R[m][u] = 0.f;
                if (smp == 0) rz[u] += (double)Zg[m][u];
                Zg[m][u] = 0.f;
            }
        }
#pragma unroll
        for (int j = 0; j < kKW; ++j) {
            const int k = warp + j * NW;
#pragma unroll
            for (int u = 0; u < 6; ++u) {
                const float v = pwa::warp_sum(q[j][u]);
                q[j][u] = 0.f;
                if (lane == 0 && k < K) rec[offQ + ((size_t)smp * K + k) * 6 + u] += (double)v;
            }
        }
        const float v = pwa::warp_sum(sc);
        sc = 0.f;
        if (lane == 0) rec[offS + 2 * warp + smp] += (double)v;
    };

    int st = 0;
    uint32_t ph = 0;
    int win = 0;
    int cur_smp = 0;
    long long i = 0;
    for (long long t = gb; t < T; t += G, ++i) {
        int smp;
        long long lt;
        tile_src(t, smp, lt);
        if (smp != cur_smp) {  // the data tiles are done: their sums go to the data record
            fold(0);
            win = 0;
            cur_smp = smp;
        }
        const bool ok = pwa::mbar_wait(&mbar[st], ph, a.timeout_cycles);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) s_abort = 1;
            break;
        }
        const float* Ft = reinterpret_cast<const float*>(stages + (size_t)st * a.stage_bytes);
        const float* m2s = Ft + (size_t)2 * K * S * kE;
        const long long e_base = lt * kE;
        const int e = lane;  // this lane's event in the tile
        const bool valid = e < (int)min((long long)kE, a.nev[smp] - e_base);

        // ---- phase 1a: the warp's resonances for this lane's event: B, F, partial A ----
        float br[kKW], bim[kKW], fr[kKW][S], fi[kKW][S];
        float Ar[S], Ai[S];
#pragma unroll
        for (int s = 0; s < S; ++s) Ar[s] = Ai[s] = 0.f;
#pragma unroll
        for (int j = 0; j < kKW; ++j) {
            const int k = warp + j * NW;
            br[j] = bim[j] = 0.f;
#pragma unroll
            for (int s = 0; s < S; ++s) fr[j][s] = fi[j][s] = 0.f;
            if (k < K) {
                const KConst c = kc[k];
                pwa::breit_wigner(c, m2s[c.ch * kE + e], br[j], bim[j]);
                const float cr = c.gre * br[j] - c.gim * bim[j], ci = c.gre * bim[j] + c.gim * br[j];
                const int p = (e + c.shift) & (kE - 1);
                if constexpr (S % 2 == 0) {
#pragma unroll
                    for (int qq = 0; qq < S / 2; ++qq) {
                        // (Re F_2q, Re F_2q+1, Im F_2q, Im F_2q+1) of (k, p): one 16-byte load
                        const float4 f4 = *reinterpret_cast<const float4*>(Ft + 4 * ((k * (S / 2) + qq) * kE + p));
                        fr[j][2 * qq] = f4.x;
                        fr[j][2 * qq + 1] = f4.y;
                        fi[j][2 * qq] = f4.z;
                        fi[j][2 * qq + 1] = f4.w;
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        const float2 f2 = *reinterpret_cast<const float2*>(Ft + 2 * ((k * S + s) * kE + p));
                        fr[j][s] = f2.x;
                        fi[j][s] = f2.y;
                    }
                }
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    Ar[s] += cr * fr[j][s] - ci * fi[j][s];
                    Ai[s] += cr * fi[j][s] + ci * fr[j][s];
                }
            }
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            PA[(warp * 2 * S + 2 * s) * 32 + e] = Ar[s];
            PA[(warp * 2 * S + 2 * s + 1) * 32 + e] = Ai[s];
        }
        __syncthreads();
        // ---- phase 1b: the coherent sums of the lane's event (every warp adds the partials) ----
#pragma unroll
        for (int s = 0; s < S; ++s) {
            float xr = 0.f, xi = 0.f;
            for (int w = 0; w < NW; ++w) {
                xr += PA[(w * 2 * S + 2 * s) * 32 + e];
                xi += PA[(w * 2 * S + 2 * s + 1) * 32 + e];
            }
            Ar[s] = xr;
            Ai[s] = xi;
        }
        float I = 0.f;
#pragma unroll
        for (int s = 0; s < S; ++s) I += Ar[s] * Ar[s] + Ai[s] * Ai[s];
        float aw = 0.f, sqa = 0.f, zw = 0.f;
        if (smp == 0) {
            const float w = m2s[3 * kE + e];
            const bool good = I > 0.f && I < INFINITY;
            if (valid && good) {
                aw = w / I;
                sqa = sqrtf(aw);
                zw = sqrtf(w) / I;
                if (warp == 0) sc += w * logf(I);
            } else if (valid && warp == 0) {
                atomicMin(a.bad, (unsigned long long)(e_base + e));
                atomicOr(a.err, pwa::ERR_NONFINITE);
                atomicOr(a.err_vec + bt, pwa::ERR_NONFINITE);
            }
        } else {
            const bool good = I < INFINITY;
            if (valid && good) {
                aw = 1.f;
                sqa = 1.f;
                if (warp == 0) sc += I;
            } else if (valid && warp == 0) {
                atomicMin(a.bad, (unsigned long long)(a.nev[0] + e_base + e));
                atomicOr(a.err, pwa::ERR_NONFINITE);
                atomicOr(a.err_vec + bt, pwa::ERR_NONFINITE);
            }
        }
        // ---- phase 1c: the warp's columns of X and z for this event, its Q sums ----
#pragma unroll
        for (int j = 0; j < kKW; ++j) {
            const int k = warp + j * NW;
            if (k >= K) continue;
            const float b1r = br[j], b1i = bim[j];
            const float b2r = b1r * b1r - b1i * b1i, b2i = 2.f * b1r * b1i;
            const float b3r = b2r * b1r - b2i * b1i, b3i = b2r * b1i + b2i * b1r;
            float* x1r = X + (size_t)(2 * k) * RS;            // column 2 k: Re (B F); 2 k + 1: Im
            float* x2r = X + (size_t)(2 * (K + k)) * RS;      // column 2 (K + k): Re (B^2 F); + 1: Im
            float Dr = 0.f, Di = 0.f;  // D = sum_s conj(A_s) F_ks
#pragma unroll
            for (int s = 0; s < S; ++s) {
                Dr += Ar[s] * fr[j][s] + Ai[s] * fi[j][s];
                Di += Ar[s] * fi[j][s] - Ai[s] * fr[j][s];
                const float v1r = b1r * fr[j][s] - b1i * fi[j][s], v1i = b1r * fi[j][s] + b1i * fr[j][s];
                const float v2r = b2r * fr[j][s] - b2i * fi[j][s], v2i = b2r * fi[j][s] + b2i * fr[j][s];
                const int r = s * 32 + e;
                x1r[r] = sqa * v1r;
                x1r[RS + r] = sqa * v1i;
                x2r[r] = sqa * v2r;
                x2r[RS + r] = sqa * v2i;
            }
            const float z1r = b1r * Dr - b1i * Di, z1i = b1r * Di + b1i * Dr;
            const float z2r = b2r * Dr - b2i * Di, z2i = b2r * Di + b2i * Dr;
            const float z3r = b3r * Dr - b3i * Di, z3i = b3r * Di + b3i * Dr;
            if (smp == 0) {
                Zs[(size_t)(2 * k) * kZStride + e] = zw * z1r;
                Zs[(size_t)(2 * k + 1) * kZStride + e] = zw * z1i;
                Zs[(size_t)(2 * (K + k)) * kZStride + e] = zw * z2r;
                Zs[(size_t)(2 * (K + k) + 1) * kZStride + e] = zw * z2i;
            }
            q[j][0] = fmaf(aw, z1r, q[j][0]);
            q[j][1] = fmaf(aw, z1i, q[j][1]);
            q[j][2] = fmaf(aw, z2r, q[j][2]);
            q[j][3] = fmaf(aw, z2i, q[j][3]);
            q[j][4] = fmaf(aw, z3r, q[j][4]);
            q[j][5] = fmaf(aw, z3i, q[j][5]);
        }
        __syncthreads();  // X and z complete; the stage has been read
        if (tid == 0) {
            const long long tn = t + 2LL * G;
            if (tn < T) {
                int s2;
                long long lt2;
                tile_src(tn, s2, lt2);
                pwa::fence_proxy_async();
                issued[st] = i + 2;
                pwa::tma_load_tile(stages + (size_t)st * a.stage_bytes, a.tiles[s2] + (size_t)lt2 * a.tile_bytes[s2],
                                   a.tile_bytes[s2], &mbar[st]);
            }
        }

        // ---- phase 2: Gram blocks over the tile's rows, 4 rows per 16-byte load ----
#pragma unroll
        for (int m = 0; m < NB; ++m) {
            if (bi[m] < 0) continue;
            const float* xi0 = X + (size_t)bi[m] * RS;
            const float* xj0 = X + (size_t)bj[m] * RS;
            const size_t cs = (size_t)K * RS;  // stride between a block's columns
#pragma unroll 2
            for (int r = 0; r < 32 * S; r += 4) {
                float4 xi[4], xj[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    xi[u] = *reinterpret_cast<const float4*>(xi0 + u * cs + r);
                    xj[u] = *reinterpret_cast<const float4*>(xj0 + u * cs + r);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        float acc = R[m][4 * u + v];
                        acc = fmaf(xi[u].x, xj[v].x, acc);
                        acc = fmaf(xi[u].y, xj[v].y, acc);
                        acc = fmaf(xi[u].z, xj[v].z, acc);
                        acc = fmaf(xi[u].w, xj[v].w, acc);
                        R[m][4 * u + v] = acc;
                    }
            }
            if (smp == 0) {
                const float* zi0 = Zs + (size_t)bi[m] * kZStride;
                const float* zj0 = Zs + (size_t)bj[m] * kZStride;
                const size_t zc = (size_t)K * kZStride;
#pragma unroll 2
                for (int r = 0; r < 32; r += 4) {
                    float4 xi[4], xj[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        xi[u] = *reinterpret_cast<const float4*>(zi0 + u * zc + r);
                        xj[u] = *reinterpret_cast<const float4*>(zj0 + u * zc + r);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            float acc = Zg[m][4 * u + v];
                            acc = fmaf(xi[u].x, xj[v].x, acc);
                            acc = fmaf(xi[u].y, xj[v].y, acc);
                            acc = fmaf(xi[u].z, xj[v].z, acc);
                            acc = fmaf(xi[u].w, xj[v].w, acc);
                            Zg[m][4 * u + v] = acc;
                        }
                }
            }
        }
        if (++win == kFold) {
            fold(smp);
            win = 0;
        }
        if (++st == 2) {
            st = 0;
            ph ^= 1u;
        }
        __syncthreads();  // phase 2 is done with X and z before the next tile rewrites them
    }
    if (s_abort) {
        // a tile never arrived: report it and wait (bounded) for the copies in flight
        if (tid == 0) {
            atomicOr(a.err, pwa::ERR_TIMEOUT);
            for (int s = 0; s < 2; ++s)
                if (issued[s] >= 0) (void)pwa::mbar_wait(&mbar[s], (uint32_t)((issued[s] / 2) & 1), a.timeout_cycles);
        }
        __syncthreads();
        return;
    }
    fold(cur_smp);
}


// ---------------------------------------------------------------------------
// The Gram matrices on the tensor cores (K <= 32: 4K <= 128 columns)
// ---------------------------------------------------------------------------
//
// The same event phase as hess_kernel, but X and z go to shared memory as
// BF16 pairs (x = hi + lo, each the nearest BF16 of what is left: 16
// significant bits) in the canonical K-major layout of a tcgen05 operand:
// element (column m, row k) in 8 x 16-byte core matrices, rows k along the
// MMA's K dimension (X row e S + s: an event's projections are adjacent, so
// a lane writes them in one store; the Gram does not depend on the order).
// The hi part is the A operand (M = 128 columns: the MMA reads past the 4K
// rounded up to 16 columns the buffer holds, into rows of D that are never
// read) and, with the lo part stored as 2 lo, the B operand (N = 4K rounded
// up to 16): per 16 rows one thread issues two kind::f16 MMAs, D += hi^T hi
// + hi^T (2 lo), whose symmetric part is hi^T hi + hi^T lo + lo^T hi (lo^T lo
// is below 2^-16 of the product; the host symmetrises).  Each tile's sums
// start in a fresh TMEM accumulator (one tile's sum stays short, so the
// tensor core's FP32 accumulation loses nothing), and the data events' z
// Gram likewise.  The tiles are pipelined over two operand buffers and two
// accumulator sets: tile i's MMAs run while the warps read tile i - 1's
// accumulators back (warp w: TMEM lanes 32 (w mod 4) + l, half w / 4 of the
// columns) into FP32 registers and build tile i + 1's operands; the FP32
// sums are folded into FP64 every kFoldG tiles (the Q sums every kFold).  (For
// S = 4 and K > 28 the two buffers do not fit in shared memory: one buffer,
// each tile read back before the next is built.)  Per-CTA record: the full
// data X Gram, the data z Gram and the MC X Gram (C x C each, row-major, not
// yet symmetric), then Q [2][K][6] and the scalars [8][2].

constexpr uint32_t kTcLbo = 144;  // core-matrix stride along the rows (16 B of padding: phase 1's
                                  // stores from 32 lanes spread over the banks)
constexpr int kTcNT = 256;  // 8 warps (16 were slower: the cross-warp sums of the event phase grow)
constexpr int kTcKW = 4;    // resonances per warp in the event phase: K <= 8 x 4 = 32

__host__ __device__ inline uint32_t tc_sbo(int rows) { return (uint32_t)(rows / 8) * kTcLbo; }
__host__ __device__ inline int hess_tc_rec_len(int K) { return 3 * 16 * K * K + 12 * K + 2 * (kTcNT / 32); }
// operand buffers per kernel instance (S, NCH = (4K rounded up to 16) / 16): two where they fit
__host__ __device__ constexpr int tc_nbuf(int S, int nch) { return (S == 4 && nch == 8) ? 1 : 2; }
// TMEM columns: per accumulator set the X Gram at [0, 128) and the z Gram at [128, 256)
__host__ __device__ constexpr int tc_tmem_cols(int nbuf) { return 256 * nbuf; }
// byte offset of (column m, row k) in a K-major BF16 operand part with stride sbo between 8-column groups
__host__ __device__ inline uint32_t tc_off(int m, int k, uint32_t sbo)
{
    return (uint32_t)(m >> 3) * sbo + (uint32_t)(k >> 3) * kTcLbo + (uint32_t)(m & 7) * 16 + (uint32_t)(k & 7) * 2;
}

// Shared-memory layout of hess_tc_kernel (byte offsets): X operand buffers
// [nbuf] (hi part, then the 2 lo part, each 4K rounded up to 16 columns) |
// z operand buffers [nbuf] | TMA stages [2] | KConst [K] | partial A
// [8 warps][2S][32] | total A [2S][32] | mbarriers (TMA 0, 1; MMA sets 0, 1)
// | TMEM address.  total covers the A operands' reads of 128 columns.
struct TcLayout {
    uint32_t sbox, sboz, pbx, pbz;  // 8-column group strides and part sizes of X and z
    uint32_t x[2], z[2], stages, kc, pa, pt, mbar, tslot, total;
};
__host__ __device__ inline TcLayout tc_layout(int K, int S, int nch, uint32_t stage_bytes)
{
    const int nbuf = tc_nbuf(S, nch), NW = kTcNT / 32;
    TcLayout L{};
    L.sbox = tc_sbo(32 * S);
    L.sboz = tc_sbo(32);
    L.pbx = (uint32_t)(2 * nch) * L.sbox;
    L.pbz = (uint32_t)(2 * nch) * L.sboz;
    L.x[0] = 0;
    L.x[1] = nbuf == 2 ? 2 * L.pbx : 0;
    uint32_t o = (uint32_t)nbuf * 2 * L.pbx;
    L.z[0] = o;
    L.z[1] = nbuf == 2 ? o + 2 * L.pbz : o;
    o += (uint32_t)nbuf * 2 * L.pbz;
    L.stages = o;  // a multiple of 16 (the parts are multiples of 144 = 9 x 16)
    o += 2 * stage_bytes;
    L.kc = o;
    o += (uint32_t)(sizeof(KConst) * K);
    L.pa = o;
    o += (uint32_t)(sizeof(float) * NW * 2 * S * 32);
    L.pt = o;
    o += (uint32_t)(sizeof(float) * 2 * S * 32);
    o = (o + 15u) & ~15u;
    L.mbar = o;
    o += 4 * 8;
    L.tslot = o;
    o += 16;
    const uint32_t ax = L.x[nbuf - 1] + 16 * L.sbox, az = L.z[nbuf - 1] + 16 * L.sboz;
    L.total = o > ax ? (o > az ? o : az) : (ax > az ? ax : az);
    return L;
}
__host__ inline size_t hess_tc_smem(int K, int S, uint32_t stage) { return tc_layout(K, S, (4 * K + 15) / 16, stage).total; }

// x as a BF16 hi part and the BF16 of 2 (x - hi) (x - hi is exact in FP32)
__device__ __forceinline__ void store_split(unsigned char* hi0, uint32_t part_bytes, uint32_t off, float x)
{
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    const __nv_bfloat16 lo2 = __float2bfloat16_rn(2.f * (x - __bfloat162float(hi)));
    *reinterpret_cast<__nv_bfloat16*>(hi0 + off) = hi;
    *reinterpret_cast<__nv_bfloat16*>(hi0 + part_bytes + off) = lo2;
}

// the same for a pair of adjacent rows, as packed BF16 pairs (the first row in the low half)
__device__ __forceinline__ void split2(float2 x, uint32_t& hi, uint32_t& lo2)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
    const float2 hf = __bfloat1622float2(h);
    const float2 d = __ffma2_rn(hf, make_float2(-2.f, -2.f), __fmul2_rn(x, make_float2(2.f, 2.f)));  // exact
    const __nv_bfloat162 l = __floats2bfloat162_rn(d.x, d.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo2 = *reinterpret_cast<const uint32_t*>(&l);
}

// The S consecutive rows (e S .. e S + S - 1) of one column, hi and 2 lo
// parts: one 8- (S = 4) or 4-byte (S = 2) store per part (the rows share a
// 16-byte core row); odd S one 2-byte store per row and part.
template <int S>
__device__ __forceinline__ void store_rows(unsigned char* hi0, uint32_t part_bytes, uint32_t off, const float (&x)[S])
{
    if constexpr (S == 4) {
        uint32_t h0, l0, h1, l1;
        split2(make_float2(x[0], x[1]), h0, l0);
        split2(make_float2(x[2], x[3]), h1, l1);
        *reinterpret_cast<uint2*>(hi0 + off) = make_uint2(h0, h1);
        *reinterpret_cast<uint2*>(hi0 + part_bytes + off) = make_uint2(l0, l1);
    } else if constexpr (S == 2) {
        uint32_t h0, l0;
        split2(make_float2(x[0], x[1]), h0, l0);
        *reinterpret_cast<uint32_t*>(hi0 + off) = h0;
        *reinterpret_cast<uint32_t*>(hi0 + part_bytes + off) = l0;
    } else {
        // odd S: the rows may cross a 16-byte core row
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int r = (int)((off >> 1) & 7) + s;  // row within its core row, from the first's offset
            const uint32_t o = off + (uint32_t)(r >> 3) * kTcLbo + (uint32_t)((r & 7) - ((off >> 1) & 7)) * 2;
            store_split(hi0, part_bytes, o, x[s]);
        }
    }
}

template <int S, int NCH>  // NCH = (4K rounded up to 16) / 16
__global__ void __launch_bounds__(kTcNT, 1) hess_tc_kernel(const HessArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int NT = kTcNT, NW = NT / 32, R = 32 * S, Cp = NCH * 16;
    constexpr int NBUF = tc_nbuf(S, NCH);
    constexpr int CPT = Cp / (NW / 4);  // Gram columns per thread: the warps of a TMEM lane quarter split them
    static_assert(kTcKW * NW >= 32 && CPT % 8 == 0 && 2 * S <= NW, "tile shape");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = a.K, C = 4 * K;
    const int bt = (int)(blockIdx.x % (unsigned)a.B), gb = (int)(blockIdx.x / (unsigned)a.B), G = a.Gb;
    const TcLayout L = tc_layout(K, S, NCH, a.stage_bytes);
    unsigned char* stages = smem + L.stages;
    KConst* kc = reinterpret_cast<KConst*>(smem + L.kc);
    float* PA = reinterpret_cast<float*>(smem + L.pa);
    float* PT = reinterpret_cast<float*>(smem + L.pt);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.mbar);  // TMA stages 0, 1; MMA sets 0, 1
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.tslot);
    __shared__ long long issued[2];

    const long long T = (long long)a.ntiles[0] + a.ntiles[1];
    auto tile_src = [&](long long t, int& smp, long long& lt) {
        smp = t < a.ntiles[0] ? 0 : 1;
        lt = smp ? t - a.ntiles[0] : t;
    };
    if (tid == 0) {
        for (int s = 0; s < 4; ++s) pwa::mbar_init(&mbar[s], 1);
        issued[0] = issued[1] = -1;
        pwa::fence_mbar_init();
        for (int i = 0; i < 2; ++i) {
            const long long t = gb + (long long)i * G;
            if (t < T) {
                int smp;
                long long lt;
                tile_src(t, smp, lt);
                pwa::tma_load_tile(stages + (size_t)i * a.stage_bytes, a.tiles[smp] + (size_t)lt * a.tile_bytes[smp],
                                   a.tile_bytes[smp], &mbar[i]);
                issued[i] = i;
            }
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(pwa::tc::sa(tslot)),
                     "r"(tc_tmem_cols(NBUF)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    {
        pwa::PassArgs pa;
        pa.res = a.res;
        for (int k = tid; k < K; k += NT) kc[k] = pwa::make_kconst(pa, a.theta + (size_t)bt * a.P, nullptr, k, false, a.ev);
        // the operands start at zero (columns past 4K only ever meet D entries that are not read)
        uint4* z4 = reinterpret_cast<uint4*>(smem);
        for (uint32_t i = tid; i < L.stages / 16; i += NT) z4[i] = make_uint4(0, 0, 0, 0);
    }
    pwa::fence_proxy_async();
    pwa::tc::fence_before();
    __syncthreads();
    pwa::tc::fence_after();
    const uint32_t tm = *tslot;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Cp >> 3) << 17) | ((128u >> 4) << 24);

    // this thread's Gram entries: row m = 32 (warp mod 4) + lane, columns c0 .. c0 + CPT - 1
    const int qd = warp & 3, m = 32 * qd + lane, c0 = (warp >> 2) * CPT;
    const uint32_t tlane = (uint32_t)(32 * qd) << 16;
    float ax[CPT], az[CPT];
#pragma unroll
    for (int j = 0; j < CPT; ++j) ax[j] = az[j] = 0.f;
    float q[kTcKW][6];
#pragma unroll
    for (int j = 0; j < kTcKW; ++j)
#pragma unroll
        for (int u = 0; u < 6; ++u) q[j][u] = 0.f;
    float sc = 0.f;

    double* rec = a.rec + (size_t)blockIdx.x * a.rec_len;
    const int CC = C * C;
    const int offQ = 3 * CC, offS = offQ + 12 * K;
    // FP32 Gram sums of sample set smp into the FP64 record
    auto fold_g = [&](int smp) {
        double* rx = rec + (smp == 0 ? 0 : 2 * CC);
        double* rz = rec + CC;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int c = c0 + j;
            if (m < C && c < C) {
                rx[m * C + c] += (double)ax[j];
                if (smp == 0) rz[m * C + c] += (double)az[j];
            }
            ax[j] = az[j] = 0.f;
        }
    };
    // FP32 Q and scalar sums of sample set smp into the FP64 record
    auto fold_q = [&](int smp) {
#pragma unroll
        for (int j = 0; j < kTcKW; ++j) {
            const int k = warp + j * NW;
#pragma unroll
            for (int u = 0; u < 6; ++u) {
                const float v = pwa::warp_sum(q[j][u]);
                q[j][u] = 0.f;
                if (lane == 0 && k < K) rec[offQ + ((size_t)smp * K + k) * 6 + u] += (double)v;
            }
        }
        const float v = pwa::warp_sum(sc);
        sc = 0.f;
        if (lane == 0) rec[offS + 2 * warp + smp] += (double)v;
    };
    // accumulator set sb (a finished tile's MMAs) into the FP32 sums; z only for data tiles
    auto read_back = [&](int sb, bool with_z) {
        const uint32_t base = tm + (uint32_t)(256 * sb) + tlane + (uint32_t)c0;
        {
            uint32_t v[CPT / 8][8];
#pragma unroll
            for (int ch = 0; ch < CPT / 8; ++ch) pwa::tc::tmem_ld8(base + 8 * ch, v[ch]);
            pwa::tc::tmem_wait();
#pragma unroll
            for (int ch = 0; ch < CPT / 8; ++ch)
#pragma unroll
                for (int u = 0; u < 8; ++u) ax[8 * ch + u] += __uint_as_float(v[ch][u]);
        }
        if (with_z) {
            uint32_t v[CPT / 8][8];
#pragma unroll
            for (int ch = 0; ch < CPT / 8; ++ch) pwa::tc::tmem_ld8(base + 128 + 8 * ch, v[ch]);
            pwa::tc::tmem_wait();
#pragma unroll
            for (int ch = 0; ch < CPT / 8; ++ch)
#pragma unroll
                for (int u = 0; u < 8; ++u) az[8 * ch + u] += __uint_as_float(v[ch][u]);
        }
    };

    int st = 0;
    uint32_t ph = 0;
    int win_q = 0, win_g = 0;
    int cur_q = 0, cur_g = 0;  // sample sets of the Q/scalar sums and of the Gram sums in registers
    int pend_smp = -1;         // two buffers: sample set of the tile whose read-back is pending (-1: none)
    long long i = 0;
    bool aborted = false;      // the same in every thread (decided at a barrier)
    bool failed = false;       // this thread's last wait gave up
    long long last_mma = -1;   // the last tile whose MMAs were issued
    const bool issuer = tid == NT - 32;  // lane 0 of the last warp (the fewest resonances) issues copies and MMAs
    // this thread's wait for tile j's MMAs (accumulator set j mod NBUF, the (j / NBUF)-th commit there)
    auto wait_mma = [&](long long j) -> bool {
        const int sb = NBUF == 2 ? (int)(j & 1) : 0;
        const uint32_t par = (uint32_t)((NBUF == 2 ? (j >> 1) : j) & 1);
        return pwa::mbar_wait(&mbar[2 + sb], par, a.timeout_cycles);
    };
    // tile j's accumulators (sample set smp) into the FP32 sums, once its MMAs are done
    auto finish_tile = [&](long long j, int smp) {
        failed |= !wait_mma(j);
        pwa::tc::fence_after();
        if (smp != cur_g) {
            fold_g(cur_g);
            win_g = 0;
            cur_g = smp;
        }
        read_back(NBUF == 2 ? (int)(j & 1) : 0, smp == 0);
        if (++win_g == kFoldG) {
            fold_g(cur_g);
            win_g = 0;
        }
        pwa::tc::fence_before();
    };
    for (long long t = gb; t < T; t += G, ++i) {
        int smp;
        long long lt;
        tile_src(t, smp, lt);
        if (smp != cur_q) {
            fold_q(cur_q);
            win_q = 0;
            cur_q = smp;
        }
        // the tile's copy (each thread waits; a failure is acted on at the next barrier)
        failed |= !pwa::mbar_wait(&mbar[st], ph, a.timeout_cycles);
        const int b = NBUF == 2 ? (int)(i & 1) : 0;
        unsigned char* xo = smem + (b ? L.x[1] : L.x[0]);
        unsigned char* zo = smem + (b ? L.z[1] : L.z[0]);
        const float* Ft = reinterpret_cast<const float*>(stages + (size_t)st * a.stage_bytes);
        const float* m2s = Ft + (size_t)2 * K * S * kE;
        const long long e_base = lt * kE;
        const int e = lane;
        const bool valid = e < (int)min((long long)kE, a.nev[smp] - e_base);

        // ---- event phase: BW and the coherent sums A_s over this warp's resonances ----
        float br[kTcKW], bim[kTcKW];
        // even S: F as packed pairs over two projections, fv[j][2q] = (Re F_2q, Re F_2q+1),
        // fv[j][2q+1] = (Im F_2q, Im F_2q+1), and A likewise; odd S: fv[j][s] = (Re F_s, Im F_s)
        float2 fv[kTcKW][S];
        float2 Ap[S];
#pragma unroll
        for (int s = 0; s < S; ++s) Ap[s] = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < kTcKW; ++j) {
            const int k = warp + j * NW;
            br[j] = bim[j] = 0.f;
#pragma unroll
            for (int s = 0; s < S; ++s) fv[j][s] = make_float2(0.f, 0.f);
            if (k < K) {
                const KConst c = kc[k];
                pwa::breit_wigner(c, m2s[c.ch * kE + e], br[j], bim[j]);
                const float cr = c.gre * br[j] - c.gim * bim[j], ci = c.gre * bim[j] + c.gim * br[j];
                const int p = (e + c.shift) & (kE - 1);
                if constexpr (S % 2 == 0) {
                    const float2 crr = make_float2(cr, cr), cii = make_float2(ci, ci), ncc = make_float2(-ci, -ci);
#pragma unroll
                    for (int qq = 0; qq < S / 2; ++qq) {
                        const float4 f4 = *reinterpret_cast<const float4*>(Ft + 4 * ((k * (S / 2) + qq) * kE + p));
                        const float2 R2 = make_float2(f4.x, f4.y), I2 = make_float2(f4.z, f4.w);
                        fv[j][2 * qq] = R2;
                        fv[j][2 * qq + 1] = I2;
                        Ap[2 * qq] = __ffma2_rn(I2, ncc, __ffma2_rn(R2, crr, Ap[2 * qq]));
                        Ap[2 * qq + 1] = __ffma2_rn(I2, crr, __ffma2_rn(R2, cii, Ap[2 * qq + 1]));
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        const float2 f2 = *reinterpret_cast<const float2*>(Ft + 2 * ((k * S + s) * kE + p));
                        fv[j][s] = f2;
                        Ap[s].x += cr * f2.x - ci * f2.y;
                        Ap[s].y += cr * f2.y + ci * f2.x;
                    }
                }
            }
        }
        // the warps' partial sums: warp c < 2S adds up component c over the warps (fixed order)
#pragma unroll
        for (int s = 0; s < S; ++s) {
            PA[(warp * 2 * S + 2 * s) * 32 + e] = Ap[s].x;
            PA[(warp * 2 * S + 2 * s + 1) * 32 + e] = Ap[s].y;
        }
        if (__syncthreads_or(failed)) {  // a copy or the previous tile's MMAs never completed
            aborted = true;
            break;
        }
        if (warp < 2 * S) {
            float x = 0.f;
#pragma unroll
            for (int w = 0; w < NW; ++w) x += PA[(w * 2 * S + warp) * 32 + e];
            PT[warp * 32 + e] = x;
        }
        __syncthreads();
        float I = 0.f;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            Ap[s] = make_float2(PT[(2 * s) * 32 + e], PT[(2 * s + 1) * 32 + e]);
            I += Ap[s].x * Ap[s].x + Ap[s].y * Ap[s].y;
        }
        float aw = 0.f, sqa = 0.f, zw = 0.f;
        if (smp == 0) {
            const float w = m2s[3 * kE + e];
            const bool good = I > 0.f && I < INFINITY;
            if (valid && good) {
                aw = w / I;
                sqa = sqrtf(aw);
                zw = sqrtf(w) / I;
                if (warp == 0) sc += w * logf(I);
            } else if (valid && warp == 0) {
                atomicMin(a.bad, (unsigned long long)(e_base + e));
                atomicOr(a.err, pwa::ERR_NONFINITE);
                atomicOr(a.err_vec + bt, pwa::ERR_NONFINITE);
            }
        } else {
            const bool good = I < INFINITY;
            if (valid && good) {
                aw = 1.f;
                sqa = 1.f;
                if (warp == 0) sc += I;
            } else if (valid && warp == 0) {
                atomicMin(a.bad, (unsigned long long)(a.nev[0] + e_base + e));
                atomicOr(a.err, pwa::ERR_NONFINITE);
                atomicOr(a.err_vec + bt, pwa::ERR_NONFINITE);
            }
        }
        // ---- per resonance: the X columns (sqrt a (B F, B^2 F)), D, the z columns and Q ----
        float2 nAi[S];  // even S: minus the imaginary pairs of A (for Im D)
        if constexpr (S % 2 == 0) {
#pragma unroll
            for (int qq = 0; qq < S / 2; ++qq) nAi[qq] = make_float2(-Ap[2 * qq + 1].x, -Ap[2 * qq + 1].y);
        }
#pragma unroll
        for (int j = 0; j < kTcKW; ++j) {
            const int k = warp + j * NW;
            if (k >= K) continue;
            const float b1r = br[j], b1i = bim[j];
            const float b2r = b1r * b1r - b1i * b1i, b2i = 2.f * b1r * b1i;
            const float b3r = b2r * b1r - b2i * b1i, b3i = b2r * b1i + b2i * b1r;
            const float p1r = sqa * b1r, p1i = sqa * b1i, p2r = sqa * b2r, p2i = sqa * b2i;
            const int c1 = 2 * k, c2 = 2 * (K + k);  // columns of Re (B F), Re (B^2 F); Im at + 1
            float v[4][S];
            float Dr, Di;
            if constexpr (S % 2 == 0) {
                float2 DR = make_float2(0.f, 0.f), DI = DR;
#pragma unroll
                for (int qq = 0; qq < S / 2; ++qq) {
                    const float2 R2 = fv[j][2 * qq], I2 = fv[j][2 * qq + 1];
                    // D = sum_s conj(A_s) F_s
                    DR = __ffma2_rn(Ap[2 * qq + 1], I2, __ffma2_rn(Ap[2 * qq], R2, DR));
                    DI = __ffma2_rn(nAi[qq], R2, __ffma2_rn(Ap[2 * qq], I2, DI));
                    const float2 x0 = __ffma2_rn(I2, make_float2(-p1i, -p1i), __fmul2_rn(R2, make_float2(p1r, p1r)));
                    const float2 x1 = __ffma2_rn(I2, make_float2(p1r, p1r), __fmul2_rn(R2, make_float2(p1i, p1i)));
                    const float2 x2 = __ffma2_rn(I2, make_float2(-p2i, -p2i), __fmul2_rn(R2, make_float2(p2r, p2r)));
                    const float2 x3 = __ffma2_rn(I2, make_float2(p2r, p2r), __fmul2_rn(R2, make_float2(p2i, p2i)));
                    v[0][2 * qq] = x0.x;
                    v[0][2 * qq + 1] = x0.y;
                    v[1][2 * qq] = x1.x;
                    v[1][2 * qq + 1] = x1.y;
                    v[2][2 * qq] = x2.x;
                    v[2][2 * qq + 1] = x2.y;
                    v[3][2 * qq] = x3.x;
                    v[3][2 * qq + 1] = x3.y;
                }
                Dr = DR.x + DR.y;
                Di = DI.x + DI.y;
            } else {
                Dr = Di = 0.f;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const float fr = fv[j][s].x, fi = fv[j][s].y;
                    Dr += Ap[s].x * fr + Ap[s].y * fi;
                    Di += Ap[s].x * fi - Ap[s].y * fr;
                    v[0][s] = p1r * fr - p1i * fi;
                    v[1][s] = p1r * fi + p1i * fr;
                    v[2][s] = p2r * fr - p2i * fi;
                    v[3][s] = p2r * fi + p2i * fr;
                }
            }
            const int cols[4] = {c1, c1 + 1, c2, c2 + 1};
#pragma unroll
            for (int u = 0; u < 4; ++u) store_rows<S>(xo, L.pbx, tc_off(cols[u], e * S, L.sbox), v[u]);
            const float z1r = b1r * Dr - b1i * Di, z1i = b1r * Di + b1i * Dr;
            const float z2r = b2r * Dr - b2i * Di, z2i = b2r * Di + b2i * Dr;
            const float z3r = b3r * Dr - b3i * Di, z3i = b3r * Di + b3i * Dr;
            if (smp == 0) {
                store_split(zo, L.pbz, tc_off(c1, e, L.sboz), zw * z1r);
                store_split(zo, L.pbz, tc_off(c1 + 1, e, L.sboz), zw * z1i);
                store_split(zo, L.pbz, tc_off(c2, e, L.sboz), zw * z2r);
                store_split(zo, L.pbz, tc_off(c2 + 1, e, L.sboz), zw * z2i);
            }
            q[j][0] = fmaf(aw, z1r, q[j][0]);
            q[j][1] = fmaf(aw, z1i, q[j][1]);
            q[j][2] = fmaf(aw, z2r, q[j][2]);
            q[j][3] = fmaf(aw, z2i, q[j][3]);
            q[j][4] = fmaf(aw, z3r, q[j][4]);
            q[j][5] = fmaf(aw, z3i, q[j][5]);
        }
        // the operands are complete (generic writes, read by the tensor cores' async proxy)
        pwa::fence_proxy_async();
        pwa::tc::fence_before();
        __syncthreads();
        if (issuer) {
            const long long tn = t + 2LL * G;
            if (tn < T) {
                int s2;
                long long lt2;
                tile_src(tn, s2, lt2);
                issued[st] = i + 2;
                pwa::tma_load_tile(stages + (size_t)st * a.stage_bytes, a.tiles[s2] + (size_t)lt2 * a.tile_bytes[s2],
                                   a.tile_bytes[s2], &mbar[st]);
            }
            pwa::tc::fence_after();
            // D = hi^T hi + hi^T (2 lo) over the tile's rows, 16 rows per step
            const uint32_t xa = pwa::tc::sa(xo), za = pwa::tc::sa(zo), dx = tm + (uint32_t)(256 * b);
#pragma unroll 1
            for (int ks = 0; ks < R / 16; ++ks) {
                const uint64_t dh = pwa::tc::sdesc(xa + ks * 2 * kTcLbo, kTcLbo, L.sbox);
                const uint64_t dl = pwa::tc::sdesc(xa + L.pbx + ks * 2 * kTcLbo, kTcLbo, L.sbox);
                pwa::tc::mma_bf16(dx, dh, dh, idesc, ks > 0);
                pwa::tc::mma_bf16(dx, dh, dl, idesc, 1);
            }
            if (smp == 0) {
#pragma unroll 1
                for (int ks = 0; ks < 2; ++ks) {
                    const uint64_t dh = pwa::tc::sdesc(za + ks * 2 * kTcLbo, kTcLbo, L.sboz);
                    const uint64_t dl = pwa::tc::sdesc(za + L.pbz + ks * 2 * kTcLbo, kTcLbo, L.sboz);
                    pwa::tc::mma_bf16(dx + 128, dh, dh, idesc, ks > 0);
                    pwa::tc::mma_bf16(dx + 128, dh, dl, idesc, 1);
                }
            }
            pwa::tc::mma_commit(&mbar[2 + b]);
        }
        last_mma = i;
        if (++win_q == kFold) {
            fold_q(cur_q);
            win_q = 0;
        }
        if (++st == 2) {
            st = 0;
            ph ^= 1u;
        }
        // read back: two buffers, the previous tile's accumulators (this tile's MMAs
        // meanwhile run); one buffer, this tile's.  Each thread waits for the MMAs
        // itself, so its next operand writes and the next MMAs into the set it
        // read (issued after the next barriers) follow its loads.
        if constexpr (NBUF == 2) {
            if (pend_smp >= 0) finish_tile(i - 1, pend_smp);
            pend_smp = smp;
        } else {
            finish_tile(i, smp);
        }
    }
    if (!aborted && NBUF == 2 && pend_smp >= 0) finish_tile(i - 1, pend_smp);
    if (__syncthreads_or(failed)) aborted = true;
    if (aborted) {
        // a copy or a tile's MMAs never completed: report it, wait (bounded)
        // for what is still in flight, free TMEM
        if (tid == 0) {
            atomicOr(a.err, pwa::ERR_TIMEOUT);
            for (int s = 0; s < 2; ++s)
                if (issued[s] >= 0) (void)pwa::mbar_wait(&mbar[s], (uint32_t)((issued[s] / 2) & 1), a.timeout_cycles);
            for (long long j = last_mma; j >= 0 && j > last_mma - 2; --j) (void)wait_mma(j);
        }
    } else {
        fold_g(cur_g);
        fold_q(cur_q);
    }
    pwa::tc::fence_before();
    __syncthreads();
    pwa::tc::fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(tc_tmem_cols(NBUF)));
}

// Fixed-order sum of the per-CTA records of each vector: out[bt] = sum over
// gb of the record of CTA gb B + bt.
__global__ void hess_reduce_kernel(const double* __restrict__ rec, int B, int Gb, int rec_len,
                                   double* __restrict__ out)
{
    const long long n = (long long)B * rec_len;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const int bt = (int)(j / rec_len), i = (int)(j % rec_len);
        double s = 0.0;
        for (int g = 0; g < Gb; ++g) s += rec[((size_t)g * B + bt) * rec_len + i];
        out[j] = s;
    }
}

using KernelH = void (*)(const HessArgs);

template <int S>
KernelH pick_s(int NT)
{
    return NT == 256 ? hess_kernel<S, 256, 1> : hess_kernel<S, 512, 2>;
}

KernelH pick_hess(int S, int NT)
{
    switch (S) {
        case 1: return pick_s<1>(NT);
        case 2: return pick_s<2>(NT);
        case 3: return pick_s<3>(NT);
        case 4: return pick_s<4>(NT);
        default: return nullptr;
    }
}

template <int S>
KernelH pick_tc_s(int nch)
{
    switch (nch) {
        case 1: return hess_tc_kernel<S, 1>;
        case 2: return hess_tc_kernel<S, 2>;
        case 3: return hess_tc_kernel<S, 3>;
        case 4: return hess_tc_kernel<S, 4>;
        case 5: return hess_tc_kernel<S, 5>;
        case 6: return hess_tc_kernel<S, 6>;
        case 7: return hess_tc_kernel<S, 7>;
        case 8: return hess_tc_kernel<S, 8>;
        default: return nullptr;
    }
}

KernelH pick_tc(int S, int K)
{
    const int nch = (4 * K + 15) / 16;
    switch (S) {
        case 1: return pick_tc_s<1>(nch);
        case 2: return pick_tc_s<2>(nch);
        case 3: return pick_tc_s<3>(nch);
        case 4: return pick_tc_s<4>(nch);
        default: return nullptr;
    }
}

using cplx = std::complex<double>;

// Combine the summed records into NLL, gradient and Hessian in the free
// parameters (FP64, host).
void combine(const pwa_handle* h, const double* theta, const double* sum, int NW, bool tc, double* nll,
             double* grad, double* hess)
{
    const int K = h->K, P = h->P, nb = K * (K + 1) / 2, C = 4 * K;
    // the three symmetric 4K x 4K Gram matrices (0: data X, 1: data z, 2: MC X):
    // the tensor-core records hold each full and not yet symmetric, read as
    // (x_ab + x_ba) / 2 in place; the CUDA-core records hold upper-triangle
    // blocks, expanded once
    const int CC = C * C;
    std::vector<double> Gx[3];
    if (!tc) {
        const int offs[3] = {0, 16 * nb, 32 * nb};
        for (int m = 0; m < 3; ++m) {
            Gx[m].assign((size_t)C * C, 0.0);
            for (int b = 0; b < nb; ++b) {
                int bi, bj;
                block_of(b, K, bi, bj);
                for (int u = 0; u < 4; ++u)
                    for (int v = 0; v < 4; ++v) {
                        const double x = sum[offs[m] + 16 * b + 4 * u + v];
                        const int ca = bi + u * K, cb = bj + v * K;
                        Gx[m][(size_t)ca * C + cb] = x;
                        Gx[m][(size_t)cb * C + ca] = x;
                    }
            }
        }
    }
    auto at = [&](int m, int a, int b) -> double {
        if (tc) {
            const double* x = sum + (size_t)m * CC;
            return 0.5 * (x[(size_t)a * C + b] + x[(size_t)b * C + a]);
        }
        return Gx[m][(size_t)a * C + b];
    };
    // C[c][c'] = sum a sum_s conj(V_c) V_c', c = p K + k, from Gram matrix m (0 data, 2 MC)
    auto cgram = [&](int m, int c, int cp) {
        return cplx(at(m, 2 * c, 2 * cp) + at(m, 2 * c + 1, 2 * cp + 1),
                    at(m, 2 * c, 2 * cp + 1) - at(m, 2 * c + 1, 2 * cp));
    };
    const int offQ = tc ? 3 * CC : 48 * nb, offS = offQ + 12 * K;
    std::vector<cplx> Q[2][3];
    for (int smp = 0; smp < 2; ++smp)
        for (int pp = 0; pp < 3; ++pp) Q[smp][pp].assign(K, cplx(0, 0));
    for (int smp = 0; smp < 2; ++smp)
        for (int k = 0; k < K; ++k) {
            const double* qq = sum + offQ + ((size_t)smp * K + k) * 6;
            for (int pp = 0; pp < 3; ++pp) Q[smp][pp][k] = cplx(qq[2 * pp], qq[2 * pp + 1]);
        }
    double SlnI = 0.0, Gm = 0.0;
    for (int w = 0; w < NW; ++w) {
        SlnI += sum[offS + 2 * w];
        Gm += sum[offS + 2 * w + 1];
    }
    const double Nd = h->Nd;
    *nll = -SlnI + Nd * std::log(Gm / h->Nmc);

    // per free parameter: resonance, kind, kappa1, kappa2
    struct ParInfo {
        int k, j;
        cplx k1, k2;
    };
    std::vector<ParInfo> par(P);
    std::vector<double> rho(K), phi(K), M(K), Gw(K);
    for (int k = 0; k < K; ++k) {
        const pwa::ResParam& r = h->res[k];
        double v[4];
        for (int j = 0; j < 4; ++j) v[j] = r.idx[j] >= 0 ? theta[r.idx[j]] : r.fixed[j];
        rho[k] = v[0];
        phi[k] = v[1];
        M[k] = v[2];
        Gw[k] = v[3];
        const cplx E1 = std::polar(1.0, v[1]), g = v[0] * E1;
        const cplx a1(-2.0 * v[2], v[3]), a2(0.0, v[2]);
        const cplx kap1[4] = {E1, cplx(0, 1) * g, 0.0, 0.0};
        const cplx kap2[4] = {0.0, 0.0, g * a1, g * a2};
        for (int j = 0; j < 4; ++j)
            if (r.idx[j] >= 0) par[r.idx[j]] = ParInfo{k, j, kap1[j], kap2[j]};
    }
    // second-derivative coefficients mu1, mu2, mu3 of d2c_k / dtheta_j dtheta_j'
    auto mu = [&](int k, int j, int jp, cplx& m1, cplx& m2, cplx& m3) {
        const cplx E1 = std::polar(1.0, phi[k]), g = rho[k] * E1, I1(0, 1);
        const cplx a1(-2.0 * M[k], Gw[k]), a2(0.0, M[k]);
        if (j > jp) std::swap(j, jp);
        m1 = m2 = m3 = 0.0;
        if (j == 0 && jp == 1) m1 = I1 * E1;
        else if (j == 0 && jp == 2) m2 = E1 * a1;
        else if (j == 0 && jp == 3) m2 = E1 * a2;
        else if (j == 1 && jp == 1) m1 = -g;
        else if (j == 1 && jp == 2) m2 = I1 * g * a1;
        else if (j == 1 && jp == 3) m2 = I1 * g * a2;
        else if (j == 2 && jp == 2) {
            m2 = -2.0 * g;
            m3 = 2.0 * g * a1 * a1;
        } else if (j == 2 && jp == 3) {
            m2 = I1 * g;
            m3 = 2.0 * g * a1 * a2;
        } else if (j == 3 && jp == 3) {
            m3 = 2.0 * g * a2 * a2;
        }
    };
    // gradients of the data and MC sums: dI sums = 2 Re (kappa1 Q1 + kappa2 Q2)
    std::vector<double> gD(P), gM(P);
    for (int i = 0; i < P; ++i) {
        const ParInfo& pi = par[i];
        gD[i] = 2.0 * std::real(pi.k1 * Q[0][0][pi.k] + pi.k2 * Q[0][1][pi.k]);
        gM[i] = 2.0 * std::real(pi.k1 * Q[1][0][pi.k] + pi.k2 * Q[1][1][pi.k]);
        if (grad) grad[i] = -gD[i] + Nd * gM[i] / Gm;
    }
    if (!hess) return;
    // z coefficients: dI/dtheta_i = c_i . z with c at columns 2 (p K + k) + (0, 1)
    for (int i = 0; i < P; ++i)
        for (int ip = i; ip < P; ++ip) {
            const ParInfo &a = par[i], &b = par[ip];
            const cplx ka[2] = {a.k1, a.k2}, kb[2] = {b.k1, b.k2};
            double s2d = 0.0, s2m = 0.0, jg = 0.0;
            for (int p = 0; p < 2; ++p)
                for (int pp = 0; pp < 2; ++pp) {
                    if (ka[p] == 0.0 || kb[pp] == 0.0) continue;
                    const int c = p * K + a.k, cp = pp * K + b.k;
                    s2d += 2.0 * std::real(std::conj(ka[p]) * kb[pp] * cgram(0, c, cp));
                    s2m += 2.0 * std::real(std::conj(ka[p]) * kb[pp] * cgram(2, c, cp));
                    // c_a^T Zg c_b with c = (2 Re kappa, -2 Im kappa) at the z columns of (p, k)
                    const double ca[2] = {2.0 * ka[p].real(), -2.0 * ka[p].imag()};
                    const double cb[2] = {2.0 * kb[pp].real(), -2.0 * kb[pp].imag()};
                    for (int u = 0; u < 2; ++u)
                        for (int v = 0; v < 2; ++v)
                            jg += ca[u] * cb[v] * at(1, 2 * c + u, 2 * cp + v);
                }
            if (a.k == b.k) {
                cplx m1, m2, m3;
                mu(a.k, a.j, b.j, m1, m2, m3);
                s2d += 2.0 * std::real(m1 * Q[0][0][a.k] + m2 * Q[0][1][a.k] + m3 * Q[0][2][a.k]);
                s2m += 2.0 * std::real(m1 * Q[1][0][a.k] + m2 * Q[1][1][a.k] + m3 * Q[1][2][a.k]);
            }
            const double hval = -(s2d - jg) + Nd * (s2m / Gm - gM[i] * gM[ip] / (Gm * Gm));
            hess[(size_t)i * P + ip] = hval;
            hess[(size_t)ip * P + i] = hval;
        }
}

}  // namespace

namespace pwa {

// Enqueue the Hessian pass of B parameter vectors (host theta [B][P]) on the
// handle's stream: theta upload, the pass, the per-vector reduction and the
// download of the sums and error words.  hessian_finish waits and combines.
pwa_status hessian_issue(pwa_handle* h, int B, const double* theta)
{
    const int K = h->K, S = h->S, P = h->P;
    if (K > kMaxKHess)
        return set_error(h, PWA_EINVAL, "the Hessian pass supports K <= " + std::to_string(kMaxKHess));
    if (h->broken) return set_error(h, PWA_ETIMEOUT, "handle is unusable after a device-side timeout");
    if (B < 1) return set_error(h, PWA_EINVAL, "B must be at least 1");
    const int nblk = K * (K + 1) / 2;
    // the tensor-core Gram for K <= 32 (unless the CUDA-core kernel is asked for), else the CUDA-core one
    const bool tc = K <= kMaxKTensor && !h->hess_cuda_cores;
    const int NT = tc ? kTcNT : (nblk <= 256 ? 256 : 512);
    const int NW = NT / 32;
    KernelH fn = tc ? pick_tc(S, K) : pick_hess(S, NT);
    if (!fn) return set_error(h, PWA_EINVAL, "no Hessian kernel for this S");
    const Tiling& t = h->tiling;
    const uint32_t stage = (uint32_t)((std::max(h->tile_bytes[0], h->tile_bytes[1]) + 127) / 128 * 128);
    const int C = 4 * K;
    const size_t smem = tc ? hess_tc_smem(K, S, stage)
                           : 2 * (size_t)stage + sizeof(KConst) * K +
                                 sizeof(float) * ((size_t)C * (x_stride(S) + kZStride) + (size_t)NW * 2 * S * 32) + 16;
    HessState& hs = h->hess;
    cudaError_t e = cudaSuccess;
    if (hs.fn != reinterpret_cast<const void*>(fn) || hs.smem != smem) {
        int dev = 0, max_optin = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return cuda_error(h, e, "cudaDeviceGetAttribute");
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(fn));
        if (e != cudaSuccess) return cuda_error(h, e, "cudaFuncGetAttributes");
        const int dyn_max = max_optin - (int)fa.sharedSizeBytes;
        if ((int)smem > dyn_max)
            return set_error(h, PWA_EINVAL, "the Hessian pass needs " + std::to_string(smem) +
                                                " bytes of shared memory per block (max " + std::to_string(dyn_max) +
                                                ")");
        e = cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dyn_max);
        if (e != cudaSuccess) return cuda_error(h, e, "cudaFuncSetAttribute");
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<const void*>(fn), NT, smem);
        if (e != cudaSuccess) return cuda_error(h, e, "occupancy");
        if (occ < 1) return set_error(h, PWA_EINVAL, "the Hessian pass does not fit on an SM");
        hs.fn = reinterpret_cast<const void*>(fn);
        hs.smem = smem;
        hs.resident = h->num_sms * occ;
        hs.rec_len = tc ? hess_tc_rec_len(K) : hess_rec_len(K, nblk, NW);
    }
    // CTAs per vector: the vectors share one wave of resident CTAs (at least one each)
    const long long T = (long long)h->ntiles[0] + h->ntiles[1];
    const int Gb = (int)std::max(1LL, std::min((long long)std::max(1, hs.resident / B), T));
    const size_t rl = (size_t)hs.rec_len;
    const size_t need = sizeof(double) * ((size_t)B * Gb * rl + (size_t)B * rl + (size_t)B * P) + sizeof(int) * B;
    const size_t need_h = sizeof(double) * ((size_t)B * rl + (size_t)B * P) + sizeof(int) * B;
    if (need > hs.cap_bytes || need_h > hs.cap_host) {
        if (hs.d_rec) cudaFree(hs.d_rec);
        if (hs.h_buf) cudaFreeHost(hs.h_buf);
        hs.d_rec = nullptr;
        hs.h_buf = nullptr;
        hs.cap_bytes = hs.cap_host = 0;
        if (cudaMalloc(reinterpret_cast<void**>(&hs.d_rec), need) != cudaSuccess) {
            cudaGetLastError();
            return set_error(h, PWA_ENOMEM, "cudaMalloc failed for the Hessian records");
        }
        if (cudaMallocHost(reinterpret_cast<void**>(&hs.h_buf), need_h) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(hs.d_rec);
            hs.d_rec = nullptr;
            return set_error(h, PWA_ENOMEM, "pinned allocation failed for the Hessian sums");
        }
        hs.cap_bytes = need;
        hs.cap_host = need_h;
    }
    HessArgs a;
    for (int s = 0; s < 2; ++s) {
        a.tiles[s] = h->d_tiles[s];
        a.tile_bytes[s] = h->tile_bytes[s];
        a.ntiles[s] = h->ntiles[s];
        a.nev[s] = h->n[s];
        if (h->tile_bytes[s] > stage || h->tile_bytes[s] % 16 != 0 || (long long)h->ntiles[s] * kE < h->n[s])
            return set_error(h, PWA_EINVAL, "inconsistent tile geometry");
    }
    // device: records [B Gb][rl] | sums [B][rl] | theta [B][P] | error words [B]
    double* d_sum = hs.d_rec + (size_t)B * Gb * rl;
    double* d_th = d_sum + (size_t)B * rl;
    int* d_ev = reinterpret_cast<int*>(d_th + (size_t)B * P);
    // host (pinned): sums [B][rl] | theta [B][P] | error words [B]
    double* h_th = hs.h_buf + (size_t)B * rl;
    int* h_ev = reinterpret_cast<int*>(h_th + (size_t)B * P);
    a.K = K;
    a.ev = 32 / t.W;
    a.stage_bytes = stage;
    a.res = h->d_res;
    a.theta = d_th;
    a.P = P;
    a.B = B;
    a.Gb = Gb;
    a.nblk = nblk;
    a.rec = hs.d_rec;
    a.rec_len = hs.rec_len;
    a.bad = h->d_bad;
    a.err = h->d_err;
    a.err_vec = d_ev;
    a.timeout_cycles = h->timeout_cycles;

    std::memcpy(h_th, theta, sizeof(double) * (size_t)B * P);
    e = cudaMemcpyAsync(d_th, h_th, sizeof(double) * (size_t)B * P, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(hs.d_rec, 0, sizeof(double) * (size_t)B * Gb * rl, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ev, 0, sizeof(int) * B, h->stream);
    if (e != cudaSuccess) return cuda_error(h, e, "Hessian inputs");
    fn<<<B * Gb, NT, smem, h->stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(h, e, "Hessian kernel launch");
    const long long nred = (long long)B * rl;
    const int rgrid = (int)std::min<long long>((nred + 255) / 256, 4LL * h->num_sms);
    hess_reduce_kernel<<<rgrid, 256, 0, h->stream>>>(hs.d_rec, B, Gb, hs.rec_len, d_sum);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hs.h_buf, d_sum, sizeof(double) * (size_t)B * rl, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_ev, d_ev, sizeof(int) * B, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_pin + P, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_error(h, e, "Hessian pass");
    hs.B = B;
    hs.NW = NW;
    hs.tc = tc;
    return PWA_OK;
}

// Wait for the pass that hessian_issue enqueued for these B vectors and
// combine each vector's sums.  status[b] (when given) receives PWA_OK or
// PWA_ENONFINITE per vector; without it a non-finite vector fails the call.
// nll, grad may be NULL; hess [B][P][P].
pwa_status hessian_finish(pwa_handle* h, int B, const double* theta, double* nll, double* grad, double* hess,
                          pwa_status* status)
{
    HessState& hs = h->hess;
    if (B != hs.B) return set_error(h, PWA_EINVAL, "hessian_finish does not match the issued batch");
    const int P = h->P;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_error(h, e, "Hessian pass");
    const size_t rl = (size_t)hs.rec_len;
    const int* h_ev = reinterpret_cast<const int*>(hs.h_buf + (size_t)B * rl + (size_t)B * P);
    int errw = 0;
    std::memcpy(&errw, h->h_pin + P, sizeof(int));
    if (errw) {
        // a timeout fails the batch; non-finite intensities fail only their vectors
        pwa_status st = check_device_errors(h);
        if (st != PWA_OK && st != PWA_ENONFINITE) return st;
        if (st == PWA_ENONFINITE && !status) return st;
    }
    for (int b = 0; b < B; ++b) {
        if (status) status[b] = h_ev[b] ? PWA_ENONFINITE : PWA_OK;
        if (h_ev[b]) continue;
        double f = 0.0;
        combine(h, theta + (size_t)b * P, hs.h_buf + (size_t)b * rl, hs.NW, hs.tc, &f,
                grad ? grad + (size_t)b * P : nullptr, hess + (size_t)b * P * P);
        if (nll) nll[b] = f;
    }
    return PWA_OK;
}

pwa_status hessian_device(pwa_handle* h, const double* theta, double* nll, double* grad, double* hess)
{
    pwa_status st = hessian_issue(h, 1, theta);
    if (st != PWA_OK) return st;
    return hessian_finish(h, 1, theta, nll, grad, hess, nullptr);
}

void free_hessian(pwa_handle* h)
{
    if (h->hess.d_rec) cudaFree(h->hess.d_rec);
    if (h->hess.h_buf) cudaFreeHost(h->hess.h_buf);
    h->hess = HessState();
}

}  // namespace pwa

extern "C" pwa_status pwa_set_hessian_cuda_cores(pwa_handle* h, int cuda_cores)
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    h->hess_cuda_cores = cuda_cores != 0;
    return PWA_OK;
}

extern "C" pwa_status pwa_hessian(pwa_handle* h, const double* theta, double* nll, double* grad, double* hess)
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    if (!theta || !hess) return pwa::set_error(h, PWA_EINVAL, "theta and hess must not be NULL");
    for (int i = 0; i < h->P; ++i)
        if (!std::isfinite(theta[i])) return pwa::set_error(h, PWA_EINVAL, "theta must be finite");
    return pwa::hessian_device(h, theta, nll, grad, hess);
}

extern "C" pwa_status pwa_hessian_batch(pwa_handle* h, int B, const double* theta, double* nll, double* grad,
                                        double* hess, pwa_status* status)
{
    if (!h) return PWA_EINVAL;
    h->err.clear();
    if (B < 1 || !theta || !hess) return pwa::set_error(h, PWA_EINVAL, "B >= 1, theta and hess are required");
    for (size_t i = 0; i < (size_t)B * h->P; ++i)
        if (!std::isfinite(theta[i])) return pwa::set_error(h, PWA_EINVAL, "theta must be finite");
    pwa_status st = pwa::hessian_issue(h, B, theta);
    if (st != PWA_OK) return st;
    return pwa::hessian_finish(h, B, theta, nll, grad, hess, status);
}
