// variant.cu -- physics variants of the likelihood: line shapes beyond the
// constant-width Breit-Wigner (a mass-dependent width, the Flatte form) and one
// coupling per (resonance, projection), with the NLL, its gradient and the exact
// H v (paper Eqs. 1, 3, 6, 7) from one pass over the events.
//
// Kernel layout: a warp walks tiles of 32 events one event at a time; lane k
// owns resonance k: it evaluates BW_k and its derivatives in the resonance's
// shape parameters for the event, forms its terms of the coherent sums
// A_s = sum_k g_ks BW_k F_ks (and of the directional sums Adot_s), which a
// butterfly over the warp adds up, and accumulates the gradient and H v
// contributions of its own parameters in registers (FP32 over a tile, FP64
// across tiles).  Every warp writes one FP64 record; a second kernel sums the
// records in fixed order and the host combines them (Eqs. 3, 6, 7).
//
// Line shapes, D = BW^-1 with m^2 the resonance's channel invariant:
//   constant width   D = M^2 - m^2 - i M Gamma
//   mass-dependent   D = M^2 - m^2 - i Gamma0 h(M) rho(m),
//                    rho(m) = q(m) F_L(q(m))^2 / m, h(M) = M^2 / (q(M) F_L(q(M))^2)
//                    (i.e. M Gamma(m) with Gamma(m) = Gamma0 (q/q0)(M/m)(F_L(q)/F_L(q0))^2)
//   Flatte           D = M^2 - m^2 - i (gamma1 rho1(m) + gamma2 rho2(m)), rho_i = 2 q_i / m,
//                    q_i = i sqrt(-q_i^2) below the channel's threshold.
// All three are D = (M^2 - m^2) - i (A0 + A1 rho_a + A2 rho_b) with event
// factors rho_a, rho_b and parameter-only coefficients, and so are their first
// and second derivatives in (M, w1, w2); the host evaluates those coefficients
// in FP64 for each theta (h, h', h'' by second-order forward differentiation).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pwa_internal.h"

namespace {

constexpr int kVarWarps = 4;  // warps per block
constexpr int kVarE = 32;     // events per tile
// Events per thread (a warp step takes kVarEV tiles).  Two were measured slower
// than one on the paper-scale model (3.68 against 3.51 ms per pass with one
// coupling per resonance, 5.82 against 4.54 with one per projection): the
// registers they need cost more occupancy than the shared per-resonance work
// saves.
constexpr int kVarEV = 1;

// A complex linear form of the event factors, X = al - i (e0 + e1 rho_a + e2 rho_b).
struct Lin {
    float al, e0, e1, e2;
};

// Per-resonance constants of one evaluation (FP32, host-computed from theta and v).
struct VarRes {
    int ch, kind, L, pad;
    float M2hi, M2lo;        // M^2 = hi + lo
    float A0, A1, A2;        // D = (M^2 - m^2) - i (A0 + A1 rho_a + A2 rho_b)
    float a_pp, a_pm, r2;    // rho_a: (m_a + m_b)^2, (m_a - m_b)^2, barrier radius^2 (kind 1)
    float b_pp, b_pm;        // rho_b (Flatte channel 2)
    Lin dD[3];               // dD / d(M, w1, w2)
    Lin Dv;                  // sum_j dD_j v_j
    Lin ddv[3];              // sum_i d2D / d theta_j d theta_i v_i
    float2 g[4], eph[4], gd[4];      // per projection: g = rho e^{i phi}, e^{i phi}, gdot = v_rho e + v_phi i g
    float rho[4], vrho[4], vphi[4];  // per projection: rho and the direction's components
};

struct VarArgs {
    const float* m2[2];     // [3][n]
    const float2* F[2];     // tiles: [ceil(n / 32)][K S][32 events], zero past the last event
    const float* w;         // data weights or null
    long long n[2];
    int K;
    // B parameter vectors per launch: block i works for vector i / nbv, as
    // block i mod nbv of that vector's nbv blocks
    int nbv;
    int blocks0;            // blocks of the data sample per vector (the rest take the MC sample)
    const VarRes* res;      // [B][K]
    double* rec;            // [B][nbv warps][rec_len], per vector data warps first
    int rec_len;
    int* err;               // [B]
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// Re(a b)
__device__ __forceinline__ float re_mul(float2 a, float2 b) { return a.x * b.x - a.y * b.y; }

// al - i (e0 + e1 ra + e2 rb) for complex ra, rb
__device__ __forceinline__ float2 lin_form(Lin c, float2 ra, float2 rb)
{
    const float wr = c.e0 + c.e1 * ra.x + c.e2 * rb.x, wi = c.e1 * ra.y + c.e2 * rb.y;
    return make_float2(c.al + wi, -wr);
}

__device__ __forceinline__ float barrier_sq(int L, float z)
{
    switch (L) {
    case 0: return 1.f;
    case 1: return 2.f * z / (1.f + z);
    case 2: return 13.f * z * z / ((z - 3.f) * (z - 3.f) + 9.f * z);
    case 3: return 277.f * z * z * z / (z * (z - 15.f) * (z - 15.f) + 9.f * (2.f * z - 5.f) * (2.f * z - 5.f));
    default: {
        const float a = z * z - 45.f * z + 105.f, b = 2.f * z - 21.f;
        return 12746.f * z * z * z * z / (a * a + 25.f * z * b * b);
    }
    }
}

// 2 q / m for masses with (m_a + m_b)^2 = pp, (m_a - m_b)^2 = pm, continued below threshold
__device__ __forceinline__ float2 rho_flatte(float m2, float pp, float pm)
{
    const float q2 = (m2 - pp) * (m2 - pm) / (4.f * m2);
    const float r = 2.f * sqrtf(fabsf(q2)) * rsqrtf(m2);
    return q2 >= 0.f ? make_float2(r, 0.f) : make_float2(0.f, r);
}

// Shared memory of a block: the K resonances' constants, then per warp a
// [2 NP][33] FP32 transpose tile and [32][2 NP] FP64 accumulators.
template <int NP>
__host__ __device__ constexpr size_t var_smem_bytes()
{
    return ((32 * sizeof(VarRes) + 15) / 16) * 16 + kVarWarps * (2 * NP * 33 * sizeof(float)) +
           kVarWarps * (32 * 2 * NP * sizeof(double));
}

// event factors of resonance r's line shape at pair mass^2 m2v
__device__ __forceinline__ void shape_factors(const VarRes& r, float m2v, float2& ra, float2& rb)
{
    ra = make_float2(0.f, 0.f);
    rb = make_float2(0.f, 0.f);
    if (r.kind == 1) {
        const float q2 = (m2v - r.a_pp) * (m2v - r.a_pm) / (4.f * m2v);
        const float q = sqrtf(fmaxf(q2, 0.f));
        ra.x = q * barrier_sq(r.L, q2 * r.r2) * rsqrtf(m2v);
    } else if (r.kind == 2) {
        ra = rho_flatte(m2v, r.a_pp, r.a_pm);
        rb = rho_flatte(m2v, r.b_pp, r.b_pm);
    }
}

// BW = 1 / D for D = (M^2 - m^2) - i (A0 + A1 ra + A2 rb)
__device__ __forceinline__ float2 breit_wigner_v(const VarRes& r, float m2v, float2 ra, float2 rb)
{
    const float wr = r.A0 + r.A1 * ra.x + r.A2 * rb.x, wi = r.A1 * ra.y + r.A2 * rb.y;
    const float2 D = make_float2(((r.M2hi - m2v) + r.M2lo) + wi, -wr);
    const float inv = 1.f / (D.x * D.x + D.y * D.y);
    return make_float2(D.x * inv, -D.y * inv);
}

// Per-resonance terms of one event (pass 2): the 2 NP weighted contributions
// (gradient, then H v) of resonance r's parameters, added to val.
template <int S, bool PKS, bool HV>
__device__ __forceinline__ void add_contributions(const VarRes& r, float m2v, const float2* __restrict__ Fk,
                                                  const float2 (&A)[S], const float2 (&Ad)[S], float wa, float wb,
                                                  float (&val)[2 * (2 * (PKS ? S : 1) + 3)])
{
    constexpr int NC = PKS ? S : 1;
    constexpr int NP = 2 * NC + 3;
    float2 ra, rb;
    shape_factors(r, m2v, ra, rb);
    const float2 BW = breit_wigner_v(r, m2v, ra, rb);
    const float2 BW2 = cmul(BW, BW);
    float2 Dv = make_float2(0.f, 0.f), BWv = Dv;
    if (HV) {
        Dv = lin_form(r.Dv, ra, rb);
        BWv = cscale(cmul(BW2, Dv), -1.f);
    }
    float2 Dk[S], Ddk[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float2 F = Fk[s * kVarE];
        Dk[s] = cmul(cconj(A[s]), F);
        Ddk[s] = HV ? cmul(cconj(Ad[s]), F) : make_float2(0.f, 0.f);
    }
    // couplings: with dmag = dc/d rho = e^{i phi} BW, dc/d phi = i rho dmag, and
    // z1 = Ddot dmag, z2 = D dmag, z3 = D e^{i phi} BWv:
    //   g_rho = 2 Re z2,                      g_phi = -2 rho Im z2,
    //   h_rho = 2 (Re z1 - v_phi Im z2 + Re z3),
    //   h_phi = -2 (rho Im z1 + v_rho Im z2 + v_phi rho Re z2 + rho Im z3)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        float2 Dc = Dk[c], Ddc = Ddk[c];
        if (!PKS) {
#pragma unroll
            for (int s = 1; s < S; ++s) {
                Dc = cadd(Dc, Dk[s]);
                Ddc = cadd(Ddc, Ddk[s]);
            }
        }
        const float2 dmag = cmul(r.eph[c], BW);
        const float2 z2 = cmul(Dc, dmag);
        const float rho = r.rho[c];
        const float gm = 2.f * z2.x, gp = -2.f * rho * z2.y;
        val[c] += wa * gm;
        val[NC + c] += wa * gp;
        if (HV) {
            const float2 z1 = cmul(Ddc, dmag), z3 = cmul(Dc, cmul(r.eph[c], BWv));
            const float hm = 2.f * (z1.x - r.vphi[c] * z2.y + z3.x);
            const float hp = -2.f * (rho * (z1.y + z3.y) + r.vrho[c] * z2.y + r.vphi[c] * rho * z2.x);
            val[NP + c] += wa * hm - wb * gm;
            val[NP + NC + c] += wa * hp - wb * gp;
        }
    }
    float2 E = make_float2(0.f, 0.f), Ed = E;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int c = PKS ? s : 0;
        E = cadd(E, cmul(Dk[s], r.g[c]));
        if (HV) Ed = cadd(Ed, cadd(cmul(Ddk[s], r.g[c]), cmul(Dk[s], r.gd[c])));
    }
    // shape parameters: dBW_j = -BW^2 dD_j and d(BWv)/d theta_j = 2 BW^3 Dv dD_j - BW^2 ddv_j, so with
    // W = E BW^2, X = Edot BW^2 (Edot = sum_s Ddot_s g_s + D_s gdot_s) and Y = 2 W BW Dv:
    //   g_j = -2 Re(W dD_j),   h_j = 2 Re((Y - X) dD_j - W ddv_j)
    const float2 Wm = cmul(E, BW2);
    float2 YX = make_float2(0.f, 0.f);
    if (HV) YX = cadd(cscale(cmul(cmul(Wm, BW), Dv), 2.f), cscale(cmul(Ed, BW2), -1.f));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        // the second width parameter exists for Flatte shapes only (the branch is the
        // same for the whole warp: its threads all work on resonance r)
        if (j == 2 && r.kind != 2) break;
        const float2 dD = lin_form(r.dD[j], ra, rb);
        const float gj = -2.f * re_mul(Wm, dD);
        val[2 * NC + j] += wa * gj;
        if (HV) {
            const float hj = 2.f * (re_mul(YX, dD) - re_mul(Wm, lin_form(r.ddv[j], ra, rb)));
            val[NP + 2 * NC + j] += wa * hj - wb * gj;
        }
    }
}

// kVarEV events per thread: a warp takes groups of kVarEV 32-event tiles
// (thread `lane` has event lane of each).  Pass 1 over the resonances forms
// A_s and Adot_s of its events in registers; pass 2 recomputes each
// resonance's terms and adds the events' 2 NP weighted parameter
// contributions, which go through the warp's transpose tile: one lane per
// contribution sums the 32 threads' values into the warp's FP64 accumulators.
template <int S, bool PKS, bool HV>
__global__ void __launch_bounds__(32 * kVarWarps) variant_kernel(const VarArgs a)
{
    constexpr int NC = PKS ? S : 1;     // distinct couplings per resonance
    constexpr int NP = 2 * NC + 3;      // parameter slots per resonance: mags, phases, M, w1, w2
    constexpr int NV = 2 * NP;          // gradient and H v contribution per slot
    constexpr int EV = kVarEV;          // events per thread
    extern __shared__ __align__(16) unsigned char var_smem[];
    VarRes* sres = reinterpret_cast<VarRes*>(var_smem);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* tile = reinterpret_cast<float*>(var_smem + ((32 * sizeof(VarRes) + 15) / 16) * 16) + warp * (NV * 33);
    double* acc = reinterpret_cast<double*>(var_smem + ((32 * sizeof(VarRes) + 15) / 16) * 16 +
                                            kVarWarps * (NV * 33 * sizeof(float))) + warp * (32 * NV);
    const int K = a.K;
    const int vec = blockIdx.x / a.nbv, bx = blockIdx.x - vec * a.nbv;
    for (int i = threadIdx.x; i < K; i += blockDim.x) sres[i] = a.res[(size_t)vec * K + i];
    for (int i = lane; i < 32 * NV; i += 32) acc[i] = 0.0;
    __syncthreads();

    const int sample = bx < a.blocks0 ? 0 : 1;
    const int blk = sample ? bx - a.blocks0 : bx;
    const int nblk = sample ? a.nbv - a.blocks0 : a.blocks0;
    const int wg = blk * kVarWarps + warp, nw = nblk * kVarWarps;
    const long long n = a.n[sample];
    const long long ntiles = (n + kVarE - 1) / kVarE;
    const long long ngroups = (ntiles + EV - 1) / EV;
    const float* m2p = a.m2[sample];
    const float2* Fp = a.F[sample];
    const float* wp = sample == 0 ? a.w : nullptr;
    double s0 = 0.0, s1 = 0.0;  // per thread: sum w ln I (data) or sum I, sum Idot (MC)
    float f0 = 0.f, f1 = 0.f;   // FP32 partial of the last (up to) 16 / EV tile groups
    int nf = 0;
    int bad = 0;

    for (long long tg = wg; tg < ngroups; tg += nw) {
        if (++nf == 16 / EV) {
            s0 += (double)f0;
            s1 += (double)f1;
            f0 = f1 = 0.f;
            nf = 0;
        }
        bool live[EV];
        float m2e[EV][3];
        const float2* Fe[EV];
#pragma unroll
        for (int u = 0; u < EV; ++u) {
            // a tile past the last one, or an event past the last one, repeats valid memory and contributes nothing
            const long long t = min(tg * EV + u, ntiles - 1);
            const long long e = (tg * EV + u) * kVarE + lane;
            live[u] = e < n;
            const long long ec = live[u] ? e : n - 1;
            m2e[u][0] = m2p[ec];
            m2e[u][1] = m2p[n + ec];
            m2e[u][2] = m2p[2 * n + ec];
            Fe[u] = Fp + t * (long long)K * S * kVarE + lane;  // entry (k, s) at Fe[(k S + s) 32]
        }
        // pass 1: coherent sums
        float2 A[EV][S], Ad[EV][S];
#pragma unroll
        for (int u = 0; u < EV; ++u)
#pragma unroll
            for (int s = 0; s < S; ++s) A[u][s] = Ad[u][s] = make_float2(0.f, 0.f);
        for (int k = 0; k < K; ++k) {
            const VarRes& r = sres[k];
#pragma unroll
            for (int u = 0; u < EV; ++u) {
                const float m2v = r.ch == 0 ? m2e[u][0] : (r.ch == 1 ? m2e[u][1] : m2e[u][2]);
                float2 ra, rb;
                shape_factors(r, m2v, ra, rb);
                const float2 BW = breit_wigner_v(r, m2v, ra, rb);
                float2 BWv = make_float2(0.f, 0.f);
                if (HV) BWv = cscale(cmul(cmul(BW, BW), lin_form(r.Dv, ra, rb)), -1.f);
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const int c = PKS ? s : 0;
                    const float2 F = Fe[u][(k * S + s) * kVarE];
                    A[u][s] = cadd(A[u][s], cmul(cmul(r.g[c], BW), F));
                    if (HV) Ad[u][s] = cadd(Ad[u][s], cmul(cadd(cmul(r.gd[c], BW), cmul(r.g[c], BWv)), F));
                }
            }
        }
        float wa[EV], wb[EV];
#pragma unroll
        for (int u = 0; u < EV; ++u) {
            float I = 0.f, Id = 0.f;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                I += A[u][s].x * A[u][s].x + A[u][s].y * A[u][s].y;
                if (HV) Id += 2.f * (A[u][s].x * Ad[u][s].x + A[u][s].y * Ad[u][s].y);
            }
            wa[u] = wb[u] = 0.f;
            if (live[u]) {
                const long long e = (tg * EV + u) * kVarE + lane;
                if (sample == 0) {
                    const float we = wp ? wp[e] : 1.f;
                    if (!(I > 0.f) || !isfinite(I)) {
                        bad = 1;
                    } else {
                        wa[u] = we / I;
                        wb[u] = HV ? we * Id / (I * I) : 0.f;
                        f0 += we * logf(I);
                    }
                } else if (!isfinite(I)) {
                    bad = 1;
                } else {
                    wa[u] = 1.f;
                    f0 += I;
                    f1 += Id;
                }
            }
        }
        // pass 2: parameter contributions, transposed through shared memory
        for (int k = 0; k < K; ++k) {
            const VarRes& r = sres[k];
            float val[NV];
#pragma unroll
            for (int j = 0; j < NV; ++j) val[j] = 0.f;
#pragma unroll
            for (int u = 0; u < EV; ++u) {
                const float m2v = r.ch == 0 ? m2e[u][0] : (r.ch == 1 ? m2e[u][1] : m2e[u][2]);
                add_contributions<S, PKS, HV>(r, m2v, Fe[u] + k * S * kVarE, A[u], Ad[u], wa[u], wb[u], val);
            }
            // contribution j of this thread's events at tile[j][lane] (row stride 33: no bank conflicts)
#pragma unroll
            for (int j = 0; j < NV; ++j) tile[j * 33 + lane] = val[j];
            __syncwarp();
            if (lane < NV) {
                float sum = 0.f;
#pragma unroll 8
                for (int q = 0; q < 32; ++q) sum += tile[lane * 33 + q];
                acc[k * NV + lane] += (double)sum;
            }
            __syncwarp();
        }
    }
    // scalars: sum over the warp's threads (FP64)
    s0 += (double)f0;
    s1 += (double)f1;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    __syncwarp();
    double* rec = a.rec + ((long long)vec * a.nbv * kVarWarps + (sample ? a.blocks0 * kVarWarps : 0) + wg) * a.rec_len;
    for (int i = lane; i < 32 * NV; i += 32) rec[i] = acc[i];
    if (lane == 0) {
        rec[32 * NV] = s0;
        rec[32 * NV + 1] = s1;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.err + vec, 1);
}

// Integral matrices of the MC sample at fixed line shapes:
// Phi_s,kk' = sum_mc conj(U_ks) U_k's, U_ks = BW_k F_ks.  A block takes 32-event
// tiles in turn: its threads write U of the tile to shared memory ([K S] rows of
// 32 events, row stride 33 against bank conflicts), then thread i accumulates
// the entries q = i, i + blockDim, ... of the S K K matrix over the tile's
// events in FP32 and adds the tile's sum to its FP64 totals.  Each block writes
// one FP64 record [S K K][2].
constexpr int kPhiThreads = 256;
constexpr int kPhiMaxPerThread = 16;  // S K K <= 4 * 32 * 32 = 16 kPhiThreads

__global__ void __launch_bounds__(kPhiThreads) variant_phi_kernel(const float* __restrict__ m2, const float2* __restrict__ Ft,
                                                                 long long n, int K, int S,
                                                                 const VarRes* __restrict__ res,
                                                                 double* __restrict__ rec)
{
    extern __shared__ __align__(16) unsigned char phi_smem[];
    VarRes* sres = reinterpret_cast<VarRes*>(phi_smem);
    float2* U = reinterpret_cast<float2*>(phi_smem + ((32 * sizeof(VarRes) + 15) / 16) * 16);  // [K S][33]
    const int tid = threadIdx.x;
    for (int i = tid; i < K; i += blockDim.x) sres[i] = res[i];
    __syncthreads();
    const int KS = K * S, NQ = S * K * K;
    double accr[kPhiMaxPerThread], acci[kPhiMaxPerThread];
#pragma unroll
    for (int j = 0; j < kPhiMaxPerThread; ++j) accr[j] = acci[j] = 0.0;
    const long long ntiles = (n + kVarE - 1) / kVarE;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        // U of the tile's events (zero past the last event: F is zero there)
        for (int i = tid; i < K * kVarE; i += blockDim.x) {
            const int k = i / kVarE, l = i % kVarE;
            const long long e = min(t * kVarE + l, n - 1);
            const VarRes& r = sres[k];
            const float m2v = m2[(long long)r.ch * n + e];
            float2 ra, rb;
            shape_factors(r, m2v, ra, rb);
            const float2 BW = breit_wigner_v(r, m2v, ra, rb);
            for (int s = 0; s < S; ++s) U[(k * S + s) * 33 + l] = cmul(BW, Ft[(t * KS + k * S + s) * kVarE + l]);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPhiMaxPerThread; ++j) {
            const int q = tid + j * kPhiThreads;
            if (q < NQ) {
                const int s = q / (K * K), kk = q % (K * K), k = kk / K, kp = kk % K;
                const float2* Ua = U + (k * S + s) * 33;
                const float2* Ub = U + (kp * S + s) * 33;
                float sr = 0.f, si = 0.f;
#pragma unroll 8
                for (int l = 0; l < kVarE; ++l) {
                    const float2 a = Ua[l], b = Ub[l];  // conj(a) b
                    sr += a.x * b.x + a.y * b.y;
                    si += a.x * b.y - a.y * b.x;
                }
                accr[j] += (double)sr;
                acci[j] += (double)si;
            }
        }
        __syncthreads();
    }
    double* out = rec + (size_t)blockIdx.x * 2 * NQ;
#pragma unroll
    for (int j = 0; j < kPhiMaxPerThread; ++j) {
        const int q = tid + j * kPhiThreads;
        if (q < NQ) {
            out[2 * q] = accr[j];
            out[2 * q + 1] = acci[j];
        }
    }
}

// out[j] = sum over the blocks' records of rec[b][j], in block order
__global__ void variant_phi_reduce_kernel(const double* __restrict__ rec, int nblocks, int len, double* __restrict__ out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= len) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += rec[(size_t)b * len + j];
    out[j] = s;
}

// F [n][KS] -> tiles [ceil(n / 32)][KS][32], zero past the last event
__global__ void variant_tile_kernel(const float2* __restrict__ F, long long n, int KS, float2* __restrict__ out)
{
    const long long total = (n + kVarE - 1) / kVarE * kVarE * KS;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(i % kVarE);
        const long long rest = i / kVarE;
        const int q = (int)(rest % KS);
        const long long t = rest / KS;
        const long long e = t * kVarE + l;
        out[i] = e < n ? F[e * KS + q] : make_float2(0.f, 0.f);
    }
}

// out[sample][j] = sum over the sample's warps of rec[warp][j], in a fixed order:
// block x takes 32 consecutive slots (threadIdx.x, coalesced reads), and
// thread row y sums the warps y, y + 32, ...; the 32 row sums are then added
// in row order.  Vector blockIdx.y: records [warps0 + warps1][rec_len] from
// rec + y (warps0 + warps1) rec_len, sums [2 rec_len] at out + y 2 rec_len.
__global__ void __launch_bounds__(1024) variant_reduce_kernel(const double* __restrict__ rec, int rec_len, int warps0,
                                                              int warps1, double* __restrict__ out)
{
    __shared__ double part[32][33];
    rec += (size_t)blockIdx.y * (warps0 + warps1) * rec_len;
    out += (size_t)blockIdx.y * 2 * rec_len;
    const int j = blockIdx.x * 32 + threadIdx.x;
    const bool ok = j < 2 * rec_len;
    const int sample = ok ? j / rec_len : 0, slot = ok ? j % rec_len : 0;
    const int w0 = sample ? warps0 : 0, nw = sample ? warps1 : warps0;
    double s = 0.0;
    if (ok)
        for (int w = threadIdx.y; w < nw; w += 32) s += rec[(long long)(w0 + w) * rec_len + slot];
    part[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && ok) {
        double t = 0.0;
        for (int y = 0; y < 32; ++y) t += part[y][threadIdx.x];
        out[j] = t;
    }
}

using VarKernel = void (*)(const VarArgs);

template <int S>
VarKernel pick_s(bool pks, bool hv)
{
    if (pks) return hv ? variant_kernel<S, true, true> : variant_kernel<S, true, false>;
    return hv ? variant_kernel<S, false, true> : variant_kernel<S, false, false>;
}

size_t var_smem_for(int S, bool pks)
{
    switch (pks ? S : 1) {
    case 1: return var_smem_bytes<5>();
    case 2: return var_smem_bytes<7>();
    case 3: return var_smem_bytes<9>();
    default: return var_smem_bytes<11>();
    }
}

VarKernel pick(int S, bool pks, bool hv)
{
    switch (S) {
    case 1: return pick_s<1>(pks, hv);
    case 2: return pick_s<2>(pks, hv);
    case 3: return pick_s<3>(pks, hv);
    case 4: return pick_s<4>(pks, hv);
    }
    return nullptr;
}

// value, first and second derivative of a function of one variable
struct Jet {
    double v, d, dd;
};
Jet operator+(Jet a, Jet b) { return {a.v + b.v, a.d + b.d, a.dd + b.dd}; }
Jet operator-(Jet a, Jet b) { return {a.v - b.v, a.d - b.d, a.dd - b.dd}; }
Jet operator*(Jet a, Jet b) { return {a.v * b.v, a.d * b.v + a.v * b.d, a.dd * b.v + 2 * a.d * b.d + a.v * b.dd}; }
Jet operator*(double s, Jet a) { return {s * a.v, s * a.d, s * a.dd}; }
Jet operator+(Jet a, double s) { return {a.v + s, a.d, a.dd}; }
Jet recip(Jet a)
{
    const double r = 1.0 / a.v;
    return {r, -a.d * r * r, (2 * a.d * a.d * r - a.dd) * r * r};
}
Jet operator/(Jet a, Jet b) { return a * recip(b); }
Jet jsqrt(Jet a)
{
    const double r = std::sqrt(a.v);
    return {r, a.d / (2 * r), a.dd / (2 * r) - a.d * a.d / (4 * r * a.v)};
}

Jet barrier_sq_jet(int L, Jet z)
{
    switch (L) {
    case 0: return {1.0, 0.0, 0.0};
    case 1: return (2.0 * z) / (z + 1.0);
    case 2: {
        const Jet a = z + (-3.0);
        return (13.0 * (z * z)) / (a * a + 9.0 * z);
    }
    case 3: {
        const Jet a = z + (-15.0), b = 2.0 * z + (-5.0);
        return (277.0 * (z * z * z)) / (z * a * a + 9.0 * (b * b));
    }
    default: {
        const Jet a = z * z - 45.0 * z + 105.0, b = 2.0 * z + (-21.0);
        return (12746.0 * (z * z * z * z)) / (a * a + 25.0 * (z * b * b));
    }
    }
}

}  // namespace

struct pwa_variant {
    pwa_handle base;  // stream, error text, K, S, P for the shared fit machinery
    int per_projection = 0;
    // plain arrays: the header's structs are unnamed typedefs, which the CUDA
    // front end does not place in standard containers in C++20 mode
    pwa_resonance* table = nullptr;  // [K]
    pwa_lineshape* shapes = nullptr; // [K]
    // theta layout: (what, k, s) with what 0 mag, 1 phase, 2 mass, 3 w1, 4 w2
    std::vector<int> lay_what, lay_k, lay_s;
    float* d_m2[2] = {nullptr, nullptr};
    float2* d_F[2] = {nullptr, nullptr};
    float* d_w = nullptr;
    // per-vector buffers, room for vcap parameter vectors (one pass evaluates up to vcap)
    VarRes* d_res = nullptr;   // [vcap][K]
    double* d_rec = nullptr;   // [vcap][(blocks0 + blocks1) warps][rec_len]
    double* d_sums = nullptr;  // [vcap][2 rec_len]
    int* d_err = nullptr;      // [vcap]
    double* h_sums = nullptr;  // pinned: [vcap][2 rec_len] sums, then vcap error words
    int rec_len = 0, blocks0 = 0, blocks1 = 0, vcap = 0;
    VarRes* h_res = nullptr;   // pinned [vcap][K]
    // coupling-only evaluation at fixed line shapes: the shape parameters and
    // the MC integral matrices Phi [S][K][K] (complex FP64, host)
    int Pc = 0;                       // coupling parameters at the head of theta
    std::vector<double> shape_theta;  // theta[Pc ..] of the last pwa_variant_set_shapes
    std::vector<double> phi;          // [S][K][K][2]
    bool have_phi = false;
};

namespace {

pwa_status vfail(pwa_variant* v, pwa_status st, const std::string& msg) { return pwa::set_error(&v->base, st, msg); }

#define VAR_TRY(call)                 \
    do {                              \
        pwa_status s_ = (call);       \
        if (s_ != PWA_OK) return s_;  \
    } while (0)

#define VAR_CUDA(v, call)                                                   \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return pwa::cuda_error(&(v)->base, e_, #call); \
    } while (0)

int NC_of(const pwa_variant* v) { return v->per_projection ? v->base.S : 1; }

// room for B parameter vectors in the per-vector buffers (grown, never shrunk;
// the error words start at zero)
pwa_status reserve_vectors(pwa_variant* v, int B)
{
    if (B <= v->vcap) return PWA_OK;
    cudaStream_t st = v->base.stream;
    VAR_CUDA(v, cudaStreamSynchronize(st));
    if (v->d_rec) cudaFree(v->d_rec);
    if (v->d_sums) cudaFree(v->d_sums);
    if (v->d_res) cudaFree(v->d_res);
    if (v->d_err) cudaFree(v->d_err);
    if (v->h_sums) cudaFreeHost(v->h_sums);
    if (v->h_res) cudaFreeHost(v->h_res);
    v->d_rec = v->d_sums = v->h_sums = nullptr;
    v->d_res = v->h_res = nullptr;
    v->d_err = nullptr;
    v->vcap = 0;
    const int K = v->base.K;
    const size_t warps = (size_t)(v->blocks0 + v->blocks1) * kVarWarps, rl = (size_t)v->rec_len;
    VAR_CUDA(v, cudaMalloc(&v->d_rec, sizeof(double) * B * warps * rl));
    VAR_CUDA(v, cudaMalloc(&v->d_sums, sizeof(double) * B * 2 * rl));
    VAR_CUDA(v, cudaMalloc(&v->d_res, sizeof(VarRes) * B * K));
    VAR_CUDA(v, cudaMalloc(&v->d_err, sizeof(int) * B));
    VAR_CUDA(v, cudaMemsetAsync(v->d_err, 0, sizeof(int) * B, st));
    VAR_CUDA(v, cudaMallocHost(&v->h_sums, sizeof(double) * B * (2 * rl + 1)));
    VAR_CUDA(v, cudaMallocHost(&v->h_res, sizeof(VarRes) * B * K));
    VAR_CUDA(v, cudaStreamSynchronize(st));
    v->vcap = B;
    return PWA_OK;
}

// host: per-resonance constants for theta (and direction v, may be null) into
// out [K] (the first vector's slot when null)
pwa_status fill_res(pwa_variant* vv, const double* theta, const double* dir, VarRes* out = nullptr)
{
    if (!out) out = vv->h_res;
    const int K = vv->base.K, S = vv->base.S, NC = NC_of(vv);
    std::vector<double> mag((size_t)K * NC), ph((size_t)K * NC), M(K), w1(K), w2(K);
    std::vector<double> vmag((size_t)K * NC, 0.0), vph((size_t)K * NC, 0.0), vM(K, 0.0), vw1(K, 0.0), vw2(K, 0.0);
    for (int k = 0; k < K; ++k) {
        for (int c = 0; c < NC; ++c) {
            mag[k * NC + c] = vv->table[k].mag;
            ph[k * NC + c] = vv->table[k].phase;
        }
        M[k] = vv->table[k].mass;
        w1[k] = vv->table[k].width;
        w2[k] = vv->shapes[k].width2;
    }
    for (size_t i = 0; i < vv->lay_what.size(); ++i) {
        const int k = vv->lay_k[i], c = vv->lay_s[i];
        const double x = theta[i], d = dir ? dir[i] : 0.0;
        switch (vv->lay_what[i]) {
        case 0: mag[k * NC + c] = x; vmag[k * NC + c] = d; break;
        case 1: ph[k * NC + c] = x; vph[k * NC + c] = d; break;
        case 2: M[k] = x; vM[k] = d; break;
        case 3: w1[k] = x; vw1[k] = d; break;
        default: w2[k] = x; vw2[k] = d; break;
        }
    }
    for (int k = 0; k < K; ++k) {
        VarRes& r = out[k];
        std::memset(&r, 0, sizeof(r));
        const pwa_lineshape& sh = vv->shapes[k];
        r.ch = vv->table[k].channel;
        r.kind = sh.kind;
        r.L = vv->table[k].spin;
        const double Mk = M[k];
        if (!(Mk > 0.0)) return vfail(vv, PWA_EINVAL, "masses must be positive");
        const double M2 = Mk * Mk;
        r.M2hi = (float)M2;
        r.M2lo = (float)(M2 - (double)r.M2hi);
        // dD[j] = {al, e0, e1, e2}; second derivatives d2[j][i] likewise
        double dD[3][4] = {{0}}, d2[3][3][4] = {{{0}}};
        dD[0][0] = 2 * Mk;
        d2[0][0][0] = 2.0;
        if (sh.kind == PWA_SHAPE_CONSTANT) {
            r.A0 = (float)(Mk * w1[k]);
            dD[0][1] = w1[k];  // d(M Gamma)/dM
            dD[1][1] = Mk;     // d(M Gamma)/dGamma
            d2[0][1][1] = d2[1][0][1] = 1.0;
        } else if (sh.kind == PWA_SHAPE_MASS_DEPENDENT) {
            const double pp = (sh.ma + sh.mb) * (sh.ma + sh.mb), pm = (sh.ma - sh.mb) * (sh.ma - sh.mb);
            r.a_pp = (float)pp;
            r.a_pm = (float)pm;
            r.r2 = (float)(sh.radius * sh.radius);
            // h(M) = M^2 / (q(M) F_L(q(M))^2) with its first two derivatives
            const Jet Mj{Mk, 1.0, 0.0};
            const Jet M2j = Mj * Mj;
            const Jet q2 = ((M2j + (-pp)) * (M2j + (-pm))) / (4.0 * M2j);
            if (!(q2.v > 0.0)) return vfail(vv, PWA_EINVAL, "a mass-dependent width needs M above the pair threshold");
            const Jet h = M2j / (jsqrt(q2) * barrier_sq_jet(r.L, (sh.radius * sh.radius) * q2));
            r.A1 = (float)(w1[k] * h.v);
            dD[0][2] = w1[k] * h.d;
            dD[1][2] = h.v;
            d2[0][0][2] = w1[k] * h.dd;
            d2[0][1][2] = d2[1][0][2] = h.d;
        } else {
            r.a_pp = (float)((sh.ma + sh.mb) * (sh.ma + sh.mb));
            r.a_pm = (float)((sh.ma - sh.mb) * (sh.ma - sh.mb));
            r.b_pp = (float)((sh.mc + sh.md) * (sh.mc + sh.md));
            r.b_pm = (float)((sh.mc - sh.md) * (sh.mc - sh.md));
            r.A1 = (float)w1[k];
            r.A2 = (float)w2[k];
            dD[1][2] = 1.0;
            dD[2][3] = 1.0;
        }
        const double vs[3] = {vM[k], vw1[k], vw2[k]};
        auto lin = [](const double c[4]) { return Lin{(float)c[0], (float)c[1], (float)c[2], (float)c[3]}; };
        double dv[4] = {0, 0, 0, 0};
        for (int j = 0; j < 3; ++j) {
            double ddvj[4] = {0, 0, 0, 0};
            for (int q = 0; q < 4; ++q) {
                dv[q] += dD[j][q] * vs[j];
                for (int i = 0; i < 3; ++i) ddvj[q] += d2[j][i][q] * vs[i];
            }
            r.dD[j] = lin(dD[j]);
            r.ddv[j] = lin(ddvj);
        }
        r.Dv = lin(dv);
        for (int s = 0; s < S && s < 4; ++s) {
            const int c = vv->per_projection ? s : 0;
            const double rho = mag[k * NC + c], phi = ph[k * NC + c], vr = vmag[k * NC + c], vp = vph[k * NC + c];
            const double er = std::cos(phi), ei = std::sin(phi);
            const double gr_ = rho * er, gi_ = rho * ei;                        // g = rho e^{i phi}
            const double gdr = vr * er - vp * gi_, gdi = vr * ei + vp * gr_;    // gdot = vr e + vp i g
            r.g[s] = make_float2((float)gr_, (float)gi_);
            r.eph[s] = make_float2((float)er, (float)ei);
            r.gd[s] = make_float2((float)gdr, (float)gdi);
            r.rho[s] = (float)rho;
            r.vrho[s] = (float)vr;
            r.vphi[s] = (float)vp;
        }
    }
    return PWA_OK;
}

pwa_status copy_sample(pwa_variant* v, int s, const pwa_events* ev, bool is_data)
{
    const int K = v->base.K, S = v->base.S;
    const long long n = ev->n;
    const size_t nF = (size_t)n * K * S;
    const size_t nT = (size_t)((n + kVarE - 1) / kVarE) * kVarE * K * S;
    VAR_CUDA(v, cudaMalloc(&v->d_m2[s], sizeof(float) * 3 * (size_t)n));
    VAR_CUDA(v, cudaMalloc(&v->d_F[s], sizeof(float2) * nT));
    const cudaMemcpyKind kind = ev->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    VAR_CUDA(v, cudaMemcpyAsync(v->d_m2[s], ev->m2, sizeof(float) * 3 * (size_t)n, kind, v->base.stream));
    // F in the caller's [n][K][S] layout, then into event tiles (SoA within a tile)
    const float2* src = reinterpret_cast<const float2*>(ev->F);
    float2* raw = nullptr;
    if (!ev->on_device) {
        VAR_CUDA(v, cudaMalloc(&raw, sizeof(float2) * nF));
        cudaError_t e = cudaMemcpyAsync(raw, ev->F, sizeof(float2) * nF, cudaMemcpyHostToDevice, v->base.stream);
        if (e != cudaSuccess) {
            cudaFree(raw);
            return pwa::cuda_error(&v->base, e, "copy of F");
        }
        src = raw;
    }
    variant_tile_kernel<<<1184, 256, 0, v->base.stream>>>(src, n, K * S, v->d_F[s]);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(v->base.stream);
    if (raw) cudaFree(raw);
    if (e != cudaSuccess) return pwa::cuda_error(&v->base, e, "tiling of F");
    if (is_data && ev->w) {
        VAR_CUDA(v, cudaMalloc(&v->d_w, sizeof(float) * (size_t)n));
        VAR_CUDA(v, cudaMemcpyAsync(v->d_w, ev->w, sizeof(float) * (size_t)n, kind, v->base.stream));
    }
    return PWA_OK;
}

// host checks of a sample given in host memory (device inputs are taken as given: the kernel flags a
// non-finite or non-positive intensity at evaluation time)
pwa_status check_sample(pwa_variant* v, const pwa_events* ev, bool is_data, double& weight_sum)
{
    if (!ev || ev->n < 1 || !ev->m2 || !ev->F) return vfail(v, PWA_EINVAL, "every sample needs n >= 1, m2 and F");
    weight_sum = (double)ev->n;
    if (!is_data && ev->w) return vfail(v, PWA_EINVAL, "the MC sample takes no weights");
    if (ev->on_device) return PWA_OK;
    const long long n = ev->n;
    const size_t nF = (size_t)n * v->base.K * v->base.S * 2;
    for (size_t i = 0; i < 3 * (size_t)n; ++i)
        if (!std::isfinite(ev->m2[i]) || !(ev->m2[i] > 0.f)) return vfail(v, PWA_EINVAL, "m2 must be finite and > 0");
    for (size_t i = 0; i < nF; ++i)
        if (!std::isfinite(ev->F[i])) return vfail(v, PWA_EINVAL, "F must be finite");
    if (is_data && ev->w) {
        weight_sum = 0.0;
        for (long long i = 0; i < n; ++i) {
            if (!std::isfinite(ev->w[i]) || ev->w[i] < 0.f) return vfail(v, PWA_EINVAL, "weights must be finite, >= 0");
            weight_sum += ev->w[i];
        }
    }
    return PWA_OK;
}

pwa_status create_impl(pwa_variant* v, const pwa_events* data, const pwa_events* mc, const pwa_resonance* table,
                       const pwa_lineshape* shapes, int K, int S, int per_projection)
{
    if (!data || !mc || !table) return vfail(v, PWA_EINVAL, "data, mc and table must not be NULL");
    if (K < 1 || K > 32 || S < 1 || S > 4) return vfail(v, PWA_EINVAL, "need 1 <= K <= 32 and 1 <= S <= 4");
    v->base.K = K;
    v->base.S = S;
    v->per_projection = per_projection ? 1 : 0;
    v->table = new (std::nothrow) pwa_resonance[K];
    v->shapes = new (std::nothrow) pwa_lineshape[K];
    if (!v->table || !v->shapes) return vfail(v, PWA_ENOMEM, "host allocation failed");
    for (int k = 0; k < K; ++k) v->table[k] = table[k];
    for (int k = 0; k < K; ++k) {
        pwa_lineshape sh{};
        sh.kind = PWA_SHAPE_CONSTANT;
        if (shapes) sh = shapes[k];
        const pwa_resonance& r = table[k];
        if (r.channel < 0 || r.channel > 2) return vfail(v, PWA_EINVAL, "channels are 0..2");
        if (sh.kind < 0 || sh.kind > 2) return vfail(v, PWA_EINVAL, "unknown line shape");
        if (sh.kind == PWA_SHAPE_MASS_DEPENDENT && (r.spin < 0 || r.spin > 4 || !(sh.radius > 0.0) ||
                                                     !(sh.ma >= 0.0) || !(sh.mb >= 0.0)))
            return vfail(v, PWA_EINVAL, "a mass-dependent width needs spin 0..4, radius > 0, daughter masses >= 0");
        if (sh.kind == PWA_SHAPE_FLATTE && !(sh.ma >= 0.0 && sh.mb >= 0.0 && sh.mc >= 0.0 && sh.md >= 0.0))
            return vfail(v, PWA_EINVAL, "Flatte channel masses must be >= 0");
        if (!std::isfinite(r.mass) || !(r.mass > 0.0) || !std::isfinite(r.width) || !std::isfinite(r.mag) ||
            !std::isfinite(r.phase) || !std::isfinite(sh.width2))
            return vfail(v, PWA_EINVAL, "table values must be finite, masses positive");
        v->shapes[k] = sh;
    }
    // theta layout
    const int NC = NC_of(v);
    for (int what = 0; what < 2; ++what)
        for (int k = 0; k < K; ++k)
            if (!table[k].fix_coupling)
                for (int c = 0; c < NC; ++c) {
                    v->lay_what.push_back(what);
                    v->lay_k.push_back(k);
                    v->lay_s.push_back(c);
                }
    for (int k = 0; k < K; ++k)
        if (!table[k].fix_mass) {
            v->lay_what.push_back(2);
            v->lay_k.push_back(k);
            v->lay_s.push_back(0);
        }
    for (int k = 0; k < K; ++k)
        if (!table[k].fix_width) {
            v->lay_what.push_back(3);
            v->lay_k.push_back(k);
            v->lay_s.push_back(0);
        }
    for (int k = 0; k < K; ++k)
        if (!table[k].fix_width && v->shapes[k].kind == PWA_SHAPE_FLATTE) {
            v->lay_what.push_back(4);
            v->lay_k.push_back(k);
            v->lay_s.push_back(0);
        }
    v->base.P = (int)v->lay_what.size();
    for (int w : v->lay_what) v->Pc += (w <= 1) ? 1 : 0;
    double wsum = 0.0, dummy = 0.0;
    pwa_status st = check_sample(v, data, true, wsum);
    if (st != PWA_OK) return st;
    st = check_sample(v, mc, false, dummy);
    if (st != PWA_OK) return st;
    v->base.n[0] = data->n;
    v->base.n[1] = mc->n;
    v->base.Nd = wsum;
    v->base.Nmc = (double)mc->n;
    if (data->on_device && data->w) {
        // the weight sum of device weights
        std::vector<float> hw((size_t)data->n);
        VAR_CUDA(v, cudaMemcpy(hw.data(), data->w, sizeof(float) * (size_t)data->n, cudaMemcpyDeviceToHost));
        v->base.Nd = 0.0;
        for (float x : hw) v->base.Nd += x;
    }
    st = copy_sample(v, 0, data, true);
    if (st != PWA_OK) return st;
    st = copy_sample(v, 1, mc, false);
    if (st != PWA_OK) return st;
    // grid: as many blocks as fit on the SMs (shared memory and registers of the
    // H v instance), split between the samples by their tile counts
    int dev = 0, sms = 148, per_sm = 2;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    {
        VarKernel fh = pick(S, v->per_projection != 0, true);
        const size_t smem = var_smem_for(S, v->per_projection != 0);
        VAR_CUDA(v, cudaFuncSetAttribute(fh, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        VAR_CUDA(v, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fh, 32 * kVarWarps, smem));
        per_sm = std::max(per_sm, 1);
    }
    // work units: groups of kVarEV 32-event tiles (one per warp step)
    const long long ge = (long long)kVarEV * kVarE;
    const long long t0 = (data->n + ge - 1) / ge, t1 = (mc->n + ge - 1) / ge;
    const long long total =
        std::max(2LL, std::min((long long)per_sm * sms, (t0 + kVarWarps - 1) / kVarWarps + (t1 + kVarWarps - 1) / kVarWarps));
    long long b0 = std::max(1LL, std::llround((double)total * t0 / (double)(t0 + t1)));
    b0 = std::min(b0, std::max(1LL, (t0 + kVarWarps - 1) / kVarWarps));
    long long b1 = std::max(1LL, std::min(total - b0, (t1 + kVarWarps - 1) / kVarWarps));
    v->blocks0 = (int)b0;
    v->blocks1 = (int)b1;
    const int NP = 2 * NC + 3;
    v->rec_len = 32 * 2 * NP + 2;
    VAR_TRY(reserve_vectors(v, 1));
    return PWA_OK;
}

}  // namespace

namespace pwa {

// One pass of the variant kernel for B parameter vectors (host theta [B][P],
// direction dir [B][P] when hv): the data sample, and the MC sample unless
// data_only; leaves the summed records in v->h_sums (per vector: data, then
// MC) and a per-vector error word (non-finite intensity) in bad[B].  A vector
// whose parameters are outside the model's domain (fill_res fails) gets
// PWA_EINVAL in vstat and the constants of another vector (its sums are not
// used); vstat [B] receives PWA_OK, PWA_EINVAL or PWA_ENONFINITE.
static pwa_status run_pass_b(pwa_variant* v, int B, const double* theta, const double* dir, bool hv, bool data_only,
                             pwa_status* vstat)
{
    const int K = v->base.K, S = v->base.S, P = v->base.P;
    VAR_TRY(reserve_vectors(v, B));
    int valid = -1;
    for (int b = 0; b < B; ++b) {
        vstat[b] = fill_res(v, theta + (size_t)b * P, hv ? dir + (size_t)b * P : nullptr, v->h_res + (size_t)b * K);
        if (vstat[b] == PWA_OK && valid < 0) valid = b;
    }
    if (valid < 0) return vstat[0];
    for (int b = 0; b < B; ++b)
        if (vstat[b] != PWA_OK) std::memcpy(v->h_res + (size_t)b * K, v->h_res + (size_t)valid * K, sizeof(VarRes) * K);
    v->base.err.clear();
    cudaStream_t st = v->base.stream;
    VAR_CUDA(v, cudaMemcpyAsync(v->d_res, v->h_res, sizeof(VarRes) * K * B, cudaMemcpyHostToDevice, st));
    VarArgs a{};
    a.m2[0] = v->d_m2[0];
    a.m2[1] = v->d_m2[1];
    a.F[0] = v->d_F[0];
    a.F[1] = v->d_F[1];
    a.w = v->d_w;
    a.n[0] = v->base.n[0];
    a.n[1] = v->base.n[1];
    a.K = K;
    // data only: the whole grid takes the data sample (the records hold that many warps)
    const int blocks0 = data_only ? v->blocks0 + v->blocks1 : v->blocks0;
    const int blocks1 = data_only ? 0 : v->blocks1;
    a.nbv = blocks0 + blocks1;
    a.blocks0 = blocks0;
    a.res = v->d_res;
    a.rec = v->d_rec;
    a.rec_len = v->rec_len;
    a.err = v->d_err;
    VarKernel fn = pick(S, v->per_projection != 0, hv);
    if (!fn) return vfail(v, PWA_EINVAL, "no variant kernel for this S");
    const size_t smem = var_smem_for(S, v->per_projection != 0);
    VAR_CUDA(v, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    fn<<<a.nbv * B, 32 * kVarWarps, smem, st>>>(a);
    VAR_CUDA(v, cudaGetLastError());
    variant_reduce_kernel<<<dim3((2 * v->rec_len + 31) / 32, B), dim3(32, 32), 0, st>>>(
        v->d_rec, v->rec_len, blocks0 * kVarWarps, blocks1 * kVarWarps, v->d_sums);
    VAR_CUDA(v, cudaGetLastError());
    const size_t ns = (size_t)B * 2 * v->rec_len;
    int* h_err = reinterpret_cast<int*>(v->h_sums + ns);
    VAR_CUDA(v, cudaMemcpyAsync(v->h_sums, v->d_sums, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
    VAR_CUDA(v, cudaMemcpyAsync(h_err, v->d_err, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
    VAR_CUDA(v, cudaMemsetAsync(v->d_err, 0, sizeof(int) * B, st));
    VAR_CUDA(v, cudaStreamSynchronize(st));
    for (int b = 0; b < B; ++b)
        if (vstat[b] == PWA_OK && h_err[b]) vstat[b] = PWA_ENONFINITE;
    return PWA_OK;
}

// The single-vector pass: an error status (with its message) when the vector failed.
static pwa_status run_pass(pwa_variant* v, const double* theta, const double* dir, bool hv, bool data_only)
{
    pwa_status vs = PWA_OK;
    VAR_TRY(run_pass_b(v, 1, theta, dir, hv, data_only, &vs));
    if (vs == PWA_ENONFINITE)
        return vfail(v, PWA_ENONFINITE, "an event's intensity is not finite, or not positive for a data event");
    if (vs != PWA_OK) return fill_res(v, theta, hv ? dir : nullptr);  // repeats the domain error with its message
    return PWA_OK;
}

// Eqs. 3, 6, 7 from one vector's sums (data sd, MC sm: per resonance
// [G NP][H NP], then sum w ln I for data and sum I, sum Idot for MC).
static pwa_status combine_sums(pwa_variant* v, const double* sd, const double* sm, double* nll, double* grad,
                               double* hv)
{
    const int P = v->base.P, NC = NC_of(v), NP = 2 * NC + 3;
    const double SL = sd[32 * 2 * NP], G = sm[32 * 2 * NP], Gd = sm[32 * 2 * NP + 1];
    if (!(G > 0.0) || !std::isfinite(SL)) return vfail(v, PWA_ENONFINITE, "the MC normalisation is not positive");
    const double Nd = v->base.Nd;
    *nll = -SL + Nd * std::log(G / v->base.Nmc);
    if (grad || hv) {
        for (int i = 0; i < P; ++i) {
            const int what = v->lay_what[i], k = v->lay_k[i], c = v->lay_s[i];
            const int slot = what == 0 ? c : what == 1 ? NC + c : 2 * NC + (what - 2);
            const double gD = sd[k * 2 * NP + slot], hD = sd[k * 2 * NP + NP + slot];
            const double gM = sm[k * 2 * NP + slot], hM = sm[k * 2 * NP + NP + slot];
            if (grad) grad[i] = -gD + Nd * gM / G;
            if (hv) hv[i] = -hD + Nd * (hM / G - gM * Gd / (G * G));
        }
    }
    return PWA_OK;
}

// One evaluation (NLL, and the gradient and H v when asked) at host theta, v.
pwa_status variant_eval(pwa_variant* v, const double* theta, const double* dir, double* nll, double* grad, double* hv)
{
    VAR_TRY(run_pass(v, theta, dir, hv != nullptr, false));
    return combine_sums(v, v->h_sums, v->h_sums + v->rec_len, nll, grad, hv);
}

// B evaluations in one launch (theta, dir [B][P]; nll [B]; grad, hv [B][P] or
// null): each vector runs the single pass's blocks, so its results equal
// variant_eval's.  status [B]: PWA_OK, PWA_EINVAL (outside the model's
// domain) or PWA_ENONFINITE per vector; the call fails only on CUDA or
// allocation errors.
pwa_status variant_eval_batch(pwa_variant* v, int B, const double* theta, const double* dir, double* nll,
                              double* grad, double* hv, pwa_status* status)
{
    const int P = v->base.P;
    VAR_TRY(run_pass_b(v, B, theta, dir, hv != nullptr, false, status));
    const size_t rl = (size_t)v->rec_len;
    for (int b = 0; b < B; ++b) {
        if (status[b] != PWA_OK) continue;
        const double* sd = v->h_sums + (size_t)b * 2 * rl;
        status[b] = combine_sums(v, sd, sd + rl, nll + b, grad ? grad + (size_t)b * P : nullptr,
                                 hv ? hv + (size_t)b * P : nullptr);
    }
    v->base.err.clear();
    return PWA_OK;
}

// The MC integral matrices at the line shapes of theta (kept in v with theta's shape part).
pwa_status variant_set_shapes(pwa_variant* v, const double* theta)
{
    const int K = v->base.K, S = v->base.S, NQ = S * K * K;
    VAR_TRY(fill_res(v, theta, nullptr));
    cudaStream_t st = v->base.stream;
    VAR_CUDA(v, cudaMemcpyAsync(v->d_res, v->h_res, sizeof(VarRes) * K, cudaMemcpyHostToDevice, st));
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long ntiles = (v->base.n[1] + kVarE - 1) / kVarE;
    const int nb = (int)std::max(1LL, std::min((long long)2 * sms, ntiles));
    const size_t smem = ((32 * sizeof(VarRes) + 15) / 16) * 16 + sizeof(float2) * (size_t)K * S * 33;
    double* d_rec = nullptr;
    double* d_out = nullptr;
    VAR_CUDA(v, cudaMallocAsync(&d_rec, sizeof(double) * 2 * (size_t)NQ * nb, st));
    cudaError_t e = cudaMallocAsync(&d_out, sizeof(double) * 2 * (size_t)NQ, st);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(variant_phi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        variant_phi_kernel<<<nb, kPhiThreads, smem, st>>>(v->d_m2[1], v->d_F[1], v->base.n[1], K, S, v->d_res, d_rec);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        variant_phi_reduce_kernel<<<(2 * NQ + 255) / 256, 256, 0, st>>>(d_rec, nb, 2 * NQ, d_out);
        e = cudaGetLastError();
    }
    v->phi.assign(2 * (size_t)NQ, 0.0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(v->phi.data(), d_out, sizeof(double) * 2 * NQ, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d_rec, st);
    if (d_out) cudaFreeAsync(d_out, st);
    if (e != cudaSuccess) return pwa::cuda_error(&v->base, e, "integral matrices");
    VAR_CUDA(v, cudaStreamSynchronize(st));
    for (double x : v->phi)
        if (!std::isfinite(x)) return vfail(v, PWA_ENONFINITE, "an integral matrix entry is not finite");
    v->shape_theta.assign(theta + v->Pc, theta + v->base.P);
    v->have_phi = true;
    return PWA_OK;
}

// Coupling-only evaluation at the fixed line shapes: the data by the variant
// kernel, the MC term from the integral matrices, sum_mc I = sum_s g_s^H Phi_s g_s.
pwa_status variant_coupling_eval(pwa_variant* v, const double* theta_c, const double* dir_c, double* nll, double* grad,
                                 double* hv)
{
    if (!v->have_phi) return vfail(v, PWA_EINVAL, "call pwa_variant_set_shapes first");
    const int K = v->base.K, S = v->base.S, P = v->base.P, Pc = v->Pc, NC = NC_of(v), NP = 2 * NC + 3;
    std::vector<double> th(P), dv(P, 0.0);
    std::copy(theta_c, theta_c + Pc, th.begin());
    std::copy(v->shape_theta.begin(), v->shape_theta.end(), th.begin() + Pc);
    if (hv) std::copy(dir_c, dir_c + Pc, dv.begin());
    VAR_TRY(run_pass(v, th.data(), dv.data(), hv != nullptr, true));
    const double* sd = v->h_sums;
    const double SL = sd[32 * 2 * NP];
    if (!std::isfinite(SL)) return vfail(v, PWA_ENONFINITE, "a data term is not finite");
    // couplings g_ks and directions gdot_ks for every (k, s) (fixed ones from the table)
    const size_t KS = (size_t)K * S;
    std::vector<double> gr(KS), gi(KS), er(KS), ei(KS), dr(KS, 0.0), di(KS, 0.0), vrh(KS, 0.0), vph(KS, 0.0);
    std::vector<double> mag((size_t)K * NC), ph((size_t)K * NC), vm((size_t)K * NC, 0.0), vp((size_t)K * NC, 0.0);
    for (int k = 0; k < K; ++k)
        for (int c = 0; c < NC; ++c) {
            mag[k * NC + c] = v->table[k].mag;
            ph[k * NC + c] = v->table[k].phase;
        }
    for (int i = 0; i < Pc; ++i) {
        const int k = v->lay_k[i], c = v->lay_s[i];
        if (v->lay_what[i] == 0) {
            mag[k * NC + c] = theta_c[i];
            if (hv) vm[k * NC + c] = dir_c[i];
        } else {
            ph[k * NC + c] = theta_c[i];
            if (hv) vp[k * NC + c] = dir_c[i];
        }
    }
    for (int k = 0; k < K; ++k)
        for (int s2 = 0; s2 < S; ++s2) {
            const int c = v->per_projection ? s2 : 0;
            const size_t q = (size_t)k * S + s2;
            const double rho = mag[k * NC + c];
            er[q] = std::cos(ph[k * NC + c]);
            ei[q] = std::sin(ph[k * NC + c]);
            gr[q] = rho * er[q];
            gi[q] = rho * ei[q];
            vrh[q] = vm[k * NC + c];
            vph[q] = vp[k * NC + c];
            dr[q] = vrh[q] * er[q] - vph[q] * gi[q];  // gdot = v_rho e + v_phi i g
            di[q] = vrh[q] * ei[q] + vph[q] * gr[q];
        }
    // (Phi_s g_s)_k and (Phi_s gdot_s)_k; G = sum_s g_s^H Phi_s g_s, Gdot = 2 Re sum_s gdot_s^H Phi_s g_s
    std::vector<double> pgr(KS), pgi(KS), pdr(KS), pdi(KS);
    double G = 0.0, Gd = 0.0;
    for (int s2 = 0; s2 < S; ++s2)
        for (int k = 0; k < K; ++k) {
            double ar = 0, ai = 0, br = 0, bi = 0;
            for (int kp = 0; kp < K; ++kp) {
                const size_t o = 2 * (((size_t)s2 * K + k) * K + kp);
                const double fr = v->phi[o], fi = v->phi[o + 1];
                const size_t q = (size_t)kp * S + s2;
                ar += fr * gr[q] - fi * gi[q];
                ai += fr * gi[q] + fi * gr[q];
                br += fr * dr[q] - fi * di[q];
                bi += fr * di[q] + fi * dr[q];
            }
            const size_t q = (size_t)k * S + s2;
            pgr[q] = ar;
            pgi[q] = ai;
            pdr[q] = br;
            pdi[q] = bi;
            G += gr[q] * ar + gi[q] * ai;          // Re conj(g) (Phi g)
            Gd += 2.0 * (dr[q] * ar + di[q] * ai);  // 2 Re conj(gdot) (Phi g)
        }
    if (!(G > 0.0)) return vfail(v, PWA_ENONFINITE, "the MC normalisation is not positive");
    const double Nd = v->base.Nd;
    *nll = -SL + Nd * std::log(G / v->base.Nmc);
    if (grad || hv) {
        for (int i = 0; i < Pc; ++i) {
            const int what = v->lay_what[i], k = v->lay_k[i], c = v->lay_s[i];
            const int slot = what == 0 ? c : NC + c;
            const double gD = sd[k * 2 * NP + slot], hD = sd[k * 2 * NP + NP + slot];
            double gM = 0.0, hM = 0.0;
            for (int s2 = 0; s2 < S; ++s2) {
                if (v->per_projection && s2 != c) continue;
                const size_t q = (size_t)k * S + s2;
                // dg and d gdot of this parameter (rho: e and v_phi i e; phi: i g and v_rho i e - v_phi g)
                double ar, ai, br, bi;
                if (what == 0) {
                    ar = er[q];
                    ai = ei[q];
                    br = -vph[q] * ei[q];
                    bi = vph[q] * er[q];
                } else {
                    ar = -gi[q];
                    ai = gr[q];
                    br = -vrh[q] * ei[q] - vph[q] * gr[q];
                    bi = vrh[q] * er[q] - vph[q] * gi[q];
                }
                gM += 2.0 * (ar * pgr[q] + ai * pgi[q]);  // 2 Re conj(dg) (Phi g)
                hM += 2.0 * (br * pgr[q] + bi * pgi[q]) + 2.0 * (ar * pdr[q] + ai * pdi[q]);
            }
            if (grad) grad[i] = -gD + Nd * gM / G;
            if (hv) hv[i] = -hD + Nd * (hM / G - gM * Gd / (G * G));
        }
    }
    return PWA_OK;
}

}  // namespace pwa

extern "C" {

thread_local std::string g_variant_create_error;

pwa_status pwa_variant_create(pwa_variant** out, const pwa_events* data, const pwa_events* mc,
                              const pwa_resonance* table, const pwa_lineshape* shapes, int K, int S, int per_projection,
                              void* cuda_stream)
{
    g_variant_create_error.clear();
    if (!out) return PWA_EINVAL;
    *out = nullptr;
    auto* v = new (std::nothrow) pwa_variant();
    if (!v) return PWA_ENOMEM;
    v->base.stream = static_cast<cudaStream_t>(cuda_stream);
    pwa_status st;
    try {
        st = create_impl(v, data, mc, table, shapes, K, S, per_projection);
    } catch (...) {
        st = vfail(v, PWA_ENOMEM, "host exception during create");
    }
    if (st != PWA_OK) {
        g_variant_create_error = v->base.err;
        pwa_variant_destroy(v);
        return st;
    }
    *out = v;
    return PWA_OK;
}

int pwa_variant_num_params(const pwa_variant* v) { return v ? v->base.P : -1; }

pwa_status pwa_variant_eval(pwa_variant* v, const double* theta, const double* dir, double* nll, double* grad,
                            double* hv)
{
    if (!v) return PWA_EINVAL;
    v->base.err.clear();
    if (!theta || !nll) return vfail(v, PWA_EINVAL, "theta and nll must not be NULL");
    if (hv && !dir) return vfail(v, PWA_EINVAL, "v is required for hv");
    for (int i = 0; i < v->base.P; ++i)
        if (!std::isfinite(theta[i]) || (hv && !std::isfinite(dir[i])))
            return vfail(v, PWA_EINVAL, "theta and v must be finite");
    std::vector<double> g_tmp;
    if (hv && !grad) {
        g_tmp.resize(v->base.P);
        grad = g_tmp.data();
    }
    return pwa::variant_eval(v, theta, dir, nll, grad, hv);
}

pwa_status pwa_variant_eval_batch(pwa_variant* v, int B, const double* theta, const double* dir, double* nll,
                                  double* grad, double* hv, pwa_status* status)
{
    if (!v) return PWA_EINVAL;
    v->base.err.clear();
    if (B < 1 || !theta || !nll || !status) return vfail(v, PWA_EINVAL, "B >= 1, theta, nll and status are required");
    if (hv && !dir) return vfail(v, PWA_EINVAL, "v is required for hv");
    for (size_t i = 0; i < (size_t)B * v->base.P; ++i)
        if (!std::isfinite(theta[i]) || (hv && !std::isfinite(dir[i])))
            return vfail(v, PWA_EINVAL, "theta and v must be finite");
    return pwa::variant_eval_batch(v, B, theta, dir, nll, grad, hv, status);
}

pwa_status pwa_variant_set_shapes(pwa_variant* v, const double* theta, double* phi_out)
{
    if (!v) return PWA_EINVAL;
    v->base.err.clear();
    if (!theta) return vfail(v, PWA_EINVAL, "theta must not be NULL");
    for (int i = 0; i < v->base.P; ++i)
        if (!std::isfinite(theta[i])) return vfail(v, PWA_EINVAL, "theta must be finite");
    v->have_phi = false;
    pwa_status st = pwa::variant_set_shapes(v, theta);
    if (st == PWA_OK && phi_out) std::memcpy(phi_out, v->phi.data(), sizeof(double) * v->phi.size());
    return st;
}

int pwa_variant_coupling_num_params(const pwa_variant* v) { return v ? v->Pc : -1; }

pwa_status pwa_variant_coupling_eval(pwa_variant* v, const double* theta_c, const double* dir_c, double* nll,
                                     double* grad, double* hv)
{
    if (!v) return PWA_EINVAL;
    v->base.err.clear();
    if (!theta_c || !nll) return vfail(v, PWA_EINVAL, "theta_c and nll must not be NULL");
    if (hv && !dir_c) return vfail(v, PWA_EINVAL, "v is required for hv");
    for (int i = 0; i < v->Pc; ++i)
        if (!std::isfinite(theta_c[i]) || (hv && !std::isfinite(dir_c[i])))
            return vfail(v, PWA_EINVAL, "theta_c and v must be finite");
    std::vector<double> g_tmp;
    if (hv && !grad) {
        g_tmp.resize(v->Pc);
        grad = g_tmp.data();
    }
    return pwa::variant_coupling_eval(v, theta_c, dir_c, nll, grad, hv);
}

const char* pwa_variant_last_error(const pwa_variant* v)
{
    return v ? v->base.err.c_str() : g_variant_create_error.c_str();
}

void pwa_variant_destroy(pwa_variant* v)
{
    if (!v) return;
    if (v->base.stream) cudaStreamSynchronize(v->base.stream);
    else cudaDeviceSynchronize();
    for (int s = 0; s < 2; ++s) {
        if (v->d_m2[s]) cudaFree(v->d_m2[s]);
        if (v->d_F[s]) cudaFree(v->d_F[s]);
    }
    void* ps[] = {v->d_w, v->d_res, v->d_rec, v->d_sums, v->d_err};
    for (void* p : ps)
        if (p) cudaFree(p);
    if (v->h_sums) cudaFreeHost(v->h_sums);
    if (v->h_res) cudaFreeHost(v->h_res);
    delete[] v->table;
    delete[] v->shapes;
    cudaGetLastError();
    delete v;
}

}  // extern "C"

namespace pwa {
pwa_handle* variant_base(pwa_variant* v) { return v ? &v->base : nullptr; }
}  // namespace pwa
