// pass_kernel.cuh -- the fused streaming pass of libpwa (sm_103a).
//
// One launch reads every event tile of F exactly once and produces the NLL,
// its gradient and a Hessian-vector product (paper Eqs. 3, 6, 7).  Per event
// e and resonance k (all FP32, in registers):
//   BW_k   = 1 / (M_k^2 - m^2_{ch(k)}(e) - i M_k Gamma_k)           (a-3)
//   c_k    = g_k BW_k,   cdot_k = BW_k (alpha_k + BW_k beta_k)       (a-3, a-6)
//   A_s    = sum_k c_k F_{k,s},  Adot_s = sum_k cdot_k F_{k,s}       (sweep 1, Eq. 1)
//   I      = sum_s |A_s|^2,      Idot = 2 Re sum_s conj(A_s) Adot_s
//   D_k    = sum_s conj(A_s) F_{k,s},  Ddot_k = sum_s conj(Adot_s) F_{k,s}   (sweep 2)
// and the event's contribution to five complex sums per resonance,
//   Q1 += Dh B, Q2 += Dh B^2, Q3 += Dh B^3, P1 += Dt B, P2 += Dt B^2,
// with Dh = a D, Dt = a Ddot - b D, (a, b) = (w/I, w Idot/I^2) for data and
// (1, 0) for MC.  Every derivative of the NLL with respect to resonance k's
// (rho, phi, M, Gamma) is a fixed complex combination of these sums, applied
// once per pass in FP64 (see combine()); no per-event intermediate is stored.
//
// Data layout (built by pwa_create): events are cut into tiles of E events;
// one tile record is contiguous in HBM:
//   F   float2 [K][S][E]   position p = (e + shift_k) mod E   (shift: bank-conflict
//                          free sweeps when several lanes share an event)
//   m2  float  [3][E]
//   w   float  [E]         (data tiles only)
// A block streams whole tile records into shared memory with the TMA bulk
// copy engine (cp.async.bulk + mbarrier transaction counts), NST tiles in
// flight, and works on them in two phases:
//   phase 1: H lanes per event (butterfly-reduced) build A, Adot, I, Idot;
//   phase 2: each warp owns KPW resonances and sweeps the tile's events.
// Per-lane FP32 sums are folded into FP64 every kWindow tiles; each block
// writes FP64 partials; a two-level "last block done" reduction (fixed order,
// hence run-to-run bit-identical) adds them and the final block evaluates the
// combination of Eqs. 4, 6, 7 in FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace pwa {

constexpr int kNV = 10;        // FP64 values per resonance and sample set
constexpr int kNScal = 3;      // per-set scalars: data (sum w ln I, -, -), MC (G, Gdot, -)
constexpr int kWindow = 64;    // tiles between FP32 -> FP64 folds
constexpr int kMaxThreads = 512;

// MODE_HVP_REUSE: H v at the theta of the last full HVP pass, taking the
// per-resonance Q sums, G and the data NLL sum from that pass (they do not
// depend on v) and accumulating only P1 and P2
enum { MODE_NLL = 0, MODE_GRAD = 1, MODE_HVP = 2, MODE_HVP_REUSE = 3 };
enum { ERR_TIMEOUT = 1, ERR_NONFINITE = 2, ERR_STALE = 4 };

struct ResParam {       // parameter map of one resonance
    int idx[4];         // theta index of rho, phi, M, Gamma; -1 when fixed
    int channel;
    int pad;
    double fixed[4];    // values of fixed parameters
};

struct __align__(16) KConst {  // FP32 per-resonance constants (48 bytes)
    float m2hi, m2lo, mg;      // M^2 = m2hi + m2lo (FP32 pair), M Gamma
    int ch;                    // channel of m^2
    float gre, gim;            // g = rho e^{i phi}
    float are, aim;            // alpha = v_rho e^{i phi} + i v_phi g
    float bre, bim;            // beta = g (v_M (-2M + i Gamma) + v_Gamma (i M))
    int shift;                 // rotation of the event position in the tile
    float mg2;                 // (M Gamma)^2
};

// Layout of a tile's F block.  Even S: for each (k, projection pair q = s/2, tile
// position p) one 16-byte group holds (Re F_{2q}, Re F_{2q+1}, Im F_{2q}, Im F_{2q+1}),
// so that the real parts and the imaginary parts of two projections load as packed
// FP32 pairs; the groups are ordered [k][q][p].  Odd S: (Re F, Im F) at [k][s][p].
// f_slot: float2 index of the group of (k, s, p) (even S) or of its (Re, Im) pair (odd S).
__host__ __device__ inline int f_slot(int k, int s, int p, int S, int E)
{
    return (S % 2 == 0) ? ((k * (S / 2) + s / 2) * E + p) * 2 : (k * S + s) * E + p;
}
// f_re: float index of Re F_{k,s} at tile position p; Im F is f_im_off(S) floats further.
__host__ __device__ inline int f_re(int k, int s, int p, int S, int E)
{
    return (S % 2 == 0) ? ((k * (S / 2) + s / 2) * E + p) * 4 + (s & 1) : ((k * S + s) * E + p) * 2;
}
__host__ __device__ inline int f_im_off(int S) { return S % 2 == 0 ? 2 : 1; }

struct PassArgs {
    const unsigned char* tiles[2];  // data, MC tile records
    uint32_t tile_bytes[2];
    int ntiles[2];
    long long nev[2];
    int K, E, H, W, NST;
    uint32_t stage_bytes;
    int P;
    const ResParam* res;
    const double* theta;  // [B][P]
    const double* v;      // [B][P] (HVP) or null
    double Nd, Nmc;
    // B parameter vectors are evaluated in one launch: block i works for vector
    // i % B and is block i / B of the Gb blocks that share its events
    int B = 1, Gb = 0;
    double* block_rec;      // [B][Gb][rec_len]
    double* group_rec;      // [B][ngroups][rec_len]
    unsigned* group_count;  // [B][ngroups]
    unsigned* top_count;    // [B]
    int group_size, ngroups, rec_len;  // ngroups = groups per vector
    double* out;                       // [B][1 + 2P]
    unsigned long long* bad;
    int* err;
    long long timeout_cycles;
    const int* skip = nullptr;  // when set and non-zero at launch, the pass does nothing
    int* err_vec = nullptr;     // when set: per-vector error words [B] (besides err)
    // [rec_len] totals then [P] theta of the last full HVP pass: written by a
    // single-vector MODE_HVP pass, read (and checked against theta) by MODE_HVP_REUSE
    double* cache = nullptr;
    // events per warp of the tiling the tile records were laid out for (their
    // resonance rotation, tile_shift); a kernel instance with H lanes per
    // event reads them when 16 / ev divides H (always for H = 4 and 8)
    int ev = 8;
    int S = 0;  // projections (the instance is compiled for S; a launch over several handles dispatches on it)
};

// ---------------------------------------------------------------------------
// small PTX helpers: mbarrier, TMA bulk copy
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arm the barrier for `bytes` of transactions and start one bulk copy of a
// contiguous tile record from global into shared memory.
__device__ __forceinline__ void tma_load_tile(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Wait for the barrier phase with the given parity; gives up after `budget`
// SM cycles and returns false (the caller reports ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget)
{
    const uint32_t a = smem_addr(bar);
    long long t0 = -1;  // the clock is read only once the first try has failed
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        const long long now = clock64();
        if (t0 < 0) t0 = now;
        else if (now - t0 > budget) return false;
    }
}

// acc = (hi, lo) += x with Knuth's TwoSum: hi + lo stays the exact sum up to the
// rounding of lo (about 2^-48 relative), without the FP64 pipe
__device__ __forceinline__ void two_sum_add(float2& acc, float x)
{
    const float s = __fadd_rn(acc.x, x);
    const float bp = __fsub_rn(s, acc.x);
    const float ap = __fsub_rn(s, bp);
    const float err = __fadd_rn(__fsub_rn(acc.x, ap), __fsub_rn(x, bp));
    acc = make_float2(s, __fadd_rn(acc.y, err));
}

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ---------------------------------------------------------------------------
// per-resonance constants (a-1): FP64 in, FP32 out
// ---------------------------------------------------------------------------

struct ResValues {
    double rho, phi, M, G;     // parameter values
    double vr, vp, vm, vg;     // direction components (0 for fixed parameters)
};

__device__ __forceinline__ ResValues res_values(const PassArgs& a, const double* theta, const double* v, int k,
                                                bool with_v)
{
    const ResParam r = a.res[k];
    double p[4], d[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        p[j] = r.idx[j] >= 0 ? theta[r.idx[j]] : r.fixed[j];
        d[j] = (with_v && r.idx[j] >= 0) ? v[r.idx[j]] : 0.0;
    }
    return ResValues{p[0], p[1], p[2], p[3], d[0], d[1], d[2], d[3]};
}

__device__ __forceinline__ KConst make_kconst(const PassArgs& a, const double* theta, const double* v, int k,
                                              bool with_v, int ev)
{
    // FP64 only where FP32 would lose the narrow peaks (M^2 as an FP32 pair,
    // M Gamma) and for the phase's range reduction; the FP32 constants are
    // otherwise computed in FP32 (the FP64 pipe is narrow on this GPU)
    const ResValues rv = res_values(a, theta, v, k, with_v);
    const double phr = rv.phi - 6.283185307179586 * rint(rv.phi * 0.15915494309189535);
    float s, c;
    sincosf((float)phr, &s, &c);
    const float rho = (float)rv.rho;
    const float gre = rho * c, gim = rho * s;
    const double M2 = rv.M * rv.M;
    const double MG = rv.M * rv.G;
    KConst kc;
    kc.m2hi = (float)M2;
    kc.m2lo = (float)(M2 - (double)kc.m2hi);
    kc.mg = (float)MG;
    kc.mg2 = (float)(MG * MG);
    kc.ch = a.res[k].channel;
    kc.gre = gre;
    kc.gim = gim;
    // alpha = v_rho E + i v_phi g
    const float vr = (float)rv.vr, vp = (float)rv.vp, vm = (float)rv.vm, vg = (float)rv.vg;
    const float M = (float)rv.M, G = (float)rv.G;
    kc.are = vr * c - vp * gim;
    kc.aim = vr * s + vp * gre;
    // u = v_M a1 + v_G a2, a1 = -2M + i G, a2 = i M;  beta = g u
    const float ure = -2.f * M * vm, uim = G * vm + M * vg;
    kc.bre = gre * ure - gim * uim;
    kc.bim = gre * uim + gim * ure;
    kc.shift = ev < 16 ? (k % (16 / ev)) * ev : 0;
    return kc;
}

// BW_k(e) = 1/(M^2 - m^2 - i M Gamma) = (d + i mg) / (d^2 + mg^2), d = M^2 - m^2
// with M^2 carried as an FP32 (hi, lo) pair so that narrow peaks keep their shape.
__device__ __forceinline__ void breit_wigner(const KConst& kc, float m2, float& br, float& bi)
{
    const float d = (kc.m2hi - m2) + kc.m2lo;
    const float r = __fdividef(1.0f, fmaf(d, d, kc.mg2));
    br = d * r;
    bi = kc.mg * r;
}

// The S projections of one (resonance, event) from the tile's F block; row
// points at s = 0 (see f_slot).  Even S: one 16-byte load per projection pair q,
// fv[2q] = (Re F_2q, Re F_2q+1) and fv[2q+1] = (Im F_2q, Im F_2q+1).  Odd S:
// fv[s] = (Re F_s, Im F_s).
template <int S, int E>
__device__ __forceinline__ void load_row(const float2* row, float2 (&fv)[S])
{
    if constexpr (S % 2 == 0) {
#pragma unroll
        for (int q = 0; q < S / 2; ++q) {
            const float4 v = *reinterpret_cast<const float4*>(row + 2 * E * q);
            fv[2 * q] = make_float2(v.x, v.y);
            fv[2 * q + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) fv[s] = row[s * E];
    }
}

// ---------------------------------------------------------------------------
// the fused pass
// ---------------------------------------------------------------------------

// Tile shape: kTileE = 32 events per tile; a block has W warps and W lanes
// share one event in the coherent-sum sweep (each takes every W-th resonance),
// so a warp covers 32/W events and the block covers the tile; in the second
// sweep lane l handles event l and warp w owns resonances [w KPW, (w+1) KPW).
constexpr int kTileE = 32;

// The pass for one block: vector bt of the batch, block gb of the a.Gb blocks
// that share that vector's events (tiles gb, gb + Gb, ...).  pass_kernel runs
// it for every block of one handle; multi_pass_kernel (multi.cu) for blocks
// of several handles in one launch.
template <int MODE, int S, int W, int KPW>
__device__ __forceinline__ void pass_body(const PassArgs& a, const int bt, const int gb, unsigned char* smem)
{
    constexpr bool HV = MODE >= MODE_HVP;
    constexpr bool RU = MODE == MODE_HVP_REUSE;  // Q sums, G, sum w ln I from the cache
    constexpr bool GR = MODE >= MODE_GRAD;
    constexpr int E = kTileE;
    constexpr int H = W;                       // lanes per event
    constexpr int EV = 32 / H;                 // events per warp (one tile = W x EV events)
    constexpr int NVM = RU ? 4 : (HV ? kNV : 4);  // accumulated reals per resonance
    constexpr int QOFF = RU ? 6 : 0;           // record slot of the first accumulated real
    constexpr int NT = 32 * W;
    using AVec = typename std::conditional<HV, float4, float2>::type;
    (void)sizeof(AVec);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = a.K, NST = a.NST;

    // shared memory: stages | KConst[K] | per-warp (hi, lo) FP32 sums [W][K*kNV + 2] | stage counters | mbarriers
    unsigned char* stages = smem;
    KConst* kc = reinterpret_cast<KConst*>(smem + (size_t)NST * a.stage_bytes);
    const int wlen = K * kNV + 2;
    float2* wacc = reinterpret_cast<float2*>(kc + K);  // (hi, lo) FP32 pairs: hi + lo is the exact running sum
    unsigned* stage_cnt = reinterpret_cast<unsigned*>(wacc + W * wlen);
    long long* issued = reinterpret_cast<long long*>(stage_cnt + 4);  // last iteration issued per stage
    uint64_t* mbar = reinterpret_cast<uint64_t*>(issued + 4);
    __shared__ int s_flag;
    __shared__ volatile int s_abort;
    __shared__ double s_part[kMaxThreads / 32];

    const long long T = (long long)a.ntiles[0] + a.ntiles[1];
    const long long G = a.Gb;
    const double* theta = a.theta + (size_t)bt * a.P;
    const double* vdir = HV ? a.v + (size_t)bt * a.P : nullptr;
    double* out = a.out + (size_t)bt * (1 + 2 * a.P);
    const int rec_block = bt * a.Gb + gb;  // index of this block's partial-sum record

    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < NST; ++s) {
            mbar_init(&mbar[s], 1);
            stage_cnt[s] = 0;
            issued[s] = -1;
        }
        fence_mbar_init();
        for (int i = 0; i < NST; ++i) {
            const long long t = gb + i * G;
            if (t < T) {
                const int smp = t < a.ntiles[0] ? 0 : 1;
                const long long lt = smp ? t - a.ntiles[0] : t;
                tma_load_tile(stages + (size_t)i * a.stage_bytes,
                              a.tiles[smp] + (size_t)lt * a.tile_bytes[smp], a.tile_bytes[smp], &mbar[i]);
                issued[i] = i;
            }
        }
    }
    for (int k = tid; k < K; k += NT) kc[k] = make_kconst(a, theta, vdir, k, HV, a.ev);
    for (int i = tid; i < W * wlen; i += NT) wacc[i] = make_float2(0.f, 0.f);
    __syncthreads();

    // lane (h, el): event e = warp * EV + el of every tile, resonances k = h + i H
    const int h = lane / EV, el = lane % EV;
    const int e = warp * EV + el;
    // all resonances of a lane share one rotation (it depends on k mod (H/2))
    const int p = (e + (h < K ? kc[h].shift : 0)) & (E - 1);
    const int kcount = h < K ? (K - 1 - h) / H + 1 : 0;  // resonances of this lane (<= KPW in GRAD/HVP)
    // channels of this lane's resonances, 2 bits each, so that the m^2 loads need no KConst load
    uint32_t chbits = 0;
    if constexpr (GR) {
#pragma unroll
        for (int j = 0; j < KPW; ++j)
            if (j < kcount) chbits |= (uint32_t)kc[h + j * H].ch << (2 * j);
    }

    // FP32 per-lane sums of the current fold window
    float acc[GR ? KPW : 1][GR ? NVM : 1];
#pragma unroll
    for (int j = 0; j < (GR ? KPW : 1); ++j)
#pragma unroll
        for (int q = 0; q < (GR ? NVM : 1); ++q) acc[j][q] = 0.f;
    float sc0 = 0.f, sc1 = 0.f;

    // fold the warp's FP32 sums into its compensated (hi, lo) sums in shared memory:
    // reduce over the EV lanes of each resonance group, lane el == 0 adds (fixed
    // order).  TwoSum keeps these sums as exact as FP64 ones without the FP64
    // pipe, which is narrow on this GPU.
    auto fold = [&]() {
        float2* wa = wacc + warp * wlen;
        if constexpr (GR) {
#pragma unroll
            for (int j = 0; j < KPW; ++j)
#pragma unroll
                for (int q = 0; q < NVM; ++q) {
                    float v = acc[j][q];
                    acc[j][q] = 0.f;
#pragma unroll
                    for (int o = 1; o < EV; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (el == 0 && j < kcount) two_sum_add(wa[(h + j * H) * kNV + QOFF + q], v);
                }
        }
        const float t0 = warp_sum(sc0), t1 = warp_sum(sc1);
        sc0 = sc1 = 0.f;
        if (lane == 0) {
            two_sum_add(wa[K * kNV + 0], t0);
            two_sum_add(wa[K * kNV + 1], t1);
        }
    };

    // the block's FP64 partials of one sample set: sum the warps in order
    auto write_set = [&](int set) {
        __syncthreads();
        double* rec = a.block_rec + (size_t)rec_block * a.rec_len + (size_t)set * (K * kNV + kNScal);
        for (int i = tid; i < K * kNV + kNScal; i += NT) {
            double v = 0.0;
            if (i < wlen)
                for (int w = 0; w < W; ++w) v += (double)wacc[w * wlen + i].x + (double)wacc[w * wlen + i].y;
            rec[i] = v;
        }
        __syncthreads();
        for (int i = tid; i < W * wlen; i += NT) wacc[i] = make_float2(0.f, 0.f);
        __syncthreads();
    };

    int win = 0;
    int st = 0;         // stage of iteration i (i mod NST), kept without 64-bit division
    uint32_t ph = 0;    // barrier phase parity of iteration i ((i / NST) & 1)
    // one tile of sample set SMP (0 data, 1 MC): global tile index t, iteration i of this block
    auto tile = [&](auto smp_c, long long t, long long i) {
        constexpr int smp = decltype(smp_c)::value;
        // the reuse pass needs A (for I, Idot and the data weights) on data events only
        constexpr bool NEED_A = !(RU && smp == 1);
        const long long lt = smp ? t - a.ntiles[0] : t;
        bool ok = false;
        if (!s_abort) {
            ok = __all_sync(0xffffffffu, mbar_wait(&mbar[st], ph, a.timeout_cycles));
            if (!ok && lane == 0) s_abort = 1;
        }
        if (ok) {
            const float2* Fs = reinterpret_cast<const float2*>(stages + (size_t)st * a.stage_bytes);
            const float* m2s = reinterpret_cast<const float*>(Fs + K * S * E);
            const long long e_base = lt * E;
            const bool valid = e < (int)min((long long)E, a.nev[smp] - e_base);
            const float2* Frow = Fs + f_slot(h, 0, p, S, E);  // F_{k,.}(e) for k = h; + i H S E for k = h + i H

            // ---- sweep 1: BW, couplings, coherent sums over this lane's resonances ----
            // packed FP32 pairs: A_s += Re(F) c + Im(F) (i c), two paired FMAs per
            // complex product (and the same for Adot with cdot)
            // PA, PD: the lane's partial sums of A_s and Adot_s as S packed pairs.  Even S:
            // PA[2q] = (Re A_2q, Re A_2q+1), PA[2q+1] = (Im A_2q, Im A_2q+1); odd S:
            // PA[s] = (Re A_s, Im A_s).  Either way I = sum of the squares of all entries.
            float2 PA[S], PD[S];
            float2 Bk[GR ? KPW : 1];
            if constexpr (S % 2 == 0) {
                // packed pairs over two projections: (Ar_s, Ar_s+1) += (ReF) c_r - (ImF) c_i, ...
                constexpr int Q = S / 2;
                float2 ARp[Q], AIp[Q], DRp[Q], DIp[Q];
#pragma unroll
                for (int q = 0; q < Q; ++q) ARp[q] = AIp[q] = DRp[q] = DIp[q] = make_float2(0.f, 0.f);
                auto visit = [&](int k, const float2* Fk, float m2v, float& br, float& bi) {
                    const KConst c = kc[k];
                    breit_wigner(c, m2v, br, bi);
                    const float cr = c.gre * br - c.gim * bi, ci = c.gre * bi + c.gim * br;
                    float dr = 0.f, di = 0.f;
                    if constexpr (HV) {
                        const float tr = c.are + (br * c.bre - bi * c.bim);
                        const float ti = c.aim + (br * c.bim + bi * c.bre);
                        dr = br * tr - bi * ti;
                        di = br * ti + bi * tr;
                    }
                    float2 fv[S];
                    load_row<S, E>(Fk, fv);  // fv[2q] = Re pair, fv[2q+1] = Im pair
                    const float2 crr = make_float2(cr, cr), cii = make_float2(ci, ci), ncc = make_float2(-ci, -ci);
                    const float2 drr = make_float2(dr, dr), dii = make_float2(di, di), ndd = make_float2(-di, -di);
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        const float2 R = fv[2 * q], Im = fv[2 * q + 1];
                        if constexpr (NEED_A) {
                            ARp[q] = __ffma2_rn(Im, ncc, __ffma2_rn(R, crr, ARp[q]));
                            AIp[q] = __ffma2_rn(Im, crr, __ffma2_rn(R, cii, AIp[q]));
                        }
                        if constexpr (HV) {
                            DRp[q] = __ffma2_rn(Im, ndd, __ffma2_rn(R, drr, DRp[q]));
                            DIp[q] = __ffma2_rn(Im, drr, __ffma2_rn(R, dii, DIp[q]));
                        }
                    }
                };
                if constexpr (GR) {
#pragma unroll
                    for (int j = 0; j < KPW; ++j) {
                        if (j >= kcount) break;
                        visit(h + j * H, Frow + j * H * S * E, m2s[((chbits >> (2 * j)) & 3u) * E + e], Bk[j].x,
                              Bk[j].y);
                    }
                } else {
#pragma unroll 2
                    for (int j = 0; j < kcount; ++j) {
                        float br, bi;
                        visit(h + j * H, Frow + j * H * S * E, m2s[kc[h + j * H].ch * E + e], br, bi);
                    }
                }
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    PA[2 * q] = ARp[q];
                    PA[2 * q + 1] = AIp[q];
                    PD[2 * q] = DRp[q];
                    PD[2 * q + 1] = DIp[q];
                }
            } else {
                float2 A2[S], D2[S];
#pragma unroll
                for (int s = 0; s < S; ++s) A2[s] = D2[s] = make_float2(0.f, 0.f);
                auto visit = [&](int k, const float2* Fk, float m2v, float& br, float& bi) {
                    const KConst c = kc[k];
                    breit_wigner(c, m2v, br, bi);
                    const float cr = c.gre * br - c.gim * bi, ci = c.gre * bi + c.gim * br;
                    float dr = 0.f, di = 0.f;
                    if constexpr (HV) {
                        const float tr = c.are + (br * c.bre - bi * c.bim);
                        const float ti = c.aim + (br * c.bim + bi * c.bre);
                        dr = br * tr - bi * ti;
                        di = br * ti + bi * tr;
                    }
                    float2 fv[S];
                    load_row<S, E>(Fk, fv);
                    const float2 c2 = make_float2(cr, ci), ic2 = make_float2(-ci, cr);
                    const float2 d2 = make_float2(dr, di), id2 = make_float2(-di, dr);
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        const float2 fxx = make_float2(fv[s].x, fv[s].x), fyy = make_float2(fv[s].y, fv[s].y);
                        if constexpr (NEED_A) A2[s] = __ffma2_rn(fyy, ic2, __ffma2_rn(fxx, c2, A2[s]));
                        if constexpr (HV) D2[s] = __ffma2_rn(fyy, id2, __ffma2_rn(fxx, d2, D2[s]));
                    }
                };
                if constexpr (GR) {
#pragma unroll
                    for (int j = 0; j < KPW; ++j) {
                        if (j >= kcount) break;
                        visit(h + j * H, Frow + j * H * S * E, m2s[((chbits >> (2 * j)) & 3u) * E + e], Bk[j].x,
                              Bk[j].y);
                    }
                } else {
                    // the NLL-only pass is compiled once per W: the trip count is runtime
#pragma unroll 2
                    for (int j = 0; j < kcount; ++j) {
                        float br, bi;
                        visit(h + j * H, Frow + j * H * S * E, m2s[kc[h + j * H].ch * E + e], br, bi);
                    }
                }
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    PA[s] = A2[s];
                    PD[s] = D2[s];
                }
            }
            // ---- the H lanes of the event combine their partial sums ----
#pragma unroll
            for (int off = EV; off < 32; off <<= 1) {
#pragma unroll
                for (int i = 0; i < S; ++i) {
                    if constexpr (NEED_A)
                        PA[i] = __fadd2_rn(PA[i], make_float2(__shfl_xor_sync(0xffffffffu, PA[i].x, off),
                                                              __shfl_xor_sync(0xffffffffu, PA[i].y, off)));
                    if constexpr (HV)
                        PD[i] = __fadd2_rn(PD[i], make_float2(__shfl_xor_sync(0xffffffffu, PD[i].x, off),
                                                              __shfl_xor_sync(0xffffffffu, PD[i].y, off)));
                }
            }
            // I = sum_s |A_s|^2, Idot = 2 Re sum_s conj(A_s) Adot_s
            float2 I2 = make_float2(0.f, 0.f), Id2 = I2;
#pragma unroll
            for (int i = 0; i < S; ++i) {
                I2 = __ffma2_rn(PA[i], PA[i], I2);
                if constexpr (HV) Id2 = __ffma2_rn(PA[i], PD[i], Id2);
            }
            const float I = I2.x + I2.y;
            const float Id = 2.f * (Id2.x + Id2.y);
            float wa = 0.f, wb = 0.f;  // (a, b) = (w/I, w Idot/I^2) for data, (1, 0) for MC
            if constexpr (smp == 0) {
                const float w = m2s[3 * E + e];
                const bool good = I > 0.f && I < INFINITY;
                if (valid && good) {
                    const float rI = __fdividef(1.0f, I);
                    wa = w * rI;
                    wb = wa * Id * rI;
                }
                if (h == 0) {
                    if (valid && !good) {
                        atomicMin(a.bad, (unsigned long long)(e_base + e));
                        atomicOr(a.err, ERR_NONFINITE);
                        if (a.err_vec) atomicOr(a.err_vec + bt, ERR_NONFINITE);
                    }
                    if (valid && good) sc0 += w * logf(I);
                }
            } else if constexpr (RU) {
                if (valid) wa = 1.f;  // G, Gdot and the finiteness check come with the cached full pass
            } else {
                if (valid) wa = 1.f;
                if (h == 0) {
                    if (valid && !(I < INFINITY)) {
                        atomicMin(a.bad, (unsigned long long)(a.nev[0] + e_base + e));
                        atomicOr(a.err, ERR_NONFINITE);
                        if (a.err_vec) atomicOr(a.err_vec + bt, ERR_NONFINITE);
                    }
                    if (valid) {
                        sc0 += I;
                        sc1 += Id;
                    }
                }
            }

            if constexpr (GR) {
                // ---- sweep 2 (packed pairs over two projections): with a = (a Ar, a Ai) and
                //      F = (ReF, ImF) pairs, Re Dh = sum (ReF a_r + ImF a_i), Im Dh = sum (ImF a_r - ReF a_i);
                //      the same for Dt with (a Adot - b A) ----
                constexpr int Q2 = S % 2 == 0 ? S / 2 : 1;
                // (each mode uses a subset: the unused ones are compiled away)
                [[maybe_unused]] float2 aR[Q2], aI[Q2], naI[Q2], dR[Q2], dI[Q2], ndI[Q2];
                [[maybe_unused]] float2 al[S], be[S], dl[S], de[S];
                const float2 waa = make_float2(wa, wa), nwaa = make_float2(-wa, -wa);
                const float2 wbb = make_float2(wb, wb), nwbb = make_float2(-wb, -wb);
                if constexpr (S % 2 == 0) {
#pragma unroll
                    for (int q = 0; q < Q2; ++q) {
                        aR[q] = __fmul2_rn(waa, PA[2 * q]);
                        aI[q] = __fmul2_rn(waa, PA[2 * q + 1]);
                        naI[q] = __fmul2_rn(nwaa, PA[2 * q + 1]);
                        if constexpr (HV && smp == 0) {
                            dR[q] = __ffma2_rn(waa, PD[2 * q], __fmul2_rn(nwbb, PA[2 * q]));
                            dI[q] = __ffma2_rn(waa, PD[2 * q + 1], __fmul2_rn(nwbb, PA[2 * q + 1]));
                            ndI[q] = __ffma2_rn(nwaa, PD[2 * q + 1], __fmul2_rn(wbb, PA[2 * q + 1]));
                        } else if constexpr (HV) {  // MC events: b = 0
                            dR[q] = __fmul2_rn(waa, PD[2 * q]);
                            dI[q] = __fmul2_rn(waa, PD[2 * q + 1]);
                            ndI[q] = __fmul2_rn(nwaa, PD[2 * q + 1]);
                        }
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        al[s] = __fmul2_rn(waa, PA[s]);
                        be[s] = make_float2(-al[s].y, al[s].x);
                        if constexpr (HV) {
                            dl[s] = __ffma2_rn(waa, PD[s], __fmul2_rn(nwbb, PA[s]));
                            de[s] = make_float2(-dl[s].y, dl[s].x);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < KPW; ++j) {
                    if (j >= kcount) break;
                    const float br = Bk[j].x, bi = Bk[j].y;
                    float2 fv[S];
                    load_row<S, E>(Frow + j * H * S * E, fv);
                    float2 X = make_float2(0.f, 0.f), Y = X, XD = X, YD = X;
                    if constexpr (S % 2 == 0) {
#pragma unroll
                        for (int q = 0; q < Q2; ++q) {
                            const float2 R = fv[2 * q], Im = fv[2 * q + 1];
                            if constexpr (!RU) {
                                X = __ffma2_rn(Im, aI[q], __ffma2_rn(R, aR[q], X));
                                Y = __ffma2_rn(R, naI[q], __ffma2_rn(Im, aR[q], Y));
                            }
                            if constexpr (HV) {
                                XD = __ffma2_rn(Im, dI[q], __ffma2_rn(R, dR[q], XD));
                                YD = __ffma2_rn(R, ndI[q], __ffma2_rn(Im, dR[q], YD));
                            }
                        }
                    } else {
#pragma unroll
                        for (int s = 0; s < S; ++s) {
                            if constexpr (!RU) {
                                X = __ffma2_rn(fv[s], al[s], X);
                                Y = __ffma2_rn(fv[s], be[s], Y);
                            }
                            if constexpr (HV) {
                                XD = __ffma2_rn(fv[s], dl[s], XD);
                                YD = __ffma2_rn(fv[s], de[s], YD);
                            }
                        }
                    }
                    [[maybe_unused]] const float hr = X.x + X.y, hi = Y.x + Y.y;
                    [[maybe_unused]] const float tr = XD.x + XD.y, ti = YD.x + YD.y;
                    const float b2r = fmaf(br, br, -bi * bi), b2i = 2.f * br * bi;
                    if constexpr (RU) {
                        // P1 += Dt B, P2 += Dt B^2 only (record slots 6..9)
                        acc[j][0] = fmaf(tr, br, fmaf(-ti, bi, acc[j][0]));
                        acc[j][1] = fmaf(tr, bi, fmaf(ti, br, acc[j][1]));
                        acc[j][2] = fmaf(tr, b2r, fmaf(-ti, b2i, acc[j][2]));
                        acc[j][3] = fmaf(tr, b2i, fmaf(ti, b2r, acc[j][3]));
                        continue;
                    }
                    acc[j][0] = fmaf(hr, br, fmaf(-hi, bi, acc[j][0]));
                    acc[j][1] = fmaf(hr, bi, fmaf(hi, br, acc[j][1]));
                    acc[j][2] = fmaf(hr, b2r, fmaf(-hi, b2i, acc[j][2]));
                    acc[j][3] = fmaf(hr, b2i, fmaf(hi, b2r, acc[j][3]));
                    if constexpr (HV) {
                        const float b3r = fmaf(b2r, br, -b2i * bi), b3i = fmaf(b2r, bi, b2i * br);
                        acc[j][4] = fmaf(hr, b3r, fmaf(-hi, b3i, acc[j][4]));
                        acc[j][5] = fmaf(hr, b3i, fmaf(hi, b3r, acc[j][5]));
                        acc[j][6] = fmaf(tr, br, fmaf(-ti, bi, acc[j][6]));
                        acc[j][7] = fmaf(tr, bi, fmaf(ti, br, acc[j][7]));
                        acc[j][8] = fmaf(tr, b2r, fmaf(-ti, b2i, acc[j][8]));
                        acc[j][9] = fmaf(tr, b2i, fmaf(ti, b2r, acc[j][9]));
                    }
                }
            }
        }
        // ---- release the stage; the last warp to do so refills it ----
        __syncwarp();
        if (lane == 0) {
            const unsigned prev = atomicAdd(&stage_cnt[st], 1u);
            if (prev == (unsigned)(W - 1)) {
                stage_cnt[st] = 0;
                const long long tn = t + (long long)NST * G;
                if (tn < T && !s_abort) {
                    fence_proxy_async();
                    const int s2 = tn < a.ntiles[0] ? 0 : 1;
                    const long long lt2 = s2 ? tn - a.ntiles[0] : tn;
                    issued[st] = i + NST;
                    tma_load_tile(stages + (size_t)st * a.stage_bytes,
                                  a.tiles[s2] + (size_t)lt2 * a.tile_bytes[s2], a.tile_bytes[s2], &mbar[st]);
                }
            }
        }
        if (++win == kWindow) {
            fold();
            win = 0;
        }
        if (++st == NST) {
            st = 0;
            ph ^= 1u;
        }
    };
    // the block's tiles are t = gb + i G, i = 0, 1, ...: data tiles first, then MC tiles
    long long t = gb, i = 0;
    for (const long long t_end = min((long long)a.ntiles[0], T); t < t_end; t += G, ++i)
        tile(std::integral_constant<int, 0>{}, t, i);
    fold();
    write_set(0);
    win = 0;
    for (; t < T; t += G, ++i) tile(std::integral_constant<int, 1>{}, t, i);
    __syncthreads();

    if (s_abort) {
        // A tile never arrived.  Report it, then wait (bounded) for the copies
        // still in flight so that none lands in a freed shared buffer.
        if (tid == 0) {
            atomicOr(a.err, ERR_TIMEOUT);
            for (int s = 0; s < NST; ++s) {
                const long long j = issued[s];
                if (j >= 0) (void)mbar_wait(&mbar[s], (uint32_t)((j / NST) & 1), a.timeout_cycles);
            }
        }
        __syncthreads();
        return;
    }

    fold();
    write_set(1);

    // ---- two-level last-block-done reduction (fixed order) ----
    __threadfence();  // every thread's record writes are visible device-wide ...
    __syncthreads();  // ... before thread 0 announces the block as done
    const int g = gb / a.group_size;                 // group of this block among the vector's blocks
    const int gi = bt * a.ngroups + g;               // its counter and record
    if (tid == 0) {
        const int members = min(a.group_size, a.Gb - g * a.group_size);
        const unsigned prev = atomicAdd(&a.group_count[gi], 1u);
        s_flag = prev == (unsigned)(members - 1);
    }
    __syncthreads();
    if (!s_flag) return;
    __threadfence();
    {
        const int b0 = bt * a.Gb + g * a.group_size, b1 = bt * a.Gb + min(a.Gb, (g + 1) * a.group_size);
        for (int i = tid; i < a.rec_len; i += NT) {
            double s = 0.0;
            for (int b = b0; b < b1; ++b) s += __ldcg(a.block_rec + (size_t)b * a.rec_len + i);
            a.group_rec[(size_t)gi * a.rec_len + i] = s;
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        a.group_count[gi] = 0;
        const unsigned prev = atomicAdd(&a.top_count[bt], 1u);
        s_flag = prev == (unsigned)(a.ngroups - 1);
    }
    __syncthreads();
    if (!s_flag) return;
    __threadfence();
    // the last group: totals into shared memory (reuse the stage area)
    double* tot = reinterpret_cast<double*>(stages);
    for (int i = tid; i < a.rec_len; i += NT) {
        double s = 0.0;
        for (int gg = 0; gg < a.ngroups; ++gg)
            s += __ldcg(a.group_rec + (size_t)(bt * a.ngroups + gg) * a.rec_len + i);
        tot[i] = s;
    }
    __syncthreads();
    if (tid == 0) a.top_count[bt] = 0;
    const int L = K * kNV + kNScal;
    if constexpr (MODE == MODE_HVP) {
        // keep this pass's totals and theta for the H v passes that reuse them
        if (a.cache && a.B == 1) {
            for (int i = tid; i < a.rec_len; i += NT) a.cache[i] = tot[i];
            for (int i = tid; i < a.P; i += NT) a.cache[a.rec_len + i] = theta[i];
        }
    }
    double Gdot = tot[L + K * kNV + 1];
    if constexpr (RU) {
        // the cached totals must belong to this theta
        if (tid == 0) s_flag = 0;
        __syncthreads();
        for (int i = tid; i < a.P; i += NT)
            if (theta[i] != a.cache[a.rec_len + i]) s_flag = 1;
        __syncthreads();
        if (s_flag) {
            if (tid == 0) atomicOr(a.err, ERR_STALE);
            for (int i = tid; i < 1 + 2 * a.P; i += NT) out[i] = __longlong_as_double(0x7ff8000000000000LL);
            return;
        }
        // cached Q sums (slots 0..5 of each resonance) and scalars; this pass's P sums (slots 6..9)
        for (int i = tid; i < a.rec_len; i += NT) {
            const int r = i % L;
            if (!(r < K * kNV && r % kNV >= 6)) tot[i] = a.cache[i];
        }
        __syncthreads();
        // Gdot = sum_mc Idot = (dG/dtheta) . v, dG/dtheta_j = 2 Re (kappa1_j Q1m + kappa2_j Q2m)
        double part = 0.0;
        for (int k = tid; k < K; k += NT) {
            const ResValues rv = res_values(a, theta, vdir, k, true);
            const ResParam rp = a.res[k];
            double sn, cs;
            sincos(rv.phi, &sn, &cs);
            const double* tm = tot + L + k * kNV;
            const double q1r = tm[0], q1i = tm[1], q2r = tm[2], q2i = tm[3];
            const double g1r = rv.rho * cs, g1i = rv.rho * sn;
            // kappa1: rho -> e^{i phi}, phi -> i g; kappa2: M -> g (-2M + i Gamma), Gamma -> g (i M)
            const double dg[4] = {2.0 * (cs * q1r - sn * q1i), 2.0 * (-g1i * q1r - g1r * q1i),
                                  2.0 * ((-2.0 * rv.M * g1r - rv.G * g1i) * q2r - (-2.0 * rv.M * g1i + rv.G * g1r) * q2i),
                                  2.0 * ((-rv.M * g1i) * q2r - (rv.M * g1r) * q2i)};
            const double vv[4] = {rv.vr, rv.vp, rv.vm, rv.vg};
            for (int j = 0; j < 4; ++j)
                if (rp.idx[j] >= 0) part += dg[j] * vv[j];
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) s_part[warp] = part;
        __syncthreads();
        Gdot = 0.0;
        for (int w = 0; w < NT / 32; ++w) Gdot += s_part[w];
    }

    // ---- combine (a-8, Eqs. 4, 6, 7) in FP64 ----
    const double SlnI = tot[K * kNV + 0];
    const double Gm = tot[L + K * kNV + 0];
    if (tid == 0) out[0] = -SlnI + a.Nd * log(Gm / a.Nmc);
    if constexpr (GR) {
        for (int k = tid; k < K; k += NT) {
            const ResValues rv = res_values(a, theta, vdir, k, HV);
            const ResParam rp = a.res[k];
            double sn, cs;
            sincos(rv.phi, &sn, &cs);
            const double2 E1 = make_double2(cs, sn);
            const double2 g1 = make_double2(rv.rho * cs, rv.rho * sn);
            const double2 a1 = make_double2(-2.0 * rv.M, rv.G), a2 = make_double2(0.0, rv.M);
            auto mul = [](double2 x, double2 y) { return make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x); };
            auto add = [](double2 x, double2 y) { return make_double2(x.x + y.x, x.y + y.y); };
            auto scl = [](double s, double2 x) { return make_double2(s * x.x, s * x.y); };
            auto ii = [](double2 x) { return make_double2(-x.y, x.x); };  // i x
            const double* td = tot + k * kNV;
            const double* tm = tot + L + k * kNV;
            const double2 Q1d = make_double2(td[0], td[1]), Q2d = make_double2(td[2], td[3]);
            const double2 Q1m = make_double2(tm[0], tm[1]), Q2m = make_double2(tm[2], tm[3]);
            // kappa_{j1}, kappa_{j2}: dc/dtheta_j = kappa1 B + kappa2 B^2
            const double2 zero = make_double2(0.0, 0.0);
            const double2 kap1[4] = {E1, ii(g1), zero, zero};
            const double2 kap2[4] = {zero, zero, mul(g1, a1), mul(g1, a2)};
            double2 lam1[4], lam2[4], lam3[4];
            if constexpr (HV) {
                const double2 al = add(scl(rv.vr, E1), scl(rv.vp, ii(g1)));
                const double2 u = add(scl(rv.vm, a1), scl(rv.vg, a2));
                const double2 be = mul(g1, u);
                lam1[0] = scl(rv.vp, ii(E1));
                lam2[0] = mul(E1, u);
                lam3[0] = zero;
                lam1[1] = add(scl(rv.vr, ii(E1)), scl(-rv.vp, g1));
                lam2[1] = ii(be);
                lam3[1] = zero;
                lam1[2] = zero;
                lam2[2] = add(mul(g1, make_double2(-2.0 * rv.vm, rv.vg)), mul(al, a1));
                lam3[2] = scl(2.0, mul(be, a1));
                lam1[3] = zero;
                lam2[3] = add(mul(g1, make_double2(0.0, rv.vm)), mul(al, a2));
                lam3[3] = scl(2.0, mul(be, a2));
            }
            for (int j = 0; j < 4; ++j) {
                const int idx = rp.idx[j];
                if (idx < 0) continue;
                const double gD = 2.0 * (mul(kap1[j], Q1d).x + mul(kap2[j], Q2d).x);
                const double gM = 2.0 * (mul(kap1[j], Q1m).x + mul(kap2[j], Q2m).x);
                out[1 + idx] = -gD + a.Nd * gM / Gm;
                if constexpr (HV) {
                    const double2 Q3d = make_double2(td[4], td[5]), P1d = make_double2(td[6], td[7]),
                                  P2d = make_double2(td[8], td[9]);
                    const double2 Q3m = make_double2(tm[4], tm[5]), P1m = make_double2(tm[6], tm[7]),
                                  P2m = make_double2(tm[8], tm[9]);
                    const double hD = 2.0 * (mul(kap1[j], P1d).x + mul(kap2[j], P2d).x + mul(lam1[j], Q1d).x +
                                             mul(lam2[j], Q2d).x + mul(lam3[j], Q3d).x);
                    const double hM = 2.0 * (mul(kap1[j], P1m).x + mul(kap2[j], P2m).x + mul(lam1[j], Q1m).x +
                                             mul(lam2[j], Q2m).x + mul(lam3[j], Q3m).x);
                    out[1 + a.P + idx] = -hD + a.Nd * (hM / Gm - gM * Gdot / (Gm * Gm));
                }
            }
        }
    }
}


// The mbarriers of pass_body in the block's shared memory (its layout for
// W warps and the arguments' K, NST and stage size).
__device__ __forceinline__ uint64_t* pass_mbarriers(unsigned char* smem, const PassArgs& a, int W)
{
    const KConst* kc = reinterpret_cast<const KConst*>(smem + (size_t)a.NST * a.stage_bytes);
    const float2* wacc = reinterpret_cast<const float2*>(kc + a.K);
    const unsigned* stage_cnt = reinterpret_cast<const unsigned*>(wacc + W * (a.K * kNV + 2));
    const long long* issued = reinterpret_cast<const long long*>(stage_cnt + 4);
    return const_cast<uint64_t*>(reinterpret_cast<const uint64_t*>(issued + 4));
}

template <int MODE, int S, int W, int KPW>
__global__ void __launch_bounds__(32 * W, 16 / W) pass_kernel(const PassArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if (a.skip && *a.skip) return;  // a device-side loop has already finished (uniform for the grid)
    // parameter vector bt of the batch; this block is block gb of the Gb that share the events
    pass_body<MODE, S, W, KPW>(a, (int)(blockIdx.x % (unsigned)a.B), (int)(blockIdx.x / (unsigned)a.B), smem);
}

}  // namespace pwa
