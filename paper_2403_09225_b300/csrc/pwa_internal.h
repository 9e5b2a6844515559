// pwa_internal.h -- handle layout shared by the libpwa translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "pwa.h"  // include/ is on the include path
#include "pass_kernel.cuh"

namespace pwa {

struct Tiling {
    int W = 4;        // warps per block (= lanes per event in the coherent-sum sweep)
    int H = 4;        // lanes per event, always W
    int NST = 2;      // tiles in flight per block
    int bps = 0;      // blocks per SM requested (0 = as many as fit)
    int E = kTileE;   // events per tile
    int KPW = 5;      // resonances owned by a warp in the second sweep
    int grid = 0;     // blocks launched
    int blocks_per_sm = 0;
    size_t smem = 0;  // dynamic shared memory per block
    uint32_t stage_bytes = 0;
};

// Rotation of resonance k's event positions inside a tile: with ev = 32/H
// events per warp, the H lanes of one event read different resonances; the
// rotation puts the rows those lanes read at the same step on different
// shared-memory banks.
__host__ __device__ inline int tile_shift(int k, int ev)
{
    return ev < 16 ? (k % (16 / ev)) * ev : 0;
}

}  // namespace pwa

namespace pwa {
// Scratch of batched evaluations (several parameter vectors in one launch),
// grown on demand: per vector Gb block records, ngroups group records and
// ngroups + 1 counters; device and pinned host buffers for the vectors and
// their results.
struct BatchState {
    int cap_B = 0;           // vectors the I/O buffers hold
    size_t cap_blocks = 0;   // block records the scratch holds
    size_t cap_groups = 0;   // group records (and group counters) it holds
    size_t cap_top = 0;      // per-vector top counters it holds
    double* d_block_rec = nullptr;
    double* d_group_rec = nullptr;
    unsigned* d_counts = nullptr;  // [cap_groups] group counters, [cap_top] top counters, [cap_top] error words
    int* d_err_vec = nullptr;      // per-vector error words (inside d_counts)
    double* d_io = nullptr;        // theta [cap_B][P] | v [cap_B][P] | out [cap_B][1 + 2P]
    double* h_io = nullptr;        // pinned, same layout, then 2 words for the error status
};
}  // namespace pwa

namespace pwa {
// Scratch of the Hessian pass: per-CTA FP64 records and their sum (device),
// the summed record on the host (pinned); sized for the kernel instance and
// grid it was set up for.
struct HessState {
    const void* fn = nullptr;  // kernel instance the geometry below belongs to
    size_t smem = 0;
    int resident = 0, rec_len = 0;  // CTAs resident on the GPU at once; FP64 record length
    size_t cap_bytes = 0, cap_host = 0;
    // device: [B Gb][rec_len] records | [B][rec_len] sums | theta [B][P] | error words [B]
    double* d_rec = nullptr;
    // pinned: [B][rec_len] sums | theta [B][P] | error words [B]
    double* h_buf = nullptr;
    int B = 0, NW = 0;  // the batch in flight (hessian_issue -> hessian_finish)
    bool tc = false;
};
}  // namespace pwa

struct pwa_handle {
    int K = 0, S = 0, P = 0;
    cudaStream_t stream = nullptr;
    long long n[2] = {0, 0};
    double Nd = 0.0, Nmc = 0.0;
    std::vector<pwa::ResParam> res;
    pwa::ResParam* d_res = nullptr;
    // device copies of the caller's events in the ABI layout (kept for re-tiling)
    float* d_F[2] = {nullptr, nullptr};
    float* d_m2[2] = {nullptr, nullptr};
    float* d_w = nullptr;
    // tiled layout streamed by the pass
    unsigned char* d_tiles[2] = {nullptr, nullptr};
    uint32_t tile_bytes[2] = {0, 0};
    int ntiles[2] = {0, 0};
    pwa::Tiling tiling;
    int num_sms = 0;
    // reduction scratch and results
    double* d_block_rec = nullptr;
    double* d_group_rec = nullptr;
    unsigned* d_counts = nullptr;  // [ngroups] group counters, then the top counter
    int group_size = 16, ngroups = 0, rec_len = 0;
    double* d_theta = nullptr;
    double* d_v = nullptr;
    double* d_out = nullptr;        // [1 + 2P]
    unsigned long long* d_bad = nullptr;
    int* d_err = nullptr;
    double* h_pin = nullptr;        // pinned staging: theta[P], v[P], out[1 + 2P], status
    double* d_cache = nullptr;      // [rec_len] totals + [P] theta of the last full HVP pass
    pwa::BatchState batch;
    pwa::HessState hess;
    long long timeout_cycles = 0;
    bool broken = false;
    bool released = false;  // d_F, d_m2, d_w freed (pwa_release_event_copies)
    bool hess_cuda_cores = false;  // the Hessian pass's Gram matrices on the CUDA cores even for K <= 32
    std::string err;
};

namespace pwa {

using KernelFn = void (*)(const PassArgs);
// compiled instances of the fused pass for (warps per block, resonances per
// warp), one function per mode and S (generated by build.py)
#define PWA_DECLARE_PICK(mode)                 \
    KernelFn pick_pass_##mode##_s1(int W, int kpw); \
    KernelFn pick_pass_##mode##_s2(int W, int kpw); \
    KernelFn pick_pass_##mode##_s3(int W, int kpw); \
    KernelFn pick_pass_##mode##_s4(int W, int kpw);
PWA_DECLARE_PICK(nll)
PWA_DECLARE_PICK(grad)
PWA_DECLARE_PICK(hvp)
PWA_DECLARE_PICK(hvpr)
#undef PWA_DECLARE_PICK

// Enqueue one fused pass on device buffers (theta, v: device [P]; out: device [1+2P]).
// skip: optional device flag; the pass does nothing when it is non-zero at launch.
pwa_status launch_pass(pwa_handle* h, const double* d_theta, const double* d_v, double* d_out, int mode,
                       const int* skip = nullptr);
// The arguments of one single-vector pass on the handle's own scratch, and the
// launch of a pass with given arguments (after the tile-geometry checks every
// launch runs); launch_pass is the two in a row.
PassArgs pass_args(pwa_handle* h, const double* d_theta, const double* d_v, double* d_out);
pwa_status launch_pass_args(pwa_handle* h, const PassArgs& a, int mode);
// Enqueue one fused pass for B parameter vectors (theta, v: device [B][P]; out:
// device [B][1 + 2P]); grows the batch scratch when needed.
// err_vec: clear and fill the per-vector error words h->batch.d_err_vec [B].
pwa_status launch_batch(pwa_handle* h, int B, const double* d_theta, const double* d_v, double* d_out, int mode,
                        bool err_vec = false);
// The arguments of a batched pass of B vectors on h without launching it:
// grows the handle's batch scratch (memsets on `stream`; when the scratch
// grows, the handle's stream and `stream` are synchronised first).
pwa_status prepare_batch(pwa_handle* h, int B, const double* d_theta, const double* d_v, double* d_out,
                         bool err_vec, cudaStream_t stream, PassArgs& a);
// Arguments of a launch over several handles: device copies and their pinned
// staging (the staging must not change until the launch's copies are done --
// a captured graph replays the copies from it).
struct MultiScratch {
    int cap = 0;
    PassArgs* d_args = nullptr;
    int* d_first = nullptr;
    unsigned char* h_stage = nullptr;
    MultiScratch() = default;
    MultiScratch(const MultiScratch&) = delete;
    MultiScratch& operator=(const MultiScratch&) = delete;
    ~MultiScratch();
};
// One batched pass (mode GRAD or HVP) over several handles in one launch on
// `stream` (multi.cu): handle i evaluates B[i] vectors d_theta[i] -> d_out[i].
// Every handle needs K <= 32.  No synchronisation: the caller keeps ms's
// staging unchanged until the launch's argument copies are done.
pwa_status launch_multi(int n, pwa_handle* const* hs, const int* B, const double* const* d_theta,
                        const double* const* d_v, double* const* d_out, int mode, bool err_vec, cudaStream_t stream,
                        MultiScratch& ms);
// Size ms for n handles (allocates; call outside a stream capture).
pwa_status launch_multi_reserve(pwa_handle* h0, int n, MultiScratch& ms);
constexpr int kMaxKMulti = 32;
// Shared memory per block of a pass instance with W warps over the handle's tiles.
size_t pass_smem_bytes(const pwa_handle* h, int W);
// Device I/O buffers of the batch state for B vectors (grown when needed).
pwa_status batch_io(pwa_handle* h, int B);
void free_batch(pwa_handle* h);
// Coupling sub-problem rows for the lockstep fits: theta, v [nb][Pc] (v may be
// null) -> out [nb][1 + 2Pc] (f, g, Hv) and per-row non-finite flags; synchronous.
pwa_status coupling_eval_rows(pwa_coupling* cp, int nb, const double* theta, const double* v, double* out,
                              int* errw);
pwa_handle* coupling_handle(const pwa_coupling* cp);
// Physics-variant likelihood: one synchronous evaluation at host theta (dir may
// be null; grad and hv may be null) and the embedded handle that carries the
// stream and the error text.
pwa_status variant_eval(pwa_variant* v, const double* theta, const double* dir, double* nll, double* grad,
                        double* hv);
// B evaluations in one launch (theta, dir [B][P]); status [B] per vector
pwa_status variant_eval_batch(pwa_variant* v, int B, const double* theta, const double* dir, double* nll,
                              double* grad, double* hv, pwa_status* status);
pwa_handle* variant_base(pwa_variant* v);
// The same with the couplings only, at the line shapes of the last pwa_variant_set_shapes.
pwa_status variant_coupling_eval(pwa_variant* v, const double* theta_c, const double* dir_c, double* nll,
                                 double* grad, double* hv);
// Largest K the Hessian pass serves (its Gram blocks fit the threads of a CTA).
constexpr int kMaxKHessian = 44;
// The full Hessian of NLL at host theta (plus NLL and gradient; either may be
// null) from one Hessian pass; synchronous.  hess: host [P][P].
pwa_status hessian_device(pwa_handle* h, const double* theta, double* nll, double* grad, double* hess);
pwa_status hessian_issue(pwa_handle* h, int B, const double* theta);
pwa_status hessian_finish(pwa_handle* h, int B, const double* theta, double* nll, double* grad, double* hess,
                          pwa_status* status);
void free_hessian(pwa_handle* h);
// Read back and clear the device error flags; turns them into a status + message.
pwa_status check_device_errors(pwa_handle* h);
pwa_status set_error(pwa_handle* h, pwa_status st, const std::string& msg);
pwa_status cuda_error(pwa_handle* h, cudaError_t e, const char* what);

}  // namespace pwa
