// fit.cu -- pwa_newton_cg_fit: truncated-Newton minimisation of the NLL.
//
// The paper fits with scipy's Newton-CG (Sec. 3), i.e. the line-search
// Newton-CG of Nocedal & Wright, Numerical Optimization, Algorithm 7.1, with
// a line search for the strong Wolfe conditions (their Algorithms 3.5/3.6).
// This is an independent C++ restatement of those textbook steps driving the
// fused GPU pass: every gradient is one pass over F, every inner CG step is
// one Hessian-vector pass.  The inner CG runs on the device (FP64 vectors and
// scalars: dot products, curvature, step lengths), replayed as a CUDA graph
// in batches of iterations; the outer loop and the line search run on the host.
//
// Differences from the textbook statement, all because the NLL is summed
// from FP32 per-event terms (its value carries rounding noise far above
// FP64 resolution, while its gradient stays accurate near the minimum):
//  * the sufficient-decrease test allows an increase up to eps_f = 1e-7 |f|
//    (the "approximate Wolfe" idea of Hager & Zhang, 2005);
//  * a failed line search whose predicted decrease |g.p| is below
//    1e-7 (1 + |f|) ends the fit as converged at the precision limit;
//  * so do 25 outer iterations in which neither the gradient norm improved
//    by 1 % nor the NLL dropped by more than ten times its resolution (the
//    noise floor of the FP32 sums).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <coroutine>
#include <exception>
#include <memory>
#include <cstring>
#include <limits>
#include <vector>

#include "pwa_internal.h"

namespace {

// ---------------------------------------------------------------------------
// inner CG on the device: every iteration is one fused HVP pass plus one
// single-block FP64 update; batches of iterations are replayed as a CUDA
// graph and only the termination word returns to the host
// ---------------------------------------------------------------------------

constexpr int kCgThreads = 256;
constexpr int kCgBatch = 8;  // CG iterations per graph launch

struct DevCG {
    double* x;      // [P] point of the Newton step
    double* g;      // [P] gradient at x
    double* z;      // [P] CG iterate (the step on exit)
    double* r;      // [P] residual
    double* d;      // [P] search direction
    double* out;    // [1 + 2P] pass output; H d at out + 1 + P
    double* scal;   // rr, eps
    int* flags;     // done (0 running, 1 negative curvature, 2 converged, 3 iteration limit), j, passes
};

// fixed-order block sum of one FP64 value per thread
__device__ double block_sum(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = kCgThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double s = sh[0];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(kCgThreads) cg_init_kernel(DevCG c, int P, double eps)
{
    __shared__ double sh[kCgThreads];
    double rr = 0.0;
    for (int i = threadIdx.x; i < P; i += kCgThreads) {
        const double gi = c.g[i];
        c.z[i] = 0.0;
        c.r[i] = gi;
        c.d[i] = -gi;
        rr += gi * gi;
    }
    rr = block_sum(rr, sh);
    if (threadIdx.x == 0) {
        c.scal[0] = rr;
        c.scal[1] = eps;
        c.flags[0] = 0;
        c.flags[1] = 0;
        c.flags[2] = 0;
    }
}

// one CG iteration (N&W Algorithm 7.1, inner loop) after H d is in c.out
__global__ void __launch_bounds__(kCgThreads) cg_step_kernel(DevCG c, int P, int maxiter)
{
    __shared__ double sh[kCgThreads];
    __shared__ int s_done;
    if (threadIdx.x == 0) s_done = c.flags[0];
    __syncthreads();
    if (s_done) return;
    const double* Bd = c.out + 1 + P;
    double curv = 0.0;
    for (int i = threadIdx.x; i < P; i += kCgThreads) curv += c.d[i] * Bd[i];
    curv = block_sum(curv, sh);
    const int j = c.flags[1];
    if (threadIdx.x == 0) c.flags[2] += 1;
    if (!(curv > 0.0)) {
        // negative curvature: steepest descent on the first iteration, else the current iterate
        if (j == 0)
            for (int i = threadIdx.x; i < P; i += kCgThreads) c.z[i] = -c.g[i];
        if (threadIdx.x == 0) c.flags[0] = 1;
        return;
    }
    const double rr = c.scal[0];
    const double alpha = rr / curv;
    double rr_new = 0.0;
    for (int i = threadIdx.x; i < P; i += kCgThreads) {
        c.z[i] += alpha * c.d[i];
        const double ri = c.r[i] + alpha * Bd[i];
        c.r[i] = ri;
        rr_new += ri * ri;
    }
    rr_new = block_sum(rr_new, sh);
    if (sqrt(rr_new) < c.scal[1]) {
        if (threadIdx.x == 0) {
            c.flags[0] = 2;
            c.flags[1] = j + 1;
            c.scal[0] = rr_new;
        }
        return;
    }
    if (j + 1 >= maxiter) {
        if (threadIdx.x == 0) {
            c.flags[0] = 3;
            c.flags[1] = j + 1;
            c.scal[0] = rr_new;
        }
        return;
    }
    const double beta = rr_new / rr;
    for (int i = threadIdx.x; i < P; i += kCgThreads) c.d[i] = -c.r[i] + beta * c.d[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        c.scal[0] = rr_new;
        c.flags[1] = j + 1;
    }
}

struct DeviceCG {
    pwa_handle* h = nullptr;
    int P = 0;
    double* block = nullptr;
    DevCG c{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;

    pwa_status init(pwa_handle* hh)
    {
        h = hh;
        P = h->P;
        const size_t n = 5 * (size_t)P + (1 + 2 * (size_t)P) + 2 + 2;
        if (cudaMalloc(&block, n * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return pwa::set_error(h, PWA_ENOMEM, "cudaMalloc failed for the CG state");
        }
        c.x = block;
        c.g = c.x + P;
        c.z = c.g + P;
        c.r = c.z + P;
        c.d = c.r + P;
        c.out = c.d + P;
        c.scal = c.out + 1 + 2 * P;
        c.flags = reinterpret_cast<int*>(c.scal + 2);
        return PWA_OK;
    }

    // capture kCgBatch iterations (H v pass at x along d, reusing the sums of
    // the solve's first, full pass at x; then the update) once
    pwa_status capture(int maxiter)
    {
        cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "cudaStreamBeginCapture");
        pwa_status st = PWA_OK;
        for (int b = 0; b < kCgBatch && st == PWA_OK; ++b) {
            st = pwa::launch_pass(h, c.x, c.d, c.out, pwa::MODE_HVP_REUSE, c.flags);
            if (st == PWA_OK) {
                cg_step_kernel<<<1, kCgThreads, 0, h->stream>>>(c, P, maxiter);
                e = cudaGetLastError();
                if (e != cudaSuccess) st = pwa::cuda_error(h, e, "cg_step launch");
            }
        }
        e = cudaStreamEndCapture(h->stream, &graph);
        if (st != PWA_OK) return st;
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "cudaGraphInstantiate");
        return PWA_OK;
    }

    // p = approximate solution of H p = -g at x (inner loop of Algorithm 7.1)
    pwa_status solve(const std::vector<double>& x, const std::vector<double>& g, double eps, int maxiter,
                     std::vector<double>& p, int& n_hvp, pwa_fit_iter* rec)
    {
        if (!exec) {
            pwa_status st = capture(maxiter);
            if (st != PWA_OK) return st;
        }
        double* pin = h->h_pin;  // 4P + 8 doubles of pinned staging
        std::memcpy(pin, x.data(), sizeof(double) * P);
        std::memcpy(pin + P, g.data(), sizeof(double) * P);
        cudaError_t e = cudaMemcpyAsync(c.x, pin, sizeof(double) * 2 * P, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "CG upload");
        cg_init_kernel<<<1, kCgThreads, 0, h->stream>>>(c, P, eps);
        e = cudaGetLastError();
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "cg_init launch");
        // the first iteration's product with the full pass, which keeps the sums at x for the others
        pwa_status st0 = pwa::launch_pass(h, c.x, c.d, c.out, pwa::MODE_HVP, c.flags);
        if (st0 != PWA_OK) return st0;
        cg_step_kernel<<<1, kCgThreads, 0, h->stream>>>(c, P, maxiter);
        e = cudaGetLastError();
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "cg_step launch");
        int flags[3] = {0, 0, 0};
        for (int done_batches = 0;; ++done_batches) {
            e = cudaGraphLaunch(exec, h->stream);
            if (e != cudaSuccess) return pwa::cuda_error(h, e, "cudaGraphLaunch");
            e = cudaMemcpyAsync(pin + 2 * P, c.flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return pwa::cuda_error(h, e, "CG flags");
            std::memcpy(flags, pin + 2 * P, sizeof(int) * 3);
            if (flags[0]) break;
            if ((done_batches + 1) * kCgBatch > maxiter + kCgBatch) break;  // guard; the step sets flag 3 first
        }
        n_hvp += flags[2];
        e = cudaMemcpyAsync(pin, c.z, sizeof(double) * P, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(pin + P, c.scal, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "CG download");
        p.assign(pin, pin + P);
        if (rec) {
            rec->cg_iters = flags[2];
            rec->cg_exit = flags[0];
            rec->cg_res = std::sqrt(pin[P]);
        }
        return pwa::check_device_errors(h);
    }

    ~DeviceCG()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (block) cudaFree(block);
        cudaGetLastError();
    }
};

double dot(const std::vector<double>& a, const std::vector<double>& b)
{
    double s = 0.0;
    for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
    return s;
}

// y = H x for the explicit Hessian H [n][n] (host FP64).  Four partial sums
// per row in a fixed order: independent chains the compiler can vectorise,
// instead of one dependent chain of n additions.
void hess_times(const double* H, int n, const double* x, double* y)
{
    for (int i = 0; i < n; ++i) {
        const double* Hi = H + (size_t)i * n;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int l = 0;
        for (; l + 4 <= n; l += 4) {
            a0 += Hi[l] * x[l];
            a1 += Hi[l + 1] * x[l + 1];
            a2 += Hi[l + 2] * x[l + 2];
            a3 += Hi[l + 3] * x[l + 3];
        }
        for (; l < n; ++l) a0 += Hi[l] * x[l];
        y[i] = (a0 + a1) + (a2 + a3);
    }
}

struct LinePoint {
    double a = 0.0, f = 0.0, df = 0.0;
    std::vector<double> x, g;
};

// minimiser of the cubic through (a, fa, dfa), (b, fb, dfb)
bool cubic_min(double a, double fa, double dfa, double b, double fb, double dfb, double& out)
{
    const double d1 = dfa + dfb - 3.0 * (fa - fb) / (a - b);
    const double disc = d1 * d1 - dfa * dfb;
    if (disc < 0) return false;
    const double d2 = std::copysign(std::sqrt(disc), b - a);
    const double den = dfb - dfa + 2.0 * d2;
    if (den == 0) return false;
    out = b - (b - a) * (dfb + d2 - d1) / den;
    return std::isfinite(out);
}

// ---------------------------------------------------------------------------
// The Newton-CG iteration as a coroutine.  It suspends whenever it needs the
// likelihood -- f and g at a point (FG), H v at a point (HV), or a whole inner
// CG solve (CG) -- and an executor serves the request and resumes it: one fit
// at a time with the device-side CG (pwa_newton_cg_fit), or many fits whose
// FG / HV requests share one batched launch (pwa_newton_cg_fit_batch).  The
// arithmetic of the iteration is written once, here.
// ---------------------------------------------------------------------------

enum class Req { None, FG, HV, CG, HESS };

struct FitState {
    int P = 0;
    pwa_fit_opts o{};
    int maxiter = 0, cg_maxiter = 0;
    bool device_cg = false;  // CG requests (device graph) instead of HV requests
    bool explicit_h = false; // one HESS request per outer iteration, the CG on its products
    std::vector<double> H;   // [P][P] Hessian at x (explicit_h)
    std::chrono::steady_clock::time_point t_start;
    std::vector<double> x, g, p;
    double f = 0.0;
    // the request posted at the last suspension, and its outcome
    Req req = Req::None;
    const double* rx = nullptr;  // FG, HV: the point
    const double* rv = nullptr;  // HV: the direction
    double* rf = nullptr;        // FG: f
    double* rg = nullptr;        // FG: g
    double* rhv = nullptr;       // HV: H v
    double* rH = nullptr;        // HESS: the Hessian [P][P] at rx
    double cg_eps = 0.0;         // CG: solve H p = -g at (x, g) to |r| < cg_eps into p
    pwa_status req_status = PWA_OK;
    // noise floor: the best |g| so far, the NLL and the outer iteration of
    // the last real progress (|g| 1 % below its best, or the NLL lower by
    // more than ten times its resolution)
    double g_best = INFINITY, f_mark = INFINITY;
    int k_best = 0;
    // per-iteration records (opts.trace); cur_it is the one being filled
    std::vector<pwa_fit_iter> trace;
    pwa_fit_iter cur_it{};
    // outcome of the fit
    pwa_status error = PWA_OK;  // an evaluation failed (the fit stopped there)
    int status = PWA_FIT_MAXITER, iters = 0, n_fev = 0, n_hvp = 0, n_hess = 0;
    double elapsed = 0.0;

    double since_start() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    }
};

struct FitTask {
    struct promise_type {
        FitTask get_return_object() { return FitTask{std::coroutine_handle<promise_type>::from_promise(*this)}; }
        std::suspend_always initial_suspend() noexcept { return {}; }
        std::suspend_always final_suspend() noexcept { return {}; }
        void return_void() {}
        // a host exception (e.g. bad_alloc) ends the coroutine; the executor reports it
        void unhandled_exception() { failed = true; }
        bool failed = false;
    };
    std::coroutine_handle<promise_type> h;
    bool failed() const { return h.promise().failed; }
    explicit FitTask(std::coroutine_handle<promise_type> hh) : h(hh) {}
    FitTask(FitTask&& o) noexcept : h(o.h) { o.h = nullptr; }
    FitTask(const FitTask&) = delete;
    ~FitTask()
    {
        if (h) h.destroy();
    }
};

// suspension point: the request is already stored in the FitState
struct Suspend {
    bool await_ready() const noexcept { return false; }
    void await_suspend(std::coroutine_handle<>) const noexcept {}
    void await_resume() const noexcept {}
};

// the record of the current iteration goes to the trace when it ends
void push_iter(FitState& s)
{
    if ((int)s.trace.size() < s.o.trace_cap) s.trace.push_back(s.cur_it);
}

// Stagnation at the FP32 noise floor: for kStall outer iterations neither has
// |g| improved by 1 % over its best nor has the NLL dropped by more than ten
// times its resolution.  Near the minimum the gradient of the FP32-summed
// NLL is dominated by rounding and the steps wander at that level without
// ever meeting xtol; the fit has then converged as far as the evaluation
// resolves.  (A long descent keeps lowering the NLL and is not cut short.)
constexpr int kStall = 25;
bool stalled(FitState& s, int k)
{
    const double gn = std::sqrt(dot(s.g, s.g));
    const double resolution = 1e-7 * (1.0 + std::fabs(s.f));
    if (gn < 0.99 * s.g_best || s.f < s.f_mark - 10.0 * resolution) {
        s.g_best = std::min(s.g_best, gn);
        s.f_mark = s.f;
        s.k_best = k;
        return false;
    }
    return k - s.k_best > kStall;
}

FitTask newton_cg(FitState& s)
{
    const int n = s.P;
    const double c1 = 1e-4, c2 = 0.9;
    s.req = Req::FG;
    s.rx = s.x.data();
    s.rf = &s.f;
    s.rg = s.g.data();
    co_await Suspend{};
    if (s.req_status != PWA_OK) {
        s.error = s.req_status;
        co_return;
    }
    s.p.assign(n, 0.0);
    std::vector<double> z, r, d, Hd;
    int k = 0;
    while (k < s.maxiter) {
        double gmax = 0.0;
        for (double v : s.g) gmax = std::max(gmax, std::fabs(v));
        if (s.o.gtol > 0 && gmax <= s.o.gtol) {
            s.status = PWA_FIT_GTOL;
            break;
        }
        // ---- inner CG on H p = -g (N&W Algorithm 7.1) ----
        const double gnorm = std::sqrt(dot(s.g, s.g));
        const double eps = std::min(0.5, std::sqrt(gnorm)) * gnorm;
        s.cur_it = pwa_fit_iter();
        s.cur_it.nll = s.f;
        s.cur_it.grad_max = gmax;
        s.cur_it.cg_eps = eps;
        if (s.explicit_h) {
            // one Hessian pass at x; every CG product below is a product with it
            s.H.resize((size_t)n * n);
            s.req = Req::HESS;
            s.rx = s.x.data();
            s.rH = s.H.data();
            co_await Suspend{};
            if (s.req_status != PWA_OK) {
                s.error = s.req_status;
                co_return;
            }
            s.cur_it.hessian = 1;
        }
        if (s.device_cg && !s.explicit_h) {
            s.req = Req::CG;
            s.cg_eps = eps;
            co_await Suspend{};
            if (s.req_status != PWA_OK) {
                s.error = s.req_status;
                co_return;
            }
        } else {
            z.assign(n, 0.0);
            r = s.g;
            d.resize(n);
            Hd.resize(n);
            for (int i = 0; i < n; ++i) d[i] = -r[i];
            double rr = dot(r, r);
            for (int j = 0;; ++j) {
                if (s.explicit_h) {
                    hess_times(s.H.data(), n, d.data(), Hd.data());
                } else {
                    s.req = Req::HV;
                    s.rx = s.x.data();
                    s.rv = d.data();
                    s.rhv = Hd.data();
                    co_await Suspend{};
                    if (s.req_status != PWA_OK) {
                        s.error = s.req_status;
                        co_return;
                    }
                    ++s.n_hvp;
                }
                s.cur_it.cg_iters = j + 1;
                const double curv = dot(d, Hd);
                if (!(curv > 0.0)) {  // negative curvature: steepest descent first, else the iterate
                    if (j == 0)
                        for (int i = 0; i < n; ++i) s.p[i] = -s.g[i];
                    else
                        s.p = z;
                    s.cur_it.cg_exit = 1;
                    s.cur_it.cg_res = std::sqrt(rr);
                    break;
                }
                const double alpha = rr / curv;
                double rr_new = 0.0;
                for (int i = 0; i < n; ++i) {
                    z[i] += alpha * d[i];
                    r[i] += alpha * Hd[i];
                    rr_new += r[i] * r[i];
                }
                if (std::sqrt(rr_new) < eps || j + 1 >= s.cg_maxiter) {
                    s.p = z;
                    s.cur_it.cg_exit = std::sqrt(rr_new) < eps ? 2 : 3;
                    s.cur_it.cg_res = std::sqrt(rr_new);
                    break;
                }
                const double beta = rr_new / rr;
                for (int i = 0; i < n; ++i) d[i] = -r[i] + beta * d[i];
                rr = rr_new;
            }
        }
        ++k;
        double pmean = 0.0;
        for (double v : s.p) pmean += std::fabs(v);
        pmean /= std::max(n, 1);
        if (pmean <= s.o.xtol) {
            s.status = PWA_FIT_XTOL;
            push_iter(s);
            break;
        }
        double df0 = dot(s.g, s.p);
        if (!(df0 < 0)) {
            for (int i = 0; i < n; ++i) s.p[i] = -s.g[i];
            df0 = dot(s.g, s.p);
        }
        s.cur_it.dir_deriv = df0;
        // ---- strong-Wolfe line search (N&W Algorithms 3.5 / 3.6) ----
        // bracketing from a = 1 (doubling), then zoom with safeguarded cubic
        // interpolation; one trial point per suspension
        const double f0 = s.f;
        const double eps_f = 1e-7 * std::fabs(f0);
        auto armijo_fails = [&](const LinePoint& lp) { return !(lp.f <= f0 + c1 * lp.a * df0 + eps_f); };
        LinePoint prev, cur, lo, hi, found;
        prev.a = 0.0;
        prev.f = f0;
        prev.df = df0;
        prev.x = s.x;
        prev.g = s.g;
        bool ok = false, zooming = false;
        int bracket_it = 0, zoom_it = 0;
        double a = 1.0;
        while (true) {
            if (zooming) {
                if (zoom_it >= 30) break;
                const double left = std::min(lo.a, hi.a), right = std::max(lo.a, hi.a), width = right - left;
                if (!std::isfinite(hi.f) || !cubic_min(lo.a, lo.f, lo.df, hi.a, hi.f, hi.df, a) ||
                    a < left + 0.1 * width || a > right - 0.1 * width)
                    a = 0.5 * (lo.a + hi.a);
            } else if (bracket_it >= 30) {
                break;
            }
            // trial point x + a p
            cur.a = a;
            cur.x.resize(n);
            cur.g.resize(n);
            for (int i = 0; i < n; ++i) cur.x[i] = s.x[i] + a * s.p[i];
            s.req = Req::FG;
            s.rx = cur.x.data();
            s.rf = &cur.f;
            s.rg = cur.g.data();
            co_await Suspend{};
            if (s.req_status == PWA_ENONFINITE) {  // the trial point left the region where I > 0
                cur.f = INFINITY;
                cur.df = 0.0;
            } else if (s.req_status != PWA_OK) {
                s.error = s.req_status;
                co_return;
            } else {
                cur.df = dot(cur.g, s.p);
            }
            if (!zooming) {
                const int it = bracket_it++;
                if (!std::isfinite(cur.f)) {
                    a = 0.5 * (prev.a + a);
                    continue;
                }
                if (armijo_fails(cur) || (it > 0 && cur.f >= prev.f + eps_f)) {
                    zooming = true;
                    lo = prev;
                    hi = cur;
                    continue;
                }
                if (std::fabs(cur.df) <= -c2 * df0) {
                    found = cur;
                    ok = true;
                    break;
                }
                if (cur.df >= 0) {
                    zooming = true;
                    lo = cur;
                    hi = prev;
                    continue;
                }
                prev = cur;
                a = std::min(2.0 * a, 1e3);
            } else {
                ++zoom_it;
                if (armijo_fails(cur) || cur.f >= lo.f + eps_f) {
                    hi = cur;
                } else {
                    if (std::fabs(cur.df) <= -c2 * df0) {
                        found = cur;
                        ok = true;
                        break;
                    }
                    if (cur.df * (hi.a - lo.a) >= 0) hi = lo;
                    lo = cur;
                }
                if (std::fabs(hi.a - lo.a) < 1e-14 * std::max(1.0, std::fabs(lo.a))) break;
            }
        }
        s.cur_it.n_fev = bracket_it + zoom_it;
        if (!ok) {
            s.status = std::fabs(df0) <= 1e-7 * (1.0 + std::fabs(f0)) ? PWA_FIT_PRECISION : PWA_FIT_LINESEARCH;
            push_iter(s);
            break;
        }
        s.cur_it.step = found.a;
        push_iter(s);
        double smean = 0.0;
        for (int i = 0; i < n; ++i) smean += std::fabs(found.x[i] - s.x[i]);
        smean /= std::max(n, 1);
        s.x = found.x;
        s.f = found.f;
        s.g = found.g;
        if (smean <= s.o.xtol) {
            s.status = PWA_FIT_XTOL;
            break;
        }
        if (stalled(s, k)) {
            s.status = PWA_FIT_PRECISION;
            break;
        }
        if (s.o.time_limit_s > 0 && s.since_start() > s.o.time_limit_s) {
            s.status = PWA_FIT_TIME_LIMIT;
            break;
        }
    }
    s.iters = k;
}

// ---------------------------------------------------------------------------
// Trust-region Newton-CG (Nocedal & Wright Algorithm 7.2, CG-Steihaug, inside
// the trust-region iteration of their Algorithm 4.1): the inner CG stops at
// the trust-region boundary instead of giving up on negative curvature, and
// no line search is needed -- one f, g evaluation per outer iteration.  The
// acceptance ratio rho = actual / predicted reduction is taken from f where
// the predicted reduction is above the NLL's FP32 resolution; below it a step
// is taken when the NLL does not rise beyond that resolution and the
// gradient along the step meets the line search's curvature test, and a
// rejected step whose predicted decrease g.p is below the resolution ends the
// fit at the precision limit -- the same concern that gives the line search
// its approximate Wolfe test.
// ---------------------------------------------------------------------------

// tau >= 0 with |z + tau d| = delta
double to_boundary(const std::vector<double>& z, const std::vector<double>& d, double delta)
{
    const double dd = dot(d, d), zd = dot(z, d), zz = dot(z, z);
    const double disc = std::max(0.0, zd * zd - dd * (zz - delta * delta));
    return dd > 0 ? (-zd + std::sqrt(disc)) / dd : 0.0;
}

FitTask newton_cg_tr(FitState& s)
{
    const int n = s.P;
    const double eta = 0.15, delta_max = 1e3;
    s.req = Req::FG;
    s.rx = s.x.data();
    s.rf = &s.f;
    s.rg = s.g.data();
    co_await Suspend{};
    if (s.req_status != PWA_OK) {
        s.error = s.req_status;
        co_return;
    }
    std::vector<double> z(n), r(n), d(n), Hd(n), Hz(n), xn(n), gn(n), p(n);
    double delta = 1.0;
    int k = 0;
    while (k < s.maxiter) {
        double gmax = 0.0;
        for (double v : s.g) gmax = std::max(gmax, std::fabs(v));
        if (s.o.gtol > 0 && gmax <= s.o.gtol) {
            s.status = PWA_FIT_GTOL;
            break;
        }
        const double gnorm = std::sqrt(dot(s.g, s.g));
        const double eps = std::min(0.5, std::sqrt(gnorm)) * gnorm;
        s.cur_it = pwa_fit_iter();
        s.cur_it.nll = s.f;
        s.cur_it.grad_max = gmax;
        s.cur_it.cg_eps = eps;
        if (s.explicit_h) {
            s.H.resize((size_t)n * n);
            s.req = Req::HESS;
            s.rx = s.x.data();
            s.rH = s.H.data();
            co_await Suspend{};
            if (s.req_status != PWA_OK) {
                s.error = s.req_status;
                co_return;
            }
            s.cur_it.hessian = 1;
        }
        // ---- CG-Steihaug on the model m(p) = g.p + p.H.p / 2 within |p| <= delta ----
        std::fill(z.begin(), z.end(), 0.0);
        std::fill(Hz.begin(), Hz.end(), 0.0);  // H z, kept for the model value
        r = s.g;
        for (int i = 0; i < n; ++i) d[i] = -r[i];
        double rr = dot(r, r);
        for (int j = 0;; ++j) {
            if (s.explicit_h) {
                hess_times(s.H.data(), n, d.data(), Hd.data());
            } else {
                s.req = Req::HV;
                s.rx = s.x.data();
                s.rv = d.data();
                s.rhv = Hd.data();
                co_await Suspend{};
                if (s.req_status != PWA_OK) {
                    s.error = s.req_status;
                    co_return;
                }
                ++s.n_hvp;
            }
            s.cur_it.cg_iters = j + 1;
            const double curv = dot(d, Hd);
            if (!(curv > 0.0)) {  // negative curvature: follow d to the boundary
                const double tau = to_boundary(z, d, delta);
                for (int i = 0; i < n; ++i) {
                    z[i] += tau * d[i];
                    Hz[i] += tau * Hd[i];
                }
                s.cur_it.cg_exit = 1;
                s.cur_it.cg_res = std::sqrt(rr);
                break;
            }
            const double alpha = rr / curv;
            double zz = 0.0;
            for (int i = 0; i < n; ++i) zz += (z[i] + alpha * d[i]) * (z[i] + alpha * d[i]);
            if (std::sqrt(zz) >= delta) {  // the step leaves the region: stop on its boundary
                const double tau = to_boundary(z, d, delta);
                for (int i = 0; i < n; ++i) {
                    z[i] += tau * d[i];
                    Hz[i] += tau * Hd[i];
                }
                s.cur_it.cg_exit = 4;
                s.cur_it.cg_res = std::sqrt(rr);
                break;
            }
            double rr_new = 0.0;
            for (int i = 0; i < n; ++i) {
                z[i] += alpha * d[i];
                Hz[i] += alpha * Hd[i];
                r[i] += alpha * Hd[i];
                rr_new += r[i] * r[i];
            }
            if (std::sqrt(rr_new) < eps || j + 1 >= s.cg_maxiter) {
                s.cur_it.cg_exit = std::sqrt(rr_new) < eps ? 2 : 3;
                s.cur_it.cg_res = std::sqrt(rr_new);
                break;
            }
            const double beta = rr_new / rr;
            for (int i = 0; i < n; ++i) d[i] = -r[i] + beta * d[i];
            rr = rr_new;
        }
        p = z;
        ++k;
        const double pred = -(dot(s.g, p) + 0.5 * dot(p, Hz));  // predicted reduction
        const double pnorm = std::sqrt(dot(p, p));
        s.cur_it.dir_deriv = dot(s.g, p);
        // ---- trial point ----
        for (int i = 0; i < n; ++i) xn[i] = s.x[i] + p[i];
        double fn = 0.0;
        s.req = Req::FG;
        s.rx = xn.data();
        s.rf = &fn;
        s.rg = gn.data();
        co_await Suspend{};
        bool finite = true;
        if (s.req_status == PWA_ENONFINITE) {
            finite = false;
        } else if (s.req_status != PWA_OK) {
            s.error = s.req_status;
            co_return;
        }
        s.cur_it.n_fev = 1;
        const double resolution = 1e-7 * (1.0 + std::fabs(s.f));
        double rho;
        bool noise = false;  // the model's reduction is below what the NLL resolves
        if (!finite || !std::isfinite(fn)) rho = -1.0;
        else if (pred > 10.0 * resolution) rho = (s.f - fn) / pred;
        else {
            // judge by the gradient along p: the curvature test of the line search
            noise = true;
            const bool fok = fn <= s.f + resolution;
            const bool curv = std::fabs(dot(gn, p)) <= 0.9 * std::fabs(dot(s.g, p));
            rho = (fok && curv) ? 1.0 : -1.0;
        }
        if (rho < 0.25) delta = 0.25 * pnorm;
        else if (rho > 0.75 && s.cur_it.cg_exit != 2 && s.cur_it.cg_exit != 3) delta = std::min(2.0 * delta, delta_max);
        if (rho > eta) {
            double smean = 0.0;
            for (int i = 0; i < n; ++i) smean += std::fabs(p[i]);
            smean /= std::max(n, 1);
            s.x = xn;
            s.f = fn;
            s.g = gn;
            s.cur_it.step = 1.0;
            push_iter(s);
            if (smean <= s.o.xtol) {
                s.status = PWA_FIT_XTOL;
                break;
            }
            if (stalled(s, k)) {
                s.status = PWA_FIT_PRECISION;
                break;
            }
        } else {
            push_iter(s);
            if (delta < 1e-12 * (1.0 + std::sqrt(dot(s.x, s.x))) ||
                (noise && std::fabs(dot(s.g, p)) <= resolution)) {
                s.status = PWA_FIT_PRECISION;  // no step the NLL can resolve
                break;
            }
        }
        if (s.o.time_limit_s > 0 && s.since_start() > s.o.time_limit_s) {
            s.status = PWA_FIT_TIME_LIMIT;
            break;
        }
    }
    s.iters = k;
}

FitTask run_fit(FitState& s) { return s.o.method == 1 ? newton_cg_tr(s) : newton_cg(s); }

void init_state(FitState& s, int n, const double* theta0, const pwa_fit_opts* opts_in)
{
    s.P = n;
    pwa_fit_opts_default(&s.o);
    if (opts_in) s.o = *opts_in;
    s.maxiter = s.o.maxiter > 0 ? s.o.maxiter : 200 * n;
    s.explicit_h = !s.o.matrix_free;  // the executor turns it off where no Hessian pass exists
    s.cg_maxiter = s.o.cg_maxiter > 0 ? s.o.cg_maxiter : 20 * n;
    s.x.assign(theta0, theta0 + n);
    s.g.assign(n, 0.0);
    s.t_start = std::chrono::steady_clock::now();
}

void fill_result(const FitState& s, pwa_fit_result* r)
{
    if (!r) return;
    double gmax = 0.0;
    for (double v : s.g) gmax = std::max(gmax, std::fabs(v));
    r->nll = s.f;
    r->grad_max = gmax;
    r->iters = s.iters;
    r->n_hvp = s.n_hvp;
    r->n_fev = s.n_fev;
    r->status = s.error != PWA_OK ? PWA_FIT_ERROR : s.status;
    r->elapsed_s = s.elapsed;
    r->n_trace = (int)s.trace.size();
    r->n_hess = s.n_hess;
}

// copy a fit's records into the caller's trace rows (fit b of a group)
void copy_trace(const FitState& s, int b)
{
    if (!s.o.trace || s.o.trace_cap <= 0 || s.trace.empty()) return;
    std::memcpy(s.o.trace + (size_t)b * s.o.trace_cap, s.trace.data(), sizeof(pwa_fit_iter) * s.trace.size());
}

bool fit_converged(const FitState& s)
{
    return s.error == PWA_OK && (s.status == PWA_FIT_XTOL || s.status == PWA_FIT_GTOL ||
                                 s.status == PWA_FIT_PRECISION || s.status == PWA_FIT_TIME_LIMIT);
}

// Run the fits' work on a private non-blocking stream (the CG graph is
// captured there); the caller's stream is restored on exit.
struct FitStream {
    pwa_handle* h;
    cudaStream_t user = nullptr, own = nullptr;
    pwa_status open(pwa_handle* hh)
    {
        h = hh;
        user = h->stream;
        if (cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            own = nullptr;
            return pwa::set_error(h, PWA_ECUDA, "cannot create the fit stream");
        }
        if (user) cudaStreamSynchronize(user);
        else cudaDeviceSynchronize();
        h->stream = own;
        return PWA_OK;
    }
    ~FitStream()
    {
        if (!own) return;
        cudaStreamSynchronize(own);
        h->stream = user;
        cudaStreamDestroy(own);
        cudaGetLastError();
    }
};

// ---------------------------------------------------------------------------
// lockstep executor: groups of fits, one group per evaluator (a handle's
// batched pass, or a coupling object); every round issues each group's
// requests (one batched evaluation per group, the groups on their own streams
// so that their kernels run concurrently), then resumes every fit
// ---------------------------------------------------------------------------

// One batched evaluation per round: rows theta [nb][P] (and v [nb][P] when any
// request wants H v; zero rows for the others) -> rows (f, g[P], Hv[P]) and a
// per-row non-finite flag.
struct RoundEvaluator {
    virtual ~RoundEvaluator() = default;
    virtual int P() const = 0;
    virtual pwa_handle* handle() const = 0;
    // staging for nb rows: theta, v (pinned where the evaluator copies from)
    virtual pwa_status reserve(int nb, double** theta, double** v) = 0;
    virtual pwa_status issue(int nb, bool any_hv) = 0;                      // asynchronous
    virtual pwa_status finish(int nb, const double** out, const int** err) = 0;  // waits
    // full Hessians at nb points [nb][P], where the evaluator has a Hessian
    // pass: issue enqueues the batched pass, finish waits and writes H
    // [nb][P][P] and a status per point
    virtual bool has_hessian() const { return false; }
    virtual pwa_status hessian_issue(int nb, const double* theta)
    {
        (void)nb;
        (void)theta;
        return PWA_EINVAL;
    }
    virtual pwa_status hessian_finish(int nb, const double* theta, double* H, pwa_status* st)
    {
        (void)nb;
        (void)theta;
        (void)H;
        (void)st;
        return PWA_EINVAL;
    }
};

// a likelihood handle: pwa_eval_batch_device's pass on the handle's batch buffers.
// A round is a fixed sequence (upload theta and v from the pinned staging, the
// batched pass, download of the results and error words); the third time a
// (rows, mode) shape comes up it is captured into a CUDA graph and replayed
// from then on.  A graph is dropped when the handle's buffers, tiling or
// stream are no longer those it was captured with (the batch scratch grows
// in the eager rounds that precede a capture).
struct HandleRounds final : RoundEvaluator {
    struct Captured {
        cudaGraphExec_t exec = nullptr;
        int uses = 0;
        // what the graph's nodes point at
        const void *d_io = nullptr, *h_io = nullptr, *rec = nullptr, *grec = nullptr, *cnt = nullptr;
        cudaStream_t stream = nullptr;
        int grid = 0, W = 0, kpw = 0;
    };
    pwa_handle* h;
    std::vector<Captured> cache;  // index 2 nb + any_hv
    explicit HandleRounds(pwa_handle* hh) : h(hh) {}
    ~HandleRounds() override
    {
        for (auto& c : cache)
            if (c.exec) cudaGraphExecDestroy(c.exec);
        cudaGetLastError();
    }
    int P() const override { return h->P; }
    pwa_handle* handle() const override { return h; }
    bool has_hessian() const override { return h->K <= pwa::kMaxKHessian; }
    pwa_status hessian_issue(int nb, const double* theta) override { return pwa::hessian_issue(h, nb, theta); }
    pwa_status hessian_finish(int nb, const double* theta, double* H, pwa_status* st) override
    {
        pwa_status r = pwa::hessian_finish(h, nb, theta, nullptr, nullptr, H, st);
        if (r == PWA_OK) h->err.clear();  // a non-finite point is reported in its own status
        return r;
    }
    pwa_status reserve(int nb, double** theta, double** v) override
    {
        pwa_status st = pwa::batch_io(h, nb);
        if (st != PWA_OK) return st;
        *theta = h->batch.h_io;
        *v = h->batch.h_io + (size_t)nb * h->P;
        return PWA_OK;
    }
    // upload of the rows' theta (and v) from the pinned staging
    pwa_status copy_in(int nb, bool any_hv, cudaStream_t s)
    {
        pwa::BatchState& bs = h->batch;
        const size_t BP = (size_t)nb * h->P;
        cudaError_t e = cudaMemcpyAsync(bs.d_io, bs.h_io, sizeof(double) * (any_hv ? 2 * BP : BP),
                                        cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "batch upload");
        return PWA_OK;
    }
    // download of the results and the error words into the pinned staging
    pwa_status copy_out(int nb, cudaStream_t s)
    {
        pwa::BatchState& bs = h->batch;
        const size_t BP = (size_t)nb * h->P;
        const size_t ow = (size_t)nb * (1 + 2 * (size_t)h->P);
        double* pin = bs.h_io;
        int* errw = reinterpret_cast<int*>(pin + 2 * BP + ow);  // [nb] per-vector words, then the shared one
        cudaError_t e = cudaMemcpyAsync(pin + 2 * BP, bs.d_io + 2 * BP, sizeof(double) * ow, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(errw, bs.d_err_vec, sizeof(int) * nb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(errw + nb, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "batch download");
        return PWA_OK;
    }
    // the round's operations, enqueued on the handle's stream
    pwa_status enqueue(int nb, bool any_hv)
    {
        pwa::BatchState& bs = h->batch;
        const size_t BP = (size_t)nb * h->P;
        pwa_status st = copy_in(nb, any_hv, h->stream);
        if (st != PWA_OK) return st;
        st = pwa::launch_batch(h, nb, bs.d_io, any_hv ? bs.d_io + BP : nullptr, bs.d_io + 2 * BP,
                               any_hv ? pwa::MODE_HVP : pwa::MODE_GRAD, true);
        if (st != PWA_OK) return st;
        return copy_out(nb, h->stream);
    }
    bool same_state(const Captured& c) const
    {
        const pwa::BatchState& bs = h->batch;
        return c.d_io == bs.d_io && c.h_io == bs.h_io && c.rec == bs.d_block_rec && c.grec == bs.d_group_rec &&
               c.cnt == bs.d_counts && c.stream == h->stream && c.grid == h->tiling.grid && c.W == h->tiling.W &&
               c.kpw == h->tiling.KPW;
    }
    pwa_status issue(int nb, bool any_hv) override
    {
        const size_t key = 2 * (size_t)nb + (any_hv ? 1 : 0);
        if (cache.size() <= key) cache.resize(key + 1);
        Captured& c = cache[key];
        if (c.exec && !same_state(c)) {
            cudaGraphExecDestroy(c.exec);
            c = Captured();
        }
        if (c.exec) {
            cudaError_t e = cudaGraphLaunch(c.exec, h->stream);
            if (e != cudaSuccess) return pwa::cuda_error(h, e, "round graph launch");
            return PWA_OK;
        }
        if (++c.uses < 3 || h->stream == nullptr) return enqueue(nb, any_hv);
        // capture this round (the scratch for nb rows exists: earlier rounds of the shape grew it)
        const pwa::BatchState& bs = h->batch;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return enqueue(nb, any_hv);
        }
        pwa_status st = enqueue(nb, any_hv);
        e = cudaStreamEndCapture(h->stream, &g);
        if (st != PWA_OK || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            h->err.clear();
            c.uses = -1000000;  // this shape stays eager
            return enqueue(nb, any_hv);
        }
        e = cudaGraphInstantiate(&c.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c.exec = nullptr;
            c.uses = -1000000;
            return enqueue(nb, any_hv);
        }
        c.d_io = bs.d_io;
        c.h_io = bs.h_io;
        c.rec = bs.d_block_rec;
        c.grec = bs.d_group_rec;
        c.cnt = bs.d_counts;
        c.stream = h->stream;
        c.grid = h->tiling.grid;
        c.W = h->tiling.W;
        c.kpw = h->tiling.KPW;
        e = cudaGraphLaunch(c.exec, h->stream);
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "round graph launch");
        return PWA_OK;
    }
    pwa_status finish(int nb, const double** out, const int** err) override
    {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "batch round");
        const size_t BP = (size_t)nb * h->P;
        const size_t ow = (size_t)nb * (1 + 2 * (size_t)h->P);
        double* pin = h->batch.h_io;
        const int* errw = reinterpret_cast<const int*>(pin + 2 * BP + ow);
        if (errw[nb]) {
            // the shared error word: a timeout ends everything; non-finite
            // intensities are attributed to their vectors by the per-vector words
            pwa_status st = pwa::check_device_errors(h);
            if (st != PWA_OK && st != PWA_ENONFINITE) return st;
            h->err.clear();
        }
        *out = pin + 2 * BP;
        *err = errw;
        return PWA_OK;
    }
};

// a coupling object: its tensor-core evaluation (synchronous, 16 rows per launch)
struct CouplingRounds final : RoundEvaluator {
    pwa_coupling* cp;
    pwa_handle* h;
    int Pc;
    std::vector<double> th, vv, res;
    std::vector<int> errw;
    CouplingRounds(pwa_coupling* c, pwa_handle* hh, int pc) : cp(c), h(hh), Pc(pc) {}
    int P() const override { return Pc; }
    pwa_handle* handle() const override { return h; }
    pwa_status reserve(int nb, double** theta, double** v) override
    {
        th.resize((size_t)nb * Pc);
        vv.resize((size_t)nb * Pc);
        *theta = th.data();
        *v = vv.data();
        return PWA_OK;
    }
    pwa_status issue(int nb, bool any_hv) override
    {
        res.resize((size_t)nb * (1 + 2 * Pc));
        errw.resize(nb);
        return pwa::coupling_eval_rows(cp, nb, th.data(), any_hv ? vv.data() : nullptr, res.data(), errw.data());
    }
    pwa_status finish(int nb, const double** out, const int** err) override
    {
        (void)nb;
        *out = res.data();
        *err = errw.data();
        return PWA_OK;
    }
};

// a physics-variant likelihood: one synchronous evaluation per row
struct VariantRounds final : RoundEvaluator {
    pwa_variant* v;
    pwa_handle* h;
    int Pv;
    std::vector<double> th, vv, res;
    std::vector<double> bf, bg, bh;  // batched evaluation: NLL [nb], gradient and H v [nb][P]
    std::vector<pwa_status> bst;
    std::vector<int> errw;
    bool couplings_only;
    VariantRounds(pwa_variant* vr, int p, bool conly = false)
        : v(vr), h(pwa::variant_base(vr)), Pv(p), couplings_only(conly)
    {
    }
    int P() const override { return Pv; }
    pwa_handle* handle() const override { return h; }
    pwa_status reserve(int nb, double** theta, double** dir) override
    {
        th.resize((size_t)nb * Pv);
        vv.resize((size_t)nb * Pv);
        *theta = th.data();
        *dir = vv.data();
        return PWA_OK;
    }
    pwa_status issue(int nb, bool any_hv) override
    {
        const size_t ow = 1 + 2 * (size_t)Pv;
        res.assign((size_t)nb * ow, 0.0);
        errw.assign(nb, 0);
        if (!couplings_only) {
            // every row in one launch
            bf.assign(nb, 0.0);
            bg.assign((size_t)nb * Pv, 0.0);
            bh.assign(any_hv ? (size_t)nb * Pv : 0, 0.0);
            bst.assign(nb, PWA_OK);
            pwa_status st = pwa::variant_eval_batch(v, nb, th.data(), any_hv ? vv.data() : nullptr, bf.data(),
                                                    bg.data(), any_hv ? bh.data() : nullptr, bst.data());
            if (st != PWA_OK) return st;
            for (int b = 0; b < nb; ++b) {
                double* r = res.data() + b * ow;
                if (bst[b] != PWA_OK) {
                    // a point outside the model's domain (non-finite intensity, a mass below its
                    // threshold): the fit sees an error for this row and backs off
                    errw[b] = 1;
                    r[0] = std::numeric_limits<double>::infinity();
                    continue;
                }
                r[0] = bf[b];
                std::memcpy(r + 1, bg.data() + (size_t)b * Pv, sizeof(double) * Pv);
                if (any_hv) std::memcpy(r + 1 + Pv, bh.data() + (size_t)b * Pv, sizeof(double) * Pv);
            }
            return PWA_OK;
        }
        for (int b = 0; b < nb; ++b) {
            double* r = res.data() + b * ow;
            const double* tb = th.data() + (size_t)b * Pv;
            const double* vb = any_hv ? vv.data() + (size_t)b * Pv : nullptr;
            pwa_status st = pwa::variant_coupling_eval(v, tb, vb, r, r + 1, any_hv ? r + 1 + Pv : nullptr);
            if (st == PWA_ENONFINITE || st == PWA_EINVAL) {
                // a point outside the model's domain (non-finite intensity, a mass below its threshold):
                // the fit sees an error for this row and backs off
                errw[b] = 1;
                h->err.clear();
                r[0] = std::numeric_limits<double>::infinity();
            } else if (st != PWA_OK) {
                return st;
            }
        }
        return PWA_OK;
    }
    pwa_status finish(int nb, const double** out, const int** err) override
    {
        (void)nb;
        *out = res.data();
        *err = errw.data();
        return PWA_OK;
    }
};

struct FitGroup {
    std::unique_ptr<RoundEvaluator> ev;
    int B = 0, P = 0;
    FitStream fs;
    std::vector<FitState> fits;
    std::vector<FitTask> tasks;
    std::vector<int> live;
    std::vector<double> zero;
    // the round's Hessian requests: fits, their points [n][P], Hessians [n][P][P], statuses
    std::vector<int> hrows;
    std::vector<double> htheta, hH;
    std::vector<pwa_status> hst;
    pwa_status hissue = PWA_OK;
};

pwa_status open_group(FitGroup& g, std::unique_ptr<RoundEvaluator> ev, int B, const double* theta0,
                      const pwa_fit_opts* opts)
{
    pwa_handle* h = ev->handle();
    g.ev = std::move(ev);
    g.B = B;
    g.P = g.ev->P();
    h->err.clear();
    if (B < 1) return pwa::set_error(h, PWA_EINVAL, "B must be at least 1");
    if (!theta0) return pwa::set_error(h, PWA_EINVAL, "theta0 must not be NULL");
    const int P = g.P;
    for (size_t i = 0; i < (size_t)B * P; ++i)
        if (!std::isfinite(theta0[i])) return pwa::set_error(h, PWA_EINVAL, "theta0 must be finite");
    pwa_status st = g.fs.open(h);
    if (st != PWA_OK) return st;
    g.zero.assign(P, 0.0);
    g.fits.resize(B);
    g.tasks.reserve(B);
    for (int b = 0; b < B; ++b) {
        init_state(g.fits[b], P, theta0 + (size_t)b * P, opts);
        g.fits[b].explicit_h &= g.ev->has_hessian();
        g.tasks.push_back(run_fit(g.fits[b]));
        g.tasks[b].h.resume();  // runs to its first request
    }
    return PWA_OK;
}

// A group's Hessian requests: hess_issue enqueues one batched Hessian pass
// over all of its fits that ask for one (returns whether there were any);
// hess_finish waits for it and resumes those fits (each runs its CG on the
// host and posts its next request).
bool hess_issue(FitGroup& g)
{
    g.hrows.clear();
    for (int b = 0; b < g.B; ++b)
        if (!g.tasks[b].h.done() && g.fits[b].req == Req::HESS) g.hrows.push_back(b);
    if (g.hrows.empty()) return false;
    const int P = g.P, nb = (int)g.hrows.size();
    g.htheta.resize((size_t)nb * P);
    for (int i = 0; i < nb; ++i)
        std::memcpy(g.htheta.data() + (size_t)i * P, g.fits[g.hrows[i]].rx, sizeof(double) * P);
    g.hissue = g.ev->hessian_issue(nb, g.htheta.data());
    return true;
}

void hess_finish(FitGroup& g)
{
    if (g.hrows.empty()) return;
    const int P = g.P, nb = (int)g.hrows.size();
    g.hH.resize((size_t)nb * P * P);
    g.hst.assign(nb, PWA_OK);
    pwa_status st = g.hissue;
    if (st == PWA_OK) st = g.ev->hessian_finish(nb, g.htheta.data(), g.hH.data(), g.hst.data());
    for (int i = 0; i < nb; ++i) {
        const int b = g.hrows[i];
        FitState& s = g.fits[b];
        ++s.n_hess;
        s.req_status = st != PWA_OK ? st : g.hst[i];
        if (s.req_status == PWA_OK) std::memcpy(s.rH, g.hH.data() + (size_t)i * P * P, sizeof(double) * P * P);
        g.tasks[b].h.resume();
        if (g.tasks[b].h.done()) s.elapsed = s.since_start();
    }
    g.hrows.clear();
}

// Serve the groups' Hessian requests: every group's pass enqueued before the
// first is waited for (the host's combination and CG for one group overlap
// the passes of the next); repeats while any fit asks for a Hessian.
void serve_hessians(const std::vector<FitGroup*>& gs)
{
    while (true) {
        bool any = false;
        for (FitGroup* g : gs) any |= hess_issue(*g);
        if (!any) return;
        for (FitGroup* g : gs) hess_finish(*g);
    }
}

// Enqueue the group's round: its unfinished fits' requests as one batched
// evaluation (H v for all when any asks for it, with v = 0 for the f, g requests).
// Collects the fits that wait for f, g or H v (the Hessian requests are
// served before, by serve_hessians).  Returns whether any of those wants H v.
bool collect_round(FitGroup& g)
{
    g.live.clear();
    for (int b = 0; b < g.B; ++b)
        if (!g.tasks[b].h.done() && g.fits[b].req != Req::HESS) g.live.push_back(b);
    bool any_hv = false;
    for (int b : g.live) any_hv |= g.fits[b].req == Req::HV;
    return any_hv;
}

// The live fits' rows (theta, and v when any_hv; zero v for f, g requests)
// into the evaluator's staging.
pwa_status stage_rows(FitGroup& g, bool any_hv)
{
    const int P = g.P, nb = (int)g.live.size();
    double *th = nullptr, *v = nullptr;
    pwa_status st = g.ev->reserve(nb, &th, &v);
    if (st != PWA_OK) return st;
    for (int i = 0; i < nb; ++i) {
        const FitState& s = g.fits[g.live[i]];
        std::memcpy(th + (size_t)i * P, s.rx, sizeof(double) * P);
        if (any_hv) std::memcpy(v + (size_t)i * P, s.req == Req::HV ? s.rv : g.zero.data(), sizeof(double) * P);
    }
    return PWA_OK;
}

pwa_status issue_round(FitGroup& g)
{
    const bool any_hv = collect_round(g);
    if (g.live.empty()) return PWA_OK;
    pwa_status st = stage_rows(g, any_hv);
    if (st != PWA_OK) return st;
    return g.ev->issue((int)g.live.size(), any_hv);
}

// Wait for the group's round and resume its fits with their results.
pwa_status finish_round(FitGroup& g)
{
    if (g.live.empty()) return PWA_OK;
    const int P = g.P, nb = (int)g.live.size();
    const double* res = nullptr;
    const int* errw = nullptr;
    pwa_status st = g.ev->finish(nb, &res, &errw);
    if (st != PWA_OK) return st;
    for (int i = 0; i < nb; ++i) {
        FitState& s = g.fits[g.live[i]];
        const double* r = res + (size_t)i * (1 + 2 * P);
        s.req_status = errw[i] ? PWA_ENONFINITE : PWA_OK;
        if (s.req == Req::FG) {
            ++s.n_fev;
            *s.rf = r[0];
            std::memcpy(s.rg, r + 1, sizeof(double) * P);
        } else {
            std::memcpy(s.rhv, r + 1 + P, sizeof(double) * P);
        }
        g.tasks[g.live[i]].h.resume();
        if (g.tasks[g.live[i]].h.done()) s.elapsed = s.since_start();
    }
    return PWA_OK;
}

// Lockstep rounds, one batched launch per group on its own stream: every
// group's Hessian pass is enqueued first; then, group by group, its Hessian
// is waited for, its fits run their CG on the host, and its f, g / H v round
// is enqueued at once, so that the GPU works on that round (and on the later
// groups' Hessians) while the host serves the next group.  A fit that asks
// for a Hessian again is served in the next round.
pwa_status run_lockstep(std::vector<std::unique_ptr<FitGroup>>& groups)
{
    while (true) {
        for (auto& g : groups) hess_issue(*g);
        bool any = false;
        for (auto& g : groups) {
            hess_finish(*g);
            pwa_status st = issue_round(*g);
            if (st != PWA_OK) return st;
            any |= !g->live.empty();
            for (int b = 0; b < g->B && !any; ++b) any |= !g->tasks[b].h.done();
        }
        if (!any) return PWA_OK;
        for (auto& g : groups) {
            pwa_status st = finish_round(*g);
            if (st != PWA_OK) return st;
        }
    }
}

// Lockstep rounds of several likelihood handles with one launch per round
// (pwa::launch_multi): the rows of every handle with live fits are uploaded,
// one pass over all those handles runs (H v mode when any fit anywhere asks
// for H v), and the results come back, all on one stream.  The third time a
// round of the same shape (which handles, how many rows each, the mode) comes
// up it is captured into a CUDA graph and replayed from then on; a graph is
// dropped when a buffer it points at has changed.
struct MultiRounds {
    struct Captured {
        std::vector<int> key;  // any_hv, then (group, rows) pairs
        cudaGraphExec_t exec = nullptr;
        int uses = 0;
        std::vector<const void*> ptrs;  // the buffers its nodes point at
        // the launch arguments' staging of this graph alone: its copy node
        // replays from it, so no other round may write it
        pwa::MultiScratch ms;
    };
    std::vector<std::unique_ptr<FitGroup>>& groups;
    cudaStream_t stream = nullptr;
    pwa::MultiScratch eager;  // staging of the rounds that run without a graph
    std::vector<std::unique_ptr<Captured>> cache;
    explicit MultiRounds(std::vector<std::unique_ptr<FitGroup>>& g) : groups(g) {}
    ~MultiRounds()
    {
        if (stream) cudaStreamSynchronize(stream);
        for (auto& c : cache)
            if (c->exec) cudaGraphExecDestroy(c->exec);
        cache.clear();
        if (stream) cudaStreamDestroy(stream);
        cudaGetLastError();
    }
    HandleRounds* hr(int i) { return static_cast<HandleRounds*>(groups[i]->ev.get()); }
    std::vector<const void*> buffers(const std::vector<int>& gs, const pwa::MultiScratch& ms)
    {
        std::vector<const void*> p{ms.d_args, ms.d_first, ms.h_stage};
        for (int i : gs) {
            const pwa::BatchState& bs = hr(i)->h->batch;
            p.insert(p.end(), {bs.d_io, bs.h_io, bs.d_block_rec, bs.d_group_rec, bs.d_counts});
        }
        return p;
    }
    pwa_status enqueue(const std::vector<int>& gs, bool any_hv, pwa::MultiScratch& ms)
    {
        const int n = (int)gs.size();
        std::vector<pwa_handle*> hs(n);
        std::vector<int> B(n);
        std::vector<const double*> th(n), v(n);
        std::vector<double*> out(n);
        for (int k = 0; k < n; ++k) {
            HandleRounds* r = hr(gs[k]);
            const int nb = (int)groups[gs[k]]->live.size();
            pwa_status st = r->copy_in(nb, any_hv, stream);
            if (st != PWA_OK) return st;
            const pwa::BatchState& bs = r->h->batch;
            const size_t BP = (size_t)nb * r->h->P;
            hs[k] = r->h;
            B[k] = nb;
            th[k] = bs.d_io;
            v[k] = bs.d_io + BP;
            out[k] = bs.d_io + 2 * BP;
        }
        pwa_status st = pwa::launch_multi(n, hs.data(), B.data(), th.data(), v.data(), out.data(),
                                          any_hv ? pwa::MODE_HVP : pwa::MODE_GRAD, true, stream, ms);
        if (st != PWA_OK) return st;
        for (int k = 0; k < n; ++k) {
            st = hr(gs[k])->copy_out(B[k], stream);
            if (st != PWA_OK) return st;
        }
        return PWA_OK;
    }
    pwa_status issue(const std::vector<int>& gs, bool any_hv)
    {
        std::vector<int> key{any_hv ? 1 : 0};
        for (int i : gs) key.insert(key.end(), {i, (int)groups[i]->live.size()});
        Captured* c = nullptr;
        for (auto& x : cache)
            if (x->key == key) c = x.get();
        if (!c) {
            cache.push_back(std::make_unique<Captured>());
            c = cache.back().get();
            c->key = key;
        }
        if (c->exec && c->ptrs != buffers(gs, c->ms)) {
            cudaGraphExecDestroy(c->exec);
            c->exec = nullptr;
            c->uses = 0;
        }
        if (c->exec) {
            cudaError_t e = cudaGraphLaunch(c->exec, stream);
            if (e != cudaSuccess) return pwa::cuda_error(hr(gs[0])->h, e, "multi round graph launch");
            return PWA_OK;
        }
        if (++c->uses < 3) return enqueue(gs, any_hv, eager);
        // the graph's own staging, allocated outside the capture (enqueue then reuses it)
        pwa_status st = pwa::launch_multi_reserve(hr(gs[0])->h, (int)gs.size(), c->ms);
        if (st != PWA_OK) return st;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return enqueue(gs, any_hv, eager);
        }
        st = enqueue(gs, any_hv, c->ms);
        e = cudaStreamEndCapture(stream, &g);
        if (st != PWA_OK || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            for (int i : gs) hr(i)->h->err.clear();
            c->uses = -1000000;  // this shape stays eager
            return enqueue(gs, any_hv, eager);
        }
        e = cudaGraphInstantiate(&c->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->exec = nullptr;
            c->uses = -1000000;
            return enqueue(gs, any_hv, eager);
        }
        c->ptrs = buffers(gs, c->ms);
        e = cudaGraphLaunch(c->exec, stream);
        if (e != cudaSuccess) return pwa::cuda_error(hr(gs[0])->h, e, "multi round graph launch");
        return PWA_OK;
    }
    pwa_status run()
    {
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            stream = nullptr;
            return pwa::set_error(hr(0)->h, PWA_ECUDA, "cannot create the multi-round stream");
        }
        std::vector<FitGroup*> all;
        for (auto& g : groups) all.push_back(g.get());
        while (true) {
            serve_hessians(all);
            bool any_hv = false;
            std::vector<int> gs;
            for (int i = 0; i < (int)groups.size(); ++i) {
                any_hv |= collect_round(*groups[i]);
                if (!groups[i]->live.empty()) gs.push_back(i);
            }
            if (gs.empty()) return PWA_OK;
            for (int i : gs) {
                pwa_status st = stage_rows(*groups[i], any_hv);
                if (st != PWA_OK) return st;
            }
            pwa_status st = issue(gs, any_hv);
            if (st != PWA_OK) return st;
            cudaError_t e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) return pwa::cuda_error(hr(gs[0])->h, e, "multi round");
            for (int i : gs) {
                st = finish_round(*groups[i]);
                if (st != PWA_OK) return st;
            }
        }
    }
};

// Results of a group; all_ok stays true when every fit converged or hit its time limit.
pwa_status close_group(FitGroup& g, double* theta_out, pwa_fit_result* results, bool& all_ok, int trace_row0 = 0)
{
    const int P = g.P;
    for (int b = 0; b < g.B; ++b)
        if (g.tasks[b].failed()) return pwa::set_error(g.ev->handle(), PWA_ENOMEM, "host exception in a fit");
    for (int b = 0; b < g.B; ++b) {
        std::memcpy(theta_out + (size_t)b * P, g.fits[b].x.data(), sizeof(double) * P);
        if (results) fill_result(g.fits[b], results + b);
        copy_trace(g.fits[b], trace_row0 + b);
        all_ok &= fit_converged(g.fits[b]);
    }
    return PWA_OK;
}

}  // namespace

extern "C" void pwa_fit_opts_default(pwa_fit_opts* o)
{
    if (!o) return;
    o->xtol = 1e-8;
    o->gtol = 0.0;
    o->maxiter = 0;
    o->cg_maxiter = 0;
    o->time_limit_s = 0.0;
    o->matrix_free = 0;
    o->method = 0;
    o->trace_cap = 0;
    o->trace = nullptr;
    o->one_launch = 0;
}

extern "C" pwa_status pwa_newton_cg_fit(pwa_handle* h, const double* theta0, const pwa_fit_opts* opts_in,
                                        double* theta_out, pwa_fit_result* result)
{
    if (!h) return PWA_EINVAL;
    if (!theta0 || !theta_out) return pwa::set_error(h, PWA_EINVAL, "theta0 and theta_out must not be NULL");
    FitState s;
    init_state(s, h->P, theta0, opts_in);
    s.device_cg = true;
    s.explicit_h &= h->K <= pwa::kMaxKHessian;
    FitStream fs;
    pwa_status st = fs.open(h);
    if (st != PWA_OK) return st;
    DeviceCG cg;
    st = cg.init(h);
    if (st != PWA_OK) return st;

    // one fit: every request is served at once
    FitTask task = run_fit(s);
    for (task.h.resume(); !task.h.done(); task.h.resume()) {
        switch (s.req) {
            case Req::FG:
                ++s.n_fev;
                s.req_status = pwa_eval(h, s.rx, nullptr, s.rf, s.rg, nullptr);
                if (s.req_status == PWA_ENONFINITE) h->err.clear();
                break;
            case Req::CG:
                s.req_status = cg.solve(s.x, s.g, s.cg_eps, s.cg_maxiter, s.p, s.n_hvp, &s.cur_it);
                break;
            case Req::HESS:
                ++s.n_hess;
                s.req_status = pwa::hessian_device(h, s.rx, nullptr, nullptr, s.rH);
                if (s.req_status == PWA_ENONFINITE) h->err.clear();
                break;
            case Req::HV: {  // matrix-free trust-region CG: one fused pass per product
                double f_unused = 0.0;
                s.req_status = pwa_eval(h, s.rx, s.rv, &f_unused, nullptr, s.rhv);
                if (s.req_status == PWA_ENONFINITE) h->err.clear();
                break;
            }
            default:
                s.req_status = pwa::set_error(h, PWA_EINVAL, "internal: unexpected fit request");
                break;
        }
    }
    s.elapsed = s.since_start();
    if (task.failed()) return pwa::set_error(h, PWA_ENOMEM, "host exception in the fit");
    std::memcpy(theta_out, s.x.data(), sizeof(double) * s.P);
    fill_result(s, result);
    copy_trace(s, 0);
    if (s.error != PWA_OK) {
        if (s.error == PWA_ENONFINITE)
            return pwa::set_error(h, PWA_ENONFINITE, "non-finite NLL at the start point");
        return s.error;
    }
    return fit_converged(s) ? PWA_OK : PWA_ENOCONV;
}

extern "C" pwa_status pwa_newton_cg_fit_batch(pwa_handle* h, int B, const double* theta0,
                                              const pwa_fit_opts* opts_in, double* theta_out,
                                              pwa_fit_result* results)
{
    if (!h) return PWA_EINVAL;
    if (!theta_out) return pwa::set_error(h, PWA_EINVAL, "theta_out must not be NULL");
    return pwa_newton_cg_fit_multi(1, &h, &B, &theta0, opts_in, &theta_out, &results);
}

extern "C" pwa_status pwa_newton_cg_fit_multi(int n_handles, pwa_handle* const* handles, const int* B,
                                              const double* const* theta0, const pwa_fit_opts* opts,
                                              double* const* theta_out, pwa_fit_result* const* results)
{
    if (n_handles < 1 || !handles || !B || !theta0 || !theta_out) return PWA_EINVAL;
    for (int i = 0; i < n_handles; ++i) {
        if (!handles[i]) return PWA_EINVAL;
        if (!theta_out[i]) return pwa::set_error(handles[i], PWA_EINVAL, "theta_out must not be NULL");
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i])
                return pwa::set_error(handles[i], PWA_EINVAL, "a handle appears twice; put its fits in one group");
    }
    std::vector<std::unique_ptr<FitGroup>> groups;
    // one launch per round over all handles (each K <= 32) when asked for
    bool multi = n_handles >= 2 && opts && opts->one_launch;
    for (int i = 0; i < n_handles; ++i) {
        multi &= handles[i]->K <= pwa::kMaxKMulti;
        groups.push_back(std::make_unique<FitGroup>());
        pwa_status st = open_group(*groups.back(), std::make_unique<HandleRounds>(handles[i]), B[i], theta0[i], opts);
        if (st != PWA_OK) return st;
    }
    pwa_status st;
    if (multi) {
        MultiRounds mr(groups);
        st = mr.run();
    } else {
        st = run_lockstep(groups);
    }
    if (st != PWA_OK) return st;
    bool all_ok = true;
    int row0 = 0;  // trace rows run over the fits of all handles in order
    for (int i = 0; i < n_handles; ++i) {
        st = close_group(*groups[i], theta_out[i], results ? results[i] : nullptr, all_ok, row0);
        if (st != PWA_OK) return st;
        row0 += B[i];
    }
    return all_ok ? PWA_OK : PWA_ENOCONV;
}

extern "C" pwa_status pwa_variant_fit(pwa_variant* v, int B, const double* theta0, const pwa_fit_opts* opts,
                                      double* theta_out, pwa_fit_result* results)
{
    if (!v) return PWA_EINVAL;
    pwa_handle* h = pwa::variant_base(v);
    if (!theta_out) return pwa::set_error(h, PWA_EINVAL, "theta_out must not be NULL");
    std::vector<std::unique_ptr<FitGroup>> groups;
    groups.push_back(std::make_unique<FitGroup>());
    pwa_status st = open_group(*groups.back(), std::make_unique<VariantRounds>(v, pwa_variant_num_params(v)), B,
                               theta0, opts);
    if (st != PWA_OK) return st;
    st = run_lockstep(groups);
    if (st != PWA_OK) return st;
    bool all_ok = true;
    st = close_group(*groups[0], theta_out, results, all_ok);
    if (st != PWA_OK) return st;
    return all_ok ? PWA_OK : PWA_ENOCONV;
}

extern "C" pwa_status pwa_variant_coupling_fit(pwa_variant* v, int B, const double* theta_c0,
                                               const pwa_fit_opts* opts, double* theta_c_out, pwa_fit_result* results)
{
    if (!v) return PWA_EINVAL;
    pwa_handle* h = pwa::variant_base(v);
    if (!theta_c_out) return pwa::set_error(h, PWA_EINVAL, "theta_c_out must not be NULL");
    std::vector<std::unique_ptr<FitGroup>> groups;
    groups.push_back(std::make_unique<FitGroup>());
    pwa_status st = open_group(*groups.back(),
                               std::make_unique<VariantRounds>(v, pwa_variant_coupling_num_params(v), true), B,
                               theta_c0, opts);
    if (st != PWA_OK) return st;
    st = run_lockstep(groups);
    if (st != PWA_OK) return st;
    bool all_ok = true;
    st = close_group(*groups[0], theta_c_out, results, all_ok);
    if (st != PWA_OK) return st;
    return all_ok ? PWA_OK : PWA_ENOCONV;
}

extern "C" pwa_status pwa_coupling_fit(pwa_coupling* cp, int C, const double* theta_c0, const pwa_fit_opts* opts,
                                       double* theta_c_out, pwa_fit_result* results)
{
    if (!cp) return PWA_EINVAL;
    pwa_handle* h = pwa::coupling_handle(cp);
    if (!theta_c_out) return pwa::set_error(h, PWA_EINVAL, "theta_c_out must not be NULL");
    std::vector<std::unique_ptr<FitGroup>> groups;
    groups.push_back(std::make_unique<FitGroup>());
    pwa_status st = open_group(*groups.back(), std::make_unique<CouplingRounds>(cp, h, pwa_coupling_num_params(cp)), C,
                               theta_c0, opts);
    if (st != PWA_OK) return st;
    st = run_lockstep(groups);
    if (st != PWA_OK) return st;
    bool all_ok = true;
    st = close_group(*groups[0], theta_c_out, results, all_ok);
    if (st != PWA_OK) return st;
    return all_ok ? PWA_OK : PWA_ENOCONV;
}
