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
//    1e-7 (1 + |f|) ends the fit as converged at the precision limit.
#include <chrono>
#include <cmath>
#include <cstring>
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
        }
        return;
    }
    if (j + 1 >= maxiter) {
        if (threadIdx.x == 0) {
            c.flags[0] = 3;
            c.flags[1] = j + 1;
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

    // capture kCgBatch iterations (HVP pass at x along d, then the update) once
    pwa_status capture(int maxiter)
    {
        cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "cudaStreamBeginCapture");
        pwa_status st = PWA_OK;
        for (int b = 0; b < kCgBatch && st == PWA_OK; ++b) {
            st = pwa::launch_pass(h, c.x, c.d, c.out, pwa::MODE_HVP, c.flags);
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
                     std::vector<double>& p, int& n_hvp)
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
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return pwa::cuda_error(h, e, "CG download");
        p.assign(pin, pin + P);
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

struct Evaluator {
    pwa_handle* h;
    int n_fev = 0, n_hvp = 0;

    pwa_status fg(const std::vector<double>& x, double& f, std::vector<double>& g)
    {
        ++n_fev;
        return pwa_eval(h, x.data(), nullptr, &f, g.data(), nullptr);
    }
};

double dot(const std::vector<double>& a, const std::vector<double>& b)
{
    double s = 0.0;
    for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
    return s;
}

struct LinePoint {
    double a, f, df;
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

}  // namespace

extern "C" void pwa_fit_opts_default(pwa_fit_opts* o)
{
    if (!o) return;
    o->xtol = 1e-8;
    o->gtol = 0.0;
    o->maxiter = 0;
    o->cg_maxiter = 0;
    o->time_limit_s = 0.0;
}

extern "C" pwa_status pwa_newton_cg_fit(pwa_handle* h, const double* theta0, const pwa_fit_opts* opts_in,
                                        double* theta_out, pwa_fit_result* result)
{
    if (!h) return PWA_EINVAL;
    if (!theta0 || !theta_out) return pwa::set_error(h, PWA_EINVAL, "theta0 and theta_out must not be NULL");
    const auto t_start = std::chrono::steady_clock::now();
    auto elapsed = [&]() {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    };
    pwa_fit_opts o;
    pwa_fit_opts_default(&o);
    if (opts_in) o = *opts_in;
    const int n = h->P;
    const int maxiter = o.maxiter > 0 ? o.maxiter : 200 * n;
    const int cg_maxiter = o.cg_maxiter > 0 ? o.cg_maxiter : 20 * n;
    const double c1 = 1e-4, c2 = 0.9;

    // the CG graph is captured on a private non-default stream
    cudaStream_t user_stream = h->stream, fit_stream = nullptr;
    if (cudaStreamCreateWithFlags(&fit_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return pwa::set_error(h, PWA_ECUDA, "cannot create the fit stream");
    }
    if (user_stream) cudaStreamSynchronize(user_stream);
    else cudaDeviceSynchronize();
    h->stream = fit_stream;
    struct Restore {
        pwa_handle* h;
        cudaStream_t user, own;
        ~Restore()
        {
            cudaStreamSynchronize(own);
            h->stream = user;
            cudaStreamDestroy(own);
            cudaGetLastError();
        }
    } restore{h, user_stream, fit_stream};
    DeviceCG cg;
    pwa_status st = cg.init(h);
    if (st != PWA_OK) return st;

    Evaluator ev{h};
    std::vector<double> x(theta0, theta0 + n), g(n), p(n);
    double f = 0.0;
    st = ev.fg(x, f, g);
    if (st != PWA_OK) return st;

    int status = PWA_FIT_MAXITER;
    int k = 0;
    while (k < maxiter) {
        double gmax = 0.0;
        for (double v : g) gmax = std::max(gmax, std::fabs(v));
        if (o.gtol > 0 && gmax <= o.gtol) {
            status = PWA_FIT_GTOL;
            break;
        }
        // ---- inner CG on H p = -g (N&W Algorithm 7.1), on the device ----
        const double gnorm = std::sqrt(dot(g, g));
        const double eps = std::min(0.5, std::sqrt(gnorm)) * gnorm;
        st = cg.solve(x, g, eps, cg_maxiter, p, ev.n_hvp);
        if (st != PWA_OK) break;
        ++k;
        double pmean = 0.0;
        for (double v : p) pmean += std::fabs(v);
        pmean /= std::max(n, 1);
        if (pmean <= o.xtol) {
            status = PWA_FIT_XTOL;
            break;
        }
        double df0 = dot(g, p);
        if (!(df0 < 0)) {
            for (int i = 0; i < n; ++i) p[i] = -g[i];
            df0 = dot(g, p);
        }
        // ---- strong-Wolfe line search (N&W Algorithms 3.5 / 3.6) ----
        const double eps_f = 1e-7 * std::fabs(f);
        auto phi = [&](double a, LinePoint& lp) -> pwa_status {
            lp.a = a;
            lp.x.resize(n);
            lp.g.resize(n);
            for (int i = 0; i < n; ++i) lp.x[i] = x[i] + a * p[i];
            pwa_status s = ev.fg(lp.x, lp.f, lp.g);
            if (s == PWA_ENONFINITE) {  // the trial point left the region where I > 0
                h->err.clear();
                lp.f = INFINITY;
                lp.df = 0.0;
                return PWA_OK;
            }
            lp.df = dot(lp.g, p);
            return s;
        };
        auto armijo_fails = [&](const LinePoint& lp) { return !(lp.f <= f + c1 * lp.a * df0 + eps_f); };
        LinePoint prev{0.0, f, df0, x, g}, cur, found;
        bool ok = false;
        auto zoom = [&](LinePoint lo, LinePoint hi) -> pwa_status {
            for (int it = 0; it < 30; ++it) {
                double a;
                const double left = std::min(lo.a, hi.a), right = std::max(lo.a, hi.a), width = right - left;
                if (!std::isfinite(hi.f) || !cubic_min(lo.a, lo.f, lo.df, hi.a, hi.f, hi.df, a) ||
                    a < left + 0.1 * width || a > right - 0.1 * width)
                    a = 0.5 * (lo.a + hi.a);
                LinePoint lp;
                pwa_status s = phi(a, lp);
                if (s != PWA_OK) return s;
                if (armijo_fails(lp) || lp.f >= lo.f + eps_f) {
                    hi = lp;
                } else {
                    if (std::fabs(lp.df) <= -c2 * df0) {
                        found = lp;
                        ok = true;
                        return PWA_OK;
                    }
                    if (lp.df * (hi.a - lo.a) >= 0) hi = lo;
                    lo = lp;
                }
                if (std::fabs(hi.a - lo.a) < 1e-14 * std::max(1.0, std::fabs(lo.a))) break;
            }
            return PWA_OK;
        };
        double a = 1.0;
        for (int it = 0; it < 30 && !ok; ++it) {
            st = phi(a, cur);
            if (st != PWA_OK) return st;
            if (!std::isfinite(cur.f)) {
                a = 0.5 * (prev.a + a);
                continue;
            }
            if (armijo_fails(cur) || (it > 0 && cur.f >= prev.f + eps_f)) {
                st = zoom(prev, cur);
                if (st != PWA_OK) return st;
                break;
            }
            if (std::fabs(cur.df) <= -c2 * df0) {
                found = cur;
                ok = true;
                break;
            }
            if (cur.df >= 0) {
                st = zoom(cur, prev);
                if (st != PWA_OK) return st;
                break;
            }
            prev = cur;
            a = std::min(2.0 * a, 1e3);
        }
        if (!ok) {
            status = std::fabs(df0) <= 1e-7 * (1.0 + std::fabs(f)) ? PWA_FIT_PRECISION : PWA_FIT_LINESEARCH;
            break;
        }
        double smean = 0.0;
        for (int i = 0; i < n; ++i) smean += std::fabs(found.x[i] - x[i]);
        smean /= std::max(n, 1);
        x = found.x;
        f = found.f;
        g = found.g;
        if (smean <= o.xtol) {
            status = PWA_FIT_XTOL;
            break;
        }
        if (o.time_limit_s > 0 && elapsed() > o.time_limit_s) {
            status = PWA_FIT_TIME_LIMIT;
            break;
        }
    }
    std::memcpy(theta_out, x.data(), sizeof(double) * n);
    if (result) {
        double gmax = 0.0;
        for (double v : g) gmax = std::max(gmax, std::fabs(v));
        result->nll = f;
        result->grad_max = gmax;
        result->iters = k;
        result->n_hvp = ev.n_hvp;
        result->n_fev = ev.n_fev;
        result->status = status;
        result->elapsed_s = elapsed();
    }
    const bool converged = status == PWA_FIT_XTOL || status == PWA_FIT_GTOL || status == PWA_FIT_PRECISION ||
                           status == PWA_FIT_TIME_LIMIT;
    return converged ? PWA_OK : PWA_ENOCONV;
}
