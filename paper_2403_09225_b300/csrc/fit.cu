// fit.cu -- pwa_newton_cg_fit: truncated-Newton minimisation of the NLL.
//
// The paper fits with scipy's Newton-CG (Sec. 3), i.e. the line-search
// Newton-CG of Nocedal & Wright, Numerical Optimization, Algorithm 7.1, with
// a line search for the strong Wolfe conditions (their Algorithms 3.5/3.6).
// This is an independent C++ restatement of those textbook steps driving the
// fused GPU pass: every gradient is one pass over F, every inner CG step is
// one Hessian-vector pass.  The CG scalars (dot products, curvature, step
// lengths) and all vectors are FP64.
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

struct Evaluator {
    pwa_handle* h;
    int n_fev = 0, n_hvp = 0;

    pwa_status fg(const std::vector<double>& x, double& f, std::vector<double>& g)
    {
        ++n_fev;
        return pwa_eval(h, x.data(), nullptr, &f, g.data(), nullptr);
    }
    pwa_status hessp(const std::vector<double>& x, const std::vector<double>& d, std::vector<double>& out)
    {
        ++n_hvp;
        double f;
        std::vector<double> g(x.size());
        return pwa_eval(h, x.data(), d.data(), &f, g.data(), out.data());
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

    Evaluator ev{h};
    std::vector<double> x(theta0, theta0 + n), g(n), p(n), z(n), r(n), d(n), Bd(n);
    double f = 0.0;
    pwa_status st = ev.fg(x, f, g);
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
        // ---- inner CG on H p = -g (N&W Algorithm 7.1) ----
        const double gnorm = std::sqrt(dot(g, g));
        const double eps = std::min(0.5, std::sqrt(gnorm)) * gnorm;
        std::fill(z.begin(), z.end(), 0.0);
        r = g;
        for (int i = 0; i < n; ++i) d[i] = -r[i];
        double rr = dot(r, r);
        bool have_p = false;
        for (int j = 0; j < cg_maxiter; ++j) {
            st = ev.hessp(x, d, Bd);
            if (st != PWA_OK) return st;
            const double curv = dot(d, Bd);
            if (curv <= 0) {
                if (j == 0) for (int i = 0; i < n; ++i) p[i] = -g[i];
                else p = z;
                have_p = true;
                break;
            }
            const double alpha = rr / curv;
            for (int i = 0; i < n; ++i) {
                z[i] += alpha * d[i];
                r[i] += alpha * Bd[i];
            }
            const double rr_new = dot(r, r);
            if (std::sqrt(rr_new) < eps) {
                p = z;
                have_p = true;
                break;
            }
            const double beta = rr_new / rr;
            for (int i = 0; i < n; ++i) d[i] = -r[i] + beta * d[i];
            rr = rr_new;
        }
        if (!have_p) p = z;
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
