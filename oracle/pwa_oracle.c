/*
 * pwa_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the
 * partial-wave-analysis likelihood of PWACG (arXiv:2403.09225).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header or constant with
 * the CUDA library; both read the same FP32 input arrays, which this file
 * promotes exactly to double before any arithmetic.
 *
 * What it computes (paper Sec. 2.2 and 2.3):
 *   amplitude   A_s(e) = sum_k c_k(e) F_{k,s}(e),  c_k = rho_k e^{i phi_k} BW_k(e)
 *               (Eq. 1: the coherent sum of coupling x projection; the
 *               Breit-Wigner factor BW_k = 1/(M_k^2 - m^2_{ch(k)}(e) - i M_k G_k)
 *               is the constant-width propagator that the paper leaves inside
 *               U; it is factored out here so masses and widths are fittable)
 *   intensity   I(e) = sum_s |A_s(e)|^2                        (Eq. 1, the 1/2 cancels)
 *   log-lik.    ln L = sum_data w ln I - N_d ln((1/N_mc) sum_mc I)   (Eq. 3, weights w)
 *   shards      F_m = sum_data w ln I,  G_m = sum_mc I          (Eq. 5)
 *   gradient    d lnL = sum dF_m - N_d dG / G                   (Eq. 6)
 *   Hessian     d2 lnL = sum d2F_m - N_d/G d2G + N_d/G^2 dG dG^T (Eq. 7)
 * The oracle returns NLL = -ln L and its derivatives.
 *
 * Parameter vector ("full order", 4K doubles):
 *   par[0*K + k] = rho_k, par[1*K + k] = phi_k, par[2*K + k] = M_k, par[3*K + k] = Gamma_k.
 * Input layout (identical to what the library's C ABI accepts):
 *   m2[ch*n + e]  channel invariant mass squared, ch = 0 (m12), 1 (m13), 2 (m23)
 *   F[((e*K + k)*S + s)*2 + {0,1}]  real/imag of F_{k,s}(e), FP32
 *   w[e]  data weight (NULL means 1)
 * Derivatives of c_k are written out by hand from its definition; every
 * per-event sum is a plain loop in event order.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cd;

/* Per-resonance coupling and its first/second derivatives with respect to
 * (rho, phi, M, Gamma) at one event.  d2c is symmetric, stored fully. */
typedef struct {
    cd c;
    cd dc[4];
    cd d2c[4][4];
} coupling;

static void coupling_at(double rho, double phi, double M, double G, double m2, coupling* out)
{
    const cd E = cexp(I * phi);
    const cd B = 1.0 / (M * M - m2 - I * M * G);
    const cd B2 = B * B, B3 = B2 * B;
    const cd t = 2.0 * M - I * G; /* d/dM of (M^2 - i M G) */
    /* derivatives of B = 1/(M^2 - m^2 - i M G) */
    const cd dB_dM = -B2 * t;
    const cd dB_dG = I * M * B2;
    const cd d2B_dM2 = 2.0 * B3 * t * t - 2.0 * B2;
    const cd d2B_dMdG = -2.0 * I * M * B3 * t + I * B2;
    const cd d2B_dG2 = -2.0 * M * M * B3;

    out->c = rho * E * B;
    out->dc[0] = E * B;              /* d/d rho   */
    out->dc[1] = I * rho * E * B;    /* d/d phi   */
    out->dc[2] = rho * E * dB_dM;    /* d/d M     */
    out->dc[3] = rho * E * dB_dG;    /* d/d Gamma */

    out->d2c[0][0] = 0.0;
    out->d2c[0][1] = I * E * B;
    out->d2c[0][2] = E * dB_dM;
    out->d2c[0][3] = E * dB_dG;
    out->d2c[1][1] = -rho * E * B;
    out->d2c[1][2] = I * rho * E * dB_dM;
    out->d2c[1][3] = I * rho * E * dB_dG;
    out->d2c[2][2] = rho * E * d2B_dM2;
    out->d2c[2][3] = rho * E * d2B_dMdG;
    out->d2c[3][3] = rho * E * d2B_dG2;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < a; ++b) out->d2c[a][b] = out->d2c[b][a];
}

static cd F_at(const float* F, long e, int k, int s, int K, int S)
{
    const float* p = F + (((size_t)e * K + k) * S + s) * 2;
    return (double)p[0] + I * (double)p[1];
}

/* I(e) for every event (Eq. 1 with the 1/2 dropped). */
long or_intensity(int K, int S, const int* ch, const double* par,
                  long n, const float* m2, const float* F, double* out_I)
{
    coupling cp;
    for (long e = 0; e < n; ++e) {
        double Ie = 0.0;
        for (int s = 0; s < S; ++s) {
            cd A = 0.0;
            for (int k = 0; k < K; ++k) {
                coupling_at(par[k], par[K + k], par[2 * K + k], par[3 * K + k],
                            (double)m2[(size_t)ch[k] * n + e], &cp);
                A += cp.c * F_at(F, e, k, s, K, S);
            }
            Ie += creal(A) * creal(A) + cimag(A) * cimag(A);
        }
        out_I[e] = Ie;
    }
    return 0;
}

/*
 * Per-sample sums of Eq. 5 and their derivatives, over one event sample.
 *   is_data != 0:  out[0] = sum w ln I          (F_m)
 *                  out[1] = sum w               (N_d contribution)
 *                  out[2 + p]      = sum w dI_p / I                     (dF_m)
 *                  out[2 + 4K + p] = sum w [(d2I v)_p / I - dI_p (dI.v) / I^2]  (d2F_m v)
 *                  out[2 + 8K]     = sum w (dI.v) / I
 *   is_data == 0:  out[0] = sum I               (G_m)
 *                  out[1] = n
 *                  out[2 + p]      = sum dI_p                            (dG_m)
 *                  out[2 + 4K + p] = sum (d2I v)_p                       (d2G_m v)
 *                  out[2 + 8K]     = sum dI.v
 * v may be NULL (then the HVP entries are zero).  Returns -1, or the index
 * of the first event whose intensity is not a finite positive number.
 */
long or_sample_sums(int K, int S, const int* ch, const double* par, const double* v,
                    long n, const float* m2, const float* w, const float* F,
                    int is_data, double* out)
{
    const int P = 4 * K;
    const int nout = 2 + 2 * P + 1;
    long bad = -1;
    coupling* cp = malloc(sizeof(coupling) * (size_t)K);
    cd* A = malloc(sizeof(cd) * (size_t)S);
    cd* Jv = malloc(sizeof(cd) * (size_t)S);
    double* dI = malloc(sizeof(double) * (size_t)P);
    double* Hv = malloc(sizeof(double) * (size_t)P);
    for (int i = 0; i < nout; ++i) out[i] = 0.0;

    for (long e = 0; e < n; ++e) {
        for (int k = 0; k < K; ++k)
            coupling_at(par[k], par[K + k], par[2 * K + k], par[3 * K + k],
                        (double)m2[(size_t)ch[k] * n + e], &cp[k]);
        /* A_s and the directional derivative (dA_s . v) */
        double Ie = 0.0;
        for (int s = 0; s < S; ++s) {
            cd a = 0.0, jv = 0.0;
            for (int k = 0; k < K; ++k) {
                const cd f = F_at(F, e, k, s, K, S);
                a += cp[k].c * f;
                if (v) {
                    cd dcv = 0.0;
                    for (int j = 0; j < 4; ++j) dcv += cp[k].dc[j] * v[j * K + k];
                    jv += dcv * f;
                }
            }
            A[s] = a;
            Jv[s] = jv;
            Ie += creal(a) * creal(a) + cimag(a) * cimag(a);
        }
        /* data events need a finite positive I (ln I); MC events a finite I */
        if (!isfinite(Ie) || (is_data && !(Ie > 0.0))) {
            if (bad < 0) bad = e;
        }
        /* dI_p = 2 Re sum_s conj(A_s) dA_s/dp ;
           (d2I v)_p = 2 Re sum_s [conj(dA_s/dp) (dA_s.v) + conj(A_s) (d2A_s v)_p] */
        double dIv = 0.0;
        for (int k = 0; k < K; ++k) {
            for (int j = 0; j < 4; ++j) {
                double g = 0.0, h = 0.0;
                for (int s = 0; s < S; ++s) {
                    const cd f = F_at(F, e, k, s, K, S);
                    const cd dA = cp[k].dc[j] * f;
                    g += 2.0 * creal(conj(A[s]) * dA);
                    if (v) {
                        cd d2Av = 0.0;
                        for (int i = 0; i < 4; ++i) d2Av += cp[k].d2c[j][i] * v[i * K + k];
                        d2Av *= f;
                        h += 2.0 * creal(conj(dA) * Jv[s] + conj(A[s]) * d2Av);
                    }
                }
                dI[j * K + k] = g;
                Hv[j * K + k] = h;
                if (v) dIv += g * v[j * K + k];
            }
        }
        if (is_data) {
            const double we = w ? (double)w[e] : 1.0;
            out[0] += we * log(Ie);
            out[1] += we;
            for (int p = 0; p < P; ++p) {
                out[2 + p] += we * dI[p] / Ie;
                out[2 + P + p] += we * (Hv[p] / Ie - dI[p] * dIv / (Ie * Ie));
            }
            out[2 + 2 * P] += we * dIv / Ie;
        } else {
            out[0] += Ie;
            out[1] += 1.0;
            for (int p = 0; p < P; ++p) {
                out[2 + p] += dI[p];
                out[2 + P + p] += Hv[p];
            }
            out[2 + 2 * P] += dIv;
        }
    }
    free(cp); free(A); free(Jv); free(dI); free(Hv);
    return bad;
}

/*
 * Full Hessian sums over one sample (4K x 4K, row-major), for small cases:
 *   is_data != 0: out = sum w [d2I / I - dI dI^T / I^2]   (= sum w d2 ln I, d2F_m)
 *   is_data == 0: out = sum d2I                            (d2G_m)
 * d2I_pq = 2 Re sum_s [conj(dA_s/dp) dA_s/dq + conj(A_s) d2A_s/dp dq], where
 * d2A_s/dp dq vanishes unless p and q belong to the same resonance.
 */
long or_sample_hessian(int K, int S, const int* ch, const double* par,
                       long n, const float* m2, const float* w, const float* F,
                       int is_data, double* out)
{
    const int P = 4 * K;
    long bad = -1;
    coupling* cp = malloc(sizeof(coupling) * (size_t)K);
    cd* A = malloc(sizeof(cd) * (size_t)S);
    cd* J = malloc(sizeof(cd) * (size_t)S * P);
    double* dI = malloc(sizeof(double) * (size_t)P);
    double* H = malloc(sizeof(double) * (size_t)P * P);
    memset(out, 0, sizeof(double) * (size_t)P * P);

    for (long e = 0; e < n; ++e) {
        for (int k = 0; k < K; ++k)
            coupling_at(par[k], par[K + k], par[2 * K + k], par[3 * K + k],
                        (double)m2[(size_t)ch[k] * n + e], &cp[k]);
        double Ie = 0.0;
        for (int s = 0; s < S; ++s) {
            cd a = 0.0;
            for (int k = 0; k < K; ++k) {
                const cd f = F_at(F, e, k, s, K, S);
                a += cp[k].c * f;
                for (int j = 0; j < 4; ++j) J[(size_t)s * P + j * K + k] = cp[k].dc[j] * f;
            }
            A[s] = a;
            Ie += creal(a) * creal(a) + cimag(a) * cimag(a);
        }
        /* data events need a finite positive I (ln I); MC events a finite I */
        if (!isfinite(Ie) || (is_data && !(Ie > 0.0))) {
            if (bad < 0) bad = e;
        }
        for (int p = 0; p < P; ++p) {
            double g = 0.0;
            for (int s = 0; s < S; ++s) g += 2.0 * creal(conj(A[s]) * J[(size_t)s * P + p]);
            dI[p] = g;
        }
        for (int p = 0; p < P; ++p) {
            const int jp = p / K, kp = p % K;
            for (int q = 0; q < P; ++q) {
                const int jq = q / K, kq = q % K;
                double h = 0.0;
                for (int s = 0; s < S; ++s) {
                    h += 2.0 * creal(conj(J[(size_t)s * P + p]) * J[(size_t)s * P + q]);
                    if (kp == kq)
                        h += 2.0 * creal(conj(A[s]) * cp[kp].d2c[jp][jq] * F_at(F, e, kp, s, K, S));
                }
                H[(size_t)p * P + q] = h;
            }
        }
        if (is_data) {
            const double we = w ? (double)w[e] : 1.0;
            for (int p = 0; p < P; ++p)
                for (int q = 0; q < P; ++q)
                    out[(size_t)p * P + q] += we * (H[(size_t)p * P + q] / Ie - dI[p] * dI[q] / (Ie * Ie));
        } else {
            for (size_t i = 0; i < (size_t)P * P; ++i) out[i] += H[i];
        }
    }
    free(cp); free(A); free(J); free(dI); free(H);
    return bad;
}

/*
 * NLL = -ln L and its derivatives, all in the full 4K parameter order,
 * assembled from the per-sample sums by Eqs. 4, 6 and 7:
 *   NLL  = -F + N_d ln(G / N_mc)
 *   grad = -dF + N_d dG / G
 *   Hv   = -(d2F v) + N_d [ (d2G v) / G - dG (dG.v) / G^2 ]
 * grad and hv may be NULL.  v is required when hv is not NULL.
 * Returns -1, or the first offending event index (data events first, then
 * MC events offset by n_data).
 */
long or_nll(int K, int S, const int* ch, const double* par, const double* v,
            long nd, const float* m2d, const float* wd, const float* Fd,
            long nm, const float* m2m, const float* Fm,
            double* nll, double* grad, double* hv)
{
    const int P = 4 * K;
    const int nout = 2 + 2 * P + 1;
    double* sd = malloc(sizeof(double) * (size_t)nout);
    double* sm = malloc(sizeof(double) * (size_t)nout);
    long bd = or_sample_sums(K, S, ch, par, hv ? v : NULL, nd, m2d, wd, Fd, 1, sd);
    long bm = or_sample_sums(K, S, ch, par, hv ? v : NULL, nm, m2m, NULL, Fm, 0, sm);
    const double Fsum = sd[0], Nd = sd[1], G = sm[0], Nmc = (double)nm;
    *nll = -Fsum + Nd * log(G / Nmc);
    if (grad)
        for (int p = 0; p < P; ++p) grad[p] = -sd[2 + p] + Nd * sm[2 + p] / G;
    if (hv) {
        const double dGv = sm[2 + 2 * P];
        for (int p = 0; p < P; ++p)
            hv[p] = -sd[2 + P + p] + Nd * (sm[2 + P + p] / G - sm[2 + p] * dGv / (G * G));
    }
    free(sd); free(sm);
    if (bd >= 0) return bd;
    if (bm >= 0) return nd + bm;
    return -1;
}

/* Full NLL Hessian (4K x 4K) by Eq. 7:
 *   H = -d2F + N_d [ d2G / G - dG dG^T / G^2 ]. */
long or_hessian(int K, int S, const int* ch, const double* par,
                long nd, const float* m2d, const float* wd, const float* Fd,
                long nm, const float* m2m, const float* Fm, double* H)
{
    const int P = 4 * K;
    const int nout = 2 + 2 * P + 1;
    double* sd = malloc(sizeof(double) * (size_t)nout);
    double* sm = malloc(sizeof(double) * (size_t)nout);
    double* Hd = malloc(sizeof(double) * (size_t)P * P);
    double* Hm = malloc(sizeof(double) * (size_t)P * P);
    long bd = or_sample_sums(K, S, ch, par, NULL, nd, m2d, wd, Fd, 1, sd);
    long bm = or_sample_sums(K, S, ch, par, NULL, nm, m2m, NULL, Fm, 0, sm);
    or_sample_hessian(K, S, ch, par, nd, m2d, wd, Fd, 1, Hd);
    or_sample_hessian(K, S, ch, par, nm, m2m, NULL, Fm, 0, Hm);
    const double Nd = sd[1], G = sm[0];
    for (int p = 0; p < P; ++p)
        for (int q = 0; q < P; ++q)
            H[(size_t)p * P + q] = -Hd[(size_t)p * P + q]
                + Nd * (Hm[(size_t)p * P + q] / G - sm[2 + p] * sm[2 + q] / (G * G));
    free(sd); free(sm); free(Hd); free(Hm);
    if (bd >= 0) return bd;
    if (bm >= 0) return nd + bm;
    return -1;
}

/*
 * Integral matrix of the fixed-mass coupling problem (Eq. 1 written as a sum
 * over coupling pairs: with U_{k,s}(e) = BW_k(e) F_{k,s}(e) and c_k = g_k BW_k,
 * sum_e I(e) = sum_{k,k'} conj(g_k) g_{k'} Phi_{k k'}):
 *   Phi_{k k'} = sum_e sum_s conj(U_{k,s}(e)) U_{k',s}(e),
 * at the masses and widths of par (its couplings are not used).
 * out[(k*K + k')*2 + {0,1}] = real/imag of Phi_{k k'}.
 */
long or_integral_matrix(int K, int S, const int* ch, const double* par,
                        long n, const float* m2, const float* F, double* out)
{
    cd* phi = (cd*)calloc((size_t)K * K, sizeof(cd));
    cd* U = (cd*)malloc((size_t)K * S * sizeof(cd));
    if (!phi || !U) {
        free(phi);
        free(U);
        return -2;
    }
    coupling cp;
    for (long e = 0; e < n; ++e) {
        for (int k = 0; k < K; ++k) {
            /* rho = 1, phi = 0: the coupling is BW_k itself */
            coupling_at(1.0, 0.0, par[2 * K + k], par[3 * K + k], (double)m2[(size_t)ch[k] * n + e], &cp);
            for (int s = 0; s < S; ++s) U[k * S + s] = cp.c * F_at(F, e, k, s, K, S);
        }
        for (int k = 0; k < K; ++k)
            for (int kp = 0; kp < K; ++kp)
                for (int s = 0; s < S; ++s) phi[k * K + kp] += conj(U[k * S + s]) * U[kp * S + s];
    }
    for (int i = 0; i < K * K; ++i) {
        out[2 * i] = creal(phi[i]);
        out[2 * i + 1] = cimag(phi[i]);
    }
    free(phi);
    free(U);
    return -1;
}
