/*
 * pwa.h -- libpwa: the unbinned extended negative log-likelihood of a
 * partial-wave analysis, its gradient, its Hessian-vector products and the
 * Newton-conjugate-gradient fit they drive, evaluated on one B300 GPU.
 *
 * The method is that of PWACG (arXiv:2403.09225):
 *   Eq. 1  omega(xi) ~ sum_mu |A^mu|^2 with A^mu = sum_m Lambda_m U_m^mu
 *          (here: I(e) = sum_s |A_s(e)|^2, A_s = sum_k c_k(e) F_{k,s}(e),
 *           c_k = g_k BW_k(e), g_k = rho_k e^{i phi_k},
 *           BW_k = 1 / (M_k^2 - m^2_{ch(k)}(e) - i M_k Gamma_k));
 *   Eq. 2  normalisation by the phase-space MC sample (efficiency folded in);
 *   Eq. 3  ln L = sum_data w ln I - N_d ln((1/N_mc) sum_mc I), N_d = sum_data w;
 *   Eqs. 4-7  the decomposition of ln L, its gradient and its Hessian into
 *          per-shard sums F_m, G_m and their derivatives.
 * The library minimises NLL = -ln L.  F (the parameter-free projections U of
 * Eq. 1) is precomputed by the caller and kept resident on the device (the
 * paper's Sec. 2.2 does the same).
 *
 * Conventions for every call:
 *  - Return value is a pwa_status; no C++ exception crosses this boundary.
 *  - Calls are synchronous with respect to the handle's CUDA stream: results
 *    are valid on return.  The *_device variants are asynchronous (enqueued on
 *    the handle's stream) and read/write device memory only.
 *  - Pointers marked "host" are ordinary host memory, "device" is CUDA device
 *    memory; "either" is resolved by the on_device flag of the struct.
 *  - The caller keeps ownership of every buffer it passes; the library copies
 *    what it needs during pwa_create and never retains caller pointers.
 *  - On error, pwa_last_error(handle) describes the first failure of the last
 *    call (for pwa_create, the message is returned through *out when a handle
 *    could be allocated, otherwise via pwa_last_create_error()).
 *
 * Parameter vector theta (host or device FP64, length P = pwa_num_params):
 *   the free magnitudes rho_k, then the free phases phi_k, then the free masses
 *   M_k, then the free widths Gamma_k, each block in resonance order.  With the
 *   usual choice (resonance 0's coupling fixed to 1, everything else free)
 *   P = 4K - 2 and theta = (rho_1..rho_{K-1}, phi_1..phi_{K-1}, M_0..M_{K-1},
 *   Gamma_0..Gamma_{K-1}).
 *
 * Besides the likelihood handle: pwa_coupling (the fixed-mass coupling
 * sub-problem on the tensor cores), pwa_variant (other line shapes and one
 * coupling per projection), the pseudo-experiment generator calls and
 * pwa_mlp (the learned starting-point proposal's network).  Each section
 * below states its own arguments and errors; the conventions above hold for
 * all of them.
 */
#ifndef LIBPWA_PWA_H
#define LIBPWA_PWA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pwa_handle pwa_handle; /* opaque; owned by the library */

typedef enum {
    PWA_OK = 0,
    PWA_EINVAL = 1,      /* bad argument (shape, range, NULL, non-finite input)   */
    PWA_ENOMEM = 2,      /* device or pinned host allocation failed               */
    PWA_ECUDA = 3,       /* a CUDA runtime call failed (message has the details)  */
    PWA_ENONFINITE = 4,  /* an event's intensity is not finite, or not positive for
                            data; pwa_last_error names the first such event index
                            (data events 0..N_d-1, MC events N_d..N_d+N_mc-1)      */
    PWA_ENOCONV = 5,     /* the fit stopped without converging (see result.status) */
    PWA_ETIMEOUT = 6     /* a bounded device-side wait ran out; the handle must be
                            destroyed (its device state is no longer consistent)  */
} pwa_status;

/* One event sample (paper Eq. 3: data; Eq. 2: phase-space MC).
 *   n          number of events (>= 1)
 *   m2         [3][n] FP32, channel-major: m12^2, m13^2, m23^2 in GeV^2
 *   w          [n] FP32 data weights, or NULL for unit weights; must be NULL
 *              for the MC sample (its events enter G = sum I unweighted)
 *   F          [n][K][S] complex FP32, interleaved (re, im): F_{k,s}(e)
 *   on_device  0: the three pointers are host memory; 1: device memory      */
typedef struct {
    int64_t n;
    const float* m2;
    const float* w;
    const float* F;
    int on_device;
} pwa_events;

/* One resonance k.  channel: 0 = m12, 1 = m13, 2 = m23 (which m^2 enters
 * BW_k); spin is informational (the angular part is inside F).  mass, width
 * in GeV; mag, phase: the coupling g_k = mag e^{i phase}.  A fixed parameter
 * keeps the value given here and is left out of theta; fix_coupling fixes
 * both mag and phase. */
typedef struct {
    int channel;
    int spin;
    double mass, width;
    double mag, phase;
    int fix_coupling, fix_mass, fix_width;
} pwa_resonance;

/* One outer Newton iteration of a fit, as recorded when the caller asks for
 * a trace (pwa_fit_opts.trace).  cg_exit: 1 negative curvature, 2 residual
 * below the forcing tolerance, 3 inner iteration limit, 4 trust-region
 * boundary (method 1). */
typedef struct pwa_fit_iter {
    double nll;        /* NLL at the start of the iteration                     */
    double grad_max;   /* max |grad| there                                      */
    double cg_eps;     /* forcing tolerance min(0.5, sqrt|g|) |g| of the CG     */
    double cg_res;     /* |r| of the inner CG when it stopped                   */
    double step;       /* accepted line-search step length (0: none found)      */
    double dir_deriv;  /* g . p along the Newton direction                      */
    int cg_iters;      /* inner CG iterations (one H v each)                    */
    int cg_exit;       /* why the inner CG stopped (see above)                  */
    int n_fev;         /* line-search evaluations (one pass each)               */
    int hessian;       /* 1 when H came from an explicit Hessian pass           */
} pwa_fit_iter;

/* Options of pwa_newton_cg_fit (paper Sec. 3: scipy's Newton-CG with xtol,
 * default 1e-8, and early stopping after 500 s). */
typedef struct {
    double xtol;          /* stop when mean |delta theta| of a step <= xtol (1e-8) */
    double gtol;          /* stop when max |grad| <= gtol (0: off)                 */
    int maxiter;          /* outer iterations (0: 200 P)                            */
    int cg_maxiter;       /* inner CG iterations per outer step (0: 20 P)           */
    double time_limit_s;  /* wall-clock limit, 0: none (the paper uses 500 s)       */
    int matrix_free;      /* 1: every inner CG step is one fused H v pass (the
                             paper's setup); 0: one Hessian pass (pwa_hessian)
                             per outer iteration and the CG on its products --
                             the same iteration, far fewer passes over F (the
                             default; handles with K > 44 and the coupling and
                             variant fits always run matrix-free)            */
    int method;           /* 0: line-search Newton-CG (Nocedal & Wright Alg. 7.1,
                             scipy's Newton-CG, the paper's method; default);
                             1: trust-region Newton-CG (Alg. 7.2, CG-Steihaug,
                             scipy's trust-ncg): the CG stops on the region's
                             boundary instead of on negative curvature, one
                             f, g evaluation per outer iteration            */
    int trace_cap;        /* records per fit that trace can hold (0: no trace)      */
    pwa_fit_iter* trace;  /* host [fits][trace_cap] or NULL: per-iteration record;
                             fits are numbered in the order of theta0 (over all
                             handles in order for pwa_newton_cg_fit_multi)     */
    int one_launch;       /* pwa_newton_cg_fit_multi only: 1: every f, g round is
                             one pwa_eval_multi_device launch over all handles
                             (when each has K <= 32); 0 (default): one batched
                             launch per handle, each on its own stream (faster
                             on the measured toys: the per-handle instances
                             are tuned for their K, S)                        */
} pwa_fit_opts;

typedef enum {
    PWA_FIT_XTOL = 0,        /* converged: step below xtol                         */
    PWA_FIT_GTOL = 1,        /* converged: gradient below gtol                     */
    PWA_FIT_MAXITER = 2,     /* outer iteration limit reached                      */
    PWA_FIT_TIME_LIMIT = 3,  /* time_limit_s reached (early stopping)              */
    PWA_FIT_LINESEARCH = 4,  /* no step satisfied the Wolfe conditions             */
    PWA_FIT_PRECISION = 5,   /* converged: predicted decrease below the NLL's
                                resolution, no further step can be resolved, or
                                the fit stalled at its rounding floor (25 outer
                                iterations without a 1 % lower |grad| or an NLL
                                drop above ten times its resolution)               */
    PWA_FIT_ERROR = 6        /* stopped on an error (e.g. a non-finite NLL at its
                                start point); only pwa_newton_cg_fit_batch reports
                                it per fit, pwa_newton_cg_fit returns the error    */
} pwa_fit_status;

typedef struct {
    double nll;       /* NLL at theta_out                                  */
    double grad_max;  /* max |grad| at theta_out                           */
    int iters;        /* outer Newton iterations                           */
    int n_hvp;        /* Hessian-vector products (one pass over F each)    */
    int n_fev;        /* NLL+gradient evaluations (one pass over F each)   */
    int status;       /* pwa_fit_status                                    */
    double elapsed_s; /* wall-clock seconds inside the call                */
    int n_trace;      /* iterations recorded in opts->trace (<= trace_cap) */
    int n_hess;       /* Hessian passes (one pass over F each)             */
} pwa_fit_result;

/* Build a likelihood handle.  Copies data and MC events to the device and
 * re-lays F out in event tiles for the streaming kernel; validates that
 * K >= 1, 1 <= S <= 4, both samples are non-empty, channels are 0..2, every
 * m2, F and w value is finite, weights are >= 0, masses and widths are finite
 * and positive.  cuda_stream: a cudaStream_t, or NULL for the default stream.
 * Errors: PWA_EINVAL, PWA_ENOMEM, PWA_ECUDA.  On error *out is set to NULL. */
pwa_status pwa_create(pwa_handle** out, const pwa_events* data, const pwa_events* mc,
                      const pwa_resonance* table, int K, int S, void* cuda_stream);

/* Message of the last pwa_create failure in this thread ("" if none). */
const char* pwa_last_create_error(void);

/* Free the device copies of the caller's events in the ABI layout that
 * pwa_create keeps beside the tiled layout the passes stream (no counterpart
 * in the paper: a memory option).  Halves the handle's device memory (2 x F
 * -> 1 x F plus the tiles' m^2 and w); afterwards the tiling is fixed
 * (pwa_set_tiling and pwa_autotune return PWA_EINVAL) and pwa_coupling_create
 * refuses the handle.  Every pass, the Hessian pass and the fits are
 * unaffected.  Idempotent. */
pwa_status pwa_release_event_copies(pwa_handle* h);

/* Device bytes the handle holds: event copies (unless released), tiles,
 * reduction and batch scratch, Hessian records. */
pwa_status pwa_device_bytes(const pwa_handle* h, long long* out);

/* Number of free parameters P (length of theta, grad, v, hv). */
int pwa_num_params(const pwa_handle* h);

/* NLL = -ln L at theta (Eq. 3, negated).  theta: host [P]; nll: host. */
pwa_status pwa_nll(pwa_handle* h, const double* theta, double* nll);

/* Gradient of NLL at theta (Eq. 6, negated); nll_or_null also receives NLL.
 * theta: host [P]; grad: host [P]. */
pwa_status pwa_grad(pwa_handle* h, const double* theta, double* nll_or_null, double* grad);

/* Hessian-vector product H v of NLL at theta (Eq. 7 contracted with v).
 * theta, v, hv: host [P]. */
pwa_status pwa_hvp(pwa_handle* h, const double* theta, const double* v, double* hv);

/* The full Hessian of NLL at theta (Eq. 7 written out without the
 * contraction with a direction), with NLL and its gradient, from one pass
 * over F.  Per event it accumulates weighted Gram matrices of the first
 * derivatives of the coherent sums (B F and B^2 F for every resonance and
 * projection) and of the adjoint terms B^p D_k, plus the resonance-diagonal
 * second-derivative sums; the host combines them in FP64.  theta: host [P];
 * nll, grad: host (either may be NULL); hess: host [P][P] row-major,
 * symmetric.  For K <= 32 the Gram matrices are contractions on the tensor
 * cores (tcgen05, BF16 hi/lo splits of the FP32 columns, two products per
 * 16 rows (hi^T hi + hi^T 2lo, symmetrised), a fresh TMEM accumulator per
 * 32-event tile, tiles pipelined over two buffers, FP32 then FP64 sums
 * across tiles); for 32 < K <= 44 on the CUDA cores in FP32.  Supported for
 * K <= 44.  Errors: PWA_EINVAL (K > 44, non-finite theta), PWA_ENOMEM,
 * PWA_ECUDA, PWA_ENONFINITE, PWA_ETIMEOUT. */
pwa_status pwa_hessian(pwa_handle* h, const double* theta, double* nll, double* grad, double* hess);

/* pwa_hessian for B parameter vectors in one launch (Eq. 7 as above, for
 * each vector): the vectors share one wave of CTAs, each CTA working for one
 * vector on its share of the tiles.  theta: host [B][P]; nll: host [B] or
 * NULL; grad: host [B][P] or NULL; hess: host [B][P][P].  status: host [B]
 * or NULL; when given, a vector with a non-finite intensity gets
 * PWA_ENONFINITE there (its outputs are left untouched) and the others are
 * still combined; when NULL such a vector fails the call.  Errors as
 * pwa_hessian, plus PWA_EINVAL for B < 1. */
pwa_status pwa_hessian_batch(pwa_handle* h, int B, const double* theta, double* nll, double* grad, double* hess,
                             pwa_status* status);

/* Run the Hessian pass's Gram matrices on the CUDA cores (cuda_cores = 1)
 * even where the tensor-core kernel applies (K <= 32), for comparisons;
 * 0 restores the default. */
pwa_status pwa_set_hessian_cuda_cores(pwa_handle* h, int cuda_cores);

/* The fused pass: NLL, gradient and H v from one read of F.  Any of grad,
 * hv may be NULL (then the cheaper pass without them runs); v is required
 * when hv is not NULL.  All pointers host. */
pwa_status pwa_eval(pwa_handle* h, const double* theta, const double* v,
                    double* nll, double* grad, double* hv);

/* Asynchronous fused pass on device buffers, enqueued on the handle's stream.
 * d_theta [P], d_v [P] (may be NULL when hv is not wanted), d_out [1 + 2P]
 * receives (NLL, grad[P], hv[P]); with want_hv == 0 the hv part is left
 * untouched and v is not read; with want_grad == 0 only NLL is written.
 * Errors detected on the device (non-finite intensity, wait timeout) are
 * reported by the next synchronous call or by pwa_sync(). */
pwa_status pwa_eval_device(pwa_handle* h, const double* d_theta, const double* d_v,
                           double* d_out, int want_grad, int want_hv);

/* H v at theta from a cheaper pass that reuses what the last full H v pass
 * (pwa_eval or pwa_hvp with hv, pwa_eval_device with want_hv, or the
 * Newton-CG inner loop) computed at the SAME theta: in Eq. 7 only the sums
 * of the direction derivatives (P1 = sum a Ddot_t B, P2 = sum a Ddot_t B^2
 * with Ddot_t = a Ddot - b D) and Gdot depend on v; the Q sums, G, sum w ln I
 * and the gradient do not.  So the pass accumulates 4 reals per resonance
 * instead of 10 and, on MC events, skips the coherent sum A and the adjoint D
 * (only Adot and Ddot are formed); Gdot = (dG/dtheta) . v from the kept
 * sums.  This is the product a conjugate-gradient solve repeats at one
 * theta.  Returns the same H v as the full pass to the pass's own accuracy.
 * If the last full pass was at another theta (checked on the device, exact
 * comparison), the call fails: PWA_EINVAL (host call), or the device error
 * reported by pwa_sync (device call; d_out is then NaN).  theta, v, hv: host
 * [P]; d_theta, d_v: device [P]; d_out: device [1 + 2P] (NLL, gradient,
 * H v as pwa_eval_device writes them). */
pwa_status pwa_hvp_reuse(pwa_handle* h, const double* theta, const double* v, double* hv);
pwa_status pwa_hvp_reuse_device(pwa_handle* h, const double* d_theta, const double* d_v, double* d_out);

/* pwa_eval_device without any device allocation (the paper has no
 * counterpart: this is a deployment variant).  For callers that may not call
 * cudaMalloc while they evaluate -- e.g. code under an external memory manager
 * that has reserved the device's memory, or a loop that must not take the
 * device-wide synchronisation an allocation can imply.  Same arguments,
 * result and asynchrony as pwa_eval_device (errors are reported by pwa_sync);
 * the handle is still created beforehand with pwa_create, which allocates.
 * The reduction scratch (per-block and per-group partial sums, completion
 * counters) lives in one statically allocated 2 MiB device array that every
 * GPU loading the library holds until exit; a handle needing more
 * (grid blocks + groups) x (20 K + 6) x 8 bytes + counters is refused with
 * PWA_EINVAL.  The array's device address is looked up on the first call on
 * each device and kept for the life of the process: make that first call
 * before any stream capture, and do not use this entry point after a
 * cudaDeviceReset in the same process (the kept address belongs to the
 * destroyed context).  All calls
 * share the array and the counters are cleared at each call, so calls whose
 * kernels overlap on the GPU (e.g. on different streams) race and must not be
 * issued concurrently. */
pwa_status pwa_eval_device_noalloc(pwa_handle* h, const double* d_theta, const double* d_v,
                                   double* d_out, int want_grad, int want_hv);

/* Batched fused pass: B parameter vectors over the same events in one launch
 * (multi-start and toy fits evaluate many parameter points of one model; the
 * paper runs its 300 random starts one after another, Sec. 4).  Each vector's
 * result is the same function value, gradient and H v as pwa_eval at that
 * vector (the event sums are split over a different block grid, so the FP32
 * partial sums round differently: agreement to the pass's own accuracy, not
 * bit for bit).  theta: host [B][P] row-major; v: host [B][P] or NULL; nll:
 * host [B]; grad, hv: host [B][P] or NULL (hv needs v).  B >= 1.  Grows the
 * handle's batch scratch when B exceeds what earlier calls used.
 * Errors: PWA_EINVAL, PWA_ENOMEM, PWA_ECUDA, PWA_ENONFINITE, PWA_ETIMEOUT. */
pwa_status pwa_eval_batch(pwa_handle* h, int B, const double* theta, const double* v,
                          double* nll, double* grad, double* hv);

/* Asynchronous batched pass on device buffers, enqueued on the handle's
 * stream: d_theta [B][P], d_v [B][P] (NULL when hv is not wanted), d_out
 * [B][1 + 2P] (row b receives (NLL, grad[P], hv[P]) of vector b, with the
 * same want_grad / want_hv rules as pwa_eval_device).  May allocate batch
 * scratch (and then synchronises the stream) when B or the grid grows. */
pwa_status pwa_eval_batch_device(pwa_handle* h, int B, const double* d_theta, const double* d_v,
                                 double* d_out, int want_grad, int want_hv);

/* Wait for the handle's stream and report device-side errors of earlier
 * asynchronous calls. */
pwa_status pwa_sync(pwa_handle* h);

/* Per-event intensity I(e) = sum_s |A_s(e)|^2 (Eq. 1) of the handle's data
 * (sample = 0) or MC (sample = 1) events at theta (host [P]), in event order.
 * out: [n] FP32, host (out_on_device = 0) or device (1). */
pwa_status pwa_event_intensity(pwa_handle* h, int sample, const double* theta,
                               float* out, int out_on_device);

/* Newton-CG fit from theta0 (host [P]); theta_out (host [P]) receives the
 * final point (it may alias theta0).  opts may be NULL (defaults).  Returns
 * PWA_OK when the fit converged or hit its time limit (result->status says
 * which), PWA_ENOCONV when it stopped otherwise, or an error status. */
pwa_status pwa_newton_cg_fit(pwa_handle* h, const double* theta0, const pwa_fit_opts* opts,
                             double* theta_out, pwa_fit_result* result);

/* B Newton-CG fits of the same model (multi-start or repeated fits), run in
 * lockstep so that each round of likelihood evaluations -- one per unfinished
 * fit, f and g for the line search or H v for the inner CG -- is one batched
 * launch (pwa_eval_batch_device); the paper's multi-start runs its starts one
 * after another (Sec. 4).  Each fit follows the same iteration as
 * pwa_newton_cg_fit, with the inner CG's FP64 vector arithmetic on the host
 * instead of on the device (so the two may differ in the last bits and, on a
 * flat or multimodal surface, in where they stop).  theta0, theta_out: host
 * [B][P] (may alias); results: host [B] or NULL; opts apply to every fit (the
 * time limit to each fit's wall time since the call began).  Returns PWA_OK
 * when every fit converged or hit its time limit, PWA_ENOCONV when some fit
 * stopped otherwise (its result says why, PWA_FIT_ERROR for a fit whose start
 * point has a non-finite NLL), or an error status that stopped all fits. */
pwa_status pwa_newton_cg_fit_batch(pwa_handle* h, int B, const double* theta0,
                                   const pwa_fit_opts* opts, double* theta_out,
                                   pwa_fit_result* results);

/* One launch of the batched pass over several handles (no counterpart in the
 * paper, which fits its samples one after another): handle i evaluates B[i]
 * parameter vectors d_theta[i] ([B[i]][P_i], device) and writes d_out[i]
 * ([B[i]][1 + 2 P_i], device) as pwa_eval_batch_device does, with d_v[i]
 * ([B[i]][P_i]) when want_hv.  The work list of the launch is every (handle,
 * vector, block) of those batched passes; persistent CTAs walk it, running
 * one compiled instance per S with K a runtime value, so toys of different
 * sizes, K and S share one launch.  Every handle needs K <= 32 and a handle
 * may appear once.  Enqueued on `stream` (a cudaStream_t, NULL = default)
 * after the handles' earlier work on it; errors found on the device (per
 * vector and per handle) are reported by pwa_sync(handle) once the stream
 * has been synchronised.  Grows each handle's batch scratch as
 * pwa_eval_batch_device does.  want_grad or want_hv must be set.
 * pwa_newton_cg_fit_multi uses this launch for its rounds when asked to
 * (pwa_fit_opts.one_launch) and every handle has K <= 32. */
pwa_status pwa_eval_multi_device(int n, pwa_handle* const* handles, const int* B, const double* const* d_theta,
                                 const double* const* d_v, double* const* d_out, int want_grad, int want_hv,
                                 void* stream);

/* Lockstep fits over several handles (toy fits: different event samples,
 * sizes, K and S), B[i] fits on handles[i].  Every round issues one batched
 * pass per handle, each on a private stream of that handle, so the handles'
 * kernels run concurrently; each fit's arithmetic is that of
 * pwa_newton_cg_fit_batch on its own handle (results are identical to calling
 * it per handle).  theta0[i], theta_out[i]: host [B[i]][P_i]; results[i]: host
 * [B[i]] (results may be NULL).  A handle may appear only once.  Returns as
 * pwa_newton_cg_fit_batch; an error on one handle (its pwa_last_error says
 * which) stops all fits.  A round's f, g requests are one batched launch per
 * handle, each on its own stream; with opts->one_launch and every handle at
 * K <= 32 they are instead one pwa_eval_multi_device launch over all handles
 * (captured into a CUDA graph once its shape repeats).  Either way, each
 * handle's Hessian requests of a round are one batched Hessian pass. */
pwa_status pwa_newton_cg_fit_multi(int n_handles, pwa_handle* const* handles, const int* B,
                                   const double* const* theta0, const pwa_fit_opts* opts,
                                   double* const* theta_out, pwa_fit_result* const* results);

/* ---- fixed-mass coupling sub-problem (tensor cores) ----
 *
 * With every mass and width held at given values, U_{k,s}(e) = BW_k(e)
 * F_{k,s}(e) is fixed and the coherent sum of Eq. 1 is linear in the
 * couplings g_k = rho_k e^{i phi_k}: A_s(e) = sum_k g_k U_{k,s}(e).  The MC
 * normalisation becomes g^H Phi g with the K x K Hermitian integral matrix
 * Phi_{kk'} = sum_mc sum_s conj(U_{k,s}) U_{k',s} (computed once), and the
 * data term for many coupling vectors is a pair of GEMMs per tile of events,
 * run on the tensor cores (tcgen05 kind::f16: every FP32 operand split into
 * three BF16 parts, which represent it exactly, and the six part products
 * with i + j <= 2 accumulated in FP32 in tensor memory, the leading products
 * apart from the corrections; FP64 across tiles).  The MC events are not
 * read after the object is created.
 *
 * The coupling parameters are the first Pc entries of theta (the free
 * magnitudes, then the free phases, in resonance order); the object keeps the
 * masses, widths and fixed couplings of the theta it was created from.
 * Supported for K <= 24 (one tile's operands must fit in shared memory). */
typedef struct pwa_coupling pwa_coupling; /* opaque; owned by the library */

/* Fix the masses and widths at theta (host [P]); lay the data events out as
 * U tiles on the device and compute Phi from the MC events.  The object
 * refers to h (destroy it before h).  Errors: PWA_EINVAL (K > 24), PWA_ENOMEM,
 * PWA_ECUDA, PWA_ETIMEOUT. */
pwa_status pwa_coupling_create(pwa_handle* h, const double* theta, pwa_coupling** out);

/* Pc: the number of coupling parameters (free magnitudes and phases). */
int pwa_coupling_num_params(const pwa_coupling* cp);

/* The integral matrix: phi [K][K][2] (real, imaginary), host. */
pwa_status pwa_coupling_integral_matrix(const pwa_coupling* cp, double* phi);

/* NLL, its gradient and H v with respect to the coupling parameters for C
 * coupling vectors (rows of theta_c, host [C][Pc]) at the fixed masses and
 * widths: the same values as pwa_eval at the full theta restricted to the
 * coupling block (Eqs. 3, 6, 7), up to FP32 summation.  v: host [C][Pc] or
 * NULL (then hv must be NULL); nll: host [C]; grad, hv: host [C][Pc] or NULL.
 * Vectors are evaluated 16 per launch.  Errors: PWA_EINVAL, PWA_ECUDA,
 * PWA_ENONFINITE (a data event with I <= 0 or non-finite), PWA_ETIMEOUT. */
pwa_status pwa_coupling_eval(pwa_coupling* cp, int C, const double* theta_c, const double* v,
                             double* nll, double* grad, double* hv);

/* Newton-CG fits in the coupling parameters alone (masses and widths fixed),
 * C of them in lockstep: every round of likelihood requests is one call of the
 * tensor-core evaluation above.  The iteration is that of pwa_newton_cg_fit
 * (host-side CG as in pwa_newton_cg_fit_batch).  theta_c0, theta_c_out: host
 * [C][Pc] (may alias); results: host [C] or NULL.  Returns as
 * pwa_newton_cg_fit_batch. */
pwa_status pwa_coupling_fit(pwa_coupling* cp, int C, const double* theta_c0, const pwa_fit_opts* opts,
                            double* theta_c_out, pwa_fit_result* results);

void pwa_coupling_destroy(pwa_coupling* cp);

/* ---- physics variants (paper Sec. 2.2, Eq. 1 with other line shapes and
 * couplings; Eqs. 3, 6, 7 for the likelihood, gradient and H v) ----
 *
 * BW_k = 1 / D_k with m^2 the channel invariant of resonance k:
 *   PWA_SHAPE_CONSTANT        D = M^2 - m^2 - i M Gamma (the main path's form)
 *   PWA_SHAPE_MASS_DEPENDENT  D = M^2 - m^2 - i M Gamma(m),
 *       Gamma(m) = Gamma0 (q(m)/q(M)) (M/m) (F_L(q(m))/F_L(q(M)))^2, q the
 *       breakup momentum of the daughters (ma, mb), F_L the von Hippel-Quigg
 *       barrier factor (unnormalised, z = (q radius)^2) of the resonance's
 *       spin L = pwa_resonance.spin (0..4); M must stay above ma + mb
 *   PWA_SHAPE_FLATTE          D = M^2 - m^2 - i (gamma1 rho1(m) + gamma2 rho2(m)),
 *       rho_i = 2 q_i / m for the channel masses (ma, mb) and (mc, md),
 *       q_i = i sqrt(-q_i^2) below a channel's threshold
 * The table's width is Gamma, Gamma0 or gamma1; width2 gives gamma2.
 * per_projection = 1 gives every (resonance, projection) its own coupling
 * g_ks = mag e^{i phase} (A_s = sum_k g_ks BW_k F_ks; each projection's
 * overall phase is then unobservable, so fix the couplings of one resonance).
 * theta order: free magnitudes (resonance-major, then projection), free
 * phases (same order), free masses, free widths (Gamma, Gamma0 or gamma1),
 * free gamma2 of the Flatte resonances; fix_coupling fixes all couplings of
 * a resonance, fix_width both width parameters. */
enum { PWA_SHAPE_CONSTANT = 0, PWA_SHAPE_MASS_DEPENDENT = 1, PWA_SHAPE_FLATTE = 2 };

typedef struct {
    int kind;           /* PWA_SHAPE_*                                        */
    double ma, mb;      /* daughter masses (Flatte: channel 1), GeV           */
    double mc, md;      /* Flatte channel 2 masses, GeV                       */
    double radius;      /* barrier radius, GeV^-1 (mass-dependent width)      */
    double width2;      /* Flatte gamma2 (start or fixed value)               */
} pwa_lineshape;

typedef struct pwa_variant pwa_variant; /* opaque; owned by the library */

/* Build a variant likelihood: events as for pwa_create (copied to the device),
 * shapes [K] (NULL: all constant width), K <= 32, S <= 4.
 * Errors: PWA_EINVAL, PWA_ENOMEM, PWA_ECUDA (message: pwa_variant_last_error(NULL)). */
pwa_status pwa_variant_create(pwa_variant** out, const pwa_events* data, const pwa_events* mc,
                              const pwa_resonance* table, const pwa_lineshape* shapes, int K, int S,
                              int per_projection, void* cuda_stream);

int pwa_variant_num_params(const pwa_variant* v);

/* NLL, and the gradient [P] and H v [P] when the pointers are non-NULL (hv
 * needs v), in one pass over the events (host arrays; synchronous).
 * Errors: PWA_EINVAL (bad theta, a mass below its pair threshold),
 * PWA_ENONFINITE, PWA_ECUDA. */
pwa_status pwa_variant_eval(pwa_variant* v, const double* theta, const double* dir, double* nll,
                            double* grad, double* hv);

/* pwa_variant_eval for B parameter vectors in one launch (each vector runs
 * the single evaluation's blocks, so its results equal pwa_variant_eval's).
 * theta, dir: host [B][P] (dir required when hv is non-NULL); nll: host [B];
 * grad, hv: host [B][P] or NULL.  status: host [B], per vector PWA_OK,
 * PWA_EINVAL (outside the model's domain, e.g. a mass below its pair
 * threshold) or PWA_ENONFINITE; such a vector's outputs are not written.
 * The call itself fails with PWA_EINVAL (B < 1, NULL or non-finite inputs),
 * PWA_ENOMEM or PWA_ECUDA. */
pwa_status pwa_variant_eval_batch(pwa_variant* v, int B, const double* theta, const double* dir, double* nll,
                                  double* grad, double* hv, pwa_status* status);

/* B Newton-CG fits (rows of theta0 [B][P]) in lockstep on the variant
 * likelihood; results as pwa_newton_cg_fit_batch. */
pwa_status pwa_variant_fit(pwa_variant* v, int B, const double* theta0, const pwa_fit_opts* opts,
                           double* theta_out, pwa_fit_result* results);

/* Coupling-only evaluation at fixed line shapes (the K S x K S integral
 * matrix of per-projection couplings, block-diagonal in s): computes, at the
 * masses and widths of theta (host [P]), Phi_s,kk' = sum_mc conj(U_ks) U_k's
 * with U_ks = BW_k F_ks, so that sum_mc I = sum_s g_s^H Phi_s g_s and the MC
 * events are not read again by the coupling-only calls below.  phi_out
 * (host [S][K][K] complex as (re, im) pairs, or NULL) receives the matrices.
 * Errors: PWA_EINVAL, PWA_ENONFINITE, PWA_ECUDA. */
pwa_status pwa_variant_set_shapes(pwa_variant* v, const double* theta, double* phi_out);

/* Number of coupling parameters: the free magnitudes and phases at the head of theta. */
int pwa_variant_coupling_num_params(const pwa_variant* v);

/* NLL, gradient and H v in the coupling parameters theta_c [Pc] (line shapes
 * as given to pwa_variant_set_shapes, which must come first): one pass over
 * the data events plus the integral matrices.  Errors as pwa_variant_eval. */
pwa_status pwa_variant_coupling_eval(pwa_variant* v, const double* theta_c, const double* dir_c,
                                     double* nll, double* grad, double* hv);

/* B coupling-only Newton-CG fits in lockstep (rows of theta_c0 [B][Pc]). */
pwa_status pwa_variant_coupling_fit(pwa_variant* v, int B, const double* theta_c0, const pwa_fit_opts* opts,
                                    double* theta_c_out, pwa_fit_result* results);

/* Message of the last failure of v (of the last pwa_variant_create when v is NULL). */
const char* pwa_variant_last_error(const pwa_variant* v);

void pwa_variant_destroy(pwa_variant* v);

/* ---- pseudo-experiment generation (paper Sec. 3 draws its test samples
 * from the PWA model itself) ----
 *
 * A pool of phase-space events (m2 [3][n], F [n][K][S] as in pwa_events) and
 * their intensities I(e; theta) (pwa_event_intensity of a handle whose MC
 * sample is the pool) define a pseudo-experiment by accept-reject: event j is
 * kept when u_j C < I_j, with u_j = (z >> 11) 2^-53 and z output j + 1 of
 * splitmix64 started at `seed` (Steele, Lea and Flood 2014), compared in
 * double precision.  All three calls work on device arrays and synchronise
 * cuda_stream (a cudaStream_t or NULL) before they return.  Errors go to
 * pwa_last_generate_error(). */

/* Pool indices of the first n_target kept events in the order
 * start, start + 1, ..., n - 1, 0, ..., start - 1, written to d_idx
 * [n_target]; *n_out = how many were kept (<= n_target).  C <= 0 takes
 * C = max_j I_j; *C_used (may be NULL) receives the C applied.
 * Errors: PWA_EINVAL (n < 1 or >= 2^31, start outside [0, n), n_target < 0,
 * C not finite), PWA_ENONFINITE (an I_j negative or not finite), PWA_ECUDA. */
pwa_status pwa_accept_reject(const float* d_I, long long n, double C, unsigned long long seed,
                             long long start, int n_target, int* d_idx, int* n_out,
                             double* C_used, void* cuda_stream);

/* Binned Dalitz plot of the events d_idx [n] of a pool with m2 [3][ld]:
 * x = m12^2, y = m23^2, nb x nb bins over [x0, x1) x [y0, y1),
 * bx = floor((x - x0) nb / (x1 - x0)) clamped to 0 .. nb - 1 (double
 * precision), likewise by; d_out [nb * nb] FP32 at bx * nb + by holds the
 * count, or log(1 + count nb^2 / n) when log_scale is 1.
 * Errors: PWA_EINVAL, PWA_ECUDA. */
pwa_status pwa_dalitz_histogram(const float* d_m2, long long ld, const int* d_idx, int n, int nb,
                                double x0, double x1, double y0, double y1, int log_scale,
                                float* d_out, void* cuda_stream);

/* Gather events d_idx [n] of a pool (m2 [3][ld], F [ld][KS] complex) into a
 * sample: m2_out [3][n], F_out [n][KS] complex.  Errors: PWA_EINVAL, PWA_ECUDA. */
pwa_status pwa_gather_events(const float* d_m2, long long ld, const float* d_F, int KS,
                             const int* d_idx, int n, float* d_m2_out, float* d_F_out,
                             void* cuda_stream);

/* Message of the last failure of the three calls above in this thread. */
const char* pwa_last_generate_error(void);

/* ---- learned starting-point proposal (no counterpart in the paper) ----
 *
 * A multilayer perceptron that maps a binned Dalitz histogram of a data set
 * to a starting theta for Newton-CG, trained on pseudo-experiments the method
 * generates (sample theta, accept-reject events from I, fit).  in inputs ->
 * `layers` hidden layers of `hidden` units with GELU (tanh form) -> out
 * outputs.  BF16 weights and activations, FP32 accumulation: every matrix
 * product is one tcgen05 tensor-core kernel of this library; Adam on FP32
 * master weights.  Loss: weighted squared error per output, or 1 - cos of the
 * difference for outputs flagged periodic (phases), averaged over the rows.
 * Sizes: in % 64 == 0, hidden % 128 == 0, batches a multiple of 128 up to
 * max_batch.  Initial weights uniform in +-sqrt(6 / (fan_in + fan_out)) from a
 * splitmix64 stream seeded with `seed`; biases 0.  All array arguments of the
 * forward and training calls are device pointers (FP32, row-major). */
typedef struct pwa_mlp pwa_mlp; /* opaque; owned by the library */

pwa_status pwa_mlp_create(int in, int hidden, int layers, int out, int max_batch,
                          unsigned long long seed, const int* periodic /* host [out] or NULL */,
                          const float* loss_weight /* host [out] or NULL (= 1) */,
                          void* cuda_stream, pwa_mlp** out_m);

/* y [B][out] = network(x [B][in]); synchronous on the network's stream. */
pwa_status pwa_mlp_forward(pwa_mlp* m, int B, const float* d_x, float* d_y);

/* Loss (host, mean over the B rows) and the gradients of every parameter for
 * inputs x [B][in] and targets t [B][out]; the gradients stay in the object
 * (pwa_mlp_params, which = 2 and 3). */
pwa_status pwa_mlp_gradients(pwa_mlp* m, int B, const float* d_x, const float* d_t, double* loss);

/* pwa_mlp_gradients followed by one Adam step (beta 0.9, 0.999, eps 1e-8). */
pwa_status pwa_mlp_train_step(pwa_mlp* m, int B, const float* d_x, const float* d_t, float lr, double* loss);

/* Copy parameters between the object and host memory.  layer 0 .. layers
 * (the last is the output layer); which: 0 W [fan_out][fan_in], 1 bias
 * [fan_out], 2 the last weight gradient, 3 the last bias gradient (2 and 3
 * read only).  to_device = 1 writes the object (0 and 1 only). */
pwa_status pwa_mlp_params(pwa_mlp* m, int layer, int which, float* host, int to_device);

/* The tensor-core product alone: C [M][N] = A [M][K] B [N][K]^T for host FP32
 * arrays rounded to BF16 (M % 128, N % 64, K % 64 == 0); for tests. */
pwa_status pwa_mlp_gemm_check(pwa_mlp* m, int M, int N, int K, const float* A, const float* B, float* C);

/* Message of the last failure of m (or of the last pwa_mlp_create when m is NULL). */
const char* pwa_mlp_last_error(const pwa_mlp* m);

void pwa_mlp_destroy(pwa_mlp* m);

/* Default options: xtol 1e-8, gtol 0, maxiter 0 (= 200 P), cg_maxiter 0
 * (= 20 P), no time limit. */
void pwa_fit_opts_default(pwa_fit_opts* opts);

/* Use another CUDA stream (cudaStream_t, NULL = default) for later calls. */
pwa_status pwa_set_stream(pwa_handle* h, void* cuda_stream);

/* Tiling of the streaming kernel (the autotuner's knobs).  Events are cut
 * into tiles of 32; warps: warps per block (1, 2, 4 or 8) -- the block shares
 * one tile, W lanes share an event in the coherent-sum sweep and each warp
 * owns ceil(K / warps) <= 8 resonances in the second sweep; stages: tiles in
 * flight per block (2..4); blocks_per_sm: 0 = as many as fit.  Re-lays the
 * events out on the device.  Errors: PWA_EINVAL when the combination is not
 * compiled or does not fit in shared memory (the previous tiling stays). */
pwa_status pwa_set_tiling(pwa_handle* h, int warps, int stages, int blocks_per_sm);

/* Current tiling and geometry: fills (warps, stages, blocks_per_sm,
 * events_per_tile, grid_blocks, smem_bytes_per_block). */
pwa_status pwa_get_tiling(const pwa_handle* h, int out6[6]);

/* Choose the tiling by measurement (no counterpart in the paper): times a
 * batched HVP pass of B copies of theta (host [P]) under every tiling the
 * model admits (warps 1, 2, 4, 8 with at most 8 resonances per warp; 2 or 3
 * stages; the most blocks per SM that fit, and half as many), keeps the
 * fastest and writes (warps, stages, blocks_per_sm) to out3 (may be NULL).
 * Re-tiles the events for each candidate (as pwa_set_tiling does) and
 * synchronises the handle's stream.  Timing noise can make two calls choose
 * different tilings, and another tiling splits the FP32 event sums
 * differently (results then agree to the pass's accuracy, not bit for bit).
 * Errors: PWA_EINVAL, PWA_ECUDA, PWA_ENONFINITE (theta has a non-finite NLL). */
pwa_status pwa_autotune(pwa_handle* h, const double* theta, int B, int out3[3]);

/* Diagnostic of the device-side failure detection (no counterpart in the
 * paper).  Launches one block that waits on an mbarrier which nothing ever
 * completes, using the same bounded wait the streaming kernel applies to its
 * tile copies, limited to `seconds` (0 < seconds <= 10) of SM clock.  Returns
 * PWA_ETIMEOUT when the wait ran out -- the expected outcome -- with the CUDA
 * context still usable; PWA_OK would mean the wait completed, PWA_EINVAL a
 * bad argument, PWA_ECUDA / PWA_ENOMEM a runtime failure. */
pwa_status pwa_selftest_bounded_wait(double seconds);

/* Message describing the first failure of the handle's last call. */
const char* pwa_last_error(const pwa_handle* h);

/* Free every resource of the handle (NULL is allowed). */
void pwa_destroy(pwa_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* LIBPWA_PWA_H */
