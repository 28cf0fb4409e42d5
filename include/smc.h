/*
 * smc.h -- C ABI of the B300 (sm_103a) tempered sequential Monte Carlo sampler
 * for Bayesian peak-count selection and peak-parameter estimation.
 *
 * Method (the paper's Sec. II): for every candidate peak count K the sampler
 * moves T particles from the prior (beta = 0) to the posterior (beta = 1)
 * through the tempered sequence pi_l ~ p(D|theta)^beta_l p(theta) (Eq. (9)).
 * Each stage reweights by the incremental weights of Eq. (10), accumulates
 * log Z by Eq. (11), resamples and rejuvenates with component-wise random-walk
 * Metropolis (Sec. II B 4).  The free energy is F(K) = -log Z (Eq. (3)) and
 * the posterior over K follows Eq. (2).
 *
 * Forward model (Eq. (1)): f(x) = sum_k g_k(x) + b(x) with
 *   SMC_GAUSS          g = A exp(-(x-mu)^2 / (2 w^2))          w: standard deviation
 *   SMC_LORENTZ        g = A w^2 / (w^2 + (x-mu)^2)            w: HWHM
 *   SMC_PSEUDO_VOIGT   g = A [eta exp(-ln2 (x-mu)^2/w^2)
 *                             + (1-eta) w^2/(w^2 + (x-mu)^2)]   w: shared HWHM,
 *                                                               eta: Gaussian fraction (Eq. (E1))
 *   SMC_GAUSS_PRECISION g = A exp(-b/2 (x-mu)^2)               b: precision (App. C Eq. (C1))
 *   SMC_XRD_PHASE      phase k of the App. D powder model, components
 *                      (A, d2theta, alpha, r, u, v, w, s, t):
 *                      A sum_j I_j [(1 - r) exp(-4 ln2 (x - m_j)^2 / S^2)
 *                                   + r / (1 + 4 (x - m_j)^2 / W^2)],
 *                      m_j = ref_j + d2theta, S = a sqrt(u T^2 - v T + w),
 *                      W = a (s / cos(x/2) + t T), T = tan(x/2) (x in degrees
 *                      2 theta), a = alpha for x >= m_j, 1 below; a part whose
 *                      width is not positive is 0.  Reference positions ref_j
 *                      and relative intensities I_j per phase are inputs
 *                      (smc_request.ref_*); phase k of a K-phase model is the
 *                      k-th listed phase; phases are not sorted in summaries.
 * and background b(x) = sum_j c_j T_j(t), T_j Chebyshev polynomials of the first
 * kind, t = (2x - (x_min + x_max)) / (x_max - x_min), or the Shirley background
 * of App. E (SMC_BG_SHIRLEY, components a, b):
 *   B_i = a + (b - a) C_i / C_N,  C_i = sum_{1 < j <= i} P_j |x_j - x_{j-1}|,
 * P the peak sum, points in data order: the running integral of the peak signal
 * from the first point (right-end rectangle rule), B = a at the first point and
 * b at the last (B = a if C_N = 0); or the App. D background (SMC_BG_XRD_PV,
 * components a, s_bg, r_bg, b): a [(1 - r_bg) exp(-4 ln2 x^2 / s_bg^2)
 * + r_bg / (1 + 4 x^2 / s_bg^2)] + b.
 * Components per job, in this order (the Metropolis sweep order): for each peak
 * (A, mu, w[, eta]), then c_0 .. c_{nbg-1}.  d = p K + nbg, p = 3 or 4.
 *
 * Likelihood (smc_request.noise): SMC_NOISE_KNOWN, Gaussian with known per-point
 * sigma_i, energy E(theta) = 1/2 sum_i ((y_i - f_i)/sigma_i)^2, the returned
 * log Z including the normaliser -sum_i log(sqrt(2 pi) sigma_i); or
 * SMC_NOISE_MODEL (App. E), variance following the model value,
 *   sigma_i^2 = s0^2 f_i + s1^2 f_i^2 + s2^2   (noise_par = {s0, s1, s2}),
 * E = sum_i [1/2 ln(2 pi sigma_i^2) + 1/2 (y_i - f_i)^2 / sigma_i^2] (+inf where
 * sigma_i^2 <= 0), sigma unused; or SMC_NOISE_POISSON (App. D), counts y_i >= 0,
 * E = sum_i [(f_i - y_i) - y_i ln(f_i / y_i)] (f_i for y_i = 0, +inf where
 * f_i <= 0) with the normaliser sum_i [y_i ln y_i - y_i - ln Gamma(y_i + 1)] in
 * log Z.  Poisson requests with FP32 energies (energy_fp64 = 0), a Gaussian
 * peak family (SMC_GAUSS, SMC_GAUSS_PRECISION) and no background are rejected
 * with SMC_EINVAL: far from every peak the model falls below FP32's range, and
 * a positive count there has an infinite FP32 energy where the FP64 one is
 * finite; such requests take energy_fp64 = 1 or 2, or a background.  Either way log Z is the log marginal likelihood of Eq. (5) and
 * F = -log Z.  The Shirley background and the model variance run
 * in the coupled-grid Metropolis kernel and are combined with no Chebyshev
 * background.
 *
 * Errors: every call returns an int status (SMC_OK = 0 or an SMC_E* code).
 * On error nothing is allocated on the caller's behalf and output arguments
 * are left untouched.  smc_strerror() gives a static message.
 *
 * Threading: one smc_ctx may be used from several threads; calls are
 * serialised internally.  smc_submit / smc_poll / smc_wait are the serving
 * interface: submitted requests run concurrently on the device with
 * continuous batching (admitted as slots and the memory budget free up).
 */
#ifndef SMC_H
#define SMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SMC_MAX_BG 8     /* background coefficients (polynomial degree <= 7) */
#define SMC_MAX_DIM 128  /* components per job: p K + nbg <= 128              */
#define SMC_MAX_K 32     /* peaks per job                                     */
#define SMC_MAX_REFS 64  /* reflections per phase (SMC_XRD_PHASE)            */

typedef struct smc_ctx smc_ctx;
typedef uint64_t smc_job;

enum smc_status {
    SMC_OK = 0,
    SMC_EINVAL = 1,       /* invalid argument (sizes, priors, sigma <= 0, ...)     */
    SMC_ENOMEM = 2,       /* device or host allocation failed / over budget        */
    SMC_ECUDA = 3,        /* a CUDA runtime call failed                            */
    SMC_ETIMEOUT = 4,     /* smc_wait ran out of time                              */
    SMC_EMAXSTAGES = 5,   /* beta did not reach 1 within max_stages                */
    SMC_ENOTREADY = 6,    /* result requested before the job finished              */
    SMC_ECANCELLED = 7,   /* request cancelled (context destroyed while queued)    */
    SMC_ENUMERIC = 8      /* every particle's energy is non-finite                 */
};

enum smc_family { SMC_GAUSS = 0, SMC_LORENTZ = 1, SMC_PSEUDO_VOIGT = 2, SMC_GAUSS_PRECISION = 3,
                  SMC_XRD_PHASE = 4 };
enum smc_bg { SMC_BG_NONE = 0, SMC_BG_CONST = 1, SMC_BG_LINEAR = 2, SMC_BG_POLY = 3, SMC_BG_SHIRLEY = 4,
              SMC_BG_XRD_PV = 5 };
enum smc_noise { SMC_NOISE_KNOWN = 0, SMC_NOISE_MODEL = 1, SMC_NOISE_POISSON = 2 };

/* Prior kinds.  Sampling coordinates: log v for LOG_UNIFORM, v otherwise.
 *   SMC_UNIFORM      p1 = lower, p2 = upper
 *   SMC_LOG_UNIFORM  log v ~ U(log p1, log p2), 0 < p1 < p2
 *   SMC_NORMAL       p1 = mean, p2 = standard deviation
 *   SMC_GAMMA        p1 = shape, p2 = rate            (App. C and D priors)
 *   SMC_FIXED        v = p1, never proposed
 * Centres accept UNIFORM, NORMAL or FIXED; widths must have positive support. */
enum smc_prior_kind { SMC_UNIFORM = 0, SMC_LOG_UNIFORM = 1, SMC_NORMAL = 2, SMC_GAMMA = 3, SMC_FIXED = 4 };

typedef struct {
    int32_t kind;
    double p1, p2;
} smc_prior;

/* Shared priors for every peak (peaks are exchangeable in Eq. (1)) and one per
 * background coefficient.  If n_comp > 0, comp[0..n_comp) gives one prior per
 * component instead (requires k_min == k_max and n_comp == d). */
typedef struct {
    smc_prior amp, centre, width, eta, bg[SMC_MAX_BG];
    const smc_prior *comp;
    int32_t n_comp;
    smc_prior phase[9];  /* SMC_XRD_PHASE: shared priors of the nine phase components */
} smc_priors;

/* How a batched FP32 run is launched (smc_create_opts.graph_mode).  Results
 * are identical in every mode. */
#define SMC_GRAPH_WHILE 0    /* one CUDA graph launch per run: a conditional while
                                node over the tempering stages (the default)     */
#define SMC_GRAPH_CHUNKED 1  /* host-replayed graphs of four stages each          */
#define SMC_GRAPH_NONE 2     /* every kernel launched on the stream, no graphs:
                                for kernel profilers and launch tracers, which do
                                not see kernels inside conditional graph nodes   */

typedef struct {
    int32_t device;           /* CUDA device ordinal                                 */
    size_t mem_budget_bytes;  /* device bytes the context may hold (0 = 80% of free) */
    void *cuda_stream;        /* cudaStream_t to run on (NULL = a private stream)    */
    int32_t graph_mode;       /* SMC_GRAPH_WHILE / _CHUNKED / _NONE (else SMC_EINVAL);
                                 the environment variable SMC_GRAPH_CHUNKED=1 at
                                 creation selects SMC_GRAPH_CHUNKED as well        */
} smc_create_opts;

typedef struct {
    int64_t particles;    /* T, particles per candidate K (2 .. 2^24)              */
    double ess_target;    /* rho: next beta keeps ESS >= rho T (0 < rho < 1)       */
    int32_t sweeps;       /* n, Metropolis sweeps per stage                        */
    int32_t waste_free;   /* 1: resample ceil(T/n) chains, keep every sweep (Sec. II B 3) */
    int32_t energy_fp64;  /* 0: FP32 energies, the batched fused kernels;
                             1: the plain FP64 path, one job per launch sequence
                                (thread-per-chain Metropolis, full FP64 energy per
                                proposal);
                             2: the same FP64 kernels with every FP64 job of the
                                call in the same launches                        */
    uint64_t seed;        /* Philox key                                            */
    int32_t max_stages;   /* cap on tempering stages (SMC_EMAXSTAGES beyond)       */
    int32_t keep_samples; /* 1: copy the final particle set to the host            */
    int32_t step_rule;    /* Metropolis step sizes (Sec. II B 4): 0 = lambda_j x the
                             weighted population SD, lambda_j adapted from the last
                             acceptance rate; 1 = predicted from the histories of
                             beta and of the acceptance rates (1-D Gaussian
                             acceptance model, weighted log-log regression of the
                             implied target SD on beta, acceptance 0.44 aimed at) */
} smc_options;

/* One spectrum and its candidate range, for smc_run_batch / smc_submit. */
typedef struct {
    const double *x, *y, *sigma;  /* n points each (host, or device if flagged);  */
    int64_t n;                    /* sigma may be NULL with SMC_NOISE_MODEL       */
    int32_t k_min, k_max;
    int32_t family, bg, bg_degree;
    const smc_priors *priors;
    const smc_options *opts;
    int32_t noise;                /* smc_noise (SMC_NOISE_KNOWN = 0)              */
    double noise_par[3];          /* s0, s1, s2 of SMC_NOISE_MODEL                */
    /* SMC_XRD_PHASE: reflections ref_off[k] .. ref_off[k+1] - 1 of phase k
     * (host arrays, copied at call time; n_phase >= k_max; 1 .. SMC_MAX_REFS
     * reflections per phase; positions finite, intensities finite and >= 0;
     * SMC_EINVAL otherwise)                                                  */
    const double *ref_pos, *ref_int;
    const int32_t *ref_off;
    int32_t n_phase;
} smc_request;

/* Result of one spectrum: arrays indexed by K - k_min.  Views are owned by the
 * context and stay valid until smc_release(job). */
typedef struct {
    int32_t k_min, k_max;
    int32_t dim_max;              /* row stride of post_mean / post_sd / samples       */
    int32_t status;               /* SMC_OK or the first failing job's status         */
    const double *log_z;          /* [nK] log marginal likelihood, F = -log_z          */
    const double *p_k;            /* [nK] posterior over K, uniform p(K) (Eq. (2))      */
    const int32_t *n_stages;      /* [nK] tempering stages used                        */
    const int32_t *job_status;    /* [nK]                                              */
    const double *post_mean;      /* [nK][dim_max] natural values, peaks sorted by mu  */
    const double *post_sd;        /* [nK][dim_max]                                     */
    const float *samples;         /* [nK][n_samples][dim_max] natural values, or NULL  */
    int64_t n_samples;            /* particles per K in the final set                  */
    double latency_ms;            /* submit (or run start) to completion, host clock   */
    int32_t selected_k;           /* the K of largest log Z among jobs with status
                                     SMC_OK (smallest F(K), Sec. II A); log Z values
                                     within 1e-12 of each other tie and the lower K
                                     wins; -1 if no job succeeded                     */
} smc_result_view;

/* Create / destroy a context bound to one device.  By default a batched run
 * is one CUDA graph launch (a conditional while node over the tempering
 * stages); opts->graph_mode selects host-replayed four-stage graphs or plain
 * stream launches instead (same results).  opts may be NULL (device 0,
 * defaults).  smc_destroy cancels queued requests, waits for the running ones
 * and frees everything the context holds. */
int smc_create(smc_ctx **out, const smc_create_opts *opts);
int smc_destroy(smc_ctx *ctx);

/* Blocking run of one spectrum over K = k_min..k_max: for every K, the
 * tempered sequence of Eq. (9) from the prior (beta = 0) to the posterior
 * (beta = 1) with the incremental weights of Eq. (10), the evidence of
 * Eq. (11) and Metropolis moves (Sec. II B 4); then F(K) = -log Z (Eq. (3))
 * and P(K|D) (Eq. (2)).  x, y, sigma are host arrays of n doubles (the grid,
 * the data and the known per-point noise SD of the Gaussian likelihood),
 * copied at call time; priors and opts are read at call time.  *out receives
 * a job handle whose result is read with smc_result and freed with
 * smc_release.  Returns SMC_EINVAL for invalid sizes or priors, SMC_ENOMEM if
 * the request does not fit the context's budget. */
int smc_run(smc_ctx *ctx, const double *x, const double *y, const double *sigma, int64_t n,
            int32_t k_min, int32_t k_max, int32_t family, int32_t bg, int32_t bg_degree,
            const smc_priors *priors, const smc_options *opts, smc_job *out);

/* Blocking run of several spectra (the computation of smc_run for each) in
 * one batched launch sequence: every (spectrum, K) job advances in the same
 * kernels.  If inputs_on_device is 1, the x/y/sigma pointers are device
 * pointers on the context's device (checked by the preparation kernel).
 * out[i] receives the handle of reqs[i].  On error no handle is returned. */
int smc_run_batch(smc_ctx *ctx, const smc_request *reqs, int32_t count, int32_t inputs_on_device,
                  smc_job *out);

/* Serving: enqueue a request (host arrays, copied at call time) and return at
 * once.  Requests are admitted in arrival order as the memory budget and job
 * slots free up, and run with continuous batching (requests admitted while
 * others run join their launches); their particle state stays on the device
 * until retirement.  A request larger than the whole budget finishes with
 * status SMC_ENOMEM; one that does not fit yet waits. */
int smc_submit(smc_ctx *ctx, const smc_request *req, smc_job *out);
/* Enqueue `count` requests at once, in order (as count calls of smc_submit
 * that no admission pass can separate).  On error none is enqueued. */
int smc_submit_batch(smc_ctx *ctx, const smc_request *reqs, int32_t count, smc_job *out);
int smc_poll(smc_ctx *ctx, smc_job job, int32_t *done);   /* *done = 1 once finished     */
int smc_wait(smc_ctx *ctx, smc_job job, double timeout_s); /* < 0: no limit; SMC_ETIMEOUT */

/* Device bytes a request would hold in this context while it runs (its
 * spectrum, per-K particle state and results, with the context's tiles): the
 * quantity admitted against mem_budget_bytes.  SMC_EINVAL for an invalid
 * request. */
int smc_request_bytes(smc_ctx *ctx, const smc_request *req, size_t *bytes);

/* Result of a finished job: log Z per K (Eq. (11)), P(K|D) (Eq. (2)), the
 * selected K, posterior summaries and (if keep_samples) the final particles.
 * SMC_ENOTREADY while it runs. */
int smc_result(smc_ctx *ctx, smc_job job, smc_result_view *out);
int smc_release(smc_ctx *ctx, smc_job job);

const char *smc_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* SMC_H */
