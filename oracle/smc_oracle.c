/*
 * smc_oracle.c -- plain FP64 CPU oracle of the tempered SMC sampler.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header or constant table with
 * the CUDA library.
 *
 * Every quantity is double precision, every loop is sequential, and every
 * Metropolis proposal recomputes the full forward model and energy.  Each
 * function names the passage of the paper it follows.  Where the paper is
 * silent the reading taken is written beside the code:
 *   - likelihood: Gaussian with known per-point sigma_i; the energy is
 *     E = 1/2 sum ((y_i - f_i)/sigma_i)^2 and the reported log Z adds the
 *     normaliser -sum log(sqrt(2 pi) sigma_i)          (App. C, Eq. (C2));
 *     or, for the XPS model (App. E), a variance that follows the model,
 *     sigma_i^2 = s0^2 f_i + s1^2 f_i^2 + s2^2, with
 *     E = sum [1/2 ln(2 pi sigma_i^2) + 1/2 (y_i - f_i)^2 / sigma_i^2]
 *     (the 1/N factor and the missing 1/2 of the printed formula read as
 *     garbles of the Gaussian negative log-likelihood);
 *   - XRD phase model (App. D): phase k contributes A_k sum_j I_kj
 *     V(x; mu_kj + d2theta_k, Sigma_k(x), Omega_k(x), r_k) over its reference
 *     reflections (positions mu_kj, relative intensities I_kj: inputs), with
 *     Sigma = asym sqrt(u tan^2(x/2) - v tan(x/2) + w), Omega = asym (s sec(x/2)
 *     + t tan(x/2)), asym = alpha for x >= mu, 1 below (x in degrees, halved
 *     and converted to radians), V = (1 - r) exp(-4 ln2 (x - mu)^2 / Sigma^2) +
 *     r / (1 + 4 (x - mu)^2 / Omega^2); G = 0 where the Caglioti radicand is not
 *     positive, L = 0 where Omega is not; background a V(x; 0, sbg, sbg, rbg) + b;
 *     Poisson likelihood with energy sum [(f - y) - y ln(f / y)] (f for y = 0,
 *     +inf where f <= 0) and normaliser sum [y ln y - y - ln Gamma(y + 1)];
 *   - Shirley background (App. E): B_i = a + (b - a) C_i / C_N with C_i the
 *     integral of the peak signal from the first grid point to x_i by the
 *     right-end rectangle rule, C_i = sum_{1 < j <= i} P_j |x_j - x_{j-1}|,
 *     so B = a at the first point and b at the last (B = a if C_N = 0);
 *   - tempering: next beta by bisection on the effective sample size;
 *   - resampling: systematic, on integer-quantised weights (exact);
 *   - step sizes: lambda_j * weighted population SD, lambda_j adapted from
 *     the previous stage's acceptance rate; or (step_rule 1) predicted from
 *     the histories of beta and of the acceptance rates (orc_predict_step);
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11) with
 *     key = seed and counter = (draw, particle, stage, K).
 *
 * Parity status: every function here is pinned by tests (closed forms,
 * brute force, published Philox answers, the linear-Gaussian evidence and
 * K = 1 quadrature).  The step-size rule and the waste-free branch are pinned
 * against weighted moments computed independently (row replication, numpy's
 * analytic-weight covariance), replays of standard stages, and the closed-form
 * and quadrature evidences run in waste-free mode.  tests/test_oracle_mutants.py
 * builds copies of this file with one plausible mistake planted in each and
 * checks that every copy fails one of those pins.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_EMAXSTAGES 5
#define ORC_ENUMERIC 8

enum { FAM_GAUSS = 0, FAM_LORENTZ = 1, FAM_PV = 2, FAM_GAUSS_PREC = 3, FAM_XRD_PHASE = 4 };
enum { BG_NONE = 0, BG_CONST = 1, BG_LINEAR = 2, BG_POLY = 3, BG_SHIRLEY = 4, BG_XRD_PV = 5 };
enum { NOISE_KNOWN = 0, NOISE_MODEL = 1, NOISE_POISSON = 2 };
enum { PR_UNIFORM = 0, PR_LOG_UNIFORM = 1, PR_NORMAL = 2, PR_GAMMA = 3, PR_FIXED = 4 };

typedef struct {
    int32_t kind;
    double p1, p2;
} orc_prior;

typedef struct {
    const double *x, *y, *sigma;
    int64_t n;
    int32_t family, K, bg_kind, bg_degree;
    orc_prior amp, centre, width, eta, bg[8];
    const orc_prior *comp_priors; /* optional: one prior per component (d) */
    int32_t n_comp_priors;
    int64_t particles;
    double ess_target;
    int32_t sweeps, waste_free;
    uint64_t seed;
    int32_t max_stages;
    int32_t noise;        /* NOISE_KNOWN: sigma[]; NOISE_MODEL: noise_par; NOISE_POISSON */
    double noise_par[3];  /* s0, s1, s2 of sigma_i^2 = s0^2 f + s1^2 f^2 + s2^2 */
    /* XRD phase model: reflections ref_off[k] .. ref_off[k+1] of phase k */
    const double *ref_pos, *ref_int;
    const int32_t *ref_off;
    int32_t n_phase;
    orc_prior phase[9]; /* shared priors of (A, d2theta, alpha, r, u, v, w, s, t) */
    int32_t step_rule;  /* 0: lambda x weighted SD; 1: the history predictor */
} orc_job;

typedef struct {
    double log_z;
    int32_t n_stages;
    int32_t status;
    int64_t n_out;     /* particles in the final set */
    int32_t d;
    double *samples;   /* [n_out][d] natural parameter values (caller buffer) */
    double *energies;  /* [n_out] */
    double *beta_trace;   /* [max_stages + 1], beta after each stage */
    double *logz_trace;   /* [max_stages + 1], log Z after each stage */
    double *acc_trace;    /* [max_stages + 1][d] acceptance rate per component */
    double *step_trace;   /* [max_stages + 1][d] step size used per component */
} orc_out;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw,  */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two   */
/* 32x32->64 multiplies with a Weyl-sequence key schedule.                    */
/* ------------------------------------------------------------------------- */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in (0, 1): (k + 1/2) 2^-32 */
static double u01(uint32_t k) { return ((double)k + 0.5) * 2.3283064365386963e-10; }

static void draw_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                       uint32_t w[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    orc_philox(ctr, key, w);
}

/* Box-Muller (1958): one standard normal from two uniforms. */
static double box_muller(uint32_t a, uint32_t b)
{
    return sqrt(-2.0 * log(u01(a))) * cos(2.0 * M_PI * u01(b));
}

/* ------------------------------------------------------------------------- */
/* Model layout: peak k has components (A, mu, width[, eta]), then the        */
/* background coefficients (forward model, Sec. II A, Eq. (1)).               */
/* ------------------------------------------------------------------------- */
static int peak_params(int family) { return family == FAM_XRD_PHASE ? 9 : (family == FAM_PV ? 4 : 3); }

static int bg_params(int kind, int degree)
{
    switch (kind) {
    case BG_NONE: return 0;
    case BG_CONST: return 1;
    case BG_LINEAR: return 2;
    case BG_SHIRLEY: return 2;
    case BG_XRD_PV: return 4;
    default: return degree + 1;
    }
}

int orc_dim(int family, int K, int bg_kind, int bg_degree)
{
    return peak_params(family) * K + bg_params(bg_kind, bg_degree);
}

static orc_prior comp_prior(const orc_job *job, int j)
{
    if (job->n_comp_priors > 0) return job->comp_priors[j];
    int p = peak_params(job->family);
    if (job->family == FAM_XRD_PHASE) return j < p * job->K ? job->phase[j % p] : job->bg[j - p * job->K];
    if (j < p * job->K) {
        switch (j % p) {
        case 0: return job->amp;
        case 1: return job->centre;
        case 2: return job->width;
        default: return job->eta;
        }
    }
    return job->bg[j - p * job->K];
}

/* Sampler coordinate u -> natural value (log-uniform priors are sampled in log). */
static double to_natural(orc_prior pr, double u) { return pr.kind == PR_LOG_UNIFORM ? exp(u) : u; }

static int in_support(orc_prior pr, double u)
{
    switch (pr.kind) {
    case PR_UNIFORM: return u >= pr.p1 && u <= pr.p2;
    case PR_LOG_UNIFORM: return u >= log(pr.p1) && u <= log(pr.p2);
    case PR_GAMMA: return u > 0.0;
    case PR_NORMAL: return 1;
    default: return 0;
    }
}

/* log prior density in sampler coordinates, up to an additive constant. */
static double log_prior(orc_prior pr, double u)
{
    switch (pr.kind) {
    case PR_NORMAL: {
        double z = (u - pr.p1) / pr.p2;
        return -0.5 * z * z;
    }
    case PR_GAMMA: return (pr.p1 - 1.0) * log(u) - pr.p2 * u;
    default: return 0.0;
    }
}

/* Peak profiles with natural parameters.
 * Gaussian with precision b, A exp(-b (x - mu)^2 / 2) (App. C Eq. (C1));
 * Gaussian with standard deviation w (Eq. (C1) with b = 1/w^2);
 * Lorentzian with HWHM w (the Lorentzian part of Eq. (E1));
 * pseudo-Voigt of Eq. (E1): eta * Gaussian + (1 - eta) * Lorentzian, shared HWHM. */
double orc_peak(int family, double x, double A, double mu, double w, double eta)
{
    double dx = x - mu;
    if (family == FAM_GAUSS_PREC) return A * exp(-w * dx * dx / 2.0);
    if (family == FAM_GAUSS) return A * exp(-dx * dx / (2.0 * w * w));
    double lor = w * w / (w * w + dx * dx);
    if (family == FAM_LORENTZ) return A * lor;
    double s = w / sqrt(2.0 * log(2.0));
    double gau = exp(-dx * dx / (2.0 * s * s));
    return A * (eta * gau + (1.0 - eta) * lor);
}

/* App. D pseudo-Voigt with separate Gaussian and Lorentzian FWHM:
 * (1 - r) exp(-4 ln2 dx^2 / S^2) + r / (1 + 4 dx^2 / W^2); a part whose width is
 * not positive is 0. */
static double xrd_pv(double dx, double S, double W, double r)
{
    double g = S > 0.0 ? exp(-4.0 * log(2.0) * dx * dx / (S * S)) : 0.0;
    double l = W > 0.0 ? 1.0 / (1.0 + 4.0 * dx * dx / (W * W)) : 0.0;
    return (1.0 - r) * g + r * l;
}

/* Phase k at x (degrees): sum over its reflections (App. D Eqs. (D1)-(D6)). */
double orc_xrd_phase(const double *q, const double *pos, const double *inten, int nref, double x)
{
    double A = q[0], shift = q[1], alpha = q[2], r = q[3], u = q[4], v = q[5], w = q[6], s = q[7],
           t = q[8];
    double th = x * M_PI / 360.0; /* x / 2 in radians */
    double tn = tan(th), sc = 1.0 / cos(th);
    double rad = u * tn * tn - v * tn + w;
    double S0 = rad > 0.0 ? sqrt(rad) : 0.0, W0 = s * sc + t * tn;
    double sum = 0.0;
    for (int j = 0; j < nref; ++j) {
        double mu = pos[j] + shift, dx = x - mu, asym = x >= mu ? alpha : 1.0;
        sum += inten[j] * xrd_pv(dx, asym * S0, asym * W0, r);
    }
    return A * sum;
}

/* App. D background a V(x; 0, sbg, sbg, rbg) + b. */
double orc_xrd_background(const double *bg, double x) { return bg[0] * xrd_pv(x, bg[1], bg[1], bg[2]) + bg[3]; }

/* Chebyshev polynomial T_j(t) by the three-term recurrence. */
static double chebyshev(int j, double t)
{
    double a = 1.0, b = t;
    if (j == 0) return a;
    for (int k = 2; k <= j; ++k) {
        double c = 2.0 * t * b - a;
        a = b;
        b = c;
    }
    return b;
}

/* Forward model f(x; theta) = sum_k g_k(x; theta_k) + b(x)  (Eq. (1)).
 * nat: natural parameters in component order. */
double orc_model_at(int family, int K, int nbg, const double *nat, double x, double xmin,
                    double xmax)
{
    int p = peak_params(family);
    double f = 0.0;
    for (int k = 0; k < K; ++k) {
        const double *q = nat + p * k;
        f += orc_peak(family, x, q[0], q[1], q[2], p == 4 ? q[3] : 0.0);
    }
    if (nbg > 0) {
        double t = (2.0 * x - (xmin + xmax)) / (xmax - xmin);
        for (int j = 0; j < nbg; ++j) f += nat[p * K + j] * chebyshev(j, t);
    }
    return f;
}

static void range_of(const double *x, int64_t n, double *lo, double *hi)
{
    double a = x[0], b = x[0];
    for (int64_t i = 1; i < n; ++i) {
        if (x[i] < a) a = x[i];
        if (x[i] > b) b = x[i];
    }
    *lo = a;
    *hi = b;
}

/* Energy E = 1/2 sum_i ((y_i - f_i) / sigma_i)^2 : the negative log-likelihood
 * of App. C Eq. (C2) with per-point known sigma, without the 1/N factor and
 * without the normaliser (which is added to log Z once). */
double orc_energy_nat(int family, int K, int nbg, const double *nat, const double *x,
                      const double *y, const double *sigma, int64_t n)
{
    double xmin, xmax;
    range_of(x, n, &xmin, &xmax);
    double e = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = (y[i] - orc_model_at(family, K, nbg, nat, x[i], xmin, xmax)) / sigma[i];
        e += 0.5 * r * r;
    }
    return e;
}

/* Forward model at every grid point, f[i] (Eq. (1); App. E for the Shirley
 * background, whose value at x_i integrates the peak signal up to x_i). */
/* Forward model of the XRD phase model at every grid point. */
void orc_model_vec_xrd(int K, int bg_kind, const double *nat, const double *x, int64_t n,
                       const double *ref_pos, const double *ref_int, const int32_t *ref_off,
                       double *f)
{
    for (int64_t i = 0; i < n; ++i) {
        double v = 0.0;
        for (int k = 0; k < K; ++k)
            v += orc_xrd_phase(nat + 9 * k, ref_pos + ref_off[k], ref_int + ref_off[k],
                               ref_off[k + 1] - ref_off[k], x[i]);
        if (bg_kind == BG_XRD_PV) v += orc_xrd_background(nat + 9 * K, x[i]);
        f[i] = v;
    }
}

void orc_model_vec(int family, int K, int bg_kind, int bg_degree, const double *nat,
                   const double *x, int64_t n, double *f)
{
    int p = peak_params(family), nbg = bg_params(bg_kind, bg_degree);
    if (bg_kind != BG_SHIRLEY) {
        double xmin, xmax;
        range_of(x, n, &xmin, &xmax);
        for (int64_t i = 0; i < n; ++i) f[i] = orc_model_at(family, K, nbg, nat, x[i], xmin, xmax);
        return;
    }
    /* peaks only, then the Shirley background from their running integral */
    for (int64_t i = 0; i < n; ++i) f[i] = orc_model_at(family, K, 0, nat, x[i], 0.0, 1.0);
    double a = nat[p * K], b = nat[p * K + 1], total = 0.0;
    for (int64_t i = 1; i < n; ++i) total += f[i] * fabs(x[i] - x[i - 1]);
    double run = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (i > 0) run += f[i] * fabs(x[i] - x[i - 1]);
        double shirley = total > 0.0 ? a + (b - a) * run / total : a;
        f[i] += shirley;
    }
}

/* Energy of the natural parameters for either likelihood (see the header):
 * noise = NOISE_KNOWN: 1/2 sum ((y - f)/sigma)^2 (normaliser not included);
 * noise = NOISE_MODEL: sum [1/2 ln(2 pi s^2) + 1/2 (y - f)^2 / s^2],
 * s^2 = par0^2 f + par1^2 f^2 + par2^2 (+inf where s^2 <= 0). */
double orc_energy_model(int family, int K, int bg_kind, int bg_degree, int noise,
                        const double *noise_par, const double *nat, const double *x,
                        const double *y, const double *sigma, int64_t n)
{
    double *f = (double *)malloc(sizeof(double) * (size_t)n);
    if (!f) return NAN;
    orc_model_vec(family, K, bg_kind, bg_degree, nat, x, n, f);
    double e = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = y[i] - f[i];
        if (noise == NOISE_KNOWN) {
            e += 0.5 * (r / sigma[i]) * (r / sigma[i]);
        } else {
            double s0 = noise_par[0], s1 = noise_par[1], s2 = noise_par[2];
            double v = s0 * s0 * f[i] + s1 * s1 * f[i] * f[i] + s2 * s2;
            if (!(v > 0.0)) {
                e = INFINITY;
                break;
            }
            e += 0.5 * log(2.0 * M_PI * v) + 0.5 * r * r / v;
        }
    }
    free(f);
    return e;
}

/* Poisson energy term (f - y) - y ln(f / y), f for y = 0 (App. D Eq. (D8) up
 * to the saturated-model constant y ln y - y, which the normaliser carries). */
static double poisson_term(double f, double y)
{
    if (!(f > 0.0)) return INFINITY;
    if (y == 0.0) return f;
    return (f - y) - y * log(f / y);
}

/* Energy of natural parameters for a job (any family, background and noise). */
double orc_energy_job(const orc_job *job, const double *nat)
{
    int64_t n = job->n;
    double *f = (double *)malloc(sizeof(double) * (size_t)n);
    if (!f) return NAN;
    if (job->family == FAM_XRD_PHASE)
        orc_model_vec_xrd(job->K, job->bg_kind, nat, job->x, n, job->ref_pos, job->ref_int,
                          job->ref_off, f);
    else
        orc_model_vec(job->family, job->K, job->bg_kind, job->bg_degree, nat, job->x, n, f);
    double e = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = job->y[i] - f[i];
        if (job->noise == NOISE_KNOWN) {
            e += 0.5 * (r / job->sigma[i]) * (r / job->sigma[i]);
        } else if (job->noise == NOISE_POISSON) {
            e += poisson_term(f[i], job->y[i]);
        } else {
            const double *np_ = job->noise_par;
            double v = np_[0] * np_[0] * f[i] + np_[1] * np_[1] * f[i] * f[i] + np_[2] * np_[2];
            if (!(v > 0.0)) {
                e = INFINITY;
                break;
            }
            e += 0.5 * log(2.0 * M_PI * v) + 0.5 * r * r / v;
        }
        if (!isfinite(e)) break;
    }
    free(f);
    return e;
}

typedef struct {
    const orc_job *job;
    int d, p, nbg;
    double xmin, xmax;
    orc_prior *pri;
    double *nat; /* scratch [d] */
} ctx_t;

static double energy_u(ctx_t *c, const double *u)
{
    for (int j = 0; j < c->d; ++j) c->nat[j] = to_natural(c->pri[j], u[j]);
    const orc_job *job = c->job;
    if (job->family == FAM_XRD_PHASE || job->noise == NOISE_POISSON)
        return orc_energy_job(job, c->nat);
    if (job->bg_kind == BG_SHIRLEY || job->noise == NOISE_MODEL)
        return orc_energy_model(job->family, job->K, job->bg_kind, job->bg_degree, job->noise,
                                job->noise_par, c->nat, job->x, job->y, job->sigma, job->n);
    double e = 0.0;
    for (int64_t i = 0; i < job->n; ++i) {
        double r = (job->y[i] - orc_model_at(job->family, job->K, c->nbg, c->nat, job->x[i],
                                             c->xmin, c->xmax)) /
                   job->sigma[i];
        e += 0.5 * r * r;
    }
    return e;
}

/* ------------------------------------------------------------------------- */
/* Prior draws at beta_0 = 0 (Sec. II B 2: the tempered sequence starts at the */
/* prior).  Counter (256 j + attempt, particle, 0, K).                         */
/* Gamma(shape, rate) by Marsaglia & Tsang (2000), with the u^(1/a) boost for  */
/* shape < 1.                                                                  */
/* ------------------------------------------------------------------------- */
double orc_prior_draw(orc_prior pr, uint64_t seed, uint32_t comp, uint32_t particle,
                      uint32_t tag)
{
    uint32_t w[4];
    switch (pr.kind) {
    case PR_UNIFORM:
        draw_words(seed, 256u * comp, particle, 0u, tag, w);
        return pr.p1 + (pr.p2 - pr.p1) * u01(w[0]);
    case PR_LOG_UNIFORM:
        draw_words(seed, 256u * comp, particle, 0u, tag, w);
        return log(pr.p1) + (log(pr.p2) - log(pr.p1)) * u01(w[0]);
    case PR_NORMAL:
        draw_words(seed, 256u * comp, particle, 0u, tag, w);
        return pr.p1 + pr.p2 * box_muller(w[0], w[1]);
    case PR_GAMMA: {
        double a = pr.p1 < 1.0 ? pr.p1 + 1.0 : pr.p1;
        double dd = a - 1.0 / 3.0;
        double cc = 1.0 / sqrt(9.0 * dd);
        for (uint32_t attempt = 0; attempt < 256u; ++attempt) {
            draw_words(seed, 256u * comp + attempt, particle, 0u, tag, w);
            double z = box_muller(w[0], w[1]);
            double t = 1.0 + cc * z;
            if (t <= 0.0) continue;
            double v = t * t * t;
            if (log(u01(w[2])) < 0.5 * z * z + dd - dd * v + dd * log(v)) {
                double g = dd * v;
                if (pr.p1 < 1.0) g *= pow(u01(w[3]), 1.0 / pr.p1);
                return g / pr.p2;
            }
        }
        return dd / pr.p2;
    }
    default: return pr.p1; /* FIXED */
    }
}

/* ------------------------------------------------------------------------- */
/* Tempering: ESS fraction of the incremental weights w_i = exp(-delta e_i)   */
/* (Sec. II B 2, Eq. (10)), e_i = E_i - min E; non-finite energies get w = 0.  */
/* ------------------------------------------------------------------------- */
double orc_ess_frac(const double *e, int64_t T, double delta)
{
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < T; ++i) {
        if (!isfinite(e[i])) continue;
        double w = exp(-delta * e[i]);
        s1 += w;
        s2 += w * w;
    }
    return s1 * s1 / ((double)T * s2);
}

/* Next temperature increment.  If the whole remaining step keeps ESS >= rho T
 * take it; otherwise bisect [0, 1 - beta], keeping ESS(lo) >= rho T > ESS(hi),
 * until hi - lo <= 1e-7 hi (cap 200 halvings), and return lo. */
double orc_choose_delta(const double *e, int64_t T, double beta, double rho, int *final_step,
                        int *iters)
{
    double room = 1.0 - beta;
    *iters = 0;
    if (orc_ess_frac(e, T, room) >= rho) {
        *final_step = 1;
        return room;
    }
    double lo = 0.0, hi = room;
    int it = 0;
    while (it < 200 && hi - lo > 1e-7 * hi) {
        double mid = 0.5 * (lo + hi);
        if (orc_ess_frac(e, T, mid) >= rho)
            lo = mid;
        else
            hi = mid;
        ++it;
    }
    *iters = it;
    *final_step = 0;
    return lo > 0.0 ? lo : hi;
}

/* ------------------------------------------------------------------------- */
/* Systematic resampling on integer weights (Sec. II B 2: resample by the      */
/* normalised weights).  q_i = floor(w_i 2^40), Q = sum q, r = floor(U Q/2^32), */
/* t_m = floor((m Q + r) / M), ancestor a_m = min{ i : C_i > t_m } with C the  */
/* inclusive prefix sum -- written here as a plain forward scan.               */
/* ------------------------------------------------------------------------- */
void orc_quantise(const double *w, int64_t T, uint64_t *q)
{
    for (int64_t i = 0; i < T; ++i) q[i] = (uint64_t)floor(ldexp(w[i], 40));
}

void orc_resample(const uint64_t *q, int64_t T, int64_t M, uint32_t u32, int32_t *anc)
{
    unsigned __int128 Q = 0;
    for (int64_t i = 0; i < T; ++i) Q += q[i];
    unsigned __int128 r = ((unsigned __int128)u32 * Q) >> 32;
    int64_t i = 0;
    unsigned __int128 C = q[0];
    for (int64_t m = 0; m < M; ++m) {
        unsigned __int128 t = ((unsigned __int128)m * Q + r) / (unsigned __int128)M;
        while (C <= t) {
            ++i;
            C += q[i];
        }
        anc[m] = (int32_t)i;
    }
}

/* ------------------------------------------------------------------------- */
/* Metropolis rejuvenation (Sec. II B 4): component-wise random-walk MH, one   */
/* 1-D Gaussian proposal per component in fixed order, n sweeps per chain.     */
/* Counter (t d + j, chain, stage, K); z by Box-Muller from words 0, 1; the    */
/* accept uniform from word 2.  Out-of-support proposals count as rejections.  */
/* Waste-free mode (Sec. II B 3) keeps the state after every sweep.            */
/* ------------------------------------------------------------------------- */
static void mh_chains(ctx_t *c, const double *u_start, const double *E_start, int64_t S,
                      const double *step, double beta, uint32_t stage, double *u_out,
                      double *E_out, int64_t *acc, int64_t *prop, double *cur)
{
    const orc_job *job = c->job;
    int d = c->d, n = job->sweeps;
    uint32_t tag = (uint32_t)job->K;
    for (int j = 0; j < d; ++j) acc[j] = prop[j] = 0;
    for (int64_t m = 0; m < S; ++m) {
        memcpy(cur, u_start + (size_t)m * d, sizeof(double) * d);
        double Ec = E_start[m];
        for (int t = 0; t < n; ++t) {
            for (int j = 0; j < d; ++j) {
                if (c->pri[j].kind == PR_FIXED) continue;
                uint32_t ww[4];
                draw_words(job->seed, (uint32_t)(t * d + j), (uint32_t)m, stage, tag, ww);
                double z = box_muller(ww[0], ww[1]);
                double up = cur[j] + step[j] * z;
                prop[j]++;
                if (!in_support(c->pri[j], up)) continue;
                double dlp = log_prior(c->pri[j], up) - log_prior(c->pri[j], cur[j]);
                double old = cur[j];
                cur[j] = up;
                double Ep = energy_u(c, cur);
                if (log(u01(ww[2])) < -beta * (Ep - Ec) + dlp) {
                    Ec = Ep;
                    acc[j]++;
                } else {
                    cur[j] = old;
                }
            }
            if (job->waste_free) {
                memcpy(u_out + (size_t)(m * n + t) * d, cur, sizeof(double) * d);
                E_out[m * n + t] = Ec;
            }
        }
        if (!job->waste_free) {
            memcpy(u_out + (size_t)m * d, cur, sizeof(double) * d);
            E_out[m] = Ec;
        }
    }
}

static int setup_ctx(ctx_t *c, const orc_job *job)
{
    c->job = job;
    c->p = peak_params(job->family);
    c->nbg = bg_params(job->bg_kind, job->bg_degree);
    c->d = c->p * job->K + c->nbg;
    range_of(job->x, job->n, &c->xmin, &c->xmax);
    c->pri = (orc_prior *)malloc(sizeof(orc_prior) * (c->d > 0 ? c->d : 1));
    c->nat = (double *)malloc(sizeof(double) * (c->d > 0 ? c->d : 1));
    if (!c->pri || !c->nat) return ORC_ENOMEM;
    for (int j = 0; j < c->d; ++j) c->pri[j] = comp_prior(job, j);
    return ORC_OK;
}

/* Exported pieces so that tests can replay single steps. */

/* Prior draws for particles [0, count) in sampler coordinates, with energies. */
int orc_init_particles(const orc_job *job, int64_t count, double *u, double *E)
{
    ctx_t c;
    if (setup_ctx(&c, job) != ORC_OK) return ORC_ENOMEM;
    for (int64_t i = 0; i < count; ++i) {
        for (int j = 0; j < c.d; ++j)
            u[i * c.d + j] =
                orc_prior_draw(c.pri[j], job->seed, (uint32_t)j, (uint32_t)i, (uint32_t)job->K);
        E[i] = energy_u(&c, u + i * c.d);
    }
    free(c.pri);
    free(c.nat);
    return ORC_OK;
}

/* Energy of particles given in sampler coordinates. */
int orc_energies(const orc_job *job, int64_t count, const double *u, double *E)
{
    ctx_t c;
    if (setup_ctx(&c, job) != ORC_OK) return ORC_ENOMEM;
    for (int64_t i = 0; i < count; ++i) E[i] = energy_u(&c, u + i * c.d);
    free(c.pri);
    free(c.nat);
    return ORC_OK;
}

/* One Metropolis stage on S chain starts (already resampled). */
int orc_mh_stage(const orc_job *job, const double *u_start, const double *E_start, int64_t S,
                 const double *step, double beta, uint32_t stage, double *u_out, double *E_out,
                 int64_t *acc, int64_t *prop)
{
    ctx_t c;
    if (setup_ctx(&c, job) != ORC_OK) return ORC_ENOMEM;
    double *cur = (double *)malloc(sizeof(double) * (c.d > 0 ? c.d : 1));
    mh_chains(&c, u_start, E_start, S, step, beta, stage, u_out, E_out, acc, prop, cur);
    free(cur);
    free(c.pri);
    free(c.nat);
    return ORC_OK;
}

/* Step-size predictor from the histories of the inverse temperatures and of
 * a component's acceptance rates (Sec. II B 4 names such a predictor and
 * cites it without printing it; the model below is the reading taken).
 *   - For a one-dimensional Gaussian target of SD sigma and a Gaussian
 *     random-walk proposal of SD s the acceptance rate is
 *     (2/pi) atan(2 sigma / s); the rate a observed at step s (clamped to
 *     [0.02, 0.98]) therefore estimates sigma = s tan(pi a / 2) / 2.
 *   - log sigma is regressed on log beta over the stages run so far, each
 *     older stage at half the weight of the next (h holds the weighted sums
 *     W, X, Y, XX, XY and is updated in place); the slope is clamped to
 *     [-1, 0], and is -1/2 (a likelihood-dominated posterior) while only
 *     one stage has been seen.
 *   - The fit is extrapolated to beta_next and the step is the one whose
 *     acceptance rate there is 0.44: 2 sigma / tan(0.22 pi), kept within
 *     [0.01, 10] x the weighted population SD sd_pop. */
double orc_predict_step(double h[5], double s_prev, double acc, double beta_prev, double beta_next,
                        double sd_pop)
{
    double a = acc;
    if (a < 0.02) a = 0.02;
    if (a > 0.98) a = 0.98;
    double sig = s_prev * tan(M_PI * a / 2.0) / 2.0;
    double x = log(beta_prev), y = log(sig);
    for (int k = 0; k < 5; ++k) h[k] *= 0.5;
    h[0] += 1.0;
    h[1] += x;
    h[2] += y;
    h[3] += x * x;
    h[4] += x * y;
    double xm = h[1] / h[0], ym = h[2] / h[0];
    double sxx = h[3] / h[0] - xm * xm, sxy = h[4] / h[0] - xm * ym;
    double b = -0.5;
    if (h[0] > 1.25 && sxx > 1e-12) {
        b = sxy / sxx;
        if (b < -1.0) b = -1.0;
        if (b > 0.0) b = 0.0;
    }
    double st = 2.0 * exp(ym + b * (log(beta_next) - xm)) / tan(M_PI * 0.44 / 2.0);
    if (st < 0.01 * sd_pop) st = 0.01 * sd_pop;
    if (st > 10.0 * sd_pop) st = 10.0 * sd_pop;
    return st;
}

/* Step sizes for the next Metropolis stage, from the population u[T][d] under
 * the stage's incremental weights w (need not be normalised): sd_j = max(
 * weighted SD_j, 1e-9 (1 + |weighted mean_j|)).  Without acceptance rates
 * (the first stage), and always under step_rule 0: lambda_j <-
 * clamp(lambda_j exp(acc_j - 0.44), 0.01, 10) when rates are given, step_j =
 * lambda_j sd_j.  Under step_rule 1 with rates, history h[5 d] and the
 * previous steps in step[]: step_j = orc_predict_step(h + 5 j, step_j,
 * acc_j, beta_prev, beta_next, sd_j).  FIXED components get step 0. */
void orc_step_sizes_ex(const orc_job *job, const double *u, const double *w, int64_t T,
                       const double *acc_rate, double *lam, double *step, double *hist,
                       double beta_prev, double beta_next)
{
    ctx_t c;
    if (setup_ctx(&c, job) != ORC_OK) return;
    int d = c.d;
    double sw = 0.0;
    for (int64_t i = 0; i < T; ++i) sw += w[i];
    for (int j = 0; j < d; ++j) {
        if (c.pri[j].kind == PR_FIXED) {
            step[j] = 0.0;
            continue;
        }
        double m1 = 0.0;
        for (int64_t i = 0; i < T; ++i) m1 += w[i] * u[i * d + j];
        m1 /= sw;
        double v = 0.0;
        for (int64_t i = 0; i < T; ++i) {
            double t = u[i * d + j] - m1;
            v += w[i] * t * t;
        }
        v /= sw;
        double sd = sqrt(v);
        double floor_sd = 1e-9 * (1.0 + fabs(m1));
        if (sd < floor_sd) sd = floor_sd;
        if (acc_rate && job->step_rule == 1 && hist) {
            step[j] = orc_predict_step(hist + 5 * j, step[j], acc_rate[j], beta_prev, beta_next, sd);
            continue;
        }
        if (acc_rate) {
            lam[j] *= exp(acc_rate[j] - 0.44);
            if (lam[j] < 0.01) lam[j] = 0.01;
            if (lam[j] > 10.0) lam[j] = 10.0;
        }
        step[j] = lam[j] * sd;
    }
    free(c.pri);
    free(c.nat);
}

void orc_step_sizes(const orc_job *job, const double *u, const double *w, int64_t T,
                    const double *acc_rate, double *lam, double *step)
{
    orc_step_sizes_ex(job, u, w, T, acc_rate, lam, step, NULL, 0.0, 0.0);
}

/* ------------------------------------------------------------------------- */
/* One full SMC run for one (spectrum, K) job (Sec. II B 2-4).                 */
/* ------------------------------------------------------------------------- */
static int validate(const orc_job *job, int d)
{
    if (job->n < 2 || job->K < 0 || job->particles < 2 || job->sweeps < 1) return ORC_EINVAL;
    if (!(job->ess_target > 0.0 && job->ess_target < 1.0)) return ORC_EINVAL;
    if (job->n_comp_priors > 0 && job->n_comp_priors != d) return ORC_EINVAL;
    if (job->noise != NOISE_KNOWN && job->noise != NOISE_MODEL && job->noise != NOISE_POISSON)
        return ORC_EINVAL;
    if (job->family == FAM_XRD_PHASE && (!job->ref_off || job->K > job->n_phase)) return ORC_EINVAL;
    if (job->noise == NOISE_POISSON)
        for (int64_t i = 0; i < job->n; ++i)
            if (job->y[i] < 0.0) return ORC_EINVAL;
    for (int64_t i = 0; i < job->n; ++i) {
        if (!isfinite(job->y[i]) || !isfinite(job->x[i])) return ORC_EINVAL;
        if (job->noise == NOISE_KNOWN && (!(job->sigma[i] > 0.0) || !isfinite(job->sigma[i])))
            return ORC_EINVAL;
    }
    return ORC_OK;
}

int orc_run_job(const orc_job *job, orc_out *out)
{
    ctx_t c;
    int d = orc_dim(job->family, job->K, job->bg_kind, job->bg_degree);
    out->d = d;
    out->status = validate(job, d);
    if (out->status != ORC_OK) return out->status;
    if (setup_ctx(&c, job) != ORC_OK) return out->status = ORC_ENOMEM;

    int n = job->sweeps;
    int64_t T = job->particles;
    int64_t S = job->waste_free ? (T + n - 1) / n : T; /* chains per stage */
    int64_t Tc = job->waste_free ? S * n : T;          /* particles carried */
    uint32_t tag = (uint32_t)job->K;
    size_t dd = (size_t)(d > 0 ? d : 1);

    double *u = (double *)malloc(sizeof(double) * Tc * dd);
    double *un = (double *)malloc(sizeof(double) * Tc * dd);
    double *us = (double *)malloc(sizeof(double) * S * dd);
    double *E = (double *)malloc(sizeof(double) * Tc);
    double *En = (double *)malloc(sizeof(double) * Tc);
    double *Es = (double *)malloc(sizeof(double) * S);
    double *e = (double *)malloc(sizeof(double) * Tc);
    double *w = (double *)malloc(sizeof(double) * Tc);
    uint64_t *q = (uint64_t *)malloc(sizeof(uint64_t) * Tc);
    int32_t *anc = (int32_t *)malloc(sizeof(int32_t) * S);
    double *lam = (double *)malloc(sizeof(double) * dd);
    double *hist = (double *)calloc(5 * dd, sizeof(double));
    double *step = (double *)malloc(sizeof(double) * dd);
    double *rate = (double *)malloc(sizeof(double) * dd);
    int64_t *acc = (int64_t *)calloc(dd, sizeof(int64_t));
    int64_t *prop = (int64_t *)calloc(dd, sizeof(int64_t));
    double *cur = (double *)malloc(sizeof(double) * dd);
    if (!u || !un || !us || !E || !En || !Es || !e || !w || !q || !anc || !lam || !step ||
        !rate || !acc || !prop || !cur || !hist) {
        out->status = ORC_ENOMEM;
        goto done;
    }
    for (int j = 0; j < d; ++j) lam[j] = 2.38;

    /* normaliser of the known-sigma Gaussian likelihood (reading of App. C,
     * Eq. (C2)); the model-variance energy carries its own log terms */
    double lognorm = 0.0;
    if (job->noise == NOISE_KNOWN)
        for (int64_t i = 0; i < job->n; ++i) lognorm -= log(sqrt(2.0 * M_PI) * job->sigma[i]);
    if (job->noise == NOISE_POISSON) /* log p(y | f) = -e - (y - y ln y + ln y!) */
        for (int64_t i = 0; i < job->n; ++i) {
            double y = job->y[i];
            lognorm += (y > 0.0 ? y * log(y) : 0.0) - y - lgamma(y + 1.0);
        }

    /* stage 0: prior draws, beta_0 = 0 (Eq. (9)) */
    for (int64_t i = 0; i < Tc; ++i) {
        for (int j = 0; j < d; ++j)
            u[i * d + j] = orc_prior_draw(c.pri[j], job->seed, (uint32_t)j, (uint32_t)i, tag);
        E[i] = energy_u(&c, u + i * d);
    }
    double beta = 0.0, logz = lognorm;
    if (out->beta_trace) out->beta_trace[0] = 0.0;
    if (out->logz_trace) out->logz_trace[0] = logz;
    out->status = ORC_OK;

    int stage = 0;
    for (;;) {
        ++stage;
        if (stage > job->max_stages) {
            out->status = ORC_EMAXSTAGES;
            stage = job->max_stages;
            break;
        }
        /* -- reweight: incremental weights (Eq. (10)), next beta by bisection */
        double emin = INFINITY;
        for (int64_t i = 0; i < Tc; ++i)
            if (isfinite(E[i]) && E[i] < emin) emin = E[i];
        if (!isfinite(emin)) {
            out->status = ORC_ENUMERIC;
            break;
        }
        for (int64_t i = 0; i < Tc; ++i) e[i] = isfinite(E[i]) ? E[i] - emin : INFINITY;
        int final_step = 0, iters = 0;
        double delta = orc_choose_delta(e, Tc, beta, job->ess_target, &final_step, &iters);
        double sw = 0.0;
        for (int64_t i = 0; i < Tc; ++i) {
            w[i] = isfinite(e[i]) ? exp(-delta * e[i]) : 0.0;
            sw += w[i];
        }
        /* -- evidence increment: log of the mean unnormalised weight (Eq. (11)) */
        logz += -delta * emin + log(sw / (double)Tc);
        const double beta_prev = beta;
        beta = final_step ? 1.0 : beta + delta;

        /* -- step sizes from the reweighted population and last acceptance */
        if (stage > 1)
            for (int j = 0; j < d; ++j) rate[j] = prop[j] ? (double)acc[j] / (double)prop[j] : 0.44;
        orc_step_sizes_ex(job, u, w, Tc, stage > 1 ? rate : NULL, lam, step, hist, beta_prev, beta);
        if (out->step_trace)
            for (int j = 0; j < d; ++j) out->step_trace[(size_t)stage * d + j] = step[j];

        /* -- systematic resampling of S ancestors */
        orc_quantise(w, Tc, q);
        uint32_t rw[4];
        draw_words(job->seed, 0u, 0xFFFFFFFFu, (uint32_t)stage, tag, rw);
        orc_resample(q, Tc, S, rw[0], anc);
        for (int64_t m = 0; m < S; ++m) {
            memcpy(us + (size_t)m * d, u + (size_t)anc[m] * d, sizeof(double) * d);
            Es[m] = E[anc[m]];
        }

        /* -- Metropolis rejuvenation at beta */
        mh_chains(&c, us, Es, S, step, beta, (uint32_t)stage, un, En, acc, prop, cur);
        {
            double *tp = u; u = un; un = tp;
            tp = E; E = En; En = tp;
        }
        if (out->beta_trace) out->beta_trace[stage] = beta;
        if (out->logz_trace) out->logz_trace[stage] = logz;
        if (out->acc_trace)
            for (int j = 0; j < d; ++j)
                out->acc_trace[(size_t)stage * d + j] =
                    prop[j] ? (double)acc[j] / (double)prop[j] : 0.0;
        if (beta >= 1.0) break;
    }
    out->log_z = logz;
    out->n_stages = stage;
    out->n_out = Tc;
    if (out->samples)
        for (int64_t i = 0; i < Tc; ++i)
            for (int j = 0; j < d; ++j)
                out->samples[i * d + j] = to_natural(c.pri[j], u[i * d + j]);
    if (out->energies)
        for (int64_t i = 0; i < Tc; ++i) out->energies[i] = E[i];

done:
    free(c.pri); free(c.nat); free(u); free(un); free(us); free(E); free(En); free(Es);
    free(e); free(w); free(q); free(anc); free(lam); free(step); free(rate); free(acc);
    free(prop); free(cur); free(hist);
    return out->status;
}
