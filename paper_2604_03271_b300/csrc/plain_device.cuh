// plain_device.cuh -- FP64 forward model and energy of the plain path.
// One thread evaluates a whole particle: sum over the grid of the K peaks
// (Eq. (1)) and the Chebyshev background, E = 1/2 sum ((y - f)/sigma)^2.
#pragma once
#include "smc_device.cuh"

// Gaussian: w is the standard deviation, or the precision b when wprec = 1
// (App. C Eq. (C1)); Lorentzian / pseudo-Voigt: w is the HWHM.
__device__ __forceinline__ double peak_eval_d(int fam, int wprec, double x, double A, double mu,
                                              double w, double eta)
{
    const double dx = x - mu;
    if (fam == FAM_GAUSS) return wprec ? A * exp(-0.5 * w * dx * dx) : A * exp(-dx * dx / (2.0 * w * w));
    const double lor = w * w / (w * w + dx * dx);
    if (fam == FAM_LORENTZ) return A * lor;
    const double sg = w / sqrt(2.0 * 0.69314718055994530942);
    return A * (eta * exp(-dx * dx / (2.0 * sg * sg)) + (1.0 - eta) * lor);
}

// sum of the K peaks at x (natural parameters)
__device__ __forceinline__ double peaks_at_d(const JobDev &jb, const double *nat, double x)
{
    double f = 0.0;
    for (int k = 0; k < jb.K; ++k) {
        const double *q = nat + jb.p * k;
        f += peak_eval_d(jb.family, jb.wprec, x, q[0], q[1], q[2], jb.p == 4 ? q[3] : 0.0);
    }
    return f;
}

// App. D pseudo-Voigt (1 - r) G + r L, G = exp(-4 ln 2 z^2 / S^2), L = 1 /
// (1 + 4 z^2 / W^2), from iS2 = 1/S^2 and iW2 = 1/W^2 (0 where the width is
// not positive, which makes that part 0)
__device__ __forceinline__ double xrd_pv_d(double z, double iS2, double iW2, double r)
{
    const double z2 = z * z;
    const double g = iS2 > 0.0 ? exp(-4.0 * 0.69314718055994530942 * z2 * iS2) : 0.0;
    const double l = iW2 > 0.0 ? 1.0 / (1.0 + 4.0 * z2 * iW2) : 0.0;
    return (1.0 - r) * g + r * l;
}

// App. D phases (Caglioti widths, asymmetry alpha scaling both widths right of
// each reflection) and PV background at grid point pt
__device__ __forceinline__ double xrd_model_d(const JobDev &jb, const double *nat, int pt)
{
    const double x = jb.x64[pt], tn = jb.tn64[pt], sc = jb.sc64[pt];
    double f = 0.0;
    for (int k = 0; k < jb.K; ++k) {
        const double *q = nat + 9 * k;
        const double rad = q[4] * tn * tn - q[5] * tn + q[6], W0 = q[7] * sc + q[8] * tn;
        const double iS2 = rad > 0.0 ? 1.0 / rad : 0.0, iW2 = W0 > 0.0 ? 1.0 / (W0 * W0) : 0.0;
        const double ia = 1.0 / q[2];
        double sum = 0.0;
        for (int j = jb.roff[k]; j < jb.roff[k + 1]; ++j) {
            const double mu = jb.rpos64[j] + q[1], dx = x - mu;
            sum += jb.rint64[j] * xrd_pv_d(x >= mu ? dx * ia : dx, iS2, iW2, q[3]);
        }
        f += q[0] * sum;
    }
    if (jb.bg_kind == BGK_XRD_PV) {
        const double *b = nat + 9 * jb.K;
        const double i2 = b[1] > 0.0 ? 1.0 / (b[1] * b[1]) : 0.0;
        f += b[0] * xrd_pv_d(x, i2, i2, b[2]) + b[3];
    }
    return f;
}

// Poisson energy term (f - y) - y ln(f / y) (f for y = 0, +inf for f <= 0)
__device__ __forceinline__ double poisson_term_d(double f, double y)
{
    if (!(f > 0.0)) return INFINITY;
    if (y == 0.0) return f;
    return (f - y) - y * log(f / y);
}

// Coupled-grid likelihoods (App. E): Shirley background B_i = a + (b - a)
// C_i / C_N with C_i = sum_{1 < j <= i} P_j |x_j - x_{j-1}| (B = a if C_N = 0),
// and the known-sigma or the model-variance energy
// sum [1/2 ln(2 pi v) + 1/2 (y - f)^2 / v], v = nd0 f + nd1 f^2 + nd2.
__device__ __forceinline__ double energy_plain_full(const JobDev &jb, const double *nat)
{
    const bool shir = jb.bg_kind == BGK_SHIRLEY, model = jb.noise == NZ_MODEL;
    double a = 0.0, b = 0.0, total = 0.0;
    if (shir) {
        a = nat[jb.p * jb.K];
        b = nat[jb.p * jb.K + 1];
        for (int pt = 1; pt < jb.n; ++pt)
            total += peaks_at_d(jb, nat, jb.x64[pt]) * fabs(jb.x64[pt] - jb.x64[pt - 1]);
    }
    double e = 0.0, run = 0.0;
    for (int pt = 0; pt < jb.n; ++pt) {
        const double x = jb.x64[pt];
        const double P = jb.family == FAM_XRD ? xrd_model_d(jb, nat, pt) : peaks_at_d(jb, nat, x);
        double f = P;
        if (shir) {
            if (pt > 0) run += P * fabs(x - jb.x64[pt - 1]);
            f += total > 0.0 ? a + (b - a) * run / total : a;
        }
        const double r = jb.y64[pt] - f;
        if (jb.noise == NZ_POISSON) {
            e += poisson_term_d(f, jb.y64[pt]);
            if (!(e < INFINITY)) return INFINITY;
        } else if (!model) {
            const double rs = r * jb.is64[pt];
            e += 0.5 * rs * rs;
        } else {
            const double v = jb.nd0 * f + jb.nd1 * f * f + jb.nd2;
            if (!(v > 0.0)) return INFINITY;
            e += 0.5 * log(2.0 * 3.141592653589793 * v) + 0.5 * r * r / v;
        }
    }
    return e;
}

__device__ __forceinline__ double energy_plain(const JobDev &jb, const double *nat)
{
    if (jb.full) return energy_plain_full(jb, nat);
    double e = 0.0;
    for (int pt = 0; pt < jb.n; ++pt) {
        const double x = jb.x64[pt];
        double f = 0.0;
        for (int k = 0; k < jb.K; ++k) {
            const double *q = nat + jb.p * k;
            f += peak_eval_d(jb.family, jb.wprec, x, q[0], q[1], q[2], jb.p == 4 ? q[3] : 0.0);
        }
        if (jb.nbg > 0) {
            const double t = x * jb.t_scale + jb.t_off;
            double a = 1.0, b = t;
            for (int q = 0; q < jb.nbg; ++q) {
                double tq;
                if (q == 0)
                    tq = 1.0;
                else if (q == 1)
                    tq = t;
                else {
                    tq = 2.0 * t * b - a;
                    a = b;
                    b = tq;
                }
                f += nat[jb.p * jb.K + q] * tq;
            }
        }
        const double r = (jb.y64[pt] - f) * jb.is64[pt];
        e += 0.5 * r * r;
    }
    return e;
}
