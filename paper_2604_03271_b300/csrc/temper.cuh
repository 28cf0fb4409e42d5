// temper.cuh -- per-component step-size update shared by the tempering kernels.
#pragma once
#include "smc_device.cuh"

namespace smc {

// Step predicted from the histories of the inverse temperatures and of the
// component's acceptance rates (Sec. II B 4): a rate a observed at step s on
// a one-dimensional Gaussian target of SD sigma satisfies a = (2/pi)
// atan(2 sigma / s), so sigma = s tan(pi a / 2) / 2 (a clamped to
// [0.02, 0.98]); log sigma is regressed on log beta over the stages so far,
// each older stage at half the weight of the next (h: sums W, X, Y, XX, XY,
// updated in place), slope clamped to [-1, 0] and -1/2 while one stage has
// been seen; extrapolated to beta_next, the step is the one of acceptance
// 0.44 there, 2 sigma / tan(0.22 pi), within [0.01, 10] x the population SD.
__device__ __forceinline__ double predict_step(double *h, double s_prev, double acc, double beta_prev,
                                               double beta_next, double sd_pop)
{
    const double a = fmin(fmax(acc, 0.02), 0.98);
    const double sig = s_prev * tan(SMC_PI * a / 2.0) / 2.0;
    const double x = log(beta_prev), y = log(sig);
    double h0 = 0.5 * h[0], h1 = 0.5 * h[1], h2 = 0.5 * h[2], h3 = 0.5 * h[3], h4 = 0.5 * h[4];
    h0 += 1.0;
    h1 += x;
    h2 += y;
    h3 += x * x;
    h4 += x * y;
    h[0] = h0;
    h[1] = h1;
    h[2] = h2;
    h[3] = h3;
    h[4] = h4;
    const double xm = h1 / h0, ym = h2 / h0;
    const double sxx = h3 / h0 - xm * xm, sxy = h4 / h0 - xm * ym;
    double b = -0.5;
    if (h0 > 1.25 && sxx > 1e-12) b = fmin(fmax(sxy / sxx, -1.0), 0.0);
    const double st = 2.0 * exp(ym + b * (log(beta_next) - xm)) / tan(SMC_PI * 0.44 / 2.0);
    return fmin(fmax(st, 0.01 * sd_pop), 10.0 * sd_pop);
}

// Step size of component j for the next Metropolis stage (Sec. II B 4), from
// the weighted mean and variance of the reweighted population:
// s_j = lambda_j max(SD_j, 1e-9 (1 + |mean_j|)), with lambda_j adapted from
// the previous stage's acceptance rate, lambda <- clamp(lambda e^(rate - 0.44),
// 0.01, 10); or, with step_rule 1 once a stage has run, the history
// predictor above at the move from beta_prev to beta_next.  Resets the
// acceptance counters.
__device__ __forceinline__ void update_step(JobDev &jb, int j, double mean, double var,
                                            double beta_prev, double beta_next)
{
    if (jb.pri[j].kind == PR_FIXED) {
        jb.step[j] = 0.0;
        jb.stepf[j] = 0.0f;
    } else {
        double sd = sqrt(fmax(var, 0.0));
        const double floor_sd = 1e-9 * (1.0 + fabs(mean));
        if (sd < floor_sd) sd = floor_sd;
        double lam = jb.lam[j];
        if (jb.step_rule == 1 && jb.stage >= 1) {
            const unsigned long long pr = jb.prop[j];
            const double rate = pr ? (double)jb.acc[j] / (double)pr : 0.44;
            const double st = predict_step(jb.hist + 5 * j, jb.step[j], rate, beta_prev, beta_next, sd);
            jb.step[j] = st;
            jb.stepf[j] = (float)st;
            jb.acc[j] = 0ull;
            jb.prop[j] = 0ull;
            return;
        }
        if (jb.stage >= 1) {
            const unsigned long long pr = jb.prop[j];
            const double rate = pr ? (double)jb.acc[j] / (double)pr : 0.44;
            lam *= exp(rate - 0.44);
            lam = fmin(fmax(lam, 0.01), 10.0);
            jb.lam[j] = lam;
        }
        jb.step[j] = lam * sd;
        jb.stepf[j] = (float)(lam * sd);
    }
    jb.acc[j] = 0ull;
    jb.prop[j] = 0ull;
}

}  // namespace smc
