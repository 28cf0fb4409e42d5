// temper.cuh -- per-component step-size update shared by the tempering kernels.
#pragma once
#include "smc_device.cuh"

namespace smc {

// Step size of component j for the next Metropolis stage (Sec. II B 4), from
// the weighted mean and variance of the reweighted population:
// s_j = lambda_j max(SD_j, 1e-9 (1 + |mean_j|)), with lambda_j adapted from
// the previous stage's acceptance rate, lambda <- clamp(lambda e^(rate - 0.44),
// 0.01, 10).  Resets the acceptance counters.
__device__ __forceinline__ void update_step(JobDev &jb, int j, double mean, double var)
{
    if (jb.pri[j].kind == PR_FIXED) {
        jb.step[j] = 0.0;
        jb.stepf[j] = 0.0f;
    } else {
        double sd = sqrt(fmax(var, 0.0));
        const double floor_sd = 1e-9 * (1.0 + fabs(mean));
        if (sd < floor_sd) sd = floor_sd;
        double lam = jb.lam[j];
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
