// k_plain.cu -- the plain FP64 Metropolis stage: one thread per chain, every
// proposal recomputes the whole forward model and energy in double precision.
// This is the straightforward GPU form of the component-wise random-walk
// Metropolis of Sec. II B 4, used as the one-spectrum-per-launch baseline and
// for replay parity with the FP64 oracle (same counters, same arithmetic).
#include <cmath>

#include "kernels.h"
#include "plain_device.cuh"

namespace smc {

__global__ void __launch_bounds__(128) k_mh_plain(JobDev *jobs, const int *slots)
{
    JobDev &jb = jobs[slots[blockIdx.y]];
    if (jb.state != JOB_ACTIVE || jb.status != 0) return;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= jb.S) return;
    const int d = jb.d, S = jb.S, T = jb.T, n = jb.sweeps;
    const double beta = jb.beta;
    const uint32_t stage = (uint32_t)(jb.stage + 1);
    double u[SMC_DMAX], nat[SMC_DMAX];
    unsigned acc[SMC_DMAX], prp[SMC_DMAX];
    for (int j = 0; j < d; ++j) {
        u[j] = jb.ths64[(size_t)j * S + m];
        nat[j] = natural_d(jb.pri[j], u[j]);
        acc[j] = prp[j] = 0u;
    }
    double Ec = jb.Es64[m];
    unsigned long long n_eval = 0;
    for (int t = 0; t < n; ++t) {
        for (int j = 0; j < d; ++j) {
            const PriorDev &pr = jb.pri[j];
            if (pr.kind == PR_FIXED) continue;
            const uint4 wv = draw(jb.seed, (uint32_t)(t * d + j), (uint32_t)m, stage, jb.tag);
            const double z = box_muller_d(wv.x, wv.y);
            const double up = u[j] + jb.step[j] * z;
            prp[j] += 1u;
            if (!in_support_d(pr, up)) continue;
            const double dlp = log_prior_d(pr, up) - log_prior_d(pr, u[j]);
            ++n_eval;
            const double old = u[j], oldn = nat[j];
            u[j] = up;
            nat[j] = natural_d(pr, up);
            const double Ep = energy_plain(jb, nat);
            if (log(u01d(wv.z)) < -beta * (Ep - Ec) + dlp) {
                Ec = Ep;
                acc[j] += 1u;
            } else {
                u[j] = old;
                nat[j] = oldn;
            }
        }
        if (jb.waste_free) {
            const size_t o = (size_t)m * n + t;
            for (int j = 0; j < d; ++j) jb.th64[(size_t)j * T + o] = u[j];
            jb.E64[o] = Ec;
        }
    }
    if (!jb.waste_free) {
        for (int j = 0; j < d; ++j) jb.th64[(size_t)j * T + m] = u[j];
        jb.E64[m] = Ec;
    }
    atomicAdd(&jb.point_evals, n_eval * (unsigned long long)jb.n);
    for (int j = 0; j < d; ++j)
        if (jb.pri[j].kind != PR_FIXED) {
            atomicAdd(&jb.acc[j], (unsigned long long)acc[j]);
            atomicAdd(&jb.prop[j], (unsigned long long)prp[j]);
        }
}

cudaError_t launch_mh_plain(JobDev *jobs, const int *slots, int nslots, int max_S,
                            cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    dim3 g((max_S + 127) / 128, nslots);
    k_mh_plain<<<g, 128, 0, s>>>(jobs, slots);
    return cudaGetLastError();
}

}  // namespace smc
