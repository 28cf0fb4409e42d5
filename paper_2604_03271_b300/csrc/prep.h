// prep.h -- spectrum descriptors used by the preparation kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "smc_device.cuh"

namespace smc {

struct SpecScal {
    double xmin, xmax, x_ref, t_scale, t_off, lognorm;
    int bad;
    int pad_;
};

struct SpecDev {
    float *xc, *wt, *y, *ts, *sec2;
    double *x64, *y64, *is64, *tn64, *sc64;
    SpecScal *scal;
    // App. D reflections: absolute (FP64, uploaded) and centred (FP32, by prep)
    double *rpos64, *rint64;
    float4 *rtab;
    int *roff;
    int nref;
};

// noise = NZ_MODEL: sigma is not read (wt = 1 on grid points, lognorm = 0);
// NZ_POISSON: sigma not read, wt = 1, y >= 0 required, lognorm = sum [y ln y -
// y - ln Gamma(y + 1)].  coord = 1 (Shirley): ts holds |x_i - x_{i-1}| (0 at
// the first point); coord = 2 (App. D): ts = tan(x/2), sec2 = 1/cos(x/2) (x in
// degrees; FP64 copies in tn64 / sc64) and the sd.nref reflections are centred into rtab = (x - x_ref, I, log2 I, 0); otherwise
// ts is the Chebyshev coordinate.  Padding points have wt = 0 (and ts = 0).
cudaError_t launch_spec_prep(const double *x, const double *y, const double *sg, int n, int n_pad,
                             int centre, int noise, int coord, const SpecDev &sd, cudaStream_t s);
cudaError_t launch_job_setup(JobDev *jobs, const int *slots, const SpecScal *scal,
                             int nslots, cudaStream_t s);
cudaError_t launch_posterior(const JobDev *jobs, const int *slots, const int *off, int nreq,
                             double *pk, cudaStream_t s);

}  // namespace smc
