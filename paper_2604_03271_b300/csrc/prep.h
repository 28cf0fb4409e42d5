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
    float *xc, *wt, *y, *ts;
    double *x64, *y64, *is64;
    SpecScal *scal;
};

// noise = NZ_MODEL: sigma is not read (wt = 1 on grid points, lognorm = 0);
// shirley = 1: ts holds |x_i - x_{i-1}| (0 at the first point) instead of the
// Chebyshev coordinate.  Padding points have wt = 0 (and ts = 0).
cudaError_t launch_spec_prep(const double *x, const double *y, const double *sg, int n, int n_pad,
                             int centre, int noise, int shirley, const SpecDev &sd, cudaStream_t s);
cudaError_t launch_job_setup(JobDev *jobs, const int *slots, const SpecScal *scal,
                             int nslots, cudaStream_t s);
cudaError_t launch_posterior(const JobDev *jobs, const int *slots, const int *off, int nreq,
                             double *pk, cudaStream_t s);

}  // namespace smc
