// k_prep.cu -- device-side preparation of a spectrum and its jobs, and the
// posterior over K.
//
//   spectrum prep: x range, centring offset x_ref = (x_min + x_max)/2, the
//   Chebyshev coordinate t = (2x - (x_min + x_max))/(x_max - x_min), the
//   Gaussian-likelihood normaliser -sum log(sqrt(2 pi) sigma_i), and the FP32
//   padded arrays xc = x - x_ref, wt = 1/sigma^2, y, t used by the kernels.
//   job setup: copies those scalars into each job and shifts centre priors of
//   FP32 jobs by -x_ref.
//   posterior over K: p(K|D) = exp(log Z_K) / sum_k exp(log Z_k), uniform p(K)
//   (Sec. II A, Eq. (2)).
#include <cmath>

#include "kernels.h"
#include "prep.h"

namespace smc {

__global__ void __launch_bounds__(1024) k_spec_prep(const double *x, const double *y,
                                                    const double *sg, int n, int n_pad,
                                                    int centre, int noise, int coord, SpecDev sd)
{
    __shared__ double r0[32], r1[32], r2[32];
    __shared__ double s_lo, s_hi;
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double lo = INFINITY, hi = -INFINITY, ln = 0.0;
    int bad = 0;
    for (int i = tid; i < n; i += blockDim.x) {
        const double xi = x[i], yi = y[i];
        if (!isfinite(xi) || !isfinite(yi)) bad = 1;
        if (noise == NZ_KNOWN) {
            const double si = sg[i];
            if (!isfinite(si) || !(si > 0.0)) bad = 1;
            ln -= log(sqrt(2.0 * 3.141592653589793) * si);
        } else if (noise == NZ_POISSON) {
            if (!(yi >= 0.0)) bad = 1;
            ln += (yi > 0.0 ? yi * log(yi) : 0.0) - yi - lgamma(yi + 1.0);
        }
        lo = fmin(lo, xi);
        hi = fmax(hi, xi);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(FULL_MASK, lo, o));
        hi = fmax(hi, __shfl_xor_sync(FULL_MASK, hi, o));
        ln += __shfl_xor_sync(FULL_MASK, ln, o);
    }
    bad = __syncthreads_or(bad);
    if (lane == 0) {
        r0[warp] = lo;
        r1[warp] = hi;
        r2[warp] = ln;
    }
    __syncthreads();
    if (tid == 0) {
        double a = r0[0], b = r1[0], c = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a = fmin(a, r0[w]);
            b = fmax(b, r1[w]);
            c += r2[w];
        }
        s_lo = a;
        s_hi = b;
        s_bad = bad || !(b > a);
        sd.scal->xmin = a;
        sd.scal->xmax = b;
        sd.scal->x_ref = centre ? 0.5 * (a + b) : 0.0;
        sd.scal->t_scale = 2.0 / (b - a);
        sd.scal->t_off = -(a + b) / (b - a);
        sd.scal->lognorm = c;
        sd.scal->bad = s_bad;
    }
    __syncthreads();
    const double xmin = s_lo, xmax = s_hi;
    const double xref = centre ? 0.5 * (xmin + xmax) : 0.0;
    for (int i = tid; i < n_pad; i += blockDim.x) {
        if (i < n) {
            const double xi = x[i];
            sd.xc[i] = (float)(xi - xref);
            sd.wt[i] = noise == NZ_KNOWN ? (float)(1.0 / (sg[i] * sg[i])) : 1.0f;
            sd.y[i] = (float)y[i];
            if (coord == 1) {
                sd.ts[i] = i > 0 ? (float)fabs(xi - x[i - 1]) : 0.0f;
            } else if (coord == 2) {
                const double th = xi * (3.141592653589793 / 360.0);
                const double t = tan(th), c = 1.0 / cos(th);
                sd.ts[i] = (float)t;
                sd.sec2[i] = (float)c;
                sd.tn64[i] = t;
                sd.sc64[i] = c;
            } else {
                sd.ts[i] = (float)((2.0 * xi - (xmin + xmax)) / (xmax - xmin));
            }
            sd.x64[i] = xi;
            sd.y64[i] = y[i];
            sd.is64[i] = noise == NZ_KNOWN ? 1.0 / sg[i] : 1.0;
        } else if (coord == 2) {
            sd.xc[i] = 0.0f;
            sd.wt[i] = 0.0f;
            sd.y[i] = 0.0f;
            sd.ts[i] = 0.0f;
            sd.sec2[i] = 1.0f;
        } else {
            sd.xc[i] = 0.0f;
            sd.wt[i] = 0.0f;
            sd.y[i] = 0.0f;
            sd.ts[i] = 0.0f;
        }
    }
    for (int j = tid; j < sd.nref; j += blockDim.x) {
        const double I = sd.rint64[j];
        sd.rtab[j] = make_float4((float)(sd.rpos64[j] - xref), (float)I, (float)log2(I), 0.0f);
    }
}

cudaError_t launch_spec_prep(const double *x, const double *y, const double *sg, int n, int n_pad,
                             int centre, int noise, int coord, const SpecDev &sd, cudaStream_t s)
{
    k_spec_prep<<<1, 1024, 0, s>>>(x, y, sg, n, n_pad, centre, noise, coord, sd);
    return cudaGetLastError();
}

__device__ void shift_prior(PriorDev &p, double off)
{
    if (!p.is_centre || off == 0.0) return;
    if (p.kind == PR_UNIFORM) {
        p.p1 -= off;
        p.p2 -= off;
        p.lo = p.p1;
        p.hi = p.p2;
    } else if (p.kind == PR_NORMAL || p.kind == PR_FIXED) {
        p.p1 -= off;
    }
    p.lof = (float)p.lo;
    p.hif = (float)p.hi;
    p.a = (float)p.p1;
    p.b = (float)p.p2;
}

__global__ void k_job_setup(JobDev *jobs, const int *slots, const SpecScal *scal)
{
    JobDev &jb = jobs[slots[blockIdx.x]];
    const SpecScal &sc = *scal;
    if (threadIdx.x == 0) {
        jb.x_ref = sc.x_ref;
        jb.t_scale = sc.t_scale;
        jb.t_off = sc.t_off;
        jb.lognorm = sc.lognorm;
        jb.logz = sc.lognorm;
        if (sc.bad) {
            jb.status = 1;  // SMC_EINVAL
            jb.state = JOB_DONE;
        }
    }
    PriorDev *pri = const_cast<PriorDev *>(jb.pri);
    for (int j = threadIdx.x; j < jb.d; j += blockDim.x) shift_prior(pri[j], sc.x_ref);
}

cudaError_t launch_job_setup(JobDev *jobs, const int *slots, const SpecScal *scal, int nslots,
                             cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    k_job_setup<<<nslots, 64, 0, s>>>(jobs, slots, scal);
    return cudaGetLastError();
}

// posterior over K for each request: slots[off[r] .. off[r+1]) are its jobs
__global__ void k_posterior(const JobDev *jobs, const int *slots, const int *off, int nreq,
                            double *pk)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nreq) return;
    double mx = -INFINITY;
    for (int a = off[r]; a < off[r + 1]; ++a) {
        const JobDev &jb = jobs[slots[a]];
        if (jb.status == 0) mx = fmax(mx, jb.logz);
    }
    double s = 0.0;
    for (int a = off[r]; a < off[r + 1]; ++a) {
        const JobDev &jb = jobs[slots[a]];
        s += jb.status == 0 ? exp(jb.logz - mx) : 0.0;
    }
    for (int a = off[r]; a < off[r + 1]; ++a) {
        const JobDev &jb = jobs[slots[a]];
        pk[a] = (jb.status == 0 && s > 0.0) ? exp(jb.logz - mx) / s : 0.0;
    }
}

cudaError_t launch_posterior(const JobDev *jobs, const int *slots, const int *off, int nreq,
                             double *pk, cudaStream_t s)
{
    if (nreq <= 0) return cudaSuccess;
    k_posterior<<<(nreq + 127) / 128, 128, 0, s>>>(jobs, slots, off, nreq, pk);
    return cudaGetLastError();
}

}  // namespace smc
