// smc_device.cuh -- device-side data layout and helpers shared by the kernels.
//
// Layout in HBM (one job = one (spectrum, K) sampler):
//   spectrum  xc[n_pad], wt[n_pad], y[n_pad], ts[n_pad]  FP32, padded with wt = 0
//             x64/y64/is64[n]                              FP64 originals (plain path)
//   particles th[d][T], E[T]        FP32 sampling coordinates (SoA, component-major)
//             ths[d][S], Es[S]       chain starts written by the gather kernel
//             th64/E64/ths64/Es64    same in FP64 for the plain path
//   tempering w64[T] FP64 weights, q[T] uint64, anc[S] int32, lam/step[d] FP64,
//             stepf[d] FP32, acc/prop[d] uint64 counters
// Centre components of FP32 jobs are stored relative to x_ref (the middle of
// the grid) so that FP32 differences x - mu keep their precision on offset axes.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define SMC_DMAX 128
#define SMC_KMAX 32

enum { FAM_GAUSS = 0, FAM_LORENTZ = 1, FAM_PV = 2, FAM_XRD = 4 };  // FAM_XRD: App. D phases
enum { PR_UNIFORM = 0, PR_LOG_UNIFORM = 1, PR_NORMAL = 2, PR_GAMMA = 3, PR_FIXED = 4 };
enum { JOB_FREE = 0, JOB_ACTIVE = 1, JOB_DONE = 2 };
enum { BGK_SHIRLEY = 4, BGK_XRD_PV = 5 };  // smc_bg values of the coupled backgrounds
enum { NZ_KNOWN = 0, NZ_MODEL = 1, NZ_POISSON = 2 };  // smc_noise values

// Prior of one component in sampling coordinates.
//   support [lo, hi] (UNIFORM, LOG_UNIFORM), u > 0 (GAMMA), all (NORMAL)
//   log density (up to a constant): NORMAL -(u-p1)^2/(2 p2^2); GAMMA (p1-1) log u - p2 u
// For centre components of FP32 jobs every coordinate is already shifted by -x_ref.
struct PriorDev {
    int kind;
    int is_centre;
    double p1, p2;   // natural parameters (centre ones shifted)
    double lo, hi;   // support in sampling coordinates (FP64)
    float lof, hif;  // same, FP32
    float a, b;      // log-density parameters p1, p2 in FP32
};

struct JobDev {
    // spectrum
    const float *xc, *wt, *y, *ts;
    const double *x64, *y64, *is64;
    const double *tn64, *sc64;  // App. D: tan(x/2), 1/cos(x/2) in FP64
    int n, n_pad;
    double x_ref;          // centring offset of centre coordinates
    double t_scale, t_off; // Chebyshev coordinate t = x * t_scale + t_off (raw x)
    // model (family: kernel family; wprec: Gaussian width given as precision b;
    // bg_kind: SMC_BG_*; noise: SMC_NOISE_*, variance nv0 f + nv1 f^2 + nv2 with
    // nv = squares of noise_par (FP32 and FP64 copies); full: coupled-grid kernel)
    int family, K, p, nbg, d, wprec;
    int bg_kind, noise, full;
    float nv0, nv1, nv2;
    double nd0, nd1, nd2;
    // App. D phases: per grid point tan(x/2) (in ts) and 1/cos(x/2); reflections
    // roff[k] .. roff[k+1] - 1 of phase k: centred positions and intensities
    // (FP32), absolute positions and intensities (FP64)
    const float *sec2;
    const float4 *rtab;  // App. D reflections: (centred position, I, log2 I, 0)
    const double *rpos64, *rint64;
    const int *roff;
    // tile of the Metropolis kernel (points per lane J, warps per chain G,
    // register budget R, 0 = the tile's default)
    int J, G, R;
    // particles
    int T, S, sweeps, waste_free, fp64;
    float *th, *E, *ths, *Es;
    double *th64, *E64, *ths64, *Es64;
    double *w64;           // weights (FP32 jobs: FP32 weights in the first half)
    double *rwpart;        // FP32 jobs: rw_split(T) rows of 1 + 2 d tempering partial sums
    unsigned long long *q;
    int *anc;
    double *lam, *step;
    float *stepf;
    int step_rule;   // 0: lambda x population SD; 1: history predictor
    double *hist;    // step_rule 1: per component (W, X, Y, XX, XY) regression sums
    unsigned long long *acc, *prop;
    const PriorDev *pri;
    // tempering state
    double beta, logz, lognorm, rho, delta, emin;
    int stage, max_stages, status, state, final_step, bisect_iters;
    int next_chain;  // dynamic work counter of the Metropolis kernel
    unsigned tag;
    unsigned long long seed;
    // cumulative algorithmic work of the Metropolis kernel: grid-point
    // evaluations of in-support proposals, and SFU operations of the
    // shape-changing (centre, width) proposals among them
    unsigned long long point_evals, sfu_ops, var_ops;  // var_ops: LG2 + RCP of the model variance
    unsigned long long ex2_part;  // the EX2 share of sfu_ops (App. D phase kernel)
    // grid-point evaluations of evaluated peak-component proposals (fused
    // peak kernel only): the units whose per-unit SFU cost is one EX2
    // (Gaussian), one RCP (Lorentzian) or one of each (pseudo-Voigt)
    unsigned long long peak_evals;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products, key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw(unsigned long long seed, uint32_t c0, uint32_t c1,
                                      uint32_t c2, uint32_t c3)
{
    return philox10(make_uint4(c0, c1, c2, c3), (uint32_t)seed, (uint32_t)(seed >> 32));
}

// (k + 1/2) 2^-32: FP64 exactly, FP32 to rounding.
__device__ __forceinline__ double u01d(uint32_t k) { return ((double)k + 0.5) * 2.3283064365386963e-10; }
__device__ __forceinline__ float u01f(uint32_t k)
{
    return fmaf(__uint2float_rn(k), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}

// Box-Muller: sqrt(-2 ln u1) cos(2 pi u2).
__device__ __forceinline__ double box_muller_d(uint32_t a, uint32_t b)
{
    return sqrt(-2.0 * log(u01d(a))) * cos(2.0 * 3.141592653589793 * u01d(b));
}
__device__ __forceinline__ float box_muller_f(uint32_t a, uint32_t b)
{
    return sqrtf(-2.0f * logf(u01f(a))) * cospif(2.0f * u01f(b));
}

// ---------------------------------------------------------------------------
// SFU primitives (PTX approximate instructions)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float a)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float rcp_approx(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float lg2_approx(float a)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// Poisson energy term (f - y) - y ln(f / y) = y g(z), z = (f - y) / y,
// g(z) = z - ln(1 + z): its Taylor series to z^8 for |z| < 1/8 (the dropped
// terms are below 2^-22 of g there), z - log1p(z) otherwise; f for y = 0,
// +inf where f <= 0
__device__ __forceinline__ float poisson_term_f(float f, float y)
{
    if (!(f > 0.0f)) return INFINITY;
    if (y == 0.0f) return f;
    const float z = (f - y) / y;
    float g;
    if (fabsf(z) < 0.125f) {
        float p = 0.125f;
        p = fmaf(z, p, -1.0f / 7.0f);
        p = fmaf(z, p, 1.0f / 6.0f);
        p = fmaf(z, p, -0.2f);
        p = fmaf(z, p, 0.25f);
        p = fmaf(z, p, -1.0f / 3.0f);
        p = fmaf(z, p, 0.5f);
        g = z * z * p;
    } else {
        g = z - log1pf(z);
    }
    return y * g;
}

// 1 / sqrt(2 ln 2): exp(-v^2/2) = 2^(-(v / sqrt(2 ln 2))^2)
#define SMC_INV_SQRT_2LN2 0.84932180028801904272150283410289f
#define SMC_PI 3.14159265358979323846

// ---------------------------------------------------------------------------
// Prior helpers (sampling coordinates)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool in_support_f(const PriorDev &p, float u)
{
    switch (p.kind) {
    case PR_UNIFORM:
    case PR_LOG_UNIFORM: return u >= p.lof && u <= p.hif;
    case PR_GAMMA: return u > 0.0f;
    case PR_NORMAL: return true;
    default: return false;
    }
}
__device__ __forceinline__ float log_prior_f(const PriorDev &p, float u)
{
    if (p.kind == PR_NORMAL) {
        const float z = (u - p.a) / p.b;
        return -0.5f * z * z;
    }
    if (p.kind == PR_GAMMA) return (p.a - 1.0f) * logf(u) - p.b * u;
    return 0.0f;
}
__device__ __forceinline__ bool in_support_d(const PriorDev &p, double u)
{
    switch (p.kind) {
    case PR_UNIFORM:
    case PR_LOG_UNIFORM: return u >= p.lo && u <= p.hi;
    case PR_GAMMA: return u > 0.0;
    case PR_NORMAL: return true;
    default: return false;
    }
}
__device__ __forceinline__ double log_prior_d(const PriorDev &p, double u)
{
    if (p.kind == PR_NORMAL) {
        const double z = (u - p.p1) / p.p2;
        return -0.5 * z * z;
    }
    if (p.kind == PR_GAMMA) return (p.p1 - 1.0) * log(u) - p.p2 * u;
    return 0.0;
}
__device__ __forceinline__ float natural_f(const PriorDev &p, float u)
{
    return p.kind == PR_LOG_UNIFORM ? expf(u) : u;
}
__device__ __forceinline__ double natural_d(const PriorDev &p, double u)
{
    return p.kind == PR_LOG_UNIFORM ? exp(u) : u;
}

// ---------------------------------------------------------------------------
// Warp reductions
// ---------------------------------------------------------------------------
#define FULL_MASK 0xffffffffu

// Butterfly sum: addition is commutative, so every lane ends with the
// bitwise-identical total.
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// Compensated (two-sum) merge of (s, c) pairs across the warp; the pair is
// ordered by lane bit so every lane computes the same result.
__device__ __forceinline__ void warp_sum2(float &s, float &c)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(FULL_MASK, s, o);
        const float c2 = __shfl_xor_sync(FULL_MASK, c, o);
        const bool low = (threadIdx.x & o) == 0;
        const float a = low ? s : s2, b = low ? s2 : s;
        const float ca = low ? c : c2, cb = low ? c2 : c;
        const float t = a + b;
        const float bp = t - a;
        const float err = (a - (t - bp)) + (b - bp);
        s = t;
        c = (ca + cb) + err;
    }
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

__device__ __forceinline__ void named_barrier(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
