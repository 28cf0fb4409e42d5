// k_misc.cu -- prior draws, full energies, particle copy, stage bookkeeping,
// posterior summaries.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "kernels.h"
#include "plain_device.cuh"

namespace smc {

// ---------------------------------------------------------------------------
// Philox words (for parity tests of the generator itself)
// ---------------------------------------------------------------------------
__global__ void k_philox(unsigned long long seed, const uint4 *ctr, uint4 *out, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox10(ctr[i], (uint32_t)seed, (uint32_t)(seed >> 32));
}

cudaError_t launch_philox(uint64_t seed, const uint32_t *ctr, uint32_t *out, int64_t n,
                          cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int b = 256;
    k_philox<<<(unsigned)((n + b - 1) / b), b, 0, s>>>(seed, (const uint4 *)ctr, (uint4 *)out, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Prior draws at beta_0 = 0 (start of the tempered sequence, Eq. (9)).
// Counter (256 j + attempt, particle, 0, K); Gamma by Marsaglia & Tsang (2000)
// with the u^(1/shape) boost below shape 1.  Draws are made in FP64.
// ---------------------------------------------------------------------------
__device__ double prior_draw(const PriorDev &p, unsigned long long seed, uint32_t j, uint32_t i,
                             uint32_t tag)
{
    uint4 w;
    switch (p.kind) {
    case PR_UNIFORM:
        w = draw(seed, 256u * j, i, 0u, tag);
        return p.p1 + (p.p2 - p.p1) * u01d(w.x);
    case PR_LOG_UNIFORM:
        w = draw(seed, 256u * j, i, 0u, tag);
        return p.lo + (p.hi - p.lo) * u01d(w.x);
    case PR_NORMAL:
        w = draw(seed, 256u * j, i, 0u, tag);
        return p.p1 + p.p2 * box_muller_d(w.x, w.y);
    case PR_GAMMA: {
        const double a = p.p1 < 1.0 ? p.p1 + 1.0 : p.p1;
        const double dd = a - 1.0 / 3.0;
        const double cc = 1.0 / sqrt(9.0 * dd);
        for (uint32_t att = 0; att < 256u; ++att) {
            w = draw(seed, 256u * j + att, i, 0u, tag);
            const double z = box_muller_d(w.x, w.y);
            const double t = 1.0 + cc * z;
            if (t <= 0.0) continue;
            const double v = t * t * t;
            if (log(u01d(w.z)) < 0.5 * z * z + dd - dd * v + dd * log(v)) {
                double g = dd * v;
                if (p.p1 < 1.0) g *= pow(u01d(w.w), 1.0 / p.p1);
                return g / p.p2;
            }
        }
        return dd / p.p2;
    }
    default: return p.p1;  // FIXED
    }
}

__global__ void k_prior_init(JobDev *jobs, const int *slots)
{
    JobDev &jb = jobs[slots[blockIdx.y]];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= jb.T) return;
    for (int j = 0; j < jb.d; ++j) {
        const double v = prior_draw(jb.pri[j], jb.seed, (uint32_t)j, (uint32_t)i, jb.tag);
        if (jb.fp64)
            jb.th64[(size_t)j * jb.T + i] = v;
        else
            jb.th[(size_t)j * jb.T + i] = (float)v;
    }
}

cudaError_t launch_prior_init(JobDev *jobs, const int *slots, int nslots, int max_T,
                              cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    const int b = 128;
    dim3 g((max_T + b - 1) / b, nslots);
    k_prior_init<<<g, b, 0, s>>>(jobs, slots);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Full energy E = 1/2 sum_i w_i r_i^2, r = y - f (forward model Eq. (1)).
// FP32 jobs: one warp per particle, lanes stride over grid points, FP32
// Kahan-compensated per lane and a compensated butterfly across lanes.
// ---------------------------------------------------------------------------
template <int FAM>
__device__ __forceinline__ float peak_eval(float x, float A, float mu, float s, float eta)
{
    const float dx = x - mu;
    const float t = dx * s;  // s = 1/(w sqrt(2 ln 2)) for GAUSS, 1/HWHM otherwise
    const float t2 = t * t;
    if (FAM == FAM_GAUSS) return A * ex2_approx(-t2);
    const float L = rcp_approx(1.0f + t2);
    if (FAM == FAM_LORENTZ) return A * L;
    const float G = ex2_approx(-t2);
    return A * fmaf(eta, G - L, L);
}

template <int FAM>
__device__ __forceinline__ float energy_warp(const JobDev &jb, const float *P)
{
    const int lane = threadIdx.x & 31;
    const int K = jb.K, p = jb.p, nbg = jb.nbg;
    float s = 0.0f, c = 0.0f;
    for (int pt = lane; pt < jb.n_pad; pt += 32) {
        const float x = jb.xc[pt];
        float f = 0.0f;
        for (int k = 0; k < K; ++k)
            f += peak_eval<FAM>(x, P[k * p], P[k * p + 1], P[k * p + 2],
                                FAM == FAM_PV ? P[k * p + 3] : 0.0f);
        if (nbg > 0) {
            const float t = jb.ts[pt];
            float a = 1.0f, b = t;
            f = fmaf(P[p * K], a, f);
            if (nbg > 1) f = fmaf(P[p * K + 1], b, f);
            for (int q = 2; q < nbg; ++q) {
                const float cn = fmaf(2.0f * t, b, -a);
                a = b;
                b = cn;
                f = fmaf(P[p * K + q], b, f);
            }
        }
        const float r = jb.y[pt] - f;
        const float term = 0.5f * jb.wt[pt] * r * r;
        const float yk = term - c;  // Kahan: running sum s, lost low part -c
        const float tk = s + yk;
        c = (tk - s) - yk;
        s = tk;
    }
    c = -c;
    warp_sum2(s, c);
    return s + c;
}

// Coupled-grid likelihoods (Shirley background, model variance): a lane owns a
// contiguous run of grid points; the running integral of the peak signal is a
// lane-local sum plus a warp scan; peaks are evaluated twice (total, then the
// running pass) instead of stored.
template <int FAM>
__device__ __forceinline__ float energy_warp_full(const JobDev &jb, const float *P)
{
    const int lane = threadIdx.x & 31;
    const int K = jb.K, p = jb.p, n = jb.n;
    const bool shir = jb.bg_kind == BGK_SHIRLEY;
    const int noise = jb.noise;
    const int ch = (n + 31) / 32, lo = min(n, lane * ch), hi = min(n, lo + ch);
    auto peaks = [&](int pt) {
        const float x = jb.xc[pt];
        float f = 0.0f;
        for (int k = 0; k < K; ++k)
            f += peak_eval<FAM>(x, P[k * p], P[k * p + 1], P[k * p + 2], FAM == FAM_PV ? P[k * p + 3] : 0.0f);
        return f;
    };
    float a = 0.0f, b = 0.0f, start = 0.0f, iCN = 0.0f;
    if (shir) {
        a = P[p * K];
        b = P[p * K + 1];
        float part = 0.0f;
        for (int pt = lo; pt < hi; ++pt) part = fmaf(jb.ts[pt], peaks(pt), part);
        float sc = part;
        for (int o = 1; o < 32; o <<= 1) {
            const float t = __shfl_up_sync(FULL_MASK, sc, o);
            if (lane >= o) sc += t;
        }
        start = __shfl_up_sync(FULL_MASK, sc, 1);
        if (lane == 0) start = 0.0f;
        const float CN = __shfl_sync(FULL_MASK, sc, 31);
        iCN = CN > 0.0f ? 1.0f / CN : 0.0f;
    }
    float s = 0.0f, c = 0.0f, run = start;
    for (int pt = lo; pt < hi; ++pt) {
        const float Pk = peaks(pt);
        float f = Pk;
        if (shir) {
            run = fmaf(jb.ts[pt], Pk, run);
            f += fmaf(b - a, run * iCN, a);
        }
        const float r = jb.y[pt] - f;
        float term;
        if (noise == NZ_KNOWN) {
            term = 0.5f * jb.wt[pt] * r * r;
        } else if (noise == NZ_MODEL) {
            const float v = fmaf(fmaf(jb.nv1, f, jb.nv0), f, jb.nv2);
            term = v > 0.0f ? fmaf(0.34657359027997264f, lg2_approx(v), 0.91893853320467274f) + 0.5f * r * r / v
                            : INFINITY;
        } else {
            term = poisson_term_f(f, jb.y[pt]);
        }
        const float yk = term - c;
        const float tk = s + yk;
        c = (tk - s) - yk;
        s = tk;
    }
    c = -c;
    warp_sum2(s, c);
    return s + c;
}

// App. D phase model (FP32, one warp per particle): phases with Caglioti widths
// and asymmetry from their reference reflections, the PV background, any noise
// model; P holds natural parameters.
__device__ __forceinline__ float xrd_phase_unit_f(float xc, float tn, float sc, const float *q,
                                                  const float4 *rtab, int j0, int j1)
{
    const float rad = fmaf(q[4] * tn, tn, fmaf(-q[5], tn, q[6]));
    const float W0 = fmaf(q[7], sc, q[8] * tn);
    const bool gok = rad > 0.0f, lok = W0 > 0.0f;
    const float rs = gok ? rsqrtf(rad) : 0.0f, iom = lok ? 1.0f / W0 : 0.0f, ia = 1.0f / q[2];
    float U = 0.0f;
    for (int j = j0; j < j1; ++j) {
        const float4 R = rtab[j];
        const float dx = xc - (R.x + q[1]);
        const float a = dx >= 0.0f ? ia : 1.0f;
        const float zg = dx * rs * a, zl = dx * iom * a;
        const float g = gok ? ex2_approx(-4.0f * zg * zg) : 0.0f;
        const float l = lok ? rcp_approx(fmaf(4.0f * zl, zl, 1.0f)) : 0.0f;
        U = fmaf(R.y, fmaf(q[3], l - g, g), U);
    }
    return U;
}

__device__ __forceinline__ float xrd_bg_unit_f(float xabs, float sbg, float rbg)
{
    if (!(sbg > 0.0f)) return 0.0f;
    const float z = xabs / sbg;
    const float g = ex2_approx(-4.0f * z * z), l = rcp_approx(fmaf(4.0f * z, z, 1.0f));
    return fmaf(rbg, l - g, g);
}

__device__ __forceinline__ float energy_warp_xrd(const JobDev &jb, const float *P)
{
    const int lane = threadIdx.x & 31;
    const int K = jb.K, noise = jb.noise;
    const float xref = (float)jb.x_ref;
    float s = 0.0f, c = 0.0f;
    for (int pt = lane; pt < jb.n; pt += 32) {
        const float xc = jb.xc[pt], tn = jb.ts[pt], sc = jb.sec2[pt];
        float f = 0.0f;
        for (int k = 0; k < K; ++k)
            f = fmaf(P[9 * k], xrd_phase_unit_f(xc, tn, sc, P + 9 * k, jb.rtab, jb.roff[k], jb.roff[k + 1]), f);
        if (jb.bg_kind == BGK_XRD_PV) {
            const float *b = P + 9 * K;
            f += fmaf(b[0], xrd_bg_unit_f(xc + xref, b[1], b[2]), b[3]);
        }
        const float r = jb.y[pt] - f;
        float term;
        if (noise == NZ_KNOWN) {
            term = 0.5f * jb.wt[pt] * r * r;
        } else if (noise == NZ_MODEL) {
            const float v = fmaf(fmaf(jb.nv1, f, jb.nv0), f, jb.nv2);
            term = v > 0.0f ? fmaf(0.34657359027997264f, lg2_approx(v), 0.91893853320467274f) + 0.5f * r * r / v
                            : INFINITY;
        } else {
            term = poisson_term_f(f, jb.y[pt]);
        }
        const float yk = term - c;
        const float tk = s + yk;
        c = (tk - s) - yk;
        s = tk;
    }
    c = -c;
    warp_sum2(s, c);
    return s + c;
}

__global__ void __launch_bounds__(256) k_energy_f32(JobDev *jobs, const int *slots)
{
    __shared__ float par[8][SMC_DMAX];
    JobDev &jb = jobs[slots[blockIdx.y]];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= jb.T) return;
    const int K = jb.K, p = jb.p, d = jb.d;
    float *P = par[wib];
    // natural parameters of this particle, widths turned into inverse scales
    for (int j = lane; j < d; j += 32) {
        float v = natural_f(jb.pri[j], jb.th[(size_t)j * jb.T + i]);
        if (jb.family != FAM_XRD && j < p * K && j % p == 2)
            v = (jb.family != FAM_GAUSS) ? 1.0f / v
                                         : (jb.wprec ? sqrtf(v) * SMC_INV_SQRT_2LN2 : SMC_INV_SQRT_2LN2 / v);
        P[j] = v;
    }
    __syncwarp();
    float e;
    if (jb.family == FAM_XRD) {
        e = energy_warp_xrd(jb, P);
    } else if (jb.full) {
        if (jb.family == FAM_GAUSS)
            e = energy_warp_full<FAM_GAUSS>(jb, P);
        else if (jb.family == FAM_LORENTZ)
            e = energy_warp_full<FAM_LORENTZ>(jb, P);
        else
            e = energy_warp_full<FAM_PV>(jb, P);
    } else if (jb.family == FAM_GAUSS)
        e = energy_warp<FAM_GAUSS>(jb, P);
    else if (jb.family == FAM_LORENTZ)
        e = energy_warp<FAM_LORENTZ>(jb, P);
    else
        e = energy_warp<FAM_PV>(jb, P);
    if (lane == 0) jb.E[i] = e;
}

// FP64 jobs: one thread per particle.
__global__ void k_energy_f64(JobDev *jobs, const int *slots)
{
    const JobDev &jb = jobs[slots[blockIdx.y]];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= jb.T) return;
    double nat[SMC_DMAX];
    for (int j = 0; j < jb.d; ++j) nat[j] = natural_d(jb.pri[j], jb.th64[(size_t)j * jb.T + i]);
    jb.E64[i] = energy_plain(jb, nat);
}

cudaError_t launch_energy(JobDev *jobs, const int *slots, int nslots, int max_T, bool fp64,
                          cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    if (fp64) {
        dim3 g((max_T + 127) / 128, nslots);
        k_energy_f64<<<g, 128, 0, s>>>(jobs, slots);
        return cudaGetLastError();
    }
    dim3 g((unsigned)(((long long)max_T * 32 + 255) / 256), nslots);
    k_energy_f32<<<g, 256, 0, s>>>(jobs, slots);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Particle copy: chain starts ths[:, m] = th[:, anc[m]], Es[m] = E[anc[m]]
// (the resampling of Sec. II B 2).  Component-major layout: writes are
// coalesced, reads follow the non-decreasing ancestors.
// ---------------------------------------------------------------------------
template <typename P>
__global__ void __launch_bounds__(256) k_gather(JobDev *jobs, const int *slots)
{
    const JobDev &jb = jobs[slots[blockIdx.y]];
    if (jb.state != JOB_ACTIVE || jb.status != 0) return;
    const int S = jb.S, T = jb.T, d = jb.d;
    const P *th = (const P *)(jb.fp64 ? (const void *)jb.th64 : (const void *)jb.th);
    const P *E = (const P *)(jb.fp64 ? (const void *)jb.E64 : (const void *)jb.E);
    P *ths = (P *)(jb.fp64 ? (void *)jb.ths64 : (void *)jb.ths);
    P *Es = (P *)(jb.fp64 ? (void *)jb.Es64 : (void *)jb.Es);
    const int *anc = jb.anc;
    const long long total = (long long)S * (d + 1);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / S);
        const int m = (int)(e - (long long)j * S);
        const int a = __ldg(anc + m);
        if (j < d)
            ths[(size_t)j * S + m] = __ldg(th + (size_t)j * T + a);
        else
            Es[m] = __ldg(E + a);
    }
}

cudaError_t launch_gather(JobDev *jobs, const int *slots, int nslots, int64_t max_elems,
                          bool fp64, cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    long long blocks = (max_elems + 255) / 256;
    if (blocks > 8 * 148) blocks = 8 * 148;
    if (blocks < 1) blocks = 1;
    dim3 g((unsigned)blocks, nslots);
    if (fp64)
        k_gather<double><<<g, 256, 0, s>>>(jobs, slots);
    else
        k_gather<float><<<g, 256, 0, s>>>(jobs, slots);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// End of a stage iteration: advance counters, retire finished jobs, count the
// jobs still active (for the host loop).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_stage_end(JobDev *jobs, const int *slots, int nslots,
                                                    int *n_active, int *n_active_host, int use_cond,
                                                    cudaGraphConditionalHandle cond, int *iter,
                                                    int max_iter)
{
    __shared__ int red[32];
    int cnt = 0;
    for (int a = threadIdx.x; a < nslots; a += blockDim.x) {
        JobDev &jb = jobs[slots[a]];
        if (jb.state != JOB_ACTIVE) continue;
        if (jb.status != 0) {
            jb.state = JOB_DONE;
            continue;
        }
        jb.stage += 1;
        if (jb.final_step) {
            jb.state = JOB_DONE;
            continue;
        }
        if (jb.stage >= jb.max_stages) {
            jb.status = 5;  // SMC_EMAXSTAGES
            jb.state = JOB_DONE;
            continue;
        }
        ++cnt;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL_MASK, cnt, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *n_active = t;
        if (n_active_host) *(volatile int *)n_active_host = t;
        if (use_cond) {
            // while-node condition of a whole-run graph: continue while any job
            // is active, and never beyond max_iter stages (every stage retires
            // or advances each job, so max_stages + 1 stages always suffice)
            const int it = ++(*iter);
            cudaGraphSetConditional(cond, (t > 0 && it < max_iter) ? 1u : 0u);
        }
    }
}

cudaError_t launch_stage_end(JobDev *jobs, const int *slots, int nslots, int *n_active,
                             int *n_active_host, cudaStream_t s)
{
    k_stage_end<<<1, 1024, 0, s>>>(jobs, slots, nslots, n_active, n_active_host, 0, 0ull, nullptr, 0);
    return cudaGetLastError();
}

cudaError_t launch_stage_end_cond(JobDev *jobs, const int *slots, int nslots, int *n_active,
                                  cudaGraphConditionalHandle cond, int *iter, int max_iter,
                                  cudaStream_t s)
{
    k_stage_end<<<1, 1024, 0, s>>>(jobs, slots, nslots, n_active, nullptr, 1, cond, iter, max_iter);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Posterior summaries of the final (equally weighted) particle set: each
// sample's peaks are ordered by centre (peaks are exchangeable in Eq. (1)),
// then mean and population SD per component in FP64; optional FP32 copy of the
// natural values as samples [T][dim_stride] (unsorted).
//
// A job's particles are split over `split` CTAs.  Each thread keeps its FP64
// sums of (v - c) and (v - c)^2 per sorted position in shared memory
// ([position][thread], so the dynamic position index costs no local memory),
// c being the sorted natural values of particle 0 (a shift against
// cancellation).  A CTA writes its per-position totals (threads summed in
// order) to part[job][split]; the last CTA of the job to finish (counted with
// an atomic after a fence, no waiting) adds the parts in split order and
// writes mean = c + S1/T and sd = sqrt(S2/T - (S1/T)^2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double natural_at(const JobDev &jb, int j, int i)
{
    const double u = jb.fp64 ? jb.th64[(size_t)j * jb.T + i] : (double)jb.th[(size_t)j * jb.T + i];
    double x = natural_d(jb.pri[j], u);
    if (jb.pri[j].is_centre) x += jb.x_ref;
    return x;
}

// sorted position of peak k: peaks with a smaller centre, ties by index (the
// order of a stable sort); cen[k * ld] holds the centres
__device__ __forceinline__ int peak_rank(const float *cen, int ld, int K, int k)
{
    const float ck = cen[k * ld];
    int r = 0;
    for (int m = 0; m < K; ++m) {
        const float cm = cen[m * ld];
        r += (cm < ck) || (cm == ck && m < k);
    }
    return r;
}

int finalize_split(int64_t T) { return (int)std::min<int64_t>(64, std::max<int64_t>(1, (T + 1023) / 1024)); }

static int fin_threads(int d) { return d <= 48 ? 128 : 64; }

static size_t fin_smem(int d, int K, int nt)
{
    return (size_t)nt * (16 * (size_t)d + 4 * (size_t)std::max(K, 1)) + 8 * (size_t)d + 16;
}

__global__ void k_finalize(JobDev *jobs, const int *slots, int split, double *mean, double *sd,
                           float *samples, int dstride, long long sstride, double *part,
                           int *counters)
{
    extern __shared__ __align__(16) unsigned char fin_sh[];
    const int a = blockIdx.x / split, sp = blockIdx.x - a * split;
    const JobDev &jb = jobs[slots[a]];
    // App. D phases are not exchangeable (each has its own reflections): no sorting
    const int T = jb.T, d = jb.d, K = jb.family == FAM_XRD ? 0 : jb.K, p = jb.p, NT = blockDim.x,
              tid = threadIdx.x;
    double *acc1 = (double *)fin_sh;                 // [d][NT]
    double *acc2 = acc1 + (size_t)d * NT;            // [d][NT]
    double *shift = acc2 + (size_t)d * NT;           // [d]
    float *cen = (float *)(shift + d);               // [K][NT]
    __shared__ int is_last;

    if (tid == 0) {  // shift: particle 0, sorted
        for (int k = 0; k < K; ++k) cen[k * NT] = (float)natural_at(jb, k * p + 1, 0);
        for (int k = 0; k < K; ++k) {
            const int r = peak_rank(cen, NT, K, k);
            for (int c = 0; c < p; ++c) shift[r * p + c] = natural_at(jb, k * p + c, 0);
        }
        for (int j = p * K; j < d; ++j) shift[j] = natural_at(jb, j, 0);
    }
    for (int j = 0; j < d; ++j) acc1[j * NT + tid] = acc2[j * NT + tid] = 0.0;
    __syncthreads();

    const int lo = (int)((long long)T * sp / split), hi = (int)((long long)T * (sp + 1) / split);
    for (int i = lo + tid; i < hi; i += NT) {
        for (int k = 0; k < K; ++k) cen[k * NT + tid] = (float)natural_at(jb, k * p + 1, i);
        float *row = samples ? samples + a * sstride + (long long)i * dstride : nullptr;
        for (int k = 0; k < K; ++k) {
            const int r = peak_rank(cen + tid, NT, K, k);
            for (int c = 0; c < p; ++c) {
                const int j = k * p + c, q = r * p + c;
                const double v = natural_at(jb, j, i);
                if (row) row[j] = (float)v;
                const double x = v - shift[q];
                acc1[q * NT + tid] += x;
                acc2[q * NT + tid] += x * x;
            }
        }
        for (int j = p * K; j < d; ++j) {
            const double v = natural_at(jb, j, i);
            if (row) row[j] = (float)v;
            const double x = v - shift[j];
            acc1[j * NT + tid] += x;
            acc2[j * NT + tid] += x * x;
        }
    }
    __syncthreads();
    double *mypart = part + ((size_t)a * split + sp) * 2 * dstride;
    for (int j = tid; j < d; j += NT) {
        double s1 = 0.0, s2 = 0.0;
        for (int t = 0; t < NT; ++t) {
            s1 += acc1[j * NT + t];
            s2 += acc2[j * NT + t];
        }
        mypart[j] = s1;
        mypart[dstride + j] = s2;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(&counters[a], 1) == split - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const double *jp = part + (size_t)a * split * 2 * dstride;
    for (int j = tid; j < d; j += NT) {
        double s1 = 0.0, s2 = 0.0;
        for (int t = 0; t < split; ++t) {
            s1 += __ldcg(&jp[(size_t)t * 2 * dstride + j]);
            s2 += __ldcg(&jp[(size_t)t * 2 * dstride + dstride + j]);
        }
        const double m1 = s1 / T;
        mean[(size_t)a * dstride + j] = shift[j] + m1;
        sd[(size_t)a * dstride + j] = sqrt(fmax(s2 / T - m1 * m1, 0.0));
    }
    if (tid == 0) counters[a] = 0;
}

cudaError_t launch_finalize(JobDev *jobs, const int *slots, int nslots, int d_max, int k_max, int64_t T,
                            double *mean, double *sd, float *samples, int dim_stride,
                            int64_t sample_stride, double *part, int *counters, cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    const int nt = fin_threads(d_max), split = finalize_split(T);
    const size_t smem = fin_smem(d_max, k_max, nt);
    // per device and cheap: set on every (eager, uncaptured) launch
    cudaError_t e = cudaFuncSetAttribute(k_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fin_smem(SMC_DMAX, SMC_KMAX, 64));
    if (e != cudaSuccess) return e;
    k_finalize<<<nslots * split, nt, smem, s>>>(jobs, slots, split, mean, sd, samples, dim_stride,
                                               (long long)sample_stride, part, counters);
    return cudaGetLastError();
}

}  // namespace smc
