// k_reweight.cu -- tempering step and systematic resampling.
//
// Reweighting (Sec. II B 2): incremental weights w_i = exp(-delta (E_i - E_min))
// (Eq. (10)); the next inverse temperature is found by bisection on the
// effective sample size ESS = (sum w)^2 / sum w^2 so that ESS >= rho T; the
// evidence gains log((1/T) sum_i exp(-delta E_i)) (Eq. (11)).  All of it is
// FP64.  This file holds the kernel for jobs with FP64 energies (the plain
// path, which replays the FP64 oracle); FP32-energy jobs take the kernels of
// k_temper32.cu.  One thread-block cluster works on one job: each CTA owns a
// slice of the particles and the per-iteration sums are exchanged through
// distributed shared memory in a fixed order, so the result does not depend on
// which other jobs share the launch.  The same pass produces the weighted mean
// and SD of every component (step sizes of the Metropolis kernel, Sec. II B 4).
//
// Resampling: systematic, on the integer weights q_i = floor(w_i 2^40).  For
// each particle i the kernel writes the range of output slots m whose point
// t_m = floor((m Q + r) / M) falls in [C_{i-1}, C_i), C the inclusive prefix
// sum of q -- the inverse of a_m = min{i : C_i > t_m}, exact in integers.
#include <cooperative_groups.h>

#include <cmath>

#include "kernels.h"
#include "temper.cuh"

namespace cg = cooperative_groups;

namespace smc {

constexpr int RW_THREADS = 512;
constexpr int RW_WARPS = RW_THREADS / 32;
constexpr int RW_CL = 8;  // CTAs per job (portable cluster size)

constexpr int RW_GATHER = 16;  // values per cluster_sum (nv * RW_CL <= RW_THREADS)
static_assert(RW_GATHER * RW_CL <= RW_THREADS, "cluster_sum gather size");

struct RwShared {
    double red[SMC_DMAX][RW_WARPS];
    double xch[2][SMC_DMAX];
    double mean[SMC_DMAX];
    double gat[RW_GATHER][RW_CL];
};

// Cluster-wide sum of per-thread values v[0..nv), nv <= RW_GATHER; every
// thread of every CTA receives the identical totals (fixed summation order).
// The nv x RW_CL remote reads are issued by as many threads at once (one
// distributed-shared-memory round trip), then summed from local shared memory.
__device__ void cluster_sum(cg::cluster_group &cl, RwShared &sh, int &par, const double *v, int nv,
                            double *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < nv; ++k) {
        const double t = warp_sum_d(v[k]);
        if (lane == 0) sh.red[k][warp] = t;
    }
    __syncthreads();
    if ((int)threadIdx.x < nv) {
        double t = 0.0;
        for (int w = 0; w < RW_WARPS; ++w) t += sh.red[threadIdx.x][w];
        sh.xch[par][threadIdx.x] = t;
    }
    cl.sync();
    if ((int)threadIdx.x < nv * RW_CL) {
        const int k = threadIdx.x / RW_CL, r = threadIdx.x - k * RW_CL;
        sh.gat[k][r] = *cl.map_shared_rank(&sh.xch[par][k], r);
    }
    __syncthreads();
    for (int k = 0; k < nv; ++k) {
        double t = 0.0;
#pragma unroll
        for (int r = 0; r < RW_CL; ++r) t += sh.gat[k][r];
        out[k] = t;
    }
    par ^= 1;
}

// Per-component variant: sh.red[j][warp] already holds warp partials for
// j < nv; totals land in out_sh[j] (shared), visible after the call.
__device__ void cluster_sum_rows(cg::cluster_group &cl, RwShared &sh, int &par, int nv,
                                 double *out_sh)
{
    __syncthreads();
    if ((int)threadIdx.x < nv) {
        double t = 0.0;
        for (int w = 0; w < RW_WARPS; ++w) t += sh.red[threadIdx.x][w];
        sh.xch[par][threadIdx.x] = t;
    }
    cl.sync();
    if ((int)threadIdx.x < nv) {
        double t = 0.0;
        for (int r = 0; r < RW_CL; ++r) t += *cl.map_shared_rank(&sh.xch[par][threadIdx.x], r);
        out_sh[threadIdx.x] = t;
    }
    par ^= 1;
    __syncthreads();
}

__device__ double cluster_min(cg::cluster_group &cl, RwShared &sh, int &par, double v)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(FULL_MASK, v, o));
    if (lane == 0) sh.red[0][warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = sh.red[0][0];
        for (int w = 1; w < RW_WARPS; ++w) t = fmin(t, sh.red[0][w]);
        sh.xch[par][0] = t;
    }
    cl.sync();
    if ((int)threadIdx.x < RW_CL) sh.gat[0][threadIdx.x] = *cl.map_shared_rank(&sh.xch[par][0], threadIdx.x);
    __syncthreads();
    double t = sh.gat[0][0];
    for (int r = 1; r < RW_CL; ++r) t = fmin(t, sh.gat[0][r]);
    par ^= 1;
    return t;
}

__device__ double ess_frac(cg::cluster_group &cl, RwShared &sh, int &par, const double *E, int lo,
                           int hi, int T, double emin, double delta)
{
    double v[2] = {0.0, 0.0};
    for (int i = lo + (int)threadIdx.x; i < hi; i += RW_THREADS) {
        const double e = (double)E[i];
        if (!isfinite(e)) continue;
        const double w = exp(-delta * (e - emin));
        v[0] += w;
        v[1] += w * w;
    }
    double s[2];
    cluster_sum(cl, sh, par, v, 2, s);
    return s[0] * s[0] / ((double)T * s[1]);
}

__global__ void __cluster_dims__(RW_CL, 1, 1) __launch_bounds__(RW_THREADS)
    k_reweight64(JobDev *jobs, const int *slots)
{
    __shared__ RwShared sh;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    JobDev &jb = jobs[slots[blockIdx.x / RW_CL]];
    // every CTA of the cluster reads the same state before the first sync
    if (jb.state != JOB_ACTIVE || jb.status != 0) return;
    const int T = jb.T, d = jb.d;
    const double *E = jb.E64;
    const double *th = jb.th64;
    double *w64 = jb.w64;
    const int lo = (int)((long long)T * rank / RW_CL);
    const int hi = (int)((long long)T * (rank + 1) / RW_CL);
    const double beta = jb.beta, rho = jb.rho;
    int par = 0;

    // -- minimum finite energy
    double m = INFINITY;
    for (int i = lo + (int)threadIdx.x; i < hi; i += RW_THREADS) {
        const double e = (double)E[i];
        if (isfinite(e)) m = fmin(m, e);
    }
    const double emin = cluster_min(cl, sh, par, m);
    if (!isfinite(emin)) {
        if (rank == 0 && threadIdx.x == 0) jb.status = 8;  // SMC_ENUMERIC
        cl.sync();
        return;
    }

    // -- next temperature: the whole remaining step if ESS allows, else bisection
    const double room = 1.0 - beta;
    double delta;
    int final_step = 0, iters = 0;
    if (ess_frac(cl, sh, par, E, lo, hi, T, emin, room) >= rho) {
        delta = room;
        final_step = 1;
    } else {
        double a = 0.0, b = room;
        while (iters < 200 && b - a > 1e-7 * b) {
            const double mid = 0.5 * (a + b);
            if (ess_frac(cl, sh, par, E, lo, hi, T, emin, mid) >= rho)
                a = mid;
            else
                b = mid;
            ++iters;
        }
        delta = a > 0.0 ? a : b;
    }

    // -- weights w_i (kept for the moments), quantised weights, their sum
    double v1 = 0.0, sw;
    for (int i = lo + (int)threadIdx.x; i < hi; i += RW_THREADS) {
        const double e = (double)E[i];
        const double w = isfinite(e) ? exp(-delta * (e - emin)) : 0.0;
        w64[i] = w;
        jb.q[i] = (unsigned long long)floor(ldexp(w, 40));
        v1 += w;
    }
    cluster_sum(cl, sh, par, &v1, 1, &sw);

    // -- weighted mean and SD per component in sampling coordinates
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < d; ++j) {
        double t = 0.0;
        if (jb.pri[j].kind != PR_FIXED)
            for (int i = lo + (int)threadIdx.x; i < hi; i += RW_THREADS)
                t += w64[i] * (double)th[(size_t)j * T + i];
        t = warp_sum_d(t);
        if (lane == 0) sh.red[j][warp] = t;
    }
    cluster_sum_rows(cl, sh, par, d, sh.mean);
    for (int j = (int)threadIdx.x; j < d; j += RW_THREADS) sh.mean[j] /= sw;
    __syncthreads();
    for (int j = 0; j < d; ++j) {
        double t = 0.0;
        const double mj = sh.mean[j];
        if (jb.pri[j].kind != PR_FIXED)
            for (int i = lo + (int)threadIdx.x; i < hi; i += RW_THREADS) {
                const double u = (double)th[(size_t)j * T + i] - mj;
                t += w64[i] * u * u;
            }
        t = warp_sum_d(t);
        if (lane == 0) sh.red[j][warp] = t;
    }
    __shared__ double var[SMC_DMAX];
    cluster_sum_rows(cl, sh, par, d, var);

    // -- job scalars (rank 0): step sizes from the previous stage's acceptance,
    //    evidence increment, new temperature
    if (rank == 0) {
        for (int j = (int)threadIdx.x; j < d; j += RW_THREADS)
            update_step(jb, j, sh.mean[j], var[j] / sw, beta, final_step ? 1.0 : beta + delta);
        if (threadIdx.x == 0) {
            jb.logz += -delta * emin + log(sw / (double)T);
            jb.beta = final_step ? 1.0 : beta + delta;
            jb.delta = delta;
            jb.final_step = final_step;
            jb.bisect_iters = iters;
            jb.next_chain = 0;
        }
    }
    cl.sync();  // keep this CTA's shared memory alive for remote readers
}

cudaError_t launch_reweight(JobDev *jobs, const int *slots, int nslots, bool fp64, int64_t t_max,
                            cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    if (!fp64) return launch_temper32(jobs, slots, nslots, t_max, s);
    k_reweight64<<<nslots * RW_CL, RW_THREADS, 0, s>>>(jobs, slots);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Systematic resampling on integer weights.
// ---------------------------------------------------------------------------
typedef unsigned __int128 u128;

// smallest m in [0, M] with m Q + r >= M c: an FP32 estimate of
// M c / Q - r / Q (off by a few slots at most for M <= 2^24; FP64 division
// would dominate this kernel on B300), corrected exactly in 128-bit integers.
// inv_q = 1 / Q in FP32.
__device__ __forceinline__ long long first_slot(unsigned long long c, unsigned long long Q,
                                                unsigned long long r, long long M, float inv_q)
{
    const u128 target = (u128)(unsigned long long)M * c;
    if (target <= (u128)r) return 0;
    const float est = ceilf(fmaf((float)M, (float)c * inv_q, -(float)r * inv_q));
    long long m = !(est >= 0.0f) ? 0 : (est > (float)M ? M : (long long)est);
    while (m > 0 && (u128)(unsigned long long)(m - 1) * Q + r >= target) --m;
    while (m < M && (u128)(unsigned long long)m * Q + r < target) ++m;
    return m;
}

constexpr int RS_THREADS = 1024;

__device__ __forceinline__ void resample_block(const unsigned long long *q, int T, int M,
                                               uint32_t u32, int *anc)
{
    __shared__ unsigned long long wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int chunk = (T + RS_THREADS - 1) / RS_THREADS;
    const int i0 = min(T, tid * chunk), i1 = min(T, i0 + chunk);
    unsigned long long loc = 0;
    for (int i = i0; i < i1; ++i) loc += q[i];
    // block exclusive scan of the per-thread sums
    unsigned long long x = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long v = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL_MASK, v, o);
            if (lane >= o) v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    const unsigned long long Q = wsum[31];
    unsigned long long C = x - loc + (warp > 0 ? wsum[warp - 1] : 0ull);
    const unsigned long long r = (unsigned long long)(((u128)u32 * Q) >> 32);
    const float inv_q = 1.0f / (float)Q;
    long long mprev = first_slot(C, Q, r, M, inv_q);
    for (int i = i0; i < i1; ++i) {
        C += q[i];
        const long long mnext = first_slot(C, Q, r, M, inv_q);
        for (long long m = mprev; m < mnext; ++m) anc[m] = i;
        mprev = mnext;
    }
}

__global__ void __launch_bounds__(RS_THREADS) k_resample(JobDev *jobs, const int *slots)
{
    const JobDev &jb = jobs[slots[blockIdx.x]];
    if (jb.state != JOB_ACTIVE || jb.status != 0) return;
    const uint32_t u32 = draw(jb.seed, 0u, 0xFFFFFFFFu, (uint32_t)(jb.stage + 1), jb.tag).x;
    resample_block(jb.q, jb.T, jb.S, u32, jb.anc);
}

cudaError_t launch_resample(JobDev *jobs, const int *slots, int nslots, cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    k_resample<<<nslots, RS_THREADS, 0, s>>>(jobs, slots);
    return cudaGetLastError();
}

// Stand-alone resampling of given integer weights (step-level entry point).
__global__ void __launch_bounds__(RS_THREADS) k_resample_raw(const unsigned long long *q, int T,
                                                             int M, uint32_t u32, int *anc)
{
    resample_block(q, T, M, u32, anc);
}

cudaError_t launch_resample_raw(const unsigned long long *q, int T, int M, uint32_t u32, int *anc,
                                cudaStream_t s)
{
    k_resample_raw<<<1, RS_THREADS, 0, s>>>(q, T, M, u32, anc);
    return cudaGetLastError();
}

}  // namespace smc
