// k_temper32.cu -- tempering step for jobs with FP32 energies.
//
// Same step as the FP64 kernel (Sec. II B 2): incremental weights
// w_i = exp(-delta (E_i - E_min)) (Eq. (10)), the largest increment delta with
// ESS = (sum w)^2 / sum w^2 >= rho T found by bisection on [0, 1 - beta]
// (stopping at relative width 1e-7, at most 200 halvings; the whole remaining
// step when its ESS is large enough), the evidence increment
// log((1/T) sum_i exp(-delta E_i)) (Eq. (11)), and the weighted mean / SD per
// component that set the Metropolis step sizes (Sec. II B 4).
//
// B300 executes FP64 at a small fraction of its FP32 rate, so this path keeps
// FP64 to the scalars and to the evidence, and spreads the FP64 work over the
// whole GPU:
//   k_search32   one 8-CTA cluster per job: minimum energy and the bisection.
//                Weights of the search are FP32 (ex2 on the SFU), summed with
//                per-thread Kahan and double-float (two-float) reductions; their
//                relative error (~2^-22) is below the one the FP32 energies
//                already carry.  Each pass evaluates RW_LEVELS levels at once
//                (the 2^L - 1 midpoints of the bracket's dyadic tree) and walks
//                the tree: the same brackets as one halving per pass, with a
//                third of the cluster exchanges.  Thread 0 of each CTA does the
//                FP64 scalar logic on the gathered totals (identical in every
//                CTA) and broadcasts the next candidates.
//   k_weights32  rw_split(T) CTAs per job: FP64 weights at the chosen delta,
//                their quantised form for resampling, the FP64 partial sum of
//                w, and per component the shifted moments sum w (u - c),
//                sum w (u - c)^2 (FP32 weights, Kahan per thread, c = the value
//                of particle 0), one row of partials per CTA.
//   k_finish32   one CTA per job: adds the partial rows in order (FP64), sets
//                log Z, beta and the step sizes.
#include <cooperative_groups.h>

#include <cmath>

#include "kernels.h"
#include "temper.cuh"

namespace cg = cooperative_groups;

namespace smc {

constexpr int SR_THREADS = 512;
constexpr int SR_WARPS = SR_THREADS / 32;
constexpr int SR_CL = 8;                      // CTAs per job in the search
constexpr int RW_LEVELS = 2;                  // bisection levels per pass
constexpr int RW_CAND = (1 << RW_LEVELS) - 1; // midpoints evaluated per pass
constexpr int SR_VALS = 2 * RW_CAND;          // sums per pass (w and w^2 per candidate)
constexpr double LOG2E = 1.4426950408889634;
constexpr int WT_THREADS = 256;
constexpr int WT_WARPS = WT_THREADS / 32;
static_assert(SR_VALS * SR_CL <= SR_THREADS, "one thread per gathered value");

// CTAs per job in the weights kernel (host and device copies of one formula)
__host__ __device__ __forceinline__ int rw_split_of(long long T)
{
    const long long s = (T + 2047) / 2048;
    return (int)(s < 1 ? 1 : (s > RW_SPLIT_MAX ? RW_SPLIT_MAX : s));
}
int rw_split(int64_t T) { return rw_split_of(T); }

// ---------------------------------------------------------------------------
// two-float arithmetic: a value h + l with |l| <= ulp(h) / 2 (Knuth's TwoSum)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void df_add(float &h, float &l, float bh, float bl)
{
    float s, e;
    two_sum(h, bh, s, e);
    e += l + bl;
    h = s + e;
    l = e - (h - s);
}

// butterfly: every step is symmetric in its operands, so all lanes end equal
__device__ __forceinline__ void df_warp_sum(float &h, float &l)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_xor_sync(FULL_MASK, h, o), bl = __shfl_xor_sync(FULL_MASK, l, o);
        df_add(h, l, bh, bl);
    }
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Kahan pair (s, c) -> normalised two-float value s - c
__device__ __forceinline__ void kahan_to_df(float s, float c, float &h, float &l)
{
    two_sum(s, -c, h, l);
}

// ---------------------------------------------------------------------------
// k_search32
// ---------------------------------------------------------------------------
struct SearchShared {
    float rh[SR_VALS][SR_WARPS], rl[SR_VALS][SR_WARPS];  // warp totals
    float xh[2][SR_VALS], xl[2][SR_VALS];                // CTA totals (read remotely)
    float gh[SR_VALS][SR_CL], gl[SR_VALS][SR_CL];        // gathered CTA totals
    float kc[RW_CAND];                                   // -delta log2(e) per candidate
    float mn[SR_WARPS], xmin, gmin[SR_CL];
    int nc, go;
};

__global__ void __cluster_dims__(SR_CL, 1, 1) __launch_bounds__(SR_THREADS)
    k_search32(JobDev *jobs, const int *slots)
{
    __shared__ SearchShared sh;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    JobDev &jb = jobs[slots[blockIdx.x / SR_CL]];
    // every CTA of the cluster reads the same state before the first sync
    if (jb.state != JOB_ACTIVE || jb.status != 0) return;
    const int T = jb.T;
    const float *E = jb.E;
    const int lo = (int)((long long)T * rank / SR_CL), hi = (int)((long long)T * (rank + 1) / SR_CL);

    // -- minimum finite energy (exact in any order)
    float m = INFINITY;
    for (int i = lo + tid; i < hi; i += SR_THREADS) {
        const float e = E[i];
        if (isfinite(e)) m = fminf(m, e);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(FULL_MASK, m, o));
    if (lane == 0) sh.mn[warp] = m;
    __syncthreads();
    if (tid == 0) {
        float t = sh.mn[0];
        for (int w = 1; w < SR_WARPS; ++w) t = fminf(t, sh.mn[w]);
        sh.xmin = t;
    }
    cl.sync();
    if (tid < SR_CL) sh.gmin[tid] = *cl.map_shared_rank(&sh.xmin, tid);
    __syncthreads();
    float emin = sh.gmin[0];
    for (int r = 1; r < SR_CL; ++r) emin = fminf(emin, sh.gmin[r]);
    if (!isfinite(emin)) {
        if (rank == 0 && tid == 0) jb.status = 8;  // SMC_ENUMERIC
        cl.sync();
        return;
    }

    // -- search state, kept by thread 0 (identical in every CTA)
    const double room = 1.0 - jb.beta, rho = jb.rho;
    double a = 0.0, b = room, delta = room, cand[RW_CAND];
    int iters = 0, final_step = 0, bisecting = 0;
    if (tid == 0) {
        cand[0] = room;
        sh.kc[0] = (float)(-room * LOG2E);
        sh.nc = 1;
        sh.go = 1;
    }
    int par = 0;
    for (;;) {
        __syncthreads();
        if (!sh.go) break;
        const int nc = sh.nc;
        float k[RW_CAND], s1[RW_CAND], c1[RW_CAND], s2[RW_CAND], c2[RW_CAND];
#pragma unroll
        for (int c = 0; c < RW_CAND; ++c) {
            k[c] = c < nc ? sh.kc[c] : 0.0f;
            s1[c] = c1[c] = s2[c] = c2[c] = 0.0f;
        }
        for (int i = lo + tid; i < hi; i += SR_THREADS) {
            const float e = E[i];
            if (!isfinite(e)) continue;
            const float ep = e - emin;
#pragma unroll
            for (int c = 0; c < RW_CAND; ++c) {
                if (c < nc) {
                    const float w = ex2_approx(k[c] * ep);
                    kahan_add(s1[c], c1[c], w);
                    kahan_add(s2[c], c2[c], w * w);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < RW_CAND; ++c) {
            if (c < nc) {
                float h, l;
                kahan_to_df(s1[c], c1[c], h, l);
                df_warp_sum(h, l);
                if (lane == 0) {
                    sh.rh[2 * c][warp] = h;
                    sh.rl[2 * c][warp] = l;
                }
                kahan_to_df(s2[c], c2[c], h, l);
                df_warp_sum(h, l);
                if (lane == 0) {
                    sh.rh[2 * c + 1][warp] = h;
                    sh.rl[2 * c + 1][warp] = l;
                }
            }
        }
        __syncthreads();
        if (tid < 2 * nc) {
            float h = 0.0f, l = 0.0f;
            for (int w = 0; w < SR_WARPS; ++w) df_add(h, l, sh.rh[tid][w], sh.rl[tid][w]);
            sh.xh[par][tid] = h;
            sh.xl[par][tid] = l;
        }
        cl.sync();
        if (tid < 2 * nc * SR_CL) {
            const int v = tid / SR_CL, r = tid - v * SR_CL;
            sh.gh[v][r] = *cl.map_shared_rank(&sh.xh[par][v], r);
            sh.gl[v][r] = *cl.map_shared_rank(&sh.xl[par][v], r);
        }
        __syncthreads();
        if (tid == 0) {
            double frac[RW_CAND];
            for (int c = 0; c < nc; ++c) {
                float h1 = 0.0f, l1 = 0.0f, h2 = 0.0f, l2 = 0.0f;
                for (int r = 0; r < SR_CL; ++r) {
                    df_add(h1, l1, sh.gh[2 * c][r], sh.gl[2 * c][r]);
                    df_add(h2, l2, sh.gh[2 * c + 1][r], sh.gl[2 * c + 1][r]);
                }
                const double t1 = (double)h1 + (double)l1, t2 = (double)h2 + (double)l2;
                frac[c] = t1 * t1 / ((double)T * t2);
            }
            int go = 1;
            if (!bisecting) {
                if (frac[0] >= rho) {
                    delta = room;
                    final_step = 1;
                    go = 0;
                } else {
                    bisecting = 1;
                }
            } else {
                int node = 0;
                for (int lev = 0; lev < RW_LEVELS && iters < 200 && b - a > 1e-7 * b; ++lev) {
                    if (frac[node] >= rho) {
                        a = cand[node];
                        node = 2 * node + 2;
                    } else {
                        b = cand[node];
                        node = 2 * node + 1;
                    }
                    ++iters;
                }
            }
            if (go && bisecting) {
                if (iters < 200 && b - a > 1e-7 * b) {
                    // heap of midpoints: node n splits the bracket held on reaching it
                    double la[RW_CAND], lb[RW_CAND];
                    cand[0] = 0.5 * (a + b);
                    la[0] = a;
                    lb[0] = b;
                    for (int n = 0; n < RW_CAND / 2; ++n) {
                        const int l = 2 * n + 1, r = 2 * n + 2;
                        cand[l] = 0.5 * (la[n] + cand[n]);
                        la[l] = la[n];
                        lb[l] = cand[n];
                        cand[r] = 0.5 * (cand[n] + lb[n]);
                        la[r] = cand[n];
                        lb[r] = lb[n];
                    }
                    for (int c = 0; c < RW_CAND; ++c) sh.kc[c] = (float)(-cand[c] * LOG2E);
                    sh.nc = RW_CAND;
                } else {
                    go = 0;
                    delta = a > 0.0 ? a : b;
                }
            }
            sh.go = go;
        }
        par ^= 1;
    }
    if (rank == 0 && tid == 0) {
        jb.delta = delta;
        jb.final_step = final_step;
        jb.bisect_iters = iters;
        jb.emin = (double)emin;
    }
    cl.sync();  // keep this CTA's shared memory alive for remote readers
}

// ---------------------------------------------------------------------------
// k_weights32: grid = nslots x max_split; partial row of CTA sp of a job:
//   part[sp][0] = sum w, part[sp][1 + 2j] = sum w (u_j - c_j),
//   part[sp][2 + 2j] = sum w (u_j - c_j)^2   (u: sampling coordinate)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(WT_THREADS) k_weights32(JobDev *jobs, const int *slots, int max_split)
{
    __shared__ float rh[2 * SMC_DMAX][WT_WARPS], rl[2 * SMC_DMAX][WT_WARPS];
    __shared__ double rw[WT_WARPS];
    const int a = blockIdx.x / max_split, sp = blockIdx.x - a * max_split;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    JobDev &jb = jobs[slots[a]];
    if (jb.state != JOB_ACTIVE || jb.status != 0) return;
    const int T = jb.T, d = jb.d, split = rw_split_of(T);
    if (sp >= split) return;
    const int lo = (int)((long long)T * sp / split), hi = (int)((long long)T * (sp + 1) / split);
    const double delta = jb.delta, emin = jb.emin;
    const float *E = jb.E, *th = jb.th;
    float *w32 = (float *)jb.w64;

    double v1 = 0.0;
    for (int i = lo + tid; i < hi; i += WT_THREADS) {
        const float e = E[i];
        const double w = isfinite(e) ? exp(-delta * ((double)e - emin)) : 0.0;
        jb.q[i] = (unsigned long long)floor(ldexp(w, 40));
        w32[i] = (float)w;
        v1 += w;
    }
    v1 = warp_sum_d(v1);
    if (lane == 0) rw[warp] = v1;

    // the same thread reads back the weights it wrote: no barrier needed
    for (int j = 0; j < d; ++j) {
        float h1 = 0.0f, l1 = 0.0f, h2 = 0.0f, l2 = 0.0f;
        if (jb.pri[j].kind != PR_FIXED) {
            const float *u = th + (size_t)j * T;
            const float c = u[0];
            float s1 = 0.0f, c1 = 0.0f, s2 = 0.0f, c2 = 0.0f;
            for (int i = lo + tid; i < hi; i += WT_THREADS) {
                const float x = u[i] - c, wx = w32[i] * x;
                kahan_add(s1, c1, wx);
                kahan_add(s2, c2, wx * x);
            }
            kahan_to_df(s1, c1, h1, l1);
            kahan_to_df(s2, c2, h2, l2);
            df_warp_sum(h1, l1);
            df_warp_sum(h2, l2);
        }
        if (lane == 0) {
            rh[2 * j][warp] = h1;
            rl[2 * j][warp] = l1;
            rh[2 * j + 1][warp] = h2;
            rl[2 * j + 1][warp] = l2;
        }
    }
    __syncthreads();
    double *row = jb.rwpart + (size_t)sp * (1 + 2 * d);
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < WT_WARPS; ++w) t += rw[w];
        row[0] = t;
    }
    for (int v = tid; v < 2 * d; v += WT_THREADS) {
        float h = 0.0f, l = 0.0f;
        for (int w = 0; w < WT_WARPS; ++w) df_add(h, l, rh[v][w], rl[v][w]);
        row[1 + v] = (double)h + (double)l;
    }
}

// ---------------------------------------------------------------------------
// k_finish32: one CTA per job
// ---------------------------------------------------------------------------
constexpr int FN_THREADS = 128;

__global__ void __launch_bounds__(FN_THREADS) k_finish32(JobDev *jobs, const int *slots)
{
    JobDev &jb = jobs[slots[blockIdx.x]];
    if (jb.state != JOB_ACTIVE || jb.status != 0) return;
    const int T = jb.T, d = jb.d, split = rw_split_of(T), ld = 1 + 2 * d;
    const double *part = jb.rwpart;
    double sw = 0.0;
    for (int sp = 0; sp < split; ++sp) sw += part[(size_t)sp * ld];
    for (int j = threadIdx.x; j < d; j += FN_THREADS) {
        double s1 = 0.0, s2 = 0.0;
        for (int sp = 0; sp < split; ++sp) {
            s1 += part[(size_t)sp * ld + 1 + 2 * j];
            s2 += part[(size_t)sp * ld + 2 + 2 * j];
        }
        const double c = (double)jb.th[(size_t)j * T], m1 = s1 / sw;
        update_step(jb, j, c + m1, s2 / sw - m1 * m1);
    }
    if (threadIdx.x == 0) {
        const double delta = jb.delta;
        jb.logz += -delta * jb.emin + log(sw / (double)T);
        jb.beta = jb.final_step ? 1.0 : jb.beta + delta;
        jb.next_chain = 0;
    }
}

cudaError_t launch_temper32(JobDev *jobs, const int *slots, int nslots, int64_t t_max, cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    const int max_split = rw_split_of(t_max);
    k_search32<<<nslots * SR_CL, SR_THREADS, 0, s>>>(jobs, slots);
    k_weights32<<<nslots * max_split, WT_THREADS, 0, s>>>(jobs, slots, max_split);
    k_finish32<<<nslots, FN_THREADS, 0, s>>>(jobs, slots);
    return cudaGetLastError();
}

}  // namespace smc
