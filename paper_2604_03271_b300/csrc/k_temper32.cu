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
// B300 executes FP64 at a small fraction of its FP32 rate, so this path spends
// FP64 only where the result needs it, and spreads the FP64 work over the GPU:
//   k_search32   one 8-CTA cluster per job: minimum energy and the bisection,
//                which takes exactly the decisions of the FP64 bisection.  A
//                pass first evaluates the ESS in FP32 (weights by ex2 on the
//                SFU, per-thread Kahan sums, two-float reductions; error of the
//                ESS fraction below 2^-21) at the 2^L - 1 midpoints of the
//                bracket's dyadic tree (RW_LEVELS levels per pass) and walks the
//                tree while every ESS fraction lies more than RW_MARGIN from
//                rho, so that the decision cannot differ from the FP64 one.  The
//                first undecidable midpoint (the last ~8 halvings, whose ESS
//                lies within about 2e-5 of rho T) switches the job to FP64: once
//                the bracket [a, b] is narrower than 1e-4 b, one FP64 pass at its
//                lower end computes w_a = exp(-a e') (e' = E - E_min) and the
//                moments M_k = sum w_a e'^k, N_k = sum w_a^2 e'^k, k <= 4; then
//                for every remaining midpoint m = a + h,
//                  sum w   = sum_k (-h)^k M_k / k!,  sum w^2 = sum_k (-2h)^k N_k / k!,
//                the Taylor series of sum w_a exp(-h e') (h e' <= 1e-4 a e': the
//                truncated terms are below FP64 rounding for every weight that is
//                not below e^-40 of the largest), so thread 0 finishes the
//                bisection without further passes.  (Wider brackets that cannot
//                be decided in FP32 take full FP64 passes first.)  Thread 0 of
//                each CTA does the FP64 scalar logic on the gathered totals
//                (identical in every CTA) and broadcasts the next pass.
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
constexpr double RW_MARGIN = 1e-5;            // FP32 decides only if |ESS/T - rho| > this
constexpr double RW_REBASE = 1e-4;            // FP64 moment series once b - a <= this * b
constexpr int RW_MOM = 5;                     // moments k = 0..4
enum { SR_FP32 = 0, SR_MOMENTS = 1, SR_EXP = 3 };  // kinds of search pass
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
    float rh[SR_VALS][SR_WARPS], rl[SR_VALS][SR_WARPS];  // warp totals (FP32 passes)
    float xh[2][SR_VALS], xl[2][SR_VALS];                // CTA totals (read remotely)
    float gh[SR_VALS][SR_CL], gl[SR_VALS][SR_CL];        // gathered CTA totals
    double rd[2 * RW_MOM][SR_WARPS];                     // the same for FP64 passes
    double xd[2][2 * RW_MOM], gd[2 * RW_MOM][SR_CL];
    float kc[RW_CAND];                                   // -delta log2(e) per candidate
    double m64;                                          // FP64 pass: candidate or moment base
    float mn[SR_WARPS], xmin, gmin[SR_CL];
    int nc, go, mode;
    // search state, kept and changed by thread 0 only
    double a, b, delta, cand[RW_CAND];
    int iters, final_step, bisecting;
};

// sum_k (-h)^k mom[k] / k!, k = 0..4 (Horner in -h)
__device__ __forceinline__ double moment_series(const double *mom, double h)
{
    double p = mom[4] / 24.0;
    p = fma(-h, p, mom[3] / 6.0);
    p = fma(-h, p, mom[2] / 2.0);
    p = fma(-h, p, mom[1]);
    return fma(-h, p, mom[0]);
}

// Thread 0's FP64 logic after a pass of the given kind: reads the gathered
// totals, takes the decisions and sets up the next pass (or ends the search).
__device__ __noinline__ void search_decide(SearchShared &sh, int mode, int T, double rho, double room)
{
    double a = sh.a, b = sh.b, delta = sh.delta, *cand = sh.cand;
    int iters = sh.iters, final_step = sh.final_step, bisecting = sh.bisecting;
    int go = 1, to64 = 0;
    if (mode == SR_FP32) {
        const int nc = sh.nc;
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
        if (!bisecting) {
            if (fabs(frac[0] - rho) <= RW_MARGIN) {
                to64 = 1;  // the whole-step check itself in FP64
            } else if (frac[0] >= rho) {
                delta = room;
                final_step = 1;
                go = 0;
            } else {
                bisecting = 1;
            }
        } else {
            int node = 0;
            for (int lev = 0; lev < RW_LEVELS && iters < 200 && b - a > 1e-7 * b; ++lev) {
                if (fabs(frac[node] - rho) <= RW_MARGIN) {
                    to64 = 1;
                    break;
                }
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
    } else if (mode == SR_EXP) {
        double t1 = 0.0, t2 = 0.0;
        for (int r = 0; r < SR_CL; ++r) {
            t1 += sh.gd[0][r];
            t2 += sh.gd[1][r];
        }
        const double fr = t1 * t1 / ((double)T * t2);
        if (!bisecting) {
            if (fr >= rho) {
                delta = room;
                final_step = 1;
                go = 0;
            } else {
                bisecting = 1;  // bisection starts with FP32 passes
            }
        } else {
            if (fr >= rho)
                a = sh.m64;
            else
                b = sh.m64;
            ++iters;
            to64 = 1;  // once in FP64, stay
        }
    } else {
        // moments at base = a: finish the bisection by the series
        double mw[RW_MOM], mw2[RW_MOM];
        for (int q = 0; q < RW_MOM; ++q) {
            double t1 = 0.0, t2 = 0.0;
            for (int r = 0; r < SR_CL; ++r) {
                t1 += sh.gd[q][r];
                t2 += sh.gd[RW_MOM + q][r];
            }
            mw[q] = t1;
            mw2[q] = t2;
        }
        const double base = sh.m64;
        while (iters < 200 && b - a > 1e-7 * b) {
            const double mid = 0.5 * (a + b), h = mid - base;
            const double t1 = moment_series(mw, h), t2 = moment_series(mw2, 2.0 * h);
            if (t1 * t1 / ((double)T * t2) >= rho)
                a = mid;
            else
                b = mid;
            ++iters;
        }
        to64 = 1;  // terminates below
    }
    if (go) {
        if (bisecting && !(iters < 200 && b - a > 1e-7 * b)) {
            go = 0;
            delta = a > 0.0 ? a : b;
        } else if (to64) {
            // next FP64 pass: the whole-step check or a midpoint (full
            // exponentials), or the moments once the bracket is narrow
            if (bisecting && b - a <= RW_REBASE * b) {
                sh.m64 = a;
                sh.mode = SR_MOMENTS;
            } else {
                sh.m64 = bisecting ? 0.5 * (a + b) : room;
                sh.mode = SR_EXP;
            }
        } else {
            // next FP32 pass: heap of midpoints, node n splits the
            // bracket held on reaching it
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
            sh.mode = SR_FP32;
        }
    }
    sh.go = go;

    sh.a = a;
    sh.b = b;
    sh.delta = delta;
    sh.iters = iters;
    sh.final_step = final_step;
    sh.bisecting = bisecting;
}

__global__ void __cluster_dims__(SR_CL, 1, 1) __launch_bounds__(SR_THREADS, 1)
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
    const double room = 1.0 - jb.beta, rho = jb.rho, emin_d = (double)emin;
    if (tid == 0) {
        sh.a = 0.0;
        sh.b = room;
        sh.delta = room;
        sh.iters = sh.final_step = sh.bisecting = 0;
        sh.cand[0] = room;
        sh.kc[0] = (float)(-room * LOG2E);
        sh.nc = 1;
        sh.mode = SR_FP32;
        sh.go = 1;
    }
    int par = 0;
    for (;;) {
        __syncthreads();
        if (!sh.go) break;
        const int mode = sh.mode;
        if (mode == SR_FP32) {
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
        } else {
            // FP64 pass: sum w, sum w^2 at the candidate m (SR_EXP), or the
            // moments of w_a = exp(-a e') at the bracket's lower end (SR_MOMENTS)
            const double m = sh.m64;
            const int nv = mode == SR_EXP ? 2 : 2 * RW_MOM;
            double acc[2 * RW_MOM];
#pragma unroll
            for (int v = 0; v < 2 * RW_MOM; ++v) acc[v] = 0.0;
            for (int i = lo + tid; i < hi; i += SR_THREADS) {
                const float e = E[i];
                if (!isfinite(e)) continue;
                const double ep = (double)e - emin_d;
                const double w = exp(-m * ep);
                if (mode == SR_EXP) {
                    acc[0] += w;
                    acc[1] = fma(w, w, acc[1]);
                } else {
                    double t1 = w, t2 = w * w;
#pragma unroll
                    for (int q = 0; q < RW_MOM; ++q) {
                        acc[q] += t1;
                        acc[RW_MOM + q] += t2;
                        t1 *= ep;
                        t2 *= ep;
                    }
                }
            }
            for (int v = 0; v < nv; ++v) {
                const double t = warp_sum_d(acc[v]);
                if (lane == 0) sh.rd[v][warp] = t;
            }
            __syncthreads();
            if (tid < nv) {
                double t = 0.0;
                for (int w = 0; w < SR_WARPS; ++w) t += sh.rd[tid][w];
                sh.xd[par][tid] = t;
            }
            cl.sync();
            if (tid < nv * SR_CL) {
                const int v = tid / SR_CL, r = tid - v * SR_CL;
                sh.gd[v][r] = *cl.map_shared_rank(&sh.xd[par][v], r);
            }
        }
        __syncthreads();
        if (tid == 0) search_decide(sh, mode, T, rho, room);
        par ^= 1;
    }
    if (rank == 0 && tid == 0) {
        jb.delta = sh.delta;
        jb.final_step = sh.final_step;
        jb.bisect_iters = sh.iters;
        jb.emin = emin_d;
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
    const double beta_prev = jb.beta, beta_next = jb.final_step ? 1.0 : jb.beta + jb.delta;
    double sw = 0.0;
    for (int sp = 0; sp < split; ++sp) sw += part[(size_t)sp * ld];
    for (int j = threadIdx.x; j < d; j += FN_THREADS) {
        double s1 = 0.0, s2 = 0.0;
        for (int sp = 0; sp < split; ++sp) {
            s1 += part[(size_t)sp * ld + 1 + 2 * j];
            s2 += part[(size_t)sp * ld + 2 + 2 * j];
        }
        const double c = (double)jb.th[(size_t)j * T], m1 = s1 / sw;
        update_step(jb, j, c + m1, s2 / sw - m1 * m1, beta_prev, beta_next);
    }
    __syncthreads();  // every thread has read beta before it moves on
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
