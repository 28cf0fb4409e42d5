// k_mh_impl.cuh -- fused FP32 Metropolis rejuvenation (Sec. II B 4); the kernel
// template, instantiated per peak family in k_mh_{gauss,lor,pv}.cu.
//
// One chain is owned by a group of G warps; its N grid points are spread over
// the group's lanes (J points per lane, point i = 32 g + lane + 32 G jj), and
// the chain's residual r_i = y_i - f_i stays in registers for the whole stage.
// A component-wise random-walk proposal (Sec. II B 4) therefore costs one pass
// over the lane's points and one group reduction:
//   dE = 1/2 sum_i w_i D_i (D_i - 2 r_i),   D_i = g'_i - g_i (change of the peak)
// which is E(theta') - E(theta) of the Gaussian energy (App. C Eq. (C2)).  The
// lanes keep h_i = w_i / 2 and R_i = -w_i r_i instead of w_i and r_i, so a point
// costs two FMAs, dE = sum_i D_i (h_i D_i + R_i), and an accepted change D
// updates R_i += 2 h_i D_i.  A lane's points are held and updated in pairs by
// the packed FP32 instructions (f32x2: two results per issue slot), because
// the kernel is bound by instruction issue; each half of a packed operation
// is the scalar IEEE operation, and the two halves are the even and odd
// points of the lane's split accumulation.
// Within a peak's block of components the unit-amplitude shapes of the peak
// (the Gaussian and Lorentzian parts) are cached per point, so amplitude and
// mixing-ratio proposals need no transcendental at all and centre / width
// proposals need one EX2 (+ one RCP for Lorentzian parts) per point.
//
// Random numbers: Philox4x32-10, counter (t d + j, chain, stage, K).  At the
// start of a sweep lane j draws component j's proposal (words 0,1 -> Box-Muller
// normal, word 2 -> accept uniform) and folds the prior ratio into a threshold;
// proposal j is accepted iff thr_j < -beta dE.
#pragma once
#include <cfloat>
#include <cmath>

#include "f32x2.cuh"
#include "kernels.h"

namespace smc {

constexpr int MH_MAX_GROUPS = 16;  // warps per chain at most, and chains per block at most


template <int FAM>
__device__ __forceinline__ void shape(float x, float mu, float sc, float &S0, float &S1)
{
    const float t = fmaf(x, sc, -mu * sc);
    const float t2 = t * t;
    if (FAM == FAM_GAUSS) {
        S0 = ex2_approx(-t2);
    } else if (FAM == FAM_LORENTZ) {
        S0 = rcp_approx(1.0f + t2);
    } else {
        const float L = rcp_approx(1.0f + t2);
        S0 = ex2_approx(-t2) - L;  // Gaussian minus Lorentzian part
        S1 = L;
    }
}

// Cached per point during a peak's block: S0 = G - L (PV) or the unit shape
// (Gaussian / Lorentzian), and for PV U = eta (G - L) + L, the unit-amplitude
// profile; the current peak contributes A U (A S0 for the other families).
template <int FAM>
__device__ __forceinline__ float unit_of(float S0, float S1, float eta)
{
    return FAM == FAM_PV ? fmaf(eta, S0, S1) : S0;
}

// Sum of the G warp totals of a group in a fixed tree order (pairs within
// each float4, then across the float4s): identical in every lane, depth log2 G.
template <int G>
__device__ __forceinline__ float warp_totals_sum(const float *slot)
{
    if constexpr (G % 4 == 0) {
        float t[G / 4];
#pragma unroll
        for (int i = 0; i < G / 4; ++i) {
            const float4 q = *reinterpret_cast<const float4 *>(slot + 4 * i);
            t[i] = (q.x + q.y) + (q.z + q.w);
        }
#pragma unroll
        for (int w = 1; w < G / 4; w *= 2)
#pragma unroll
            for (int i = 0; i + w < G / 4; i += 2 * w) t[i] += t[i + w];
        return t[0];
    } else if constexpr (G == 2) {
        return slot[0] + slot[1];
    } else {
        float s = slot[0];
#pragma unroll
        for (int w = 1; w < G; ++w) s += slot[w];
        return s;
    }
}

template <int G>
struct GroupCtx {
    int lane, gw, grp;
    float *red;  // [2][G] for this group
    int par;
};

template <int G>
__device__ __forceinline__ void group_sync(const GroupCtx<G> &g)
{
    if (G == 1)
        __syncwarp();
    else
        named_barrier(1 + g.grp, 32 * G);
}

// The cross-warp part of group_sum, for a value already summed over the warp.
template <int G>
__device__ __forceinline__ float group_cross(GroupCtx<G> &g, float v)
{
    if (G == 1) return v;
    float *slot = g.red + g.par * MH_MAX_GROUPS;
    if (g.lane == 0) slot[g.gw] = v;
    named_barrier(1 + g.grp, 32 * G);
    const float s = warp_totals_sum<G>(slot);
    g.par ^= 1;
    return s;
}

template <int G>
__device__ __forceinline__ float group_sum(GroupCtx<G> &g, float v)
{
    v = warp_sum(v);
    if (G == 1) return v;
    float *slot = g.red + g.par * MH_MAX_GROUPS;
    if (g.lane == 0) slot[g.gw] = v;
    named_barrier(1 + g.grp, 32 * G);
    const float s = warp_totals_sum<G>(slot);
    g.par ^= 1;
    return s;
}

// Kahan-compensated energy 1/2 sum w r^2 over the group
template <int J, int G>
__device__ __forceinline__ float group_energy(GroupCtx<G> &g, const float *w, const float *r)
{
    float s = 0.0f, c = 0.0f;
#pragma unroll
    for (int jj = 0; jj < J; ++jj) {
        // w holds h = w/2 and r holds R = -w r: 1/2 w r^2 = R^2 / (4 h)
        const float term = w[jj] > 0.0f ? r[jj] * r[jj] / (4.0f * w[jj]) : 0.0f;
        const float yk = term - c;
        const float tk = s + yk;
        c = (tk - s) - yk;
        s = tk;
    }
    c = -c;
    warp_sum2(s, c);
    if (G == 1) return s + c;
    float *slot = g.red + g.par * MH_MAX_GROUPS;
    if (g.lane == 0) slot[g.gw] = s + c;
    named_barrier(1 + g.grp, 32 * G);
    // compensated sum of the warps' totals in a fixed order
    float S = 0.0f, Cc = 0.0f;
#pragma unroll
    for (int w2 = 0; w2 < G; ++w2) {
        const float yk = slot[w2] - Cc;
        const float tk = S + yk;
        Cc = (tk - S) - yk;
        S = tk;
    }
    g.par ^= 1;
    return S - Cc;
}

// Inverse scale of the shape argument t = (x - mu) sc: Gaussian with standard
// deviation w -> 1 / (w sqrt(2 ln 2)); Gaussian with precision b (wprec = 1)
// -> sqrt(b / (2 ln 2)); Lorentzian / pseudo-Voigt HWHM w -> 1 / w.
template <int FAM>
__device__ __forceinline__ float sc2_of(float w, int wprec)
{
    if (FAM == FAM_GAUSS) return wprec ? sqrtf(w) * SMC_INV_SQRT_2LN2 : SMC_INV_SQRT_2LN2 / w;
    return 1.0f / w;
}

// Per-warp copy of the chain's component state (every warp of a group keeps
// an identical copy, so no cross-warp synchronisation is needed for it).
struct WarpComp {
    float th[SMC_DMAX];   // current value, sampling coordinate
    float nat[SMC_DMAX];  // current value, natural
    unsigned acc[SMC_DMAX];
};

// One sweep's proposals of a chain, drawn once by the group's first warp and
// read by all of its warps (double-buffered by sweep parity: the group
// barrier after each table write keeps every warp within one sweep).  An
// accepted proposal sets its flag (every lane of every warp of the group
// stores the same 1, so no lane waits on another); the first warp adds the
// flags of sweep s to its acceptance counts when it draws sweep s + 2 into the
// same buffer, and those of the last two sweeps when the chain ends.
struct PropTable {
    float2 tv[SMC_DMAX];  // (thr, vn): accept iff thr < -beta dE (INFINITY: not proposed), natural value
    float un[SMC_DMAX];   // proposal, sampling coordinate
    unsigned acc[SMC_DMAX];  // 1: accepted in this table's sweep
};

// Chebyshev T_q(t) by the three-term recurrence
__device__ __forceinline__ float cheb(int q, float t)
{
    if (q == 0) return 1.0f;
    float a = 1.0f, b = t;
    for (int e = 2; e <= q; ++e) {
        const float c = fmaf(2.0f * t, b, -a);
        a = b;
        b = c;
    }
    return b;
}

// Threads per block of a tile: four one-, two- or four-warp chains per block,
// one chain per block beyond that.
template <int G>
struct MhThreads {
    static constexpr int NT = G <= 4 ? 128 : 32 * G;
};

// Register budget per tile, as resident blocks per SM (the __launch_bounds__
// minimum).  Measured on B300 (Metropolis time of XPS-, XRD- and App. C-shaped
// runs and of the tuning spectra): a four-warp chain per 128-thread block runs
// best at 64 registers for J <= 8 (32 warps per SM, despite a few spilled
// values) and at 128 for J <= 16; blocks holding several one- or two-warp
// chains keep 128 / 170 registers (their extra per-chain state spills
// otherwise); 256- and 512-thread blocks at 64 (J <= 8) or 128 registers.
template <int FAM, int J, int G>
struct MhBounds {
    static constexpr int NT = MhThreads<G>::NT;
    static constexpr int MINB =
        (G == 4)      ? (J <= 8 ? 8 : (J <= 16 ? 4 : 2))
        : (NT == 128) ? (J <= 8 ? 4 : (J <= 12 || (J <= 16 && FAM != FAM_PV) ? 3 : 2))
        : (NT == 256) ? (J <= 8 ? 4 : 2)
                      : 2;
};

// Register budget of a tile: R = 0 takes MhBounds; R > 0 asks for at most R
// registers per thread (resident blocks per SM = 65536 / (threads x R)), a
// dimension the autotuner sweeps for four- and eight-warp chains.
template <int FAM, int J, int G, int R>
struct MhMinBlocks {
    static constexpr int NT = MhThreads<G>::NT;
    static constexpr int value = R == 0 ? MhBounds<FAM, J, G>::MINB
                                        : (65536 / (NT * R) > 0 ? 65536 / (NT * R) : 1);
};

__device__ __forceinline__ f2 neg2(f2 a) { return mul2(a, splat2(-1.0f)); }

// Packed form of shape() for two grid points: the argument in f32x2
// arithmetic, one MUFU operation per point and transcendental.  Each half is
// bit-identical to shape() of that point.  (A Newton-Raphson reciprocal on the
// FMA pipe in place of the SFU's was measured slower: the kernel is bound by
// issue and latency, not by the SFU.)
template <int FAM>
__device__ __forceinline__ void shape2(f2 x, f2 sc, f2 nmsc, f2 &S0, f2 &S1)
{
    const f2 t = fma2(x, sc, nmsc);
    const f2 t2 = mul2(t, t);
    if (FAM == FAM_GAUSS) {
        S0 = mk2(ex2_approx(-lo2(t2)), ex2_approx(-hi2(t2)));
    } else {
        const f2 q = add2(t2, splat2(1.0f));
        const f2 L = mk2(rcp_approx(lo2(q)), rcp_approx(hi2(q)));
        if (FAM == FAM_LORENTZ) {
            S0 = L;
        } else {
            S0 = sub2(mk2(ex2_approx(-lo2(t2)), ex2_approx(-hi2(t2))), L);  // G - L
            S1 = L;
        }
    }
}

// group_energy() on packed points (pair p holds points 2p and 2p + 1; the
// compensated sum runs over them in that order)
template <int JP, int G>
__device__ __forceinline__ float group_energy2(GroupCtx<G> &g, const f2 *w2, const f2 *r2)
{
    float w[2 * JP], r[2 * JP];
#pragma unroll
    for (int p = 0; p < JP; ++p) {
        w[2 * p] = lo2(w2[p]);
        w[2 * p + 1] = hi2(w2[p]);
        r[2 * p] = lo2(r2[p]);
        r[2 * p + 1] = hi2(r2[p]);
    }
    return group_energy<2 * JP, G>(g, w, r);
}

template <int FAM, int J, int G, int R>
__global__ void __launch_bounds__(MhThreads<G>::NT, (MhMinBlocks<FAM, J, G, R>::value))
    k_mh(JobDev *__restrict__ jobs, const int *__restrict__ slots, int nslots)
{
    static_assert(J % 2 == 0, "a lane's points are processed in packed pairs");
    constexpr int JP = J / 2;
    constexpr int NT = MhThreads<G>::NT;
    __shared__ __align__(16) float red_sh[MH_MAX_GROUPS][2][MH_MAX_GROUPS];
    __shared__ int work_sh[MH_MAX_GROUPS][2];
    __shared__ WarpComp comp_sh[NT / 32];
    __shared__ PropTable prop_sh[NT / 32 / G][2];  // one double-buffered table per chain
    // with J >= 16 the lane's grid abscissae (pairs) live in shared memory
    // rather than in registers: read once per shape evaluation, they free J
    // registers a lane (measured: -3 % Metropolis time at J = 16, +1.5 % at J = 8)
    constexpr bool XS = J >= 16;
    __shared__ unsigned long long xs_sh[XS ? NT / 32 : 1][XS ? J / 2 : 1][32];
    GroupCtx<G> g;
    g.lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    g.grp = warp / G;
    g.gw = warp - g.grp * G;
    g.par = 0;
    constexpr int ngroups = (NT / 32) / G;
    if (g.grp >= ngroups) return;
    g.red = &red_sh[g.grp][0][0];
    const int lane = g.lane;
    WarpComp &cs = comp_sh[warp];
    constexpr int P = (FAM == FAM_PV) ? 4 : 3;

    int li = 0;
    for (;;) {
        // ---- claim the next chain (dynamic scheduling over the bucket's jobs)
        int slot = -1, m = 0;
        if (g.gw == 0 && lane == 0) {
            while (li < nslots) {
                const int sl = slots[li];
                JobDev &jq = jobs[sl];
                if (jq.state == JOB_ACTIVE && jq.status == 0) {
                    const int c = atomicAdd(&jq.next_chain, 1);
                    if (c < jq.S) {
                        slot = sl;
                        m = c;
                        break;
                    }
                }
                ++li;
            }
            if constexpr (G > 1) {
                work_sh[g.grp][0] = slot;
                work_sh[g.grp][1] = m;
            }
        }
        if constexpr (G == 1) {
            slot = __shfl_sync(FULL_MASK, slot, 0);
            m = __shfl_sync(FULL_MASK, m, 0);
        } else {
            named_barrier(1 + g.grp, 32 * G);
            slot = work_sh[g.grp][0];
            m = work_sh[g.grp][1];
            named_barrier(1 + g.grp, 32 * G);
        }
        if (slot < 0) break;

        const JobDev &jb = jobs[slot];
        const int K = jb.K, d = jb.d, nbg = jb.nbg, S = jb.S, T = jb.T, n = jb.sweeps;
        const int wf = jb.waste_free, wprec = jb.wprec;
        const float beta = (float)jb.beta;
        const uint32_t stage = (uint32_t)(jb.stage + 1), tag = jb.tag;
        const unsigned long long seed = jb.seed;
        const int base = g.gw * 32 + lane;
        const int stride = 32 * G;

        // ---- components of the chain start
        for (int j = lane; j < d; j += 32) {
            const float u = jb.ths[(size_t)j * S + m];
            cs.th[j] = u;
            cs.nat[j] = natural_f(jb.pri[j], u);
            cs.acc[j] = 0u;
            if (g.gw == 0) {
                prop_sh[g.grp][0].acc[j] = 0u;
                prop_sh[g.grp][1].acc[j] = 0u;
            }
        }
        __syncwarp();

        // ---- grid points of this lane, in pairs (points 2p and 2p + 1 of the
        // lane), and the residual r = y - f(theta)
        f2 xr[XS ? 1 : JP], w[JP], r[JP], S0[JP], S1[JP], N0[JP], N1[JP];
        unsigned long long(&xs)[XS ? J / 2 : 1][32] = xs_sh[XS ? warp : 0];
        const auto X = [&](int p) {
            if constexpr (XS) {
                f2 v;
                v.v = xs[p][lane];
                return v;
            } else {
                return xr[p];
            }
        };
#pragma unroll
        for (int p = 0; p < JP; ++p) {
            const int i0 = base + 2 * p * stride, i1 = i0 + stride;
            if constexpr (XS)
                xs[p][lane] = mk2(__ldg(jb.xc + i0), __ldg(jb.xc + i1)).v;
            else
                xr[p] = mk2(__ldg(jb.xc + i0), __ldg(jb.xc + i1));
            w[p] = mk2(__ldg(jb.wt + i0), __ldg(jb.wt + i1));
            r[p] = mk2(__ldg(jb.y + i0), __ldg(jb.y + i1));
        }
        for (int k = 0; k < K; ++k) {
            const int j0 = k * P;
            const float A = cs.nat[j0], mu = cs.nat[j0 + 1], wd = cs.nat[j0 + 2];
            const float eta = (FAM == FAM_PV) ? cs.nat[j0 + 3] : 0.0f;
            const float sc = sc2_of<FAM>(wd, wprec);
            const f2 scv = splat2(sc), nmsc = splat2(-mu * sc), nA = splat2(-A), et = splat2(eta);
#pragma unroll
            for (int p = 0; p < JP; ++p) {
                f2 a0, a1 = splat2(0.0f);
                shape2<FAM>(X(p), scv, nmsc, a0, a1);
                r[p] = fma2(nA, FAM == FAM_PV ? fma2(et, a0, a1) : a0, r[p]);
            }
        }
        if (nbg > 0) {
            // Chebyshev terms by the three-term recurrence, carried across q
#pragma unroll
            for (int p = 0; p < JP; ++p) {
                const int i0 = base + 2 * p * stride;
                N0[p] = mk2(__ldg(jb.ts + i0), __ldg(jb.ts + i0 + stride));  // t
                S0[p] = splat2(1.0f);                                         // T_{q-1}
                S1[p] = N0[p];                                                // T_q (q = 1)
            }
            for (int q = 0; q < nbg; ++q) {
                const f2 ncq = splat2(-cs.nat[K * P + q]);
#pragma unroll
                for (int p = 0; p < JP; ++p) {
                    f2 tq;
                    if (q == 0) {
                        tq = splat2(1.0f);
                    } else if (q == 1) {
                        tq = N0[p];
                    } else {
                        tq = fma2(add2(N0[p], N0[p]), S1[p], neg2(S0[p]));
                        S0[p] = S1[p];
                        S1[p] = tq;
                    }
                    r[p] = fma2(ncq, tq, r[p]);
                }
            }
        }

        // weighted form of the residual: h = w / 2, R = -w r, so that
        // dE = 1/2 sum w D (D - 2 r) = sum D (h D + R) and, on acceptance,
        // r -> r - D is R -> R + 2 h D
#pragma unroll
        for (int p = 0; p < JP; ++p) {
            r[p] = mul2(neg2(w[p]), r[p]);
            w[p] = mul2(splat2(0.5f), w[p]);
        }
        unsigned n_eval = 0, n_shape = 0, n_peak = 0;  // evaluated proposals (group-uniform)
        for (int sw = 0; sw < n; ++sw) {
            // ---- this sweep's proposals: lane j of the first warp draws component j
            PropTable &tb = prop_sh[g.grp][sw & 1];
            if (g.gw == 0)
            for (int j = lane; j < d; j += 32) {
                const PriorDev &pr = jb.pri[j];
                float thr = INFINITY, u = 0.0f, v = 0.0f;
                if (pr.kind != PR_FIXED) {
                    const uint4 wv = draw(seed, (uint32_t)(sw * d + j), (uint32_t)m, stage, tag);
                    const float z = box_muller_f(wv.x, wv.y);
                    const float lu = logf(u01f(wv.z));
                    const float t0 = cs.th[j];
                    u = fmaf(jb.stepf[j], z, t0);
                    if (in_support_f(pr, u)) {
                        thr = lu - (log_prior_f(pr, u) - log_prior_f(pr, t0));
                        v = pr.kind == PR_LOG_UNIFORM ? expf(u) : u;
                    }
                }
                tb.tv[j] = make_float2(thr, v);
                tb.un[j] = u;
                cs.acc[j] += tb.acc[j];  // acceptances of sweep sw - 2
                tb.acc[j] = 0u;
            }
            group_sync(g);

            // ---- peak blocks
            for (int k = 0; k < K; ++k) {
                const int j0 = k * P;
                float A = cs.nat[j0], mu = cs.nat[j0 + 1], wd = cs.nat[j0 + 2];
                float eta = (FAM == FAM_PV) ? cs.nat[j0 + 3] : 0.0f;
                float sc = sc2_of<FAM>(wd, wprec);
                {
                    const f2 scv = splat2(sc), nmsc = splat2(-mu * sc), et = splat2(eta);
#pragma unroll
                    for (int p = 0; p < JP; ++p) {
                        f2 l = splat2(0.0f);
                        shape2<FAM>(X(p), scv, nmsc, S0[p], l);
                        if (FAM == FAM_PV) S1[p] = fma2(et, S0[p], l);  // U
                    }
                }
                float tq[P], vq[P];
#pragma unroll
                for (int c = 0; c < P; ++c) {
                    const float2 q2 = tb.tv[j0 + c];
                    tq[c] = q2.x;
                    vq[c] = q2.y;
                }
                bool mu_ready = false;  // the centre proposal's profile already in N0 / N1
#pragma unroll
                for (int c = 0; c < P; ++c) {
                    const int j = j0 + c;
                    const float tj = tq[c];
                    if (tj == INFINITY) continue;  // fixed or outside the prior's support
                    const float v = vq[c];
                    ++n_eval;
                    ++n_peak;
                    // lanes of the packed accumulator: even and odd points
                    f2 acc2 = splat2(0.0f);
                    if (c == 0) {  // amplitude: D = (A' - A) U
                        const f2 dA = splat2(v - A);
#pragma unroll
                        for (int p = 0; p < JP; ++p) {
                            const f2 D = mul2(dA, FAM == FAM_PV ? S1[p] : S0[p]);
                            acc2 = fma2(D, fma2(w[p], D, r[p]), acc2);
                        }
                    } else if (c == 3) {  // mixing ratio: D = A (eta' - eta) (G - L)
                        const f2 dd = splat2(A * (v - eta));
#pragma unroll
                        for (int p = 0; p < JP; ++p) {
                            const f2 D = mul2(dd, S0[p]);
                            acc2 = fma2(D, fma2(w[p], D, r[p]), acc2);
                        }
                    } else if (c == 1 && mu_ready) {  // centre, profile computed already
                        ++n_shape;
                        const f2 Av = splat2(A);
#pragma unroll
                        for (int p = 0; p < JP; ++p) {
                            const f2 D = mul2(Av, FAM == FAM_PV ? sub2(N1[p], S1[p]) : sub2(N0[p], S0[p]));
                            acc2 = fma2(D, fma2(w[p], D, r[p]), acc2);
                        }
                    } else {  // centre or width: new shape, D = A (U' - U)
                        ++n_shape;
                        const float mu2 = (c == 1) ? v : mu;
                        const float scn = (c == 2) ? sc2_of<FAM>(v, wprec) : sc;
                        const f2 scv = splat2(scn), nmsc = splat2(-mu2 * scn), et = splat2(eta),
                                 Av = splat2(A);
#pragma unroll
                        for (int p = 0; p < JP; ++p) {
                            f2 l = splat2(0.0f);
                            shape2<FAM>(X(p), scv, nmsc, N0[p], l);
                            if (FAM == FAM_PV) N1[p] = fma2(et, N0[p], l);
                            const f2 D = mul2(Av, FAM == FAM_PV ? sub2(N1[p], S1[p]) : sub2(N0[p], S0[p]));
                            acc2 = fma2(D, fma2(w[p], D, r[p]), acc2);
                        }
                    }
                    float dE;
                    if (c == 0 && tq[1] != INFINITY) {
                        // The centre proposal's new unit-amplitude profile does
                        // not depend on the amplitude's outcome: it is computed
                        // between the shuffles of the amplitude's reduction, so
                        // that its SFU and FMA work fills the reduction's latency.
                        float s0 = lo2(acc2) + hi2(acc2);
                        s0 += __shfl_xor_sync(FULL_MASK, s0, 16);
                        const f2 scv = splat2(sc), nmsc = splat2(-vq[1] * sc), et = splat2(eta);
#pragma unroll
                        for (int p = 0; p < JP; ++p) {
                            f2 l = splat2(0.0f);
                            shape2<FAM>(X(p), scv, nmsc, N0[p], l);
                            if (FAM == FAM_PV) N1[p] = fma2(et, N0[p], l);
                        }
                        s0 += __shfl_xor_sync(FULL_MASK, s0, 8);
                        s0 += __shfl_xor_sync(FULL_MASK, s0, 4);
                        s0 += __shfl_xor_sync(FULL_MASK, s0, 2);
                        s0 += __shfl_xor_sync(FULL_MASK, s0, 1);
                        dE = group_cross(g, s0);
                        mu_ready = true;
                    } else {
                        dE = group_sum(g, lo2(acc2) + hi2(acc2));
                    }
                    if (tj < -beta * dE) {
                        if (c == 0) {
                            const float dA = v - A;
                            const f2 d2 = splat2(dA + dA);
#pragma unroll
                            for (int p = 0; p < JP; ++p)
                                r[p] = fma2(w[p], mul2(d2, FAM == FAM_PV ? S1[p] : S0[p]), r[p]);
                            A = v;
                        } else if (c == 3) {
                            const float de = v - eta;
                            const float dd = A * de;
                            const f2 dd2 = splat2(dd + dd), de2 = splat2(de);
#pragma unroll
                            for (int p = 0; p < JP; ++p) {
                                r[p] = fma2(w[p], mul2(dd2, S0[p]), r[p]);
                                S1[p] = fma2(de2, S0[p], S1[p]);
                            }
                            eta = v;
                        } else {
                            const f2 AA = splat2(A + A);
#pragma unroll
                            for (int p = 0; p < JP; ++p) {
                                if (FAM == FAM_PV) {
                                    r[p] = fma2(w[p], mul2(AA, sub2(N1[p], S1[p])), r[p]);
                                    S1[p] = N1[p];
                                } else {
                                    r[p] = fma2(w[p], mul2(AA, sub2(N0[p], S0[p])), r[p]);
                                }
                                S0[p] = N0[p];
                            }
                            if (c == 1) {
                                mu = v;
                            } else {
                                wd = v;
                                sc = sc2_of<FAM>(v, wprec);
                            }
                        }
                        // every lane stores the same values (no lane waits on
                        // another); the count is the table's flag
                        cs.th[j] = tb.un[j];
                        cs.nat[j] = v;
                        tb.acc[j] = 1u;
                    }
                }
            }
            // ---- background coefficients: D = (c' - c) T_q(t), the Chebyshev
            // terms by the recurrence carried across q (N1: t, S0/S1: T_{q-1}, T_q)
            if (nbg > 0) {
#pragma unroll
                for (int p = 0; p < JP; ++p) {
                    const int i0 = base + 2 * p * stride;
                    N1[p] = mk2(__ldg(jb.ts + i0), __ldg(jb.ts + i0 + stride));
                    S0[p] = splat2(1.0f);
                    S1[p] = N1[p];
                }
            }
            for (int q = 0; q < nbg; ++q) {
                const int j = K * P + q;
                // advance the recurrence to T_q for every q, proposed or not
#pragma unroll
                for (int p = 0; p < JP; ++p) {
                    if (q == 0) {
                        N0[p] = splat2(1.0f);
                    } else if (q == 1) {
                        N0[p] = N1[p];
                    } else {
                        N0[p] = fma2(add2(N1[p], N1[p]), S1[p], neg2(S0[p]));
                        S0[p] = S1[p];
                        S1[p] = N0[p];
                    }
                }
                const float2 q2 = tb.tv[j];
                const float tj = q2.x;
                if (tj == INFINITY) continue;
                const float v = q2.y;
                const float dc = v - cs.nat[j];
                ++n_eval;
                f2 acc2 = splat2(0.0f);
                const f2 dcv = splat2(dc);
#pragma unroll
                for (int p = 0; p < JP; ++p) {
                    const f2 D = mul2(dcv, N0[p]);
                    acc2 = fma2(D, fma2(w[p], D, r[p]), acc2);
                }
                const float dE = group_sum(g, lo2(acc2) + hi2(acc2));
                if (tj < -beta * dE) {
                    const f2 d2 = splat2(dc + dc);
#pragma unroll
                    for (int p = 0; p < JP; ++p) r[p] = fma2(w[p], mul2(d2, N0[p]), r[p]);
                    cs.th[j] = tb.un[j];
                    cs.nat[j] = v;
                    tb.acc[j] = 1u;
                }
            }
            if (wf) {
                const float E = group_energy2<JP, G>(g, w, r);
                const size_t o = (size_t)m * n + sw;
                if (g.gw == 0) {
                    for (int j = lane; j < d; j += 32) jb.th[(size_t)j * T + o] = cs.th[j];
                    if (lane == 0) jb.E[o] = E;
                }
            }
        }
        if (!wf) {
            const float E = group_energy2<JP, G>(g, w, r);
            if (g.gw == 0) {
                for (int j = lane; j < d; j += 32) jb.th[(size_t)j * T + m] = cs.th[j];
                if (lane == 0) jb.E[m] = E;
            }
        }
        if (g.gw == 0) {
            for (int j = lane; j < d; j += 32)
                if (jb.pri[j].kind != PR_FIXED) {
                    atomicAdd(&jobs[slot].acc[j],
                              (unsigned long long)(cs.acc[j] + prop_sh[g.grp][0].acc[j] +
                                                   prop_sh[g.grp][1].acc[j]));
                    atomicAdd(&jobs[slot].prop[j], (unsigned long long)n);
                }
            if (lane == 0) {
                const unsigned long long npts = (unsigned long long)jb.n;
                atomicAdd(&jobs[slot].point_evals, (unsigned long long)n_eval * npts);
                atomicAdd(&jobs[slot].sfu_ops,
                          (unsigned long long)n_shape * npts * (FAM == FAM_PV ? 2ull : 1ull));
                atomicAdd(&jobs[slot].peak_evals, (unsigned long long)n_peak * npts);
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// instantiation table of one family
// ---------------------------------------------------------------------------
typedef void (*mh_fn)(JobDev *, const int *, int);

template <int FAM, int G>
static mh_fn mh_pick_j(int J)
{
    switch (J) {
    case 4: return k_mh<FAM, 4, G, 0>;
    case 8: return k_mh<FAM, 8, G, 0>;
    case 12:
        if constexpr (G <= 8) return k_mh<FAM, 12, G, 0>;
        return nullptr;
    case 16:
        if constexpr (G <= 8) return k_mh<FAM, 16, G, 0>;
        return nullptr;
    case 24:
        if constexpr (FAM != FAM_PV && G == 1) return k_mh<FAM, 24, G, 0>;
        return nullptr;
    case 32:
        if constexpr (FAM != FAM_PV && G == 1) return k_mh<FAM, 32, G, 0>;
        return nullptr;
    default: return nullptr;
    }
}

// register-budget variants (R = 64, 80, 96, 128) of four- and eight-warp
// chains with J = 4, 8, 16
template <int FAM, int J, int G>
static mh_fn mh_pick_r(int R)
{
    switch (R) {
    case 64: return k_mh<FAM, J, G, 64>;
    case 80: return k_mh<FAM, J, G, 80>;
    case 96: return k_mh<FAM, J, G, 96>;
    case 128: return k_mh<FAM, J, G, 128>;
    default: return nullptr;
    }
}

template <int FAM, int G>
static mh_fn mh_pick_jr(int J, int R)
{
    switch (J) {
    case 4: return mh_pick_r<FAM, 4, G>(R);
    case 8: return mh_pick_r<FAM, 8, G>(R);
    case 16: return mh_pick_r<FAM, 16, G>(R);
    default: return nullptr;
    }
}

template <int FAM>
static mh_fn mh_pick_family(int J, int G, int R)
{
    if (R != 0) {
        if (G == 4) return mh_pick_jr<FAM, 4>(J, R);
        if (G == 8) return mh_pick_jr<FAM, 8>(J, R);
        return nullptr;
    }
    switch (G) {
    case 1: return mh_pick_j<FAM, 1>(J);
    case 2: return mh_pick_j<FAM, 2>(J);
    case 4: return mh_pick_j<FAM, 4>(J);
    case 8: return mh_pick_j<FAM, 8>(J);
    case 16: return mh_pick_j<FAM, 16>(J);
    default: return nullptr;
    }
}

}  // namespace smc
