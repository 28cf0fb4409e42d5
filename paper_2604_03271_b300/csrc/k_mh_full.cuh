// k_mh_full.cuh -- fused FP32 Metropolis rejuvenation (Sec. II B 4) for the
// likelihoods of App. E that couple the grid points: the Shirley background,
// whose value at x_i is the running integral of the peak signal up to x_i,
//   B_i = a + (b - a) C_i / C_N,  C_i = sum_{1 < j <= i} P_j |x_j - x_{j-1}|,
// and the variance that follows the model value f_i,
//   v_i = s0^2 f_i + s1^2 f_i^2 + s2^2,
//   E = sum_i [1/2 ln(2 pi v_i) + 1/2 (y_i - f_i)^2 / v_i]
// (or the known-sigma energy 1/2 sum_i w_i (y_i - f_i)^2 with the Shirley
// background).  Instantiated per peak family in k_mh_full_{gauss,lor,pv}.cu.
//
// Layout and scheduling are those of k_mh (one chain per group of G warps,
// dynamic chain claims, the sweep's proposals drawn by the first warp into a
// shared table, the current peak's unit shape cached per point), except that a
// lane owns J consecutive grid points (i = (32 g + lane) J + jj), so that the
// running integral of a proposal's peak change D is a lane-local prefix plus a
// group scan.  A lane keeps per point: x, y, w (1/sigma^2, or 1 / 0 marking grid
// and padding points with the model variance), the Shirley increment
// |x_i - x_{i-1}|, the model value f, the running integral C and the energy term
// e.  A proposal computes the new f' = f + D + B' - B and e' at every point and
// dE = sum (e' - e) with one group reduction; acceptance copies f', e', C'.
// Background proposals (a, b) change B = a + (b - a) C / C_N at fixed C.
#pragma once
#include "k_mh_impl.cuh"

namespace smc {

constexpr float MHF_HALF_LN_2PI = 0.91893853320467274f;  // 1/2 ln(2 pi)
constexpr float MHF_HALF_LN2 = 0.34657359027997264f;     // 1/2 ln 2

// energy term of one grid point (wt = 0: padding point, term 0); the model
// variance's term is computed unconditionally and selected (no branch)
__device__ __forceinline__ float mhf_eterm(int noise, float f, float y, float wt, float nv0,
                                           float nv1, float nv2)
{
    const float r = y - f;
    if (noise == NZ_KNOWN) return 0.5f * wt * r * r;
    float t;
    if (noise == NZ_MODEL) {
        const float v = fmaf(fmaf(nv1, f, nv0), f, nv2);
        t = fmaf(MHF_HALF_LN2, lg2_approx(v), MHF_HALF_LN_2PI) + 0.5f * r * r * rcp_approx(v);
        t = v > 0.0f ? t : INFINITY;
    } else {
        t = poisson_term_f(f, y);
    }
    return wt == 0.0f ? 0.0f : t;
}

// In place: v <- inclusive prefix sums of v over the group's grid (point order
// i = (32 g + lane) J + jj); returns the group total.  The warp totals pass
// through slot (double-buffered by g.spar), summed in warp order.
template <int J, int G>
__device__ __forceinline__ float mhf_group_scan(GroupCtx<G> &g, float *scan_slots, int &spar,
                                                float (&v)[J])
{
    float run = 0.0f;
#pragma unroll
    for (int jj = 0; jj < J; ++jj) {
        run += v[jj];
        v[jj] = run;
    }
    float s = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_up_sync(FULL_MASK, s, o);
        if (g.lane >= o) s += t;
    }
    float excl = __shfl_up_sync(FULL_MASK, s, 1);
    if (g.lane == 0) excl = 0.0f;
    const float wtot = __shfl_sync(FULL_MASK, s, 31);
    float pre = 0.0f, tot = wtot;
    if constexpr (G > 1) {
        float *slot = scan_slots + spar * MH_MAX_GROUPS;
        if (g.lane == 0) slot[g.gw] = wtot;
        named_barrier(1 + g.grp, 32 * G);
        tot = 0.0f;
#pragma unroll
        for (int w = 0; w < G; ++w) {
            const float t = slot[w];
            if (w < g.gw) pre += t;
            tot += t;
        }
        spar ^= 1;
    }
    const float add = excl + pre;
#pragma unroll
    for (int jj = 0; jj < J; ++jj) v[jj] += add;
    return tot;
}

// group sum of a Kahan-compensated per-lane sum of the energy terms
template <int J, int G>
__device__ __forceinline__ float mhf_group_energy(GroupCtx<G> &g, const float (&e)[J])
{
    float s = 0.0f, c = 0.0f;
#pragma unroll
    for (int jj = 0; jj < J; ++jj) {
        const float yk = e[jj] - c;
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

// Register budget (resident blocks per SM) from a sweep on B300 with the App. E
// spectrum: 128 registers for J = 8 in 128-thread blocks, 64 for J = 4.
template <int J, int G>
struct MhfBounds {
    static constexpr int NT = MhThreads<G>::NT;
    static constexpr int MINB = (NT == 128) ? (J <= 4 ? 8 : 4) : (NT == 256) ? (J <= 4 ? 4 : 2) : 2;
};

template <int FAM, int J, int G>
__global__ void __launch_bounds__(MhThreads<G>::NT, (MhfBounds<J, G>::MINB))
    k_mh_full(JobDev *__restrict__ jobs, const int *__restrict__ slots, int nslots)
{
    constexpr int NT = MhThreads<G>::NT;
    __shared__ __align__(16) float red_sh[MH_MAX_GROUPS][2][MH_MAX_GROUPS];
    __shared__ float scan_sh[MH_MAX_GROUPS][2][MH_MAX_GROUPS];
    __shared__ int work_sh[MH_MAX_GROUPS][2];
    __shared__ WarpComp comp_sh[NT / 32];
    __shared__ PropTable prop_sh[NT / 32 / G][2];
    GroupCtx<G> g;
    g.lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    g.grp = warp / G;
    g.gw = warp - g.grp * G;
    g.par = 0;
    int spar = 0;
    constexpr int ngroups = (NT / 32) / G;
    if (g.grp >= ngroups) return;
    g.red = &red_sh[g.grp][0][0];
    float *scan_slots = &scan_sh[g.grp][0][0];
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
        const int model = jb.noise;
        const bool shir = jb.bg_kind == BGK_SHIRLEY;
        const float nv0 = jb.nv0, nv1 = jb.nv1, nv2 = jb.nv2;
        const float beta = (float)jb.beta;
        const uint32_t stage = (uint32_t)(jb.stage + 1), tag = jb.tag;
        const unsigned long long seed = jb.seed;
        const int i0 = (g.gw * 32 + lane) * J;

        for (int j = lane; j < d; j += 32) {
            const float u = jb.ths[(size_t)j * S + m];
            cs.th[j] = u;
            cs.nat[j] = natural_f(jb.pri[j], u);
            cs.acc[j] = 0u;
        }
        __syncwarp();

        // ---- grid points, peak sum, Shirley background, energy terms
        float x[J], y[J], w[J], om[J], f[J], C[J], e[J], S0[J], S1[J], N0[J], N1[J], fn[J], en[J],
            Cn[J];
#pragma unroll
        for (int jj = 0; jj < J; ++jj) {
            x[jj] = __ldg(jb.xc + i0 + jj);
            y[jj] = __ldg(jb.y + i0 + jj);
            w[jj] = __ldg(jb.wt + i0 + jj);
            om[jj] = shir ? __ldg(jb.ts + i0 + jj) : 0.0f;
            f[jj] = 0.0f;
        }
        for (int k = 0; k < K; ++k) {
            const int j0 = k * P;
            const float A = cs.nat[j0], mu = cs.nat[j0 + 1], wd = cs.nat[j0 + 2];
            const float eta = (FAM == FAM_PV) ? cs.nat[j0 + 3] : 0.0f;
            const float sc = sc2_of<FAM>(wd, wprec);
#pragma unroll
            for (int jj = 0; jj < J; ++jj) {
                float a0, a1 = 0.0f;
                shape<FAM>(x[jj], mu, sc, a0, a1);
                f[jj] = fmaf(A, unit_of<FAM>(a0, a1, eta), f[jj]);
            }
        }
        float ba = 0.0f, bb = 0.0f, CN = 0.0f, iCN = 0.0f;
        if (shir) {
            ba = cs.nat[K * P];
            bb = cs.nat[K * P + 1];
#pragma unroll
            for (int jj = 0; jj < J; ++jj) C[jj] = om[jj] * f[jj];
            CN = mhf_group_scan<J, G>(g, scan_slots, spar, C);
            iCN = CN > 0.0f ? 1.0f / CN : 0.0f;
#pragma unroll
            for (int jj = 0; jj < J; ++jj) f[jj] += fmaf(bb - ba, C[jj] * iCN, ba);
        } else {
#pragma unroll
            for (int jj = 0; jj < J; ++jj) C[jj] = 0.0f;
        }
#pragma unroll
        for (int jj = 0; jj < J; ++jj) e[jj] = mhf_eterm(model, f[jj], y[jj], w[jj], nv0, nv1, nv2);

        unsigned n_eval = 0, n_shape = 0;
        for (int sw = 0; sw < n; ++sw) {
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
                }
            group_sync(g);

            // ---- peak blocks
            for (int k = 0; k < K; ++k) {
                const int j0 = k * P;
                float A = cs.nat[j0], mu = cs.nat[j0 + 1], wd = cs.nat[j0 + 2];
                float eta = (FAM == FAM_PV) ? cs.nat[j0 + 3] : 0.0f;
                float sc = sc2_of<FAM>(wd, wprec);
#pragma unroll
                for (int jj = 0; jj < J; ++jj) {
                    float l = 0.0f;
                    shape<FAM>(x[jj], mu, sc, S0[jj], l);
                    if (FAM == FAM_PV) S1[jj] = fmaf(eta, S0[jj], l);
                }
#pragma unroll
                for (int c = 0; c < P; ++c) {
                    const int j = j0 + c;
                    const float2 q2 = tb.tv[j];
                    const float tj = q2.x;
                    if (tj == INFINITY) continue;
                    const float v = q2.y;
                    ++n_eval;
                    // D: the change of the peak at every point (kept in fn)
                    if (c == 0) {
                        const float dA = v - A;
#pragma unroll
                        for (int jj = 0; jj < J; ++jj) fn[jj] = dA * (FAM == FAM_PV ? S1[jj] : S0[jj]);
                    } else if (c == 3) {
                        const float dd = A * (v - eta);
#pragma unroll
                        for (int jj = 0; jj < J; ++jj) fn[jj] = dd * S0[jj];
                    } else {
                        ++n_shape;
                        const float mu2 = (c == 1) ? v : mu;
                        const float sc2 = (c == 2) ? sc2_of<FAM>(v, wprec) : sc;
#pragma unroll
                        for (int jj = 0; jj < J; ++jj) {
                            float l = 0.0f;
                            shape<FAM>(x[jj], mu2, sc2, N0[jj], l);
                            if (FAM == FAM_PV) N1[jj] = fmaf(eta, N0[jj], l);
                            fn[jj] = A * (FAM == FAM_PV ? N1[jj] - S1[jj] : N0[jj] - S0[jj]);
                        }
                    }
                    float CNn = CN, iCNn = iCN;
                    if (shir) {
#pragma unroll
                        for (int jj = 0; jj < J; ++jj) Cn[jj] = om[jj] * fn[jj];
                        CNn = CN + mhf_group_scan<J, G>(g, scan_slots, spar, Cn);
                        iCNn = CNn > 0.0f ? 1.0f / CNn : 0.0f;
#pragma unroll
                        for (int jj = 0; jj < J; ++jj) {
                            Cn[jj] += C[jj];
                            const float dB = (bb - ba) * (Cn[jj] * iCNn - C[jj] * iCN);
                            fn[jj] = f[jj] + fn[jj] + dB;
                        }
                    } else {
#pragma unroll
                        for (int jj = 0; jj < J; ++jj) fn[jj] += f[jj];
                    }
                    float p0 = 0.0f, p1 = 0.0f;
#pragma unroll
                    for (int jj = 0; jj < J; ++jj) {
                        en[jj] = mhf_eterm(model, fn[jj], y[jj], w[jj], nv0, nv1, nv2);
                        if (jj & 1)
                            p1 += en[jj] - e[jj];
                        else
                            p0 += en[jj] - e[jj];
                    }
                    const float dE = group_sum(g, p0 + p1);
                    if (tj < -beta * dE) {
#pragma unroll
                        for (int jj = 0; jj < J; ++jj) {
                            f[jj] = fn[jj];
                            e[jj] = en[jj];
                            if (shir) C[jj] = Cn[jj];
                        }
                        CN = CNn;
                        iCN = iCNn;
                        if (c == 0) {
                            A = v;
                        } else if (c == 3) {
                            const float de = v - eta;
#pragma unroll
                            for (int jj = 0; jj < J; ++jj) S1[jj] = fmaf(de, S0[jj], S1[jj]);
                            eta = v;
                        } else {
#pragma unroll
                            for (int jj = 0; jj < J; ++jj) {
                                if (FAM == FAM_PV) S1[jj] = N1[jj];
                                S0[jj] = N0[jj];
                            }
                            if (c == 1) {
                                mu = v;
                            } else {
                                wd = v;
                                sc = sc2_of<FAM>(v, wprec);
                            }
                        }
                        if (lane == 0) {
                            cs.th[j] = tb.un[j];
                            cs.nat[j] = v;
                            cs.acc[j] += 1u;
                        }
                        __syncwarp();
                    }
                }
            }
            // ---- Shirley end points: B = a + (b - a) C / C_N at fixed C
            for (int q = 0; q < nbg; ++q) {
                const int j = K * P + q;
                const float2 q2 = tb.tv[j];
                const float tj = q2.x;
                if (tj == INFINITY) continue;
                const float v = q2.y;
                ++n_eval;
                const float da = q == 0 ? v - ba : 0.0f, db = q == 1 ? v - bb : 0.0f;
                float p0 = 0.0f, p1 = 0.0f;
#pragma unroll
                for (int jj = 0; jj < J; ++jj) {
                    fn[jj] = f[jj] + fmaf(db - da, C[jj] * iCN, da);
                    en[jj] = mhf_eterm(model, fn[jj], y[jj], w[jj], nv0, nv1, nv2);
                    if (jj & 1)
                        p1 += en[jj] - e[jj];
                    else
                        p0 += en[jj] - e[jj];
                }
                const float dE = group_sum(g, p0 + p1);
                if (tj < -beta * dE) {
#pragma unroll
                    for (int jj = 0; jj < J; ++jj) {
                        f[jj] = fn[jj];
                        e[jj] = en[jj];
                    }
                    if (q == 0)
                        ba = v;
                    else
                        bb = v;
                    if (lane == 0) {
                        cs.th[j] = tb.un[j];
                        cs.nat[j] = v;
                        cs.acc[j] += 1u;
                    }
                    __syncwarp();
                }
            }
            if (wf) {
                const float E = mhf_group_energy<J, G>(g, e);
                const size_t o = (size_t)m * n + sw;
                if (g.gw == 0) {
                    for (int j = lane; j < d; j += 32) jb.th[(size_t)j * T + o] = cs.th[j];
                    if (lane == 0) jb.E[o] = E;
                }
            }
        }
        if (!wf) {
            const float E = mhf_group_energy<J, G>(g, e);
            if (g.gw == 0) {
                for (int j = lane; j < d; j += 32) jb.th[(size_t)j * T + m] = cs.th[j];
                if (lane == 0) jb.E[m] = E;
            }
        }
        if (g.gw == 0) {
            for (int j = lane; j < d; j += 32)
                if (jb.pri[j].kind != PR_FIXED) {
                    atomicAdd(&jobs[slot].acc[j], (unsigned long long)cs.acc[j]);
                    atomicAdd(&jobs[slot].prop[j], (unsigned long long)n);
                }
            if (lane == 0) {
                const unsigned long long npts = (unsigned long long)jb.n;
                atomicAdd(&jobs[slot].point_evals, (unsigned long long)n_eval * npts);
                atomicAdd(&jobs[slot].sfu_ops,
                          (unsigned long long)n_shape * npts * (FAM == FAM_PV ? 2ull : 1ull));
                if (model == NZ_MODEL) atomicAdd(&jobs[slot].var_ops, (unsigned long long)n_eval * npts * 2ull);
            }
        }
        __syncwarp();
    }
}

// instantiation table of one family: J in {4, 8}, G in {1, 2, 4, 8, 16}
template <int FAM, int G>
static mh_fn mhf_pick_j(int J)
{
    switch (J) {
    case 4: return k_mh_full<FAM, 4, G>;
    case 8: return k_mh_full<FAM, 8, G>;
    default: return nullptr;
    }
}

template <int FAM>
static mh_fn mhf_pick_family(int J, int G)
{
    switch (G) {
    case 1: return mhf_pick_j<FAM, 1>(J);
    case 2: return mhf_pick_j<FAM, 2>(J);
    case 4: return mhf_pick_j<FAM, 4>(J);
    case 8: return mhf_pick_j<FAM, 8>(J);
    case 16: return mhf_pick_j<FAM, 16>(J);
    default: return nullptr;
    }
}

}  // namespace smc
