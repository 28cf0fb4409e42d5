// k_mh_phase.cuh -- fused FP32 Metropolis rejuvenation (Sec. II B 4) for the
// powder-diffraction phase model of App. D: phase k contributes
//   A_k sum_j I_kj [(1 - r_k) G(x; m_kj, S_k(x)) + r_k L(x; m_kj, W_k(x))],
//   m_kj = ref_kj + d2theta_k,  S = a sqrt(u T^2 - v T + w),
//   W = a (s / cos(x/2) + t T),  T = tan(x/2),  a = alpha_k right of m_kj,
// G = 2^(-4 (dx/S)^2), L = 1 / (1 + 4 (dx/W)^2), over the phase's reference
// reflections, plus the background a_bg PV(x; 0, s_bg, s_bg, r_bg) + b; any
// noise model (known sigma, model variance, Poisson).
//
// Scheduling and the proposal table are those of k_mh / k_mh_full.  A lane owns
// J consecutive grid points and keeps per point y, w, the model value f, the
// energy term e, the current phase's unit profile U (A = 1) and the
// background's unit PV; the centred angle, tan(x/2) and 1/cos(x/2) are re-read
// (L1-resident) whenever a profile is rebuilt.  The profile is (1 - r) Gs + r Ls
// with Gs, Ls the intensity-weighted sums of the Gaussian and Lorentzian parts
// over the phase's reflections.  A proposal of the phase's amplitude changes f
// by dA U; any other phase component forms U' and changes f by A (U' - U).
// When the launch gives dynamic shared memory for the two parts of K phases
// per group, the parts are kept there across sweeps (rewritten when a shape
// proposal that changed them is accepted): a phase's block starts without a
// rebuild, r proposals remix the cached parts, u/v/w proposals rebuild Gs only
// (one EX2 per reflection and point), s/t proposals Ls only (one RCP), d2theta
// and alpha both; without that memory every shape proposal rebuilds both.
// Every proposal recomputes the energy term at every point; dE is one group
// reduction.  Phases are not exchangeable and are never reordered.
//
// Grids longer than one block's tile (32 G J points) run with CL = true: a
// chain spans a thread-block cluster of C CTAs of G = 8 warps (C = 2..16, the
// tile's warps per chain are 8 C), CTA r owning points [r, r + 1) x 256 J.  Every
// CTA draws the same proposals from the same Philox counters; per proposal each
// warp pushes its partial dE into every CTA's shared memory (distributed shared
// memory), one cluster barrier follows, and every CTA sums the 8 C partials in
// the same order, so all CTAs take the same decisions.  The first CTA claims the
// chains and alone writes the chain's results.
#pragma once
#include "k_mh_full.cuh"

namespace smc {

// The two parts of one phase's unit profile (A = 1) at the lane's J points,
// from the phase's natural components (d2theta, alpha, u, v, w, s, t);
// iam1 = 1/alpha - 1:  Gs = sum_j I_j G_j and Ls = sum_j I_j L_j, each 0 where
// its width is not positive, so that the profile is (1 - r) Gs + r Ls.
// MODE bit 1: Gs, bit 2: Ls (the other output is left alone).
// Per point: K1 = -4 / S^2 (S^2 = u T^2 - v T + w), K2 = 4 / W^2; per
// reflection (R = centred position, I, log2 I) and point: dx = x - (R.x +
// d2theta), q = dx scaled by 1/alpha right of the reflection, I G =
// 2^(K1 q^2 + log2 I) (one EX2), L = 1 / (1 + K2 q^2) (one RCP), with six ALU
// operations for one part and eight for both.  The reflections are read once
// per lane (a uniform address), outside the loop over the lane's points.
template <int J, int MODE>
__device__ __forceinline__ void mhp_sums(float (&Gs)[J], float (&Ls)[J], const float *__restrict__ gx,
                                         const float *__restrict__ gt, const float *__restrict__ gs,
                                         float shift, float iam1, float u, float v, float w, float s, float t,
                                         const float4 *__restrict__ rtab, int j0, int j1)
{
    constexpr bool DG = (MODE & 1) != 0, DL = (MODE & 2) != 0;
    float xs[J], K1[J], K2[J], Ug[J], Ul[J];
#pragma unroll
    for (int jj = 0; jj < J; ++jj) {
        const float tn = __ldg(gt + jj);
        // clamped so that q = 0 never meets an infinite factor
        if (DG) {
            const float rad = fmaf(u * tn, tn, fmaf(-v, tn, w));
            K1[jj] = rad > 0.0f ? fmaxf(-4.0f * rcp_approx(rad), -3.0e38f) : 0.0f;
        }
        if (DL) {
            const float W0 = fmaf(s, __ldg(gs + jj), t * tn);
            K2[jj] = W0 > 0.0f ? fminf(4.0f * rcp_approx(W0 * W0), 3.0e38f) : 0.0f;
        }
        xs[jj] = __ldg(gx + jj) - shift;
        Ug[jj] = 0.0f;
        Ul[jj] = 0.0f;
    }
    for (int j = j0; j < j1; ++j) {
        const float4 R = __ldg(rtab + j);
#pragma unroll
        for (int jj = 0; jj < J; ++jj) {
            const float dx = xs[jj] - R.x;
            const float q = fmaf(fmaxf(dx, 0.0f), iam1, dx);
            const float q2 = q * q;
            if (DG) Ug[jj] += ex2_approx(fmaf(q2, K1[jj], R.z));
            if (DL) Ul[jj] = fmaf(R.y, rcp_approx(fmaf(q2, K2[jj], 1.0f)), Ul[jj]);
        }
    }
#pragma unroll
    for (int jj = 0; jj < J; ++jj) {
        if (DG) Gs[jj] = K1[jj] < 0.0f ? Ug[jj] : 0.0f;
        if (DL) Ls[jj] = K2[jj] > 0.0f ? Ul[jj] : 0.0f;
    }
}

// unit background PV(x; 0, s_bg, s_bg, r_bg) at the absolute angle x
__device__ __forceinline__ float mhp_bg_unit(float xabs, float sbg, float rbg)
{
    if (!(sbg > 0.0f)) return 0.0f;
    const float z = xabs * rcp_approx(sbg);
    const float g = ex2_approx(-4.0f * z * z), l = rcp_approx(fmaf(4.0f * z, z, 1.0f));
    return fmaf(rbg, l - g, g);
}

constexpr int MHP_MAX_CL = 16;  // CTAs per cluster at most (non-portable above 8)
constexpr int MHP_CL_WARPS = 8;

__device__ __forceinline__ unsigned mhp_cl_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned mhp_cl_size()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// every thread of every CTA of the cluster; orders the shared::cluster stores
// issued before it with the reads after it
__device__ __forceinline__ void mhp_cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// store v at the address of `local` in the shared memory of CTA `rank`
__device__ __forceinline__ void mhp_cl_store(const void *local, unsigned rank, float v)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(local);
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
}
__device__ __forceinline__ void mhp_cl_store_i(const void *local, unsigned rank, int v)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(local);
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(ra), "r"(v) : "memory");
}

// Cluster-wide sum of one value per warp (v: the warp's total, equal in its
// lanes); every thread of every CTA returns the same sum.  Two levels: the
// CTA adds its warps' values in warp order (ctab: [2][G] in this CTA's shared
// memory, one CTA barrier), then its first warp pushes the CTA total into
// every CTA of the cluster (xch: [2][.] in each CTA's shared memory, one
// cluster barrier) and each CTA adds the C totals in CTA order, so every CTA
// takes the same decision from the same bits.
template <int G>
__device__ __forceinline__ float mhp_cl_sum(float (*xch)[MHP_MAX_CL * G], float (*ctab)[G], int &cpar,
                                            unsigned crank, unsigned csize, int gw, int lane, float v)
{
    if (lane == 0) ctab[cpar][gw] = v;
    __syncthreads();
    float t = 0.0f;
#pragma unroll
    for (int w = 0; w < G; w += 4) {
        const float4 q = *reinterpret_cast<const float4 *>(&ctab[cpar][w]);
        t += q.x;
        t += q.y;
        t += q.z;
        t += q.w;
    }
    if (gw == 0 && (unsigned)lane < csize) mhp_cl_store(&xch[cpar][crank], (unsigned)lane, t);
    __syncwarp();
    mhp_cl_sync();
    float s = 0.0f;
    for (unsigned r = 0; r < csize; ++r) s += xch[cpar][r];
    cpar ^= 1;
    return s;
}

// Per-phase profile parts of the lane's J points, kept in dynamic shared
// memory across sweeps ([K][2][32 G J] per group: Gs, Ls; the lane's J points
// contiguous)
template <int J>
__device__ __forceinline__ void mhp_cache_store(float *uc, const float (&U)[J])
{
#pragma unroll
    for (int jj = 0; jj < J; jj += 4)
        *reinterpret_cast<float4 *>(uc + jj) = make_float4(U[jj], U[jj + 1], U[jj + 2], U[jj + 3]);
}
template <int J>
__device__ __forceinline__ void mhp_cache_load(const float *uc, float (&U)[J])
{
#pragma unroll
    for (int jj = 0; jj < J; jj += 4) {
        const float4 q = *reinterpret_cast<const float4 *>(uc + jj);
        U[jj] = q.x;
        U[jj + 1] = q.y;
        U[jj + 2] = q.z;
        U[jj + 3] = q.w;
    }
}
__device__ __forceinline__ unsigned mhp_dyn_smem_bytes()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

// A proposal's dE: the group sum, then (clusters) the exchange between CTAs
template <int G, bool CL>
__device__ __forceinline__ float mhp_dE(GroupCtx<G> &g, float (*xch)[CL ? MHP_MAX_CL * G : 4],
                                        float (*ctab)[G], int &cpar, unsigned crank, unsigned csize,
                                        float v)
{
    if constexpr (CL)
        return mhp_cl_sum<G>(xch, ctab, cpar, crank, csize, g.gw, g.lane, warp_sum(v));
    else
        return group_sum(g, v);
}

// The chain's energy: the compensated group sum, then (clusters) the CTAs'
// totals added in CTA order
template <int J, int G, bool CL>
__device__ __forceinline__ float mhp_chain_energy(GroupCtx<G> &g, const float (&e)[J],
                                                  float (*xch)[CL ? MHP_MAX_CL * G : 4],
                                                  float (*ctab)[G], int &cpar, unsigned crank,
                                                  unsigned csize)
{
    const float E = mhf_group_energy<J, G>(g, e);
    if constexpr (CL)
        return mhp_cl_sum<G>(xch, ctab, cpar, crank, csize, g.gw, g.lane, g.gw == 0 ? E : 0.0f);
    else
        return E;
}

// Register budget (resident blocks per SM): the phase kernel holds about nine
// values per point plus a phase's nine components, so J = 4 gets up to 80
// registers and J = 8 up to 128 (no spills with the groups of four or more
// warps that grids of about a thousand points take).
template <int J, int G, bool CL>
struct MhpBounds {
    static constexpr int NT = CL ? 32 * G : MhThreads<G>::NT;
    static constexpr int MINB = (NT == 128) ? (J <= 4 ? 6 : 4) : (NT == 256) ? (J <= 4 ? 3 : 2) : 1;
};

template <int J, int G, bool CL>
__global__ void __launch_bounds__((MhpBounds<J, G, CL>::NT), (MhpBounds<J, G, CL>::MINB))
    k_mh_phase(JobDev *__restrict__ jobs, const int *__restrict__ slots, int nslots)
{
    static_assert(!CL || G == MHP_CL_WARPS, "cluster chains use 8-warp CTAs");
    constexpr int NT = MhpBounds<J, G, CL>::NT;
    constexpr int P = 9;
    __shared__ __align__(16) float red_sh[MH_MAX_GROUPS][2][MH_MAX_GROUPS];
    __shared__ int work_sh[MH_MAX_GROUPS][2];
    __shared__ WarpComp comp_sh[NT / 32];
    __shared__ PropTable prop_sh[NT / 32 / G][2];
    __shared__ __align__(16) float xch_sh[CL ? 2 : 1][CL ? MHP_MAX_CL * G : 4];
    __shared__ __align__(16) float ctab_sh[2][G < 4 ? 4 : G];  // a CTA's warp totals (clusters)
    __shared__ int claim_sh[2][2];
    unsigned crank = 0, csize = 1;
    int cpar = 0;
    if constexpr (CL) {
        crank = mhp_cl_rank();
        csize = mhp_cl_size();
        // every CTA of the cluster runs before any shared::cluster access
        mhp_cl_sync();
    }
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
    // profile-part cache: as many phases as the launch's dynamic shared memory holds
    extern __shared__ __align__(16) float ucache_sh[];
    constexpr int GP = 32 * G * J;  // points of a group (of a CTA with clusters)
    const int kcache = (int)(mhp_dyn_smem_bytes() / (8u * (unsigned)(ngroups * GP)));
    float *ucg = ucache_sh + (size_t)g.grp * kcache * 2 * GP + (g.gw * 32 + lane) * J;

    int li = 0;
    for (;;) {
        // ---- claim the next chain (dynamic scheduling over the bucket's jobs)
        int slot = -1, m = 0;
        if (g.gw == 0 && lane == 0 && crank == 0) {
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
            if constexpr (CL) {
                for (unsigned r = 0; r < csize; ++r) {
                    mhp_cl_store_i(&claim_sh[cpar][0], r, slot);
                    mhp_cl_store_i(&claim_sh[cpar][1], r, m);
                }
            } else if constexpr (G > 1) {
                work_sh[g.grp][0] = slot;
                work_sh[g.grp][1] = m;
            }
        }
        if constexpr (CL) {
            __syncwarp();
            mhp_cl_sync();
            slot = claim_sh[cpar][0];
            m = claim_sh[cpar][1];
            cpar ^= 1;
        } else if constexpr (G == 1) {
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
        const int wf = jb.waste_free, noise = jb.noise;
        const float nv0 = jb.nv0, nv1 = jb.nv1, nv2 = jb.nv2;
        const float beta = (float)jb.beta, xref = (float)jb.x_ref;
        const uint32_t stage = (uint32_t)(jb.stage + 1), tag = jb.tag;
        const unsigned long long seed = jb.seed;
        const float4 *rtab = jb.rtab;
        const int *roff = jb.roff;
        const int i0 = (((int)crank * G + g.gw) * 32 + lane) * J;

        for (int j = lane; j < d; j += 32) {
            const float u = jb.ths[(size_t)j * S + m];
            cs.th[j] = u;
            cs.nat[j] = natural_f(jb.pri[j], u);
            cs.acc[j] = 0u;
        }
        __syncwarp();

        const float *gx = jb.xc + i0, *gt = jb.ts + i0, *gs = jb.sec2 + i0;
        float y[J], w[J], f[J], e[J], U[J], Gn[J], Ln[J], en[J], Bv[J];
#pragma unroll
        for (int jj = 0; jj < J; ++jj) {
            y[jj] = __ldg(jb.y + i0 + jj);
            w[jj] = __ldg(jb.wt + i0 + jj);
            f[jj] = 0.0f;
        }
        const bool cached = K <= kcache;
        for (int k = 0; k < K; ++k) {
            const float *q = cs.nat + P * k;
            mhp_sums<J, 3>(Gn, Ln, gx, gt, gs, q[1], 1.0f / q[2] - 1.0f, q[4], q[5], q[6], q[7], q[8], rtab,
                           roff[k], roff[k + 1]);
            if (cached) {
                mhp_cache_store<J>(ucg + (2 * k) * GP, Gn);
                mhp_cache_store<J>(ucg + (2 * k + 1) * GP, Ln);
            }
#pragma unroll
            for (int jj = 0; jj < J; ++jj) f[jj] = fmaf(q[0], fmaf(q[3], Ln[jj] - Gn[jj], Gn[jj]), f[jj]);
        }
        float ba = 0.0f, bs = 0.0f, br = 0.0f, bb = 0.0f;
        if (nbg > 0) {
            ba = cs.nat[P * K];
            bs = cs.nat[P * K + 1];
            br = cs.nat[P * K + 2];
            bb = cs.nat[P * K + 3];
        }
#pragma unroll
        for (int jj = 0; jj < J; ++jj) {
            Bv[jj] = nbg > 0 ? mhp_bg_unit(__ldg(gx + jj) + xref, bs, br) : 0.0f;
            f[jj] += fmaf(ba, Bv[jj], bb);
            e[jj] = mhf_eterm(noise, f[jj], y[jj], w[jj], nv0, nv1, nv2);
        }

        unsigned n_eval = 0;
        // reflections whose Gaussian (EX2) / Lorentzian (RCP) parts the shape proposals evaluated
        unsigned long long n_ex2_ref = 0, n_rcp_ref = 0;
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

            // ---- phase blocks; the current components are read from cs.nat
            for (int k = 0; k < K; ++k) {
                const int jc0 = P * k, j0 = roff[k], j1 = roff[k + 1];
                const float *q = cs.nat + jc0;
                float *ucG = ucg + (2 * k) * GP, *ucL = ucg + (2 * k + 1) * GP;
                if (cached) {
                    mhp_cache_load<J>(ucG, Gn);
                    mhp_cache_load<J>(ucL, Ln);
                } else {
                    mhp_sums<J, 3>(Gn, Ln, gx, gt, gs, q[1], 1.0f / q[2] - 1.0f, q[4], q[5], q[6], q[7], q[8], rtab,
                                   j0, j1);
                }
#pragma unroll
                for (int jj = 0; jj < J; ++jj) U[jj] = fmaf(q[3], Ln[jj] - Gn[jj], Gn[jj]);
#pragma unroll 1
                for (int c = 0; c < P; ++c) {
                    const int j = jc0 + c;
                    const float2 q2 = tb.tv[j];
                    const float tj = q2.x;
                    if (tj == INFINITY) continue;
                    const float v = q2.y;
                    const float A = q[0];
                    ++n_eval;
                    float p0 = 0.0f, p1 = 0.0f;
                    // parts a shape proposal rebuilds: r none (the cached parts
                    // remix), u, v, w the Gaussian part, s, t the Lorentzian
                    // part, d2theta and alpha both (both always without a cache)
                    const int mode = !cached ? 3 : c == 3 ? 0 : c >= 7 ? 2 : c >= 4 ? 1 : 3;
                    if (c == 0) {
                        const float dA = v - A;
#pragma unroll
                        for (int jj = 0; jj < J; ++jj) {
                            en[jj] = mhf_eterm(noise, fmaf(dA, U[jj], f[jj]), y[jj], w[jj], nv0, nv1, nv2);
                            if (jj & 1)
                                p1 += en[jj] - e[jj];
                            else
                                p0 += en[jj] - e[jj];
                        }
                    } else {
                        // the phase's components with component c replaced by v
                        const float sh = c == 1 ? v : q[1], al = c == 2 ? v : q[2], r = c == 3 ? v : q[3];
                        const float cu = c == 4 ? v : q[4], cv = c == 5 ? v : q[5], cw = c == 6 ? v : q[6];
                        const float cs_ = c == 7 ? v : q[7], ct = c == 8 ? v : q[8];
                        const float iam1 = 1.0f / al - 1.0f;
                        if (mode == 0) {
                            mhp_cache_load<J>(ucG, Gn);
                            mhp_cache_load<J>(ucL, Ln);
                        } else if (mode == 1) {
                            mhp_sums<J, 1>(Gn, Ln, gx, gt, gs, sh, iam1, cu, cv, cw, cs_, ct, rtab, j0, j1);
                            mhp_cache_load<J>(ucL, Ln);
                            n_ex2_ref += (unsigned long long)(j1 - j0);
                        } else if (mode == 2) {
                            mhp_sums<J, 2>(Gn, Ln, gx, gt, gs, sh, iam1, cu, cv, cw, cs_, ct, rtab, j0, j1);
                            mhp_cache_load<J>(ucG, Gn);
                            n_rcp_ref += (unsigned long long)(j1 - j0);
                        } else {
                            mhp_sums<J, 3>(Gn, Ln, gx, gt, gs, sh, iam1, cu, cv, cw, cs_, ct, rtab, j0, j1);
                            n_ex2_ref += (unsigned long long)(j1 - j0);
                            n_rcp_ref += (unsigned long long)(j1 - j0);
                        }
#pragma unroll
                        for (int jj = 0; jj < J; ++jj) {
                            const float Un = fmaf(r, Ln[jj] - Gn[jj], Gn[jj]);
                            en[jj] = mhf_eterm(noise, fmaf(A, Un - U[jj], f[jj]), y[jj], w[jj], nv0, nv1, nv2);
                            if (jj & 1)
                                p1 += en[jj] - e[jj];
                            else
                                p0 += en[jj] - e[jj];
                        }
                    }
                    const float dE = mhp_dE<G, CL>(g, xch_sh, (float(*)[G])ctab_sh, cpar, crank, csize, p0 + p1);
                    if (tj < -beta * dE) {
                        if (c == 0) {
                            const float dA = v - A;
#pragma unroll
                            for (int jj = 0; jj < J; ++jj) f[jj] = fmaf(dA, U[jj], f[jj]);
                        } else {
                            const float r = c == 3 ? v : q[3];
#pragma unroll
                            for (int jj = 0; jj < J; ++jj) {
                                const float Un = fmaf(r, Ln[jj] - Gn[jj], Gn[jj]);
                                f[jj] = fmaf(A, Un - U[jj], f[jj]);
                                U[jj] = Un;
                            }
                            if (cached && (mode & 1)) mhp_cache_store<J>(ucG, Gn);
                            if (cached && (mode & 2)) mhp_cache_store<J>(ucL, Ln);
                        }
#pragma unroll
                        for (int jj = 0; jj < J; ++jj) e[jj] = en[jj];
                        __syncwarp();
                        if (lane == 0) {
                            cs.th[j] = tb.un[j];
                            cs.nat[j] = v;
                            cs.acc[j] += 1u;
                        }
                        __syncwarp();
                    }
                }
            }
            // ---- background (a, s_bg, r_bg, b)
            for (int qb = 0; qb < nbg; ++qb) {
                const int j = P * K + qb;
                const float2 q2 = tb.tv[j];
                const float tj = q2.x;
                if (tj == INFINITY) continue;
                const float v = q2.y;
                ++n_eval;
                float p0 = 0.0f, p1 = 0.0f;
#pragma unroll
                for (int jj = 0; jj < J; ++jj) {
                    float fn;
                    if (qb == 0) {
                        fn = fmaf(v - ba, Bv[jj], f[jj]);
                    } else if (qb == 3) {
                        fn = f[jj] + (v - bb);
                    } else {
                        Gn[jj] = mhp_bg_unit(__ldg(gx + jj) + xref, qb == 1 ? v : bs, qb == 2 ? v : br);
                        fn = fmaf(ba, Gn[jj] - Bv[jj], f[jj]);
                    }
                    en[jj] = mhf_eterm(noise, fn, y[jj], w[jj], nv0, nv1, nv2);
                    if (jj & 1)
                        p1 += en[jj] - e[jj];
                    else
                        p0 += en[jj] - e[jj];
                }
                const float dE = mhp_dE<G, CL>(g, xch_sh, (float(*)[G])ctab_sh, cpar, crank, csize, p0 + p1);
                if (tj < -beta * dE) {
#pragma unroll
                    for (int jj = 0; jj < J; ++jj) {
                        if (qb == 0) {
                            f[jj] = fmaf(v - ba, Bv[jj], f[jj]);
                        } else if (qb == 3) {
                            f[jj] += v - bb;
                        } else {
                            f[jj] = fmaf(ba, Gn[jj] - Bv[jj], f[jj]);
                            Bv[jj] = Gn[jj];
                        }
                        e[jj] = en[jj];
                    }
                    if (qb == 0)
                        ba = v;
                    else if (qb == 1)
                        bs = v;
                    else if (qb == 2)
                        br = v;
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
                const float E = mhp_chain_energy<J, G, CL>(g, e, xch_sh, (float(*)[G])ctab_sh, cpar, crank, csize);
                const size_t o = (size_t)m * n + sw;
                if (g.gw == 0 && crank == 0) {
                    for (int j = lane; j < d; j += 32) jb.th[(size_t)j * T + o] = cs.th[j];
                    if (lane == 0) jb.E[o] = E;
                }
            }
        }
        if (!wf) {
            const float E = mhp_chain_energy<J, G, CL>(g, e, xch_sh, (float(*)[G])ctab_sh, cpar, crank, csize);
            if (g.gw == 0 && crank == 0) {
                for (int j = lane; j < d; j += 32) jb.th[(size_t)j * T + m] = cs.th[j];
                if (lane == 0) jb.E[m] = E;
            }
        }
        if (g.gw == 0 && crank == 0) {
            for (int j = lane; j < d; j += 32)
                if (jb.pri[j].kind != PR_FIXED) {
                    atomicAdd(&jobs[slot].acc[j], (unsigned long long)cs.acc[j]);
                    atomicAdd(&jobs[slot].prop[j], (unsigned long long)n);
                }
            if (lane == 0) {
                const unsigned long long npts = (unsigned long long)jb.n;
                atomicAdd(&jobs[slot].point_evals, (unsigned long long)n_eval * npts);
                // SFU work of the proposals' profile rebuilds: an EX2 per
                // reflection and point of a Gaussian part, an RCP of a
                // Lorentzian part (the per-point reciprocals are not counted)
                atomicAdd(&jobs[slot].sfu_ops, (n_ex2_ref + n_rcp_ref) * npts);
                atomicAdd(&jobs[slot].ex2_part, n_ex2_ref * npts);
                if (noise == NZ_MODEL) atomicAdd(&jobs[slot].var_ops, (unsigned long long)n_eval * npts * 2ull);
            }
        }
        __syncwarp();
    }
    // no CTA leaves while a peer could still address its shared memory
    if constexpr (CL) mhp_cl_sync();
}

template <int G, bool CL>
static mh_fn mhp_pick_j(int J)
{
    switch (J) {
    case 4: return k_mh_phase<4, G, CL>;
    case 8: return k_mh_phase<8, G, CL>;
    default: return nullptr;
    }
}

// G warps per chain: 1..16 in one block; multiples of 8 above (a cluster of
// G / 8 CTAs of 8 warps, at most MHP_MAX_CL)
static mh_fn mhp_pick_tile(int J, int G)
{
    switch (G) {
    case 1: return mhp_pick_j<1, false>(J);
    case 2: return mhp_pick_j<2, false>(J);
    case 4: return mhp_pick_j<4, false>(J);
    case 8: return mhp_pick_j<8, false>(J);
    case 16: return mhp_pick_j<16, false>(J);
    default:
        if (G > 16 && G % MHP_CL_WARPS == 0 && G / MHP_CL_WARPS <= MHP_MAX_CL)
            return mhp_pick_j<MHP_CL_WARPS, true>(J);
        return nullptr;
    }
}

}  // namespace smc
