// engine.cpp -- requests, device memory, the batched stage loop and the
// serving loop behind the C ABI.
#include "engine.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace smc {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? SMC_OK : (e == cudaErrorMemoryAllocation ? SMC_ENOMEM : SMC_ECUDA); }

#define CK(expr)                                  \
    do {                                          \
        cudaError_t _e = (expr);                  \
        if (_e != cudaSuccess) return cuda_status(_e); \
    } while (0)

static size_t al(size_t x) { return (x + 255) & ~size_t(255); }

static int peak_params(int family)
{
    return family == SMC_XRD_PHASE ? 9 : (family == SMC_PSEUDO_VOIGT ? 4 : 3);
}
static int bg_params(int bg, int deg)
{
    switch (bg) {
    case SMC_BG_NONE: return 0;
    case SMC_BG_CONST: return 1;
    case SMC_BG_LINEAR: return 2;
    case SMC_BG_SHIRLEY: return 2;
    case SMC_BG_XRD_PV: return 4;
    default: return deg + 1;
    }
}
int job_dim(int family, int K, int bg, int deg) { return peak_params(family) * K + bg_params(bg, deg); }

// Gaussian peaks given by their precision run the Gaussian kernels with the
// width component read as b (shape scale sqrt(b / (2 ln 2)) instead of
// 1 / (w sqrt(2 ln 2))).
int kernel_family(int family) { return family == SMC_GAUSS_PRECISION ? SMC_GAUSS : family; }

// ---------------------------------------------------------------------------
// Tile of the fused Metropolis kernel: J points per lane, G warps per chain,
// 32 G J >= N.  Chosen to minimise padding, then the number of warps per chain.
// ---------------------------------------------------------------------------
Tile choose_tile(int family, int n)
{
    if (family & MH_COUPLED) {  // coupled-grid kernel: J = 8 or 4, least padding
        // G > 16 (multiples of 8): the phase kernel's cluster-spanning chains
        static const int Gs[] = {1,  2,  4,  8,  16, 24, 32, 40,  48,  56,  64,
                                 72, 80, 88, 96, 104, 112, 120, 128};
        Tile best{0, 0, 0};
        long best_pad = -1;
        for (int J : {8, 4})
            for (int G : Gs) {
                if (!mh_tile_supported(family, J, G) || 32L * G * J < n) continue;
                if (best_pad < 0 || 32L * G * J < best_pad) {
                    best = {J, G, 0};
                    best_pad = 32L * G * J;
                }
                break;
            }
        return best;
    }
    // measured on B300 (XPS-, XRD- and App. C-shaped grids): J = 8 (64
    // registers, 32 warps/SM) while four warps per chain cover the grid,
    // J = 16 (128 registers) beyond; other J only when they pad much less
    static const int Js_small[] = {8, 16, 12, 4, 24, 32};
    static const int Js_large[] = {16, 8, 12, 4, 24, 32};
    const int *Js = n <= 32 * 4 * 8 ? Js_small : Js_large;
    const int nJ = 6;  // unsupported (family, J, G) are skipped below
    Tile best{0, 0, 0};
    double best_cost = -1.0;
    for (int a = 0; a < nJ; ++a)
        for (int G : {1, 2, 4, 8, 16}) {
            const int J = Js[a];
            if (!mh_tile_supported(family, J, G)) continue;
            const long pad = 32L * G * J;
            if (pad < n) continue;
            const double cost = (double)pad * (1.0 + 0.1 * a);  // preferred J first
            if (best_cost < 0.0 || cost < best_cost) {
                best = {J, G, 0};
                best_cost = cost;
            }
            break;  // smallest G for this J
        }
    return best;
}

// role: 0 amp, 1 centre, 2 width, 3 eta, 4 background, 5 App. D phase component
static bool prior_ok(const smc_prior &p, int role)
{
    if (!std::isfinite(p.p1) || (p.kind != SMC_FIXED && !std::isfinite(p.p2))) return false;
    switch (p.kind) {
    case SMC_UNIFORM:
        if (!(p.p1 < p.p2)) return false;
        if (role == 2 && !(p.p1 > 0.0)) return false;
        return true;
    case SMC_LOG_UNIFORM: return role != 1 && p.p1 > 0.0 && p.p1 < p.p2;
    case SMC_NORMAL: return role != 2 && p.p2 > 0.0;
    case SMC_GAMMA: return role != 1 && p.p1 > 0.0 && p.p2 > 0.0;
    case SMC_FIXED: return role != 2 || p.p1 > 0.0;
    default: return false;
    }
}

static smc_prior comp_prior(const Request &r, int K, int j)
{
    if (!r.comp.empty()) return r.comp[j];
    const int p = r.p;
    if (r.family == SMC_XRD_PHASE) return j < p * K ? r.pri.phase[j % p] : r.pri.bg[j - p * K];
    if (j < p * K) {
        switch (j % p) {
        case 0: return r.pri.amp;
        case 1: return r.pri.centre;
        case 2: return r.pri.width;
        default: return r.pri.eta;
        }
    }
    return r.pri.bg[j - p * K];
}

static int comp_role(const Request &r, int K, int j)
{
    if (r.family == SMC_XRD_PHASE) return j < r.p * K ? 5 : 4;
    if (j < r.p * K) return j % r.p;
    return 4;
}

int make_request(Ctx &c, const smc_request &rq, bool on_device, Request *&out)
{
    if (!rq.priors || !rq.opts || !rq.x || !rq.y) return SMC_EINVAL;
    if (rq.noise != SMC_NOISE_KNOWN && rq.noise != SMC_NOISE_MODEL && rq.noise != SMC_NOISE_POISSON)
        return SMC_EINVAL;
    if (rq.noise == SMC_NOISE_KNOWN && !rq.sigma) return SMC_EINVAL;
    if (rq.noise == SMC_NOISE_MODEL)
        for (int q = 0; q < 3; ++q)
            if (!std::isfinite(rq.noise_par[q])) return SMC_EINVAL;
    const smc_options &o = *rq.opts;
    // FP32 Poisson energies need the model inside FP32's range wherever a count
    // is positive: Gaussian-tailed peaks with no background underflow there
    // (an infinite FP32 energy where the FP64 one is finite), so those
    // requests must take the FP64 energies
    if (rq.noise == SMC_NOISE_POISSON && o.energy_fp64 == 0 && rq.bg == SMC_BG_NONE &&
        (rq.family == SMC_GAUSS || rq.family == SMC_GAUSS_PRECISION))
        return SMC_EINVAL;
    if (rq.n < 2 || rq.n > (1 << 24)) return SMC_EINVAL;
    if (rq.family < 0 || rq.family > 4 || rq.bg < 0 || rq.bg > 5) return SMC_EINVAL;
    const bool xrd = rq.family == SMC_XRD_PHASE;
    const bool full = xrd || rq.bg == SMC_BG_SHIRLEY || rq.noise != SMC_NOISE_KNOWN;
    if (xrd && rq.bg != SMC_BG_NONE && rq.bg != SMC_BG_XRD_PV) return SMC_EINVAL;
    if (!xrd && full && rq.bg != SMC_BG_NONE && rq.bg != SMC_BG_SHIRLEY) return SMC_EINVAL;
    if (xrd) {  // reflections of every candidate phase
        if (!rq.ref_pos || !rq.ref_int || !rq.ref_off || rq.n_phase < rq.k_max || rq.ref_off[0] != 0)
            return SMC_EINVAL;
        for (int k = 0; k < rq.n_phase; ++k) {
            const int nr = rq.ref_off[k + 1] - rq.ref_off[k];
            if (nr < 1 || nr > SMC_MAX_REFS) return SMC_EINVAL;
        }
        for (int j = 0; j < rq.ref_off[rq.n_phase]; ++j)
            if (!std::isfinite(rq.ref_pos[j]) || !std::isfinite(rq.ref_int[j]) || rq.ref_int[j] < 0.0)
                return SMC_EINVAL;
    }
    if (rq.bg == SMC_BG_POLY && (rq.bg_degree < 0 || rq.bg_degree >= SMC_MAX_BG)) return SMC_EINVAL;
    if (rq.k_min < 0 || rq.k_min > rq.k_max || rq.k_max > SMC_MAX_K) return SMC_EINVAL;
    if (job_dim(rq.family, rq.k_max, rq.bg, rq.bg_degree) > SMC_MAX_DIM) return SMC_EINVAL;
    if (o.particles < 2 || o.particles > (1 << 24) || o.sweeps < 1 || o.sweeps > 100000) return SMC_EINVAL;
    if (o.energy_fp64 < 0 || o.energy_fp64 > 2) return SMC_EINVAL;
    if (o.step_rule < 0 || o.step_rule > 1) return SMC_EINVAL;
    if (!(o.ess_target > 0.0 && o.ess_target < 1.0) || o.max_stages < 1) return SMC_EINVAL;
    if (o.waste_free) {
        const int64_t S = (o.particles + o.sweeps - 1) / o.sweeps;
        if (S * o.sweeps > (1 << 24) || S < 2) return SMC_EINVAL;
    }
    Request *r = new Request();
    r->k_min = rq.k_min;
    r->k_max = rq.k_max;
    r->family = rq.family;
    r->bg = rq.bg;
    r->bg_degree = rq.bg_degree;
    r->nbg = bg_params(rq.bg, rq.bg_degree);
    r->p = peak_params(rq.family);
    r->n = (int)rq.n;
    r->noise = rq.noise;
    for (int q = 0; q < 3; ++q) r->noise_par[q] = rq.noise == SMC_NOISE_MODEL ? rq.noise_par[q] : 0.0;
    r->full = full;
    if (xrd) {
        const int nref = rq.ref_off[rq.n_phase];
        r->ref_pos.assign(rq.ref_pos, rq.ref_pos + nref);
        r->ref_int.assign(rq.ref_int, rq.ref_int + nref);
        r->ref_off.assign(rq.ref_off, rq.ref_off + rq.n_phase + 1);
    }
    r->opts = o;
    r->pri = *rq.priors;
    r->fp64 = o.energy_fp64 != 0;
    if (rq.priors->n_comp > 0) {
        if (!rq.priors->comp || rq.k_min != rq.k_max ||
            rq.priors->n_comp != job_dim(rq.family, rq.k_min, rq.bg, rq.bg_degree)) {
            delete r;
            return SMC_EINVAL;
        }
        r->comp.assign(rq.priors->comp, rq.priors->comp + rq.priors->n_comp);
    }
    r->pri.comp = nullptr;
    r->pri.n_comp = 0;
    for (int K = r->k_min; K <= r->k_max; ++K) {
        const int d = job_dim(r->family, K, r->bg, r->bg_degree);
        for (int j = 0; j < d; ++j)
            if (!prior_ok(comp_prior(*r, K, j), comp_role(*r, K, j))) {
                delete r;
                return SMC_EINVAL;
            }
    }
    if (!r->fp64) {
        const int kf = kernel_family(r->family) | (full ? MH_COUPLED : 0);
        r->tile = choose_tile(kf, r->n);
        std::lock_guard<std::mutex> tl(c.tmu);
        for (const auto &t : c.tiles)
            if (t[0] == kf && t[1] >= r->n && 32L * t[2] * t[3] >= r->n &&
                mh_tile_supported(kf, (int)t[2], (int)t[3], (int)t[4])) {
                r->tile = {(int)t[2], (int)t[3], (int)t[4]};
                break;
            }
        if (r->tile.J == 0) {
            delete r;
            return SMC_EINVAL;  // grid too long for the FP32 tiles
        }
        r->n_pad = 32 * r->tile.G * r->tile.J;
    } else {
        r->n_pad = r->n;
    }
    const bool known = rq.noise == SMC_NOISE_KNOWN;
    if (on_device) {
        r->dx = rq.x;
        r->dy = rq.y;
        r->ds = known ? rq.sigma : nullptr;
    } else {
        r->hx.assign(rq.x, rq.x + rq.n);
        r->hy.assign(rq.y, rq.y + rq.n);
        if (known) r->hs.assign(rq.sigma, rq.sigma + rq.n);
        for (int i = 0; i < r->n; ++i)
            if (!std::isfinite(r->hx[i]) || !std::isfinite(r->hy[i]) ||
                (known && (!std::isfinite(r->hs[i]) || !(r->hs[i] > 0.0)))) {
                delete r;
                return SMC_EINVAL;
            }
    }
    out = r;
    return SMC_OK;
}

// ---------------------------------------------------------------------------
// Device memory of a request: one arena for the spectrum and results, one per job.
// ---------------------------------------------------------------------------
struct SpecLayout {
    size_t raw, x64, y64, is64, tn64, sc64, xc, wt, y, ts, sec2, rpos64, rint64, rtab, roff, scal, slots, off, pk,
        mean, sd, fpart, fcnt, samples, total;
};

static SpecLayout spec_layout(const Request &r, int64_t T_out)
{
    SpecLayout L{};
    const size_t n = r.n, np = r.n_pad, nK = r.k_max - r.k_min + 1;
    const size_t dmax = std::max(1, job_dim(r.family, r.k_max, r.bg, r.bg_degree));
    size_t o = 0;
    L.raw = o;  o += al(3 * n * 8);
    L.x64 = o;  o += al(n * 8);
    L.y64 = o;  o += al(n * 8);
    L.is64 = o; o += al(n * 8);
    const size_t nx = r.family == SMC_XRD_PHASE ? n : 1;
    L.tn64 = o; o += al(nx * 8);
    L.sc64 = o; o += al(nx * 8);
    L.xc = o;   o += al(np * 4);
    L.wt = o;   o += al(np * 4);
    L.y = o;    o += al(np * 4);
    L.ts = o;   o += al(np * 4);
    const size_t nref = std::max<size_t>(1, r.ref_pos.size());
    L.sec2 = o; o += al(np * 4);
    L.rpos64 = o; o += al(nref * 8);
    L.rint64 = o; o += al(nref * 8);
    L.rtab = o; o += al(nref * 16);
    L.roff = o; o += al(std::max<size_t>(2, r.ref_off.size()) * 4);
    L.scal = o; o += al(sizeof(SpecScal));
    L.slots = o; o += al(nK * 4);
    L.off = o;  o += al(2 * 4);
    L.pk = o;   o += al(nK * 8);
    L.mean = o; o += al(nK * dmax * 8);
    L.sd = o;   o += al(nK * dmax * 8);
    L.fpart = o; o += al(nK * (size_t)finalize_split(T_out) * 2 * dmax * 8);
    L.fcnt = o; o += al(nK * 4);
    L.samples = o;
    if (r.opts.keep_samples) o += al(nK * (size_t)T_out * dmax * 4);
    L.total = o;
    return L;
}

struct JobLayout {
    size_t th, E, ths, Es, w64, rwpart, q, anc, lam, step, stepf, acc, prop, pri, hist, total;
};

static JobLayout job_layout(int d, int64_t T, int64_t S, bool fp64)
{
    JobLayout L{};
    const size_t e = fp64 ? 8 : 4, dd = std::max(d, 1);
    size_t o = 0;
    L.th = o;   o += al(dd * T * e);
    L.E = o;    o += al(T * e);
    L.ths = o;  o += al(dd * S * e);
    L.Es = o;   o += al(S * e);
    L.w64 = o;  o += al(T * 8);
    L.rwpart = o; o += al((size_t)rw_split(T) * (1 + 2 * dd) * 8);
    L.q = o;    o += al(T * 8);
    L.anc = o;  o += al(S * 4);
    L.lam = o;  o += al(dd * 8);
    L.step = o; o += al(dd * 8);
    L.stepf = o; o += al(dd * 4);
    L.acc = o;  o += al(dd * 8);
    L.prop = o; o += al(dd * 8);
    L.pri = o;  o += al(dd * sizeof(PriorDev));
    L.hist = o; o += al(5 * dd * 8);
    L.total = o;
    return L;
}

static void chains(const Request &r, int64_t &T, int64_t &S)
{
    const int64_t n = r.opts.sweeps;
    if (r.opts.waste_free) {
        S = (r.opts.particles + n - 1) / n;
        T = S * n;
    } else {
        S = T = r.opts.particles;
    }
}

size_t request_bytes(const Request &r)
{
    int64_t T, S;
    chains(r, T, S);
    size_t b = spec_layout(r, T).total;
    for (int K = r.k_min; K <= r.k_max; ++K)
        b += job_layout(job_dim(r.family, K, r.bg, r.bg_degree), T, S, r.fp64).total;
    return b;
}

static PriorDev to_dev(const smc_prior &p, int is_centre)
{
    PriorDev d{};
    d.kind = p.kind;
    d.is_centre = is_centre;
    d.p1 = p.p1;
    d.p2 = p.p2;
    d.lo = -INFINITY;
    d.hi = INFINITY;
    if (p.kind == SMC_UNIFORM) {
        d.lo = p.p1;
        d.hi = p.p2;
    } else if (p.kind == SMC_LOG_UNIFORM) {
        d.lo = std::log(p.p1);
        d.hi = std::log(p.p2);
    }
    d.lof = (float)d.lo;
    d.hif = (float)d.hi;
    d.a = (float)p.p1;
    d.b = (float)p.p2;
    return d;
}

void free_request_device(Ctx &c, Request &r)
{
    for (size_t a = 0; a < r.slots.size(); ++a) {
        const int sl = r.slots[a];
        c.h_jobs[sl].state = JOB_FREE;
        c.free_slots.push_back(sl);
        if (r.job_arena[a]) cudaFreeAsync(r.job_arena[a], c.stream);
        c.used -= r.job_bytes[a];
    }
    r.slots.clear();
    r.job_arena.clear();
    r.job_bytes.clear();
    if (r.spec_arena) {
        cudaFreeAsync(r.spec_arena, c.stream);
        c.used -= r.spec_bytes;
        r.spec_arena = nullptr;
    }
}

// Allocate, upload and prepare a request's spectrum and jobs, then draw the
// prior particles and their energies.  T_override / S_override replace the
// particle counts (step-level entry points).
int setup_request(Ctx &c, Request &r, int64_t T_override, int64_t S_override)
{
    int64_t T, S;
    chains(r, T, S);
    if (T_override > 0) {
        T = T_override;
        S = S_override > 0 ? S_override : T_override;
    }
    const int nK = r.k_max - r.k_min + 1;
    if ((int)c.free_slots.size() < nK) return ST_NO_ROOM;
    const SpecLayout SL = spec_layout(r, T);
    size_t need = SL.total;
    for (int K = r.k_min; K <= r.k_max; ++K)
        need += job_layout(job_dim(r.family, K, r.bg, r.bg_degree), T, S, r.fp64).total;
    if (c.used + need > c.budget) return ST_NO_ROOM;

    char *sa = nullptr;
    CK(cudaMallocAsync((void **)&sa, SL.total, c.stream));
    r.spec_arena = sa;
    r.spec_bytes = SL.total;
    c.used += SL.total;
    r.sd.xc = (float *)(sa + SL.xc);
    r.sd.wt = (float *)(sa + SL.wt);
    r.sd.y = (float *)(sa + SL.y);
    r.sd.ts = (float *)(sa + SL.ts);
    r.sd.sec2 = (float *)(sa + SL.sec2);
    r.sd.rpos64 = (double *)(sa + SL.rpos64);
    r.sd.rint64 = (double *)(sa + SL.rint64);
    r.sd.rtab = (float4 *)(sa + SL.rtab);
    r.sd.roff = (int *)(sa + SL.roff);
    r.sd.nref = (int)r.ref_pos.size();
    if (!r.ref_pos.empty()) {
        CK(cudaMemcpyAsync(r.sd.rpos64, r.ref_pos.data(), 8 * r.ref_pos.size(), cudaMemcpyHostToDevice, c.stream));
        CK(cudaMemcpyAsync(r.sd.rint64, r.ref_int.data(), 8 * r.ref_int.size(), cudaMemcpyHostToDevice, c.stream));
        CK(cudaMemcpyAsync(r.sd.roff, r.ref_off.data(), 4 * r.ref_off.size(), cudaMemcpyHostToDevice, c.stream));
    }
    r.sd.x64 = (double *)(sa + SL.x64);
    r.sd.y64 = (double *)(sa + SL.y64);
    r.sd.is64 = (double *)(sa + SL.is64);
    r.sd.tn64 = (double *)(sa + SL.tn64);
    r.sd.sc64 = (double *)(sa + SL.sc64);
    r.sd.scal = (SpecScal *)(sa + SL.scal);
    const double *ix = r.dx, *iy = r.dy, *is = r.ds;
    if (!ix) {
        double *raw = (double *)(sa + SL.raw);
        CK(cudaMemcpyAsync(raw, r.hx.data(), r.n * 8, cudaMemcpyHostToDevice, c.stream));
        CK(cudaMemcpyAsync(raw + r.n, r.hy.data(), r.n * 8, cudaMemcpyHostToDevice, c.stream));
        if (!r.hs.empty())
            CK(cudaMemcpyAsync(raw + 2 * r.n, r.hs.data(), r.n * 8, cudaMemcpyHostToDevice, c.stream));
        c.prof.h2d_bytes += (r.hs.empty() ? 16.0 : 24.0) * r.n;
        ix = raw;
        iy = raw + r.n;
        is = r.hs.empty() ? nullptr : raw + 2 * r.n;
    }
    const int coord = r.family == SMC_XRD_PHASE ? 2 : (r.bg == SMC_BG_SHIRLEY ? 1 : 0);
    CK(launch_spec_prep(ix, iy, is, r.n, r.n_pad, r.fp64 ? 0 : 1, r.noise, coord, r.sd, c.stream));

    std::vector<int> slots;
    for (int K = r.k_min; K <= r.k_max; ++K) {
        const int d = job_dim(r.family, K, r.bg, r.bg_degree);
        const JobLayout JL = job_layout(d, T, S, r.fp64);
        char *ja = nullptr;
        CK(cudaMallocAsync((void **)&ja, JL.total, c.stream));
        c.used += JL.total;
        const int sl = c.free_slots.back();
        c.free_slots.pop_back();
        r.slots.push_back(sl);
        r.job_arena.push_back(ja);
        r.job_bytes.push_back(JL.total);
        slots.push_back(sl);

        std::vector<PriorDev> pri(std::max(d, 1));
        for (int j = 0; j < d; ++j) {
            const int role = comp_role(r, K, j);
            pri[j] = to_dev(comp_prior(r, K, j), role == 1 ? 1 : 0);
        }
        CK(cudaMemcpyAsync(ja + JL.pri, pri.data(), sizeof(PriorDev) * std::max(d, 1),
                           cudaMemcpyHostToDevice, c.stream));
        std::vector<double> lam(std::max(d, 1), 2.38);
        CK(cudaMemcpyAsync(ja + JL.lam, lam.data(), 8 * lam.size(), cudaMemcpyHostToDevice, c.stream));
        CK(cudaMemsetAsync(ja + JL.acc, 0, 8 * std::max(d, 1), c.stream));
        CK(cudaMemsetAsync(ja + JL.prop, 0, 8 * std::max(d, 1), c.stream));
        CK(cudaMemsetAsync(ja + JL.hist, 0, 5 * 8 * std::max(d, 1), c.stream));
        JobDev jb{};
        jb.xc = r.sd.xc;
        jb.wt = r.sd.wt;
        jb.y = r.sd.y;
        jb.ts = r.sd.ts;
        jb.sec2 = r.sd.sec2;
        jb.rtab = r.sd.rtab;
        jb.rpos64 = r.sd.rpos64;
        jb.rint64 = r.sd.rint64;
        jb.roff = r.sd.roff;
        jb.x64 = r.sd.x64;
        jb.y64 = r.sd.y64;
        jb.is64 = r.sd.is64;
        jb.tn64 = r.sd.tn64;
        jb.sc64 = r.sd.sc64;
        jb.n = r.n;
        jb.n_pad = r.n_pad;
        jb.family = kernel_family(r.family);
        jb.wprec = r.family == SMC_GAUSS_PRECISION ? 1 : 0;
        jb.bg_kind = r.bg;
        jb.noise = r.noise;
        jb.full = r.full ? 1 : 0;
        jb.nd0 = r.noise_par[0] * r.noise_par[0];
        jb.nd1 = r.noise_par[1] * r.noise_par[1];
        jb.nd2 = r.noise_par[2] * r.noise_par[2];
        jb.nv0 = (float)jb.nd0;
        jb.nv1 = (float)jb.nd1;
        jb.nv2 = (float)jb.nd2;
        jb.K = K;
        jb.p = r.p;
        jb.nbg = r.nbg;
        jb.d = d;
        jb.J = r.tile.J;
        jb.G = r.tile.G;
        jb.R = r.tile.R;
        jb.T = (int)T;
        jb.S = (int)S;
        jb.sweeps = r.opts.sweeps;
        jb.waste_free = r.opts.waste_free ? 1 : 0;
        jb.fp64 = r.fp64 ? 1 : 0;
        if (r.fp64) {
            jb.th64 = (double *)(ja + JL.th);
            jb.E64 = (double *)(ja + JL.E);
            jb.ths64 = (double *)(ja + JL.ths);
            jb.Es64 = (double *)(ja + JL.Es);
        } else {
            jb.th = (float *)(ja + JL.th);
            jb.E = (float *)(ja + JL.E);
            jb.ths = (float *)(ja + JL.ths);
            jb.Es = (float *)(ja + JL.Es);
        }
        jb.w64 = (double *)(ja + JL.w64);
        jb.rwpart = (double *)(ja + JL.rwpart);
        jb.q = (unsigned long long *)(ja + JL.q);
        jb.anc = (int *)(ja + JL.anc);
        jb.lam = (double *)(ja + JL.lam);
        jb.step = (double *)(ja + JL.step);
        jb.stepf = (float *)(ja + JL.stepf);
        jb.acc = (unsigned long long *)(ja + JL.acc);
        jb.prop = (unsigned long long *)(ja + JL.prop);
        jb.pri = (const PriorDev *)(ja + JL.pri);
        jb.hist = (double *)(ja + JL.hist);
        jb.step_rule = r.opts.step_rule;
        jb.beta = 0.0;
        jb.rho = r.opts.ess_target;
        jb.stage = 0;
        jb.max_stages = r.opts.max_stages;
        jb.status = 0;
        jb.state = JOB_ACTIVE;
        jb.seed = r.opts.seed;
        jb.tag = (unsigned)K;
        c.h_jobs[sl] = jb;
        CK(cudaMemcpyAsync(c.d_jobs + sl, &c.h_jobs[sl], sizeof(JobDev), cudaMemcpyHostToDevice,
                           c.stream));
    }
    int *dslots = (int *)(sa + SL.slots);
    CK(cudaMemcpyAsync(dslots, slots.data(), 4 * nK, cudaMemcpyHostToDevice, c.stream));
    const int off[2] = {0, nK};
    CK(cudaMemcpyAsync(sa + SL.off, off, 8, cudaMemcpyHostToDevice, c.stream));
    CK(launch_job_setup(c.d_jobs, dslots, r.sd.scal, nK, c.stream));
    CK(launch_prior_init(c.d_jobs, dslots, nK, (int)T, c.stream));
    CK(launch_energy(c.d_jobs, dslots, nK, (int)T, r.fp64, c.stream));
    // pageable sources of the copies above must stay valid until consumed
    CK(cudaStreamSynchronize(c.stream));
    return SMC_OK;
}

// ---------------------------------------------------------------------------
// Stage loop.
// ---------------------------------------------------------------------------
struct Bucket {
    int family, J, G, R;
    std::vector<int> slots;
    int kcap = 0;  // most peaks (phases) of its jobs
};

struct Plan {
    int nreq = 0;  // requests with FP32 jobs in the plan
    std::vector<int> all;
    std::vector<Bucket> buckets;
    std::vector<size_t> boff;
    std::vector<int> grids;
    int64_t max_elems = 0;
    int64_t max_T = 0;
    int max_stages = 1;
};

// Slot lists of every FP32 job of the requests: all jobs (per-job kernels)
// and one list per Metropolis tile bucket, uploaded to the device list area.
static int build_plan(Ctx &c, std::vector<Request *> &reqs, Plan &P)
{
    for (Request *r : reqs) {
        if (r->fp64) continue;
        if (!r->slots.empty()) P.nreq += 1;
        for (int sl : r->slots) {
            P.all.push_back(sl);
            const JobDev &jb = c.h_jobs[sl];
            P.max_elems = std::max<int64_t>(P.max_elems, (int64_t)jb.S * (jb.d + 1));
            P.max_T = std::max<int64_t>(P.max_T, jb.T);
            P.max_stages = std::max(P.max_stages, jb.max_stages);
            Bucket *b = nullptr;
            const int kfam = jb.family | (jb.full ? MH_COUPLED : 0);
            for (Bucket &x : P.buckets)
                if (x.family == kfam && x.J == jb.J && x.G == jb.G && x.R == jb.R) b = &x;
            if (!b) {
                P.buckets.push_back({kfam, jb.J, jb.G, jb.R, {}});
                b = &P.buckets.back();
            }
            b->slots.push_back(sl);
            b->kcap = std::max(b->kcap, jb.K);
        }
    }
    if (P.all.empty()) return SMC_OK;
    c.prof.max_batch_requests = std::max<int64_t>(c.prof.max_batch_requests, P.nreq);
    // costliest chains first inside each bucket (dynamic scheduling drains them first)
    for (Bucket &b : P.buckets)
        std::stable_sort(b.slots.begin(), b.slots.end(), [&](int a, int z) {
            const JobDev &A = c.h_jobs[a], &Z = c.h_jobs[z];
            return (long)A.d * A.sweeps > (long)Z.d * Z.sweeps;
        });
    std::vector<int> host_lists(P.all);
    for (Bucket &b : P.buckets) {
        P.boff.push_back(host_lists.size());
        host_lists.insert(host_lists.end(), b.slots.begin(), b.slots.end());
        P.grids.push_back(mh_resident_grid(b.family, b.J, b.G, b.R, b.kcap));
    }
    if ((int)host_lists.size() > LIST_AREA) return SMC_ENOMEM;
    CK(cudaMemcpyAsync(c.d_lists, host_lists.data(), 4 * host_lists.size(), cudaMemcpyHostToDevice,
                       c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return SMC_OK;
}

// One tempering stage of every active job of the plan.  ev (optional) holds
// six events recorded between the kernel classes; k selects the host-mapped
// slot that receives the number of jobs still active afterwards.
static cudaError_t iteration(Ctx &c, const Plan &P, cudaEvent_t *ev, int k)
{
    const int nall = (int)P.all.size();
    cudaError_t e;
    auto mark = [&](int i) {
        // external record nodes keep the events timeable when captured in a graph
        return ev ? cudaEventRecordWithFlags(ev[i], c.stream, cudaEventRecordExternal) : cudaSuccess;
    };
    if ((e = mark(0)) != cudaSuccess) return e;
    if ((e = launch_reweight(c.d_jobs, c.d_lists, nall, false, P.max_T, c.stream)) != cudaSuccess) return e;
    if ((e = mark(1)) != cudaSuccess) return e;
    if ((e = launch_resample(c.d_jobs, c.d_lists, nall, c.stream)) != cudaSuccess) return e;
    if ((e = mark(2)) != cudaSuccess) return e;
    if ((e = launch_gather(c.d_jobs, c.d_lists, nall, P.max_elems, false, c.stream)) != cudaSuccess)
        return e;
    if ((e = mark(3)) != cudaSuccess) return e;
    for (size_t b = 0; b < P.buckets.size(); ++b)
        if ((e = launch_mh(c.d_jobs, c.d_lists + P.boff[b], (int)P.buckets[b].slots.size(),
                           P.buckets[b].family, P.buckets[b].J, P.buckets[b].G, P.buckets[b].R,
                           P.grids[b], c.stream,
                           P.buckets[b].kcap)) != cudaSuccess)
            return e;
    if ((e = mark(4)) != cudaSuccess) return e;
    if ((e = launch_stage_end(c.d_jobs, c.d_lists, nall, c.d_nactive, c.h_nactive_dev + k, c.stream)) !=
        cudaSuccess)
        return e;
    return mark(5);
}

int run_chunk(Ctx &c, std::vector<Request *> &reqs, int iters)
{
    Plan P;
    int st = build_plan(c, reqs, P);
    if (st != SMC_OK || P.all.empty()) return st;
    for (int k = 0; k < iters; ++k) CK(iteration(c, P, nullptr, 0));
    CK(cudaStreamSynchronize(c.stream));
    return SMC_OK;
}

// The whole run as one graph launch: a conditional while node whose body is
// one stage iteration; its last kernel clears the condition when no job is
// active (or after max_iter stages).  Returns false if the graph could not be
// built, so the caller falls back to replaying chunks of stages.
static bool run_whole_graph(Ctx &c, const Plan &P, int *status)
{
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = false;
    const int max_iter = P.max_stages + 2;
    do {
        if (cudaGraphCreate(&graph, 0) != cudaSuccess) break;
        cudaGraphConditionalHandle h;
        if (cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) break;
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) != cudaSuccess) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(c.stream, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            break;
        const int nall = (int)P.all.size();
        cudaError_t e = launch_reweight(c.d_jobs, c.d_lists, nall, false, P.max_T, c.stream);
        if (e == cudaSuccess) e = launch_resample(c.d_jobs, c.d_lists, nall, c.stream);
        if (e == cudaSuccess) e = launch_gather(c.d_jobs, c.d_lists, nall, P.max_elems, false, c.stream);
        for (size_t b = 0; b < P.buckets.size() && e == cudaSuccess; ++b)
            e = launch_mh(c.d_jobs, c.d_lists + P.boff[b], (int)P.buckets[b].slots.size(),
                          P.buckets[b].family, P.buckets[b].J, P.buckets[b].G, P.buckets[b].R,
                          P.grids[b], c.stream,
                          P.buckets[b].kcap);
        if (e == cudaSuccess)
            e = launch_stage_end_cond(c.d_jobs, c.d_lists, nall, c.d_nactive, h, c.d_nactive + 1,
                                      max_iter, c.stream);
        cudaGraph_t captured = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(c.stream, &captured);
        if (e != cudaSuccess || e2 != cudaSuccess) break;
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) break;
        ok = true;
    } while (false);
    cudaGetLastError();
    if (ok) {
        cudaError_t e = cudaMemsetAsync(c.d_nactive + 1, 0, sizeof(int), c.stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        int iters = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&iters, c.d_nactive + 1, sizeof(int), cudaMemcpyDeviceToHost);
        c.prof.stages += iters;
        *status = cuda_status(e);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    return ok;
}

static int run_fp32(Ctx &c, std::vector<Request *> &reqs)
{
    Plan P;
    int st = build_plan(c, reqs, P);
    if (st != SMC_OK || P.all.empty()) return st;
    // without per-kernel events the whole run is one graph launch
    if (!c.prof_events && c.graph_mode == SMC_GRAPH_WHILE && run_whole_graph(c, P, &st)) return st;
    // capture CHUNK stages into a CUDA graph and replay it until no job is active
    std::vector<cudaEvent_t> ev;
    if (c.prof_events) {
        ev.resize(6 * CHUNK);
        for (auto &x : ev) CK(cudaEventCreate(&x));
    }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = c.graph_mode != SMC_GRAPH_NONE;
    if (use_graph && cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < CHUNK && e == cudaSuccess; ++k)
            e = iteration(c, P, ev.empty() ? nullptr : &ev[6 * k], k);
        cudaError_t e2 = cudaStreamEndCapture(c.stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
            use_graph = false;
    } else {
        use_graph = false;
    }
    cudaGetLastError();
    const int max_iters = P.max_stages + 2 * CHUNK;
    int done_iters = 0;
    int status = SMC_OK;
    int prev_active = 1;
    while (done_iters < max_iters) {
        cudaError_t e = cudaSuccess;
        int ran = 0;
        if (use_graph) {
            e = cudaGraphLaunch(exec, c.stream);
            ran = CHUNK;
        } else {
            for (int k = 0; k < CHUNK && e == cudaSuccess; ++k, ++ran)
                e = iteration(c, P, ev.empty() ? nullptr : &ev[6 * k], k);
        }
        done_iters += ran;
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        if (e != cudaSuccess) {
            status = cuda_status(e);
            break;
        }
        int last = 0;
        for (int k = 0; k < ran; ++k) {
            const int now = ((volatile int *)c.h_nactive)[k];
            if (!ev.empty() && prev_active > 0) {
                for (int q = 0; q < 5; ++q) {
                    float ms = 0.0f;
                    if (cudaEventElapsedTime(&ms, ev[6 * k + q], ev[6 * k + q + 1]) != cudaSuccess) {
                        cudaGetLastError();
                        ms = 0.0f;
                    }
                    c.prof.ms[q] += ms;
                    // the tempering class is three kernels for FP32 jobs
                    c.prof.launches[q] += (q == 3) ? (int64_t)P.buckets.size() : (q == 0 ? 3 : 1);
                }
            }
            if (prev_active > 0) c.prof.stages += 1;
            prev_active = now;
            last = now;
        }
        if (last == 0) break;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto &x : ev) cudaEventDestroy(x);
    return status;
}

// FP64 jobs: the plain kernels (thread-per-chain Metropolis with a full FP64
// energy per proposal), one stage per launch sequence, the host checking
// completion after every stage.  The plain path passes one job at a time;
// the batched FP64 mode (energy_fp64 = 2) passes every FP64 job of the batch.
static int run_fp64_list(Ctx &c, const std::vector<int> &list)
{
    if (list.empty()) return SMC_OK;
    if ((int)list.size() > LIST_AREA) return SMC_ENOMEM;
    int64_t max_T = 0, max_elems = 0, max_S = 0;
    int max_stages = 1;
    for (int sl : list) {
        const JobDev &jb = c.h_jobs[sl];
        max_T = std::max<int64_t>(max_T, jb.T);
        max_S = std::max<int64_t>(max_S, jb.S);
        max_elems = std::max<int64_t>(max_elems, (int64_t)jb.S * (jb.d + 1));
        max_stages = std::max(max_stages, jb.max_stages);
    }
    const int n = (int)list.size();
    CK(cudaMemcpyAsync(c.d_lists, list.data(), 4 * list.size(), cudaMemcpyHostToDevice, c.stream));
    for (int it = 0; it < max_stages + 2; ++it) {
        CK(launch_reweight(c.d_jobs, c.d_lists, n, true, max_T, c.stream));
        CK(launch_resample(c.d_jobs, c.d_lists, n, c.stream));
        CK(launch_gather(c.d_jobs, c.d_lists, n, max_elems, true, c.stream));
        CK(launch_mh_plain(c.d_jobs, c.d_lists, n, (int)max_S, c.stream));
        CK(launch_stage_end(c.d_jobs, c.d_lists, n, c.d_nactive, c.h_nactive_dev, c.stream));
        CK(cudaStreamSynchronize(c.stream));
        c.prof.stages += 1;
        if (*(volatile int *)c.h_nactive == 0) break;
    }
    return SMC_OK;
}

int run_requests(Ctx &c, std::vector<Request *> &reqs)
{
    int st = run_fp32(c, reqs);
    if (st != SMC_OK) return st;
    std::vector<int> batched;
    for (Request *r : reqs) {
        if (!r->fp64) continue;
        if (r->opts.energy_fp64 == 2) {
            batched.insert(batched.end(), r->slots.begin(), r->slots.end());
            continue;
        }
        for (int sl : r->slots) {  // the plain path: one job per launch sequence
            st = run_fp64_list(c, std::vector<int>{sl});
            if (st != SMC_OK) return st;
        }
    }
    st = run_fp64_list(c, batched);
    if (st != SMC_OK) return st;
    return finalize_requests(c, reqs);
}

// Posterior summaries, p(K|D), results to the host; frees the request's device memory.
int finalize_requests(Ctx &c, std::vector<Request *> &reqs)
{
    for (Request *r : reqs) {
        int64_t T, S;
        chains(*r, T, S);
        const JobDev &j0 = c.h_jobs[r->slots[0]];
        T = j0.T;
        const SpecLayout SL = spec_layout(*r, T);
        char *sa = (char *)r->spec_arena;
        const int nK = r->k_max - r->k_min + 1;
        const int dmax = std::max(1, job_dim(r->family, r->k_max, r->bg, r->bg_degree));
        const int *dslots = (const int *)(sa + SL.slots);
        float *samples = r->opts.keep_samples ? (float *)(sa + SL.samples) : nullptr;
        CK(cudaMemsetAsync(sa + SL.fcnt, 0, 4 * nK, c.stream));
        CK(launch_finalize(c.d_jobs, dslots, nK, dmax, r->k_max, T, (double *)(sa + SL.mean),
                           (double *)(sa + SL.sd), samples, dmax, (int64_t)T * dmax,
                           (double *)(sa + SL.fpart), (int *)(sa + SL.fcnt), c.stream));
        CK(launch_posterior(c.d_jobs, dslots, (const int *)(sa + SL.off), 1, (double *)(sa + SL.pk),
                            c.stream));
        r->dim_max = dmax;
        r->n_samples = T;
        r->mean.resize((size_t)nK * dmax);
        r->sdv.resize((size_t)nK * dmax);
        r->p_k.resize(nK);
        CK(cudaMemcpyAsync(r->mean.data(), sa + SL.mean, 8 * r->mean.size(), cudaMemcpyDeviceToHost,
                           c.stream));
        CK(cudaMemcpyAsync(r->sdv.data(), sa + SL.sd, 8 * r->sdv.size(), cudaMemcpyDeviceToHost,
                           c.stream));
        CK(cudaMemcpyAsync(r->p_k.data(), sa + SL.pk, 8 * nK, cudaMemcpyDeviceToHost, c.stream));
        if (samples) {
            r->samples.resize((size_t)nK * T * dmax);
            CK(cudaMemcpyAsync(r->samples.data(), samples, 4 * r->samples.size(),
                               cudaMemcpyDeviceToHost, c.stream));
        }
        std::vector<JobDev> jobs(nK);
        for (int a = 0; a < nK; ++a)
            CK(cudaMemcpyAsync(&jobs[a], c.d_jobs + r->slots[a], sizeof(JobDev),
                               cudaMemcpyDeviceToHost, c.stream));
        CK(cudaStreamSynchronize(c.stream));
        c.prof.d2h_bytes += 16.0 * r->mean.size() + 8.0 * nK + (double)sizeof(JobDev) * nK +
                            4.0 * r->samples.size();
        r->log_z.resize(nK);
        r->n_stages.resize(nK);
        r->job_status.resize(nK);
        r->status = SMC_OK;
        for (int a = 0; a < nK; ++a) {
            const JobDev &jd = jobs[a];
            const double esz = jd.fp64 ? 8.0 : 4.0;
            c.prof.point_evals += (double)jd.point_evals + (double)jd.T * jd.n;
            c.prof.sfu_ops += (double)jd.sfu_ops;
            c.prof.peak_point_evals += (double)jd.peak_evals;
            if (jd.peak_evals) c.prof.peak_sfu_per_eval = jd.family == SMC_PSEUDO_VOIGT ? 2.0 : 1.0;
            c.prof.lg2_ops += 0.5 * (double)jd.var_ops;  // one LG2 and one RCP per point
            c.prof.rcp_ops += 0.5 * (double)jd.var_ops;
            if (jd.family == SMC_GAUSS) c.prof.ex2_ops += (double)jd.sfu_ops;
            else if (jd.family == SMC_LORENTZ) c.prof.rcp_ops += (double)jd.sfu_ops;
            else if (jd.family == SMC_XRD_PHASE) {
                c.prof.ex2_ops += (double)jd.ex2_part;
                c.prof.rcp_ops += (double)(jd.sfu_ops - jd.ex2_part);
            } else {
                c.prof.ex2_ops += 0.5 * (double)jd.sfu_ops;
                c.prof.rcp_ops += 0.5 * (double)jd.sfu_ops;
            }
            c.prof.gather_bytes += (double)jd.stage * ((double)jd.S * (jd.d + 1) * 2.0 * esz + 4.0 * jd.S);
            c.prof.resample_bytes += (double)jd.stage * (8.0 * jd.T + 4.0 * jd.S);
            c.prof.jobs += 1;
            r->log_z[a] = jobs[a].logz;
            r->n_stages[a] = jobs[a].stage;
            r->job_status[a] = jobs[a].status;
            if (jobs[a].status != 0 && r->status == SMC_OK) r->status = jobs[a].status;
        }
        // model selection: the K of smallest free energy F = -log Z (Sec. II A);
        // scanning K upwards and moving only on a gain beyond 1e-12 keeps the
        // lower K on ties
        r->selected_k = -1;
        double best = 0.0;
        for (int a = 0; a < nK; ++a) {
            if (r->job_status[a] != SMC_OK || !std::isfinite(r->log_z[a])) continue;
            if (r->selected_k < 0 || r->log_z[a] > best + 1e-12) {
                r->selected_k = r->k_min + a;
                best = r->log_z[a];
            }
        }
        free_request_device(c, *r);
        r->t_done = std::chrono::steady_clock::now();
        r->latency_ms =
            std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
        r->state.store(2, std::memory_order_release);
    }
    return SMC_OK;
}

}  // namespace smc
