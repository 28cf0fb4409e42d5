"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

None of these re-types the oracle's own formula: each checks a closed form,
an invariant, a published answer, a special case that reduces to a library
routine, or an independent high-precision evaluation.
"""
import math

import mpmath
import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle
from conftest import load_golden
from paper_2604_03271_b300 import workloads as W

GAUSS, LOR, PV, GPREC = 0, 1, 2, 3


# --------------------------------------------------------------------------
# Philox4x32-10: published known-answer vectors
# --------------------------------------------------------------------------

def test_philox_known_answers():
    for row in load_golden("philox4x32_10_kat.txt"):
        v = [int(t, 16) for t in row]
        got = oracle.philox(v[0:4], v[4:6])
        assert list(got) == v[6:10]


def _curand_host():
    import ctypes
    import glob
    paths = sorted(glob.glob("/usr/local/cuda/lib64/libcurand.so*")) + ["libcurand.so.10", "libcurand.so"]
    for p in paths:
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    # the same generator through cuRAND's host (CPU) Philox4x32-10 generator:
    # with the default ordering, a request of 4 B words returns as words
    # 4b .. 4b+3 the block of counter (0, 0, b, 0) -- subsequence b, offset 0
    # of its device API's curand_init -- under key (seed low, seed high)
    import ctypes
    L = _curand_host()
    if L is None:
        pytest.skip("cuRAND not available")
    B = 4096
    for seed in (0, 12345, 0x123456789ABCDEF0):
        gen = ctypes.c_void_p()
        assert L.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
        try:
            assert L.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            buf = (ctypes.c_uint * (4 * B))()
            assert L.curandGenerate(gen, buf, ctypes.c_size_t(4 * B)) == 0
        finally:
            L.curandDestroyGenerator(gen)
        lib = np.frombuffer(buf, dtype=np.uint32).reshape(B, 4)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        ours = np.array([oracle.philox([0, 0, b, 0], key) for b in range(B)], dtype=np.uint32)
        np.testing.assert_array_equal(ours, lib)


def test_uniform_mapping_is_open_interval():
    # u = (k + 1/2) 2^-32 never reaches 0 or 1; checked at the two extreme words
    # through the Uniform(0, 1) prior draw, whose value is exactly the mapping.
    lo = (0 + 0.5) * 2.0 ** -32
    hi = (2 ** 32 - 1 + 0.5) * 2.0 ** -32
    assert 0.0 < lo < hi < 1.0
    # the draw is the mapping of the first word of Philox counter
    # (256 comp, particle, 0, tag) under key (seed low, seed high), exactly
    for seed, comp, particle, tag in [(0, 0, 0, 1), (3, 2, 17, 5), (2 ** 40 + 7, 1, 123456, 3)]:
        k = int(oracle.philox([256 * comp, particle, 0, tag], [seed & 0xFFFFFFFF, seed >> 32])[0])
        got = oracle.prior_draw(W.UNIFORM, 0.0, 1.0, seed=seed, comp=comp, particle=particle, tag=tag)
        assert got == (k + 0.5) * 2.0 ** -32
    vals = [oracle.prior_draw(W.UNIFORM, 0.0, 1.0, seed=s, comp=0, particle=p, tag=1)
            for s in range(3) for p in range(200)]
    assert min(vals) > 0.0 and max(vals) < 1.0


# --------------------------------------------------------------------------
# Peak profiles (Eq. (1), Eq. (C1), Eq. (E1)): heights, half widths, areas
# --------------------------------------------------------------------------

@pytest.mark.parametrize("eta", [0.0, 0.25, 0.7, 1.0])
def test_pv_height_and_half_height(eta):
    A, mu, s = 3.0, 1.7, 0.4
    assert oracle.peak(PV, mu, A, mu, s, eta) == pytest.approx(A, rel=1e-15)
    # both the Gaussian and the Lorentzian part are 1/2 at |x - mu| = HWHM
    for x in (mu - s, mu + s):
        assert oracle.peak(PV, x, A, mu, s, eta) == pytest.approx(A / 2, rel=1e-14)


def test_gauss_lorentz_half_heights():
    A, mu, w = 2.0, -0.3, 0.6
    assert oracle.peak(GAUSS, mu, A, mu, w) == pytest.approx(A, rel=1e-15)
    hw = w * math.sqrt(2 * math.log(2))
    assert oracle.peak(GAUSS, mu + hw, A, mu, w) == pytest.approx(A / 2, rel=1e-14)
    assert oracle.peak(LOR, mu + w, A, mu, w) == pytest.approx(A / 2, rel=1e-14)
    assert oracle.peak(LOR, mu, A, mu, w) == pytest.approx(A, rel=1e-15)


def test_precision_gaussian_height_half_height_area():
    # Eq. (C1): A exp(-b/2 (x - mu)^2); half height at |x - mu| = sqrt(2 ln 2 / b),
    # area A sqrt(2 pi / b), and the standard-deviation form at w = b^(-1/2)
    A, mu, b = 1.3, 1.455, 146.837
    assert oracle.peak(GPREC, mu, A, mu, b) == pytest.approx(A, rel=1e-15)
    hw = math.sqrt(2 * math.log(2) / b)
    for x in (mu - hw, mu + hw):
        assert oracle.peak(GPREC, x, A, mu, b) == pytest.approx(A / 2, rel=1e-13)
    val, _ = integrate.quad(lambda x: oracle.peak(GPREC, x, A, mu, b), -np.inf, np.inf,
                            points=None, limit=400, epsabs=1e-14, epsrel=1e-12)
    assert val == pytest.approx(A * math.sqrt(2 * math.pi / b), rel=1e-9)
    for x in (0.9, 1.4, 2.0):
        assert oracle.peak(GPREC, x, A, mu, b) == pytest.approx(
            oracle.peak(GAUSS, x, A, mu, 1.0 / math.sqrt(b)), rel=1e-13)


@pytest.mark.parametrize("fam,eta,area", [
    (GAUSS, 0.0, lambda A, w, eta: A * w * math.sqrt(2 * math.pi)),
    (LOR, 0.0, lambda A, w, eta: A * math.pi * w),
    (PV, 0.3, lambda A, w, eta: A * (eta * w * math.sqrt(math.pi / math.log(2))
                                     + (1 - eta) * math.pi * w)),
    (PV, 0.9, lambda A, w, eta: A * (eta * w * math.sqrt(math.pi / math.log(2))
                                     + (1 - eta) * math.pi * w)),
])
def test_peak_areas(fam, eta, area):
    A, mu, w = 1.7, 0.4, 0.35
    val, err = integrate.quad(lambda x: oracle.peak(fam, x, A, mu, w, eta), -np.inf, np.inf,
                              limit=400, epsabs=1e-13, epsrel=1e-12)
    assert val == pytest.approx(area(A, w, eta), rel=1e-9)


def test_background_is_chebyshev_series():
    # b(x) = sum c_j T_j(t) on x scaled to [-1, 1]: numpy's Chebyshev series
    x = np.linspace(10.0, 90.0, 37)
    c = np.array([3.0, -1.5, 0.7, 0.2, -0.05])
    f = oracle.model(PV, 0, len(c), c, x)
    t = (2 * x - (x.min() + x.max())) / (x.max() - x.min())
    ref = np.polynomial.chebyshev.chebval(t, c)
    np.testing.assert_allclose(f, ref, rtol=1e-13, atol=1e-13)


def _mp_energy(fam, K, nbg, nat, x, y, s):
    """Energy 1/2 sum ((y-f)/sigma)^2 in 50-digit arithmetic, peaks written
    from Eq. (C1)/(E1) directly in mpmath."""
    mpmath.mp.dps = 50
    p = 4 if fam == PV else 3
    xmin, xmax = mpmath.mpf(float(min(x))), mpmath.mpf(float(max(x)))
    tot = mpmath.mpf(0)
    for xi, yi, si in zip(x, y, s):
        X = mpmath.mpf(float(xi))
        f = mpmath.mpf(0)
        for k in range(K):
            A, mu, w = [mpmath.mpf(float(v)) for v in nat[p * k:p * k + 3]]
            d2 = (X - mu) ** 2
            if fam == GAUSS:
                f += A * mpmath.e ** (-d2 / (2 * w * w))
            elif fam == GPREC:
                f += A * mpmath.e ** (-w * d2 / 2)
            else:
                lor = w * w / (w * w + d2)
                if fam == LOR:
                    f += A * lor
                else:
                    eta = mpmath.mpf(float(nat[p * k + 3]))
                    f += A * (eta * mpmath.e ** (-mpmath.log(2) * d2 / (w * w)) + (1 - eta) * lor)
        t = (2 * X - (xmin + xmax)) / (xmax - xmin)
        for j in range(nbg):
            f += mpmath.mpf(float(nat[p * K + j])) * mpmath.chebyt(j, t)
        r = (mpmath.mpf(float(yi)) - f) / mpmath.mpf(float(si))
        tot += r * r / 2
    return float(tot)


@pytest.mark.parametrize("fam", [GAUSS, LOR, PV, GPREC])
def test_energy_brute_force_high_precision(fam):
    rng = np.random.default_rng(11 + fam)
    N, K, nbg = 8, 2, 2
    x = np.sort(rng.uniform(0.0, 5.0, N))
    s = rng.uniform(0.05, 0.2, N)
    nat = []
    for k in range(K):
        nat += [rng.uniform(0.5, 2.0), rng.uniform(1.0, 4.0), rng.uniform(0.2, 0.8)]
        if fam == PV:
            nat.append(rng.uniform(0.0, 1.0))
    nat += [0.3, -0.1]
    y = rng.normal(1.0, 0.5, N)
    e = oracle.energy_natural(fam, K, nbg, nat, x, y, s)
    assert e == pytest.approx(_mp_energy(fam, K, nbg, nat, x, y, s), rel=1e-13)


# --------------------------------------------------------------------------
# Prior draws: distributions (KS against scipy)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind,p1,p2,dist,transform", [
    (W.UNIFORM, -1.0, 3.0, stats.uniform(-1.0, 4.0), None),
    (W.LOG_UNIFORM, 0.1, 3.0, stats.loguniform(0.1, 3.0), np.exp),
    (W.NORMAL, 1.5, 0.2, stats.norm(1.5, 0.2), None),
    (W.GAMMA, 2.0, 1.0, stats.gamma(2.0, scale=1.0), None),
    (W.GAMMA, 5.0, 0.04, stats.gamma(5.0, scale=25.0), None),
    (W.GAMMA, 0.5, 2.0, stats.gamma(0.5, scale=0.5), None),
])
def test_prior_draw_distributions(kind, p1, p2, dist, transform):
    v = np.array([oracle.prior_draw(kind, p1, p2, seed=77, comp=3, particle=i, tag=2)
                  for i in range(3000)])
    if transform is not None:
        v = transform(v)
    assert stats.kstest(v, dist.cdf).pvalue > 1e-3


# --------------------------------------------------------------------------
# ESS and the bisection (Eq. (10) weights)
# --------------------------------------------------------------------------

def test_ess_limits_and_monotonicity():
    rng = np.random.default_rng(4)
    e = rng.exponential(3.0, 500)
    e -= e.min()
    assert oracle.ess_frac(e, 0.0) == pytest.approx(1.0, rel=1e-15)
    assert oracle.ess_frac(np.full(40, 2.5), 7.0) == pytest.approx(1.0, rel=1e-14)
    vals = [oracle.ess_frac(e, d) for d in np.linspace(0, 5, 60)]
    assert all(b <= a + 1e-15 for a, b in zip(vals, vals[1:]))
    assert vals[-1] >= 1.0 / len(e)


def test_bisection_exponential_closed_form():
    # e_i = 10 x the quantiles of Exp(1): ESS/T -> (1+20d)/(1+10d)^2, which
    # equals 1/2 at d = (1 + sqrt(2))/10.
    T = 400000
    e = -10.0 * np.log1p(-(np.arange(T) + 0.5) / T)
    d, final, it = oracle.choose_delta(e, beta=0.0, rho=0.5)
    assert not final
    assert d == pytest.approx((1.0 + math.sqrt(2.0)) / 10.0, rel=2e-3)


def test_bisection_bracket_property():
    rng = np.random.default_rng(9)
    for scale in (1e6, 1e3, 30.0):
        e = rng.gamma(2.0, scale, 2048)
        e -= e.min()
        d, final, it = oracle.choose_delta(e, beta=0.0, rho=0.5)
        assert not final
        g = oracle.ess_frac(e, d)
        assert 0.5 <= g <= 0.5 * (1 + 1e-6)
        assert oracle.ess_frac(e, d * (1 + 3e-7)) < g + 1e-15


def test_bisection_final_step_when_flat():
    e = np.linspace(0.0, 1e-3, 100)
    d, final, it = oracle.choose_delta(e, beta=0.6, rho=0.5)
    assert final and d == pytest.approx(0.4, rel=0, abs=0)


# --------------------------------------------------------------------------
# Systematic resampling
# --------------------------------------------------------------------------

def test_quantise_is_exact():
    w = np.array([1.0, 0.5, 2.0 ** -40, 2.0 ** -41, 0.3])
    q = oracle.quantise(w)
    assert list(q[:4]) == [2 ** 40, 2 ** 39, 1, 0]
    assert int(q[4]) == math.floor(0.3 * 2 ** 40)


@pytest.mark.parametrize("T,M", [(7, 7), (64, 64), (1000, 997), (300, 30)])
def test_resample_offspring_bounds(T, M):
    rng = np.random.default_rng(T + M)
    q = oracle.quantise(rng.uniform(0, 1, T) ** 3)
    Q = int(q.astype(object).sum())
    for u32 in (0, 1, 2 ** 31, 2 ** 32 - 1, int(rng.integers(0, 2 ** 32))):
        a = oracle.resample(q, M, u32)
        assert np.all(np.diff(a) >= 0) and a.min() >= 0 and a.max() < T
        o = np.bincount(a, minlength=T)
        assert o.sum() == M
        for i in range(T):
            lo = (M * int(q[i])) // Q
            assert o[i] in (lo, lo + 1) or (o[i] == lo and M * int(q[i]) % Q == 0)
            assert q[i] > 0 or o[i] == 0


def test_resample_equal_and_zero_weights_are_exact():
    # equal weights: each particle is drawn exactly once, in order, for every U
    # (t_m lands in particle m's own interval of the cumulative sum); with
    # zero-weight particles between them, exactly the nonzero ones are drawn --
    # including U = 0, where t_m falls on an interval's left end
    T = 64
    for u32 in (0, 1, 2 ** 31, 2 ** 32 - 1):
        np.testing.assert_array_equal(oracle.resample(oracle.quantise(np.ones(T)), T, u32), np.arange(T))
        w = np.zeros(T)
        w[::3] = 0.37
        nz = np.flatnonzero(w)
        np.testing.assert_array_equal(oracle.resample(oracle.quantise(w), len(nz), u32), nz)


def test_resample_mean_offspring_is_proportional():
    rng = np.random.default_rng(3)
    T = M = 8
    q = oracle.quantise(rng.uniform(0.05, 1, T))
    Q = int(q.astype(object).sum())
    K = 4096
    acc = np.zeros(T)
    for k in range(K):
        acc += np.bincount(oracle.resample(q, M, (k << 32) // K), minlength=T)
    np.testing.assert_allclose(acc / K, M * q.astype(np.float64) / Q, atol=M / K + 1e-12)


def test_resample_matches_textbook_float_version():
    # textbook systematic resampling: points (m + U)/M on the normalised CDF
    rng = np.random.default_rng(12)
    T = M = 5000
    w = rng.uniform(0, 1, T) ** 4
    q = oracle.quantise(w)
    u32 = int(rng.integers(0, 2 ** 32))
    a = oracle.resample(q, M, u32)
    cdf = np.cumsum(q.astype(np.float64))
    cdf /= cdf[-1]
    pts = (np.arange(M) + (u32 + 0.0) / 2 ** 32) / M
    ref = np.searchsorted(cdf, pts, side="right")
    assert np.mean(a != ref) < 2e-3


# --------------------------------------------------------------------------
# Metropolis kernel: prior invariance at beta = 0; 1-D Gaussian target
# --------------------------------------------------------------------------

def test_mh_keeps_prior_at_beta_zero():
    spec = W.gaussian_small(2)
    opts = W.Options(particles=3000, sweeps=15, seed=5)
    u0, E0 = oracle.init_particles(spec, 1, opts, 3000)
    step = np.array([0.8, 2.5, 0.6])
    u1, E1, acc, prop = oracle.mh_stage(spec, 1, opts, u0, E0, step, beta=0.0, stage=1)
    assert np.all(acc > 0)
    assert stats.kstest(u1[:, 0], stats.gamma(2.0).cdf).pvalue > 1e-3
    assert stats.kstest(u1[:, 1], stats.uniform(0, 10).cdf).pvalue > 1e-3
    assert stats.kstest(u1[:, 2], stats.uniform(math.log(0.1), math.log(30)).cdf).pvalue > 1e-3


def _lin_gauss_posterior(x, y, s, mus, ws, m0, s0):
    Phi = np.stack([np.exp(-(x - m) ** 2 / (2 * w * w)) for m, w in zip(mus, ws)], axis=1)
    Sig = np.diag(s ** 2)
    S0 = np.eye(len(mus)) * s0 ** 2
    Cov = Sig + Phi @ S0 @ Phi.T
    logz = stats.multivariate_normal(mean=Phi @ np.full(len(mus), m0), cov=Cov).logpdf(y)
    Sp = np.linalg.inv(np.linalg.inv(S0) + Phi.T @ np.linalg.inv(Sig) @ Phi)
    mp = Sp @ (Phi.T @ np.linalg.inv(Sig) @ y + np.linalg.inv(S0) @ np.full(len(mus), m0))
    return logz, mp, Sp


def test_mh_keeps_gaussian_posterior_invariant():
    # Linear-Gaussian posterior of the two amplitudes (closed form): chains
    # started from exact posterior draws must stay on it at beta = 1.
    spec = W.linear_gaussian_case(3)
    t = spec.truth
    _, mp, Sp = _lin_gauss_posterior(spec.x, spec.y, spec.sigma, t["mu"], t["w"], t["m0"], t["s0"])
    opts = W.Options(particles=4000, sweeps=20, seed=8)
    rng = np.random.default_rng(21)
    A0 = rng.multivariate_normal(mp, Sp, size=4000)
    u0 = np.zeros((4000, 6))
    u0[:, 0], u0[:, 3] = A0[:, 0], A0[:, 1]
    u0[:, 1], u0[:, 2], u0[:, 4], u0[:, 5] = t["mu"][0], t["w"][0], t["mu"][1], t["w"][1]
    E0 = oracle.energies(spec, 2, opts, u0)
    sd = np.sqrt(np.diag(Sp))
    step = np.array([2.38 * sd[0], 0, 0, 2.38 * sd[1], 0, 0])
    u1, _, acc, prop = oracle.mh_stage(spec, 2, opts, u0, E0, step, beta=1.0, stage=1)
    assert np.all(acc[[0, 3]] > 0.2 * prop[[0, 3]])
    A = u1[:, [0, 3]]
    se = sd / math.sqrt(4000)
    assert np.all(np.abs(A.mean(0) - mp) < 5 * se)
    np.testing.assert_allclose(A.std(0), sd, rtol=0.06)
    np.testing.assert_allclose(np.corrcoef(A.T)[0, 1], Sp[0, 1] / (sd[0] * sd[1]), atol=0.05)


# --------------------------------------------------------------------------
# Evidence: closed form (linear-Gaussian), quadrature (K = 1), flat limit
# --------------------------------------------------------------------------

def test_evidence_linear_gaussian_closed_form():
    spec = W.linear_gaussian_case(3)
    t = spec.truth
    exact, mp, Sp = _lin_gauss_posterior(spec.x, spec.y, spec.sigma, t["mu"], t["w"], t["m0"], t["s0"])
    vals, means = [], []
    for seed in range(1, 7):
        r = oracle.run_job(spec, 2, W.Options(particles=2000, sweeps=8, seed=seed))
        assert r["status"] == 0
        vals.append(r["log_z"])
        means.append(r["samples"][:, [0, 3]].mean(0))
    vals = np.array(vals)
    se = vals.std(ddof=1) / math.sqrt(len(vals))
    assert abs(vals.mean() - exact) < max(0.05, 4 * se)
    tol = 4 * np.sqrt(np.diag(Sp)) / math.sqrt(2000) + 2e-3
    assert np.all(np.abs(np.mean(means, 0) - mp) < tol)


def _log_lik_gauss(y, s, f):
    return float(np.sum(-0.5 * ((y - f) / s) ** 2 - np.log(np.sqrt(2 * np.pi) * s)))


def test_evidence_k1_quadrature_gamma_amplitude():
    # mu and w fixed, A ~ Gamma(2, 1): Z = int Gamma(A) L(A) dA by adaptive quadrature
    spec = W.tiny_single_peak(5)
    mu, w = 0.9, 0.25
    spec.comp_priors = [W.Prior(W.GAMMA, 2.0, 1.0), W.Prior(W.FIXED, mu), W.Prior(W.FIXED, w)]
    phi = np.exp(-(spec.x - mu) ** 2 / (2 * w * w))
    ll = lambda A: _log_lik_gauss(spec.y, spec.sigma, A * phi)
    lmax = max(ll(A) for A in np.linspace(0.01, 5, 500))
    Z, _ = integrate.quad(lambda A: stats.gamma(2.0).pdf(A) * math.exp(ll(A) - lmax), 0, 20,
                          limit=400, points=[1.0, 1.2, 1.5], epsabs=0, epsrel=1e-11)
    exact = math.log(Z) + lmax
    vals = [oracle.run_job(spec, 1, W.Options(particles=3000, sweeps=8, seed=s))["log_z"]
            for s in range(1, 6)]
    se = np.std(vals, ddof=1) / math.sqrt(len(vals))
    assert abs(np.mean(vals) - exact) < max(0.05, 4 * se)


def test_evidence_k1_quadrature_free_centre():
    # w fixed, A ~ N(m0, s0^2), mu ~ U(0, 2): Z = int p(mu) Z_lin(mu) dmu
    spec = W.tiny_single_peak(5)
    w, m0, s0 = 0.25, 1.0, 0.5
    spec.comp_priors = [W.Prior(W.NORMAL, m0, s0), W.Prior(W.UNIFORM, 0.0, 2.0), W.Prior(W.FIXED, w)]

    def lz_lin(mu):
        phi = np.exp(-(spec.x - mu) ** 2 / (2 * w * w))
        cov = np.diag(spec.sigma ** 2) + s0 ** 2 * np.outer(phi, phi)
        return stats.multivariate_normal(mean=m0 * phi, cov=cov).logpdf(spec.y)

    grid = np.linspace(0, 2, 801)
    lg = np.array([lz_lin(m) for m in grid])
    lmax = lg.max()
    Z, _ = integrate.quad(lambda m: 0.5 * math.exp(lz_lin(m) - lmax), 0, 2, limit=500,
                          points=[float(grid[np.argmax(lg)])], epsabs=0, epsrel=1e-10)
    exact = math.log(Z) + lmax
    vals = [oracle.run_job(spec, 1, W.Options(particles=3000, sweeps=8, seed=s))["log_z"]
            for s in range(1, 6)]
    se = np.std(vals, ddof=1) / math.sqrt(len(vals))
    assert abs(np.mean(vals) - exact) < max(0.05, 4 * se)


def _gauss_legendre(lo, hi, panels, order=20):
    z, wq = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(lo, hi, panels + 1)
    a, b = edges[:-1, None], edges[1:, None]
    return (0.5 * (b - a) * z + 0.5 * (a + b)).ravel(), (0.5 * (b - a) * wq).ravel()


def _gamma21_amplitude_integral(a, bp):
    """int_0^inf A exp(-A) exp(-a A^2 / 2 + b A) dA with bp = b - 1: from
    I0 = int_0^inf exp(-a A^2/2 + bp A) dA = sqrt(pi / 2a) erfcx(-bp / sqrt(2a))
    and, integrating d/dA exp(...) over [0, inf), -a I1 + bp I0 = -1."""
    I0 = np.sqrt(np.pi / (2 * a)) * special.erfcx(-bp / np.sqrt(2 * a))
    return (1.0 + bp * I0) / a


def test_evidence_k1_tensor_quadrature_all_three_free():
    # the 21-point case with all three parameters free under its own priors:
    # A ~ Gamma(2, 1), mu ~ U(0, 2), w ~ log-uniform(0.1, 1).  The amplitude
    # integral is closed-form (the likelihood is Gaussian in A), the (mu, log w)
    # integral a composite Gauss-Legendre tensor rule, refined until it is
    # converged to 1e-9
    spec = W.tiny_single_peak(5)
    x, y, s = spec.x, spec.y, spec.sigma
    C0 = -np.sum(np.log(np.sqrt(2 * np.pi) * s))

    def log_z(panels):
        mu, wmu = _gauss_legendre(0.0, 2.0, panels)
        lw, wlw = _gauss_legendre(math.log(0.1), 0.0, panels // 2)
        M, LW = np.meshgrid(mu, lw, indexing="ij")
        phi = np.exp(-(x - M[..., None]) ** 2 / (2 * np.exp(LW)[..., None] ** 2))
        a = np.sum(phi ** 2 / s ** 2, axis=-1)
        b = np.sum(phi * y / s ** 2, axis=-1)
        li = C0 - 0.5 * np.sum((y / s) ** 2) + np.log(_gamma21_amplitude_integral(a, b - 1.0))
        m = li.max()
        # prior densities: 1/2 on mu, 1/ln(10) on log w
        return math.log(np.sum(wmu[:, None] * wlw[None, :] * np.exp(li - m)) / (2.0 * math.log(10.0))) + m

    # the amplitude integral against adaptive quadrature at one node
    phi = np.exp(-(x - 0.9) ** 2 / (2 * 0.25 ** 2))
    a, b = np.sum(phi ** 2 / s ** 2), np.sum(phi * y / s ** 2)
    ref, _ = integrate.quad(lambda A: A * math.exp(-A - 0.5 * a * A * A + b * A - (b - 1) ** 2 / (2 * a)),
                            0, np.inf, epsabs=0, epsrel=1e-12)
    assert _gamma21_amplitude_integral(a, b - 1.0) * math.exp(-(b - 1) ** 2 / (2 * a)) == pytest.approx(ref, rel=1e-10)
    exact = log_z(40)
    assert abs(exact - log_z(20)) < 1e-9
    vals = [oracle.run_job(spec, 1, W.Options(particles=3000, sweeps=8, seed=sd))["log_z"]
            for sd in range(1, 9)]
    se = np.std(vals, ddof=1) / math.sqrt(len(vals))
    print("all-free K = 1 log Z: mean", np.mean(vals), "exact", exact, "SE", se)
    assert 3 * se <= 0.05
    assert abs(np.mean(vals) - exact) <= 0.05


def test_evidence_k1_quadrature_gamma_precision():
    # the App. C parameterisation: A and mu fixed, precision b ~ Gamma(4, 0.25)
    # (shape, rate; mean 16): Z = int Ga(b) L(b) db by adaptive quadrature
    spec = W.tiny_single_peak(6)
    spec.family = W.GAUSS_PRECISION
    A, mu = 1.2, 0.9
    spec.comp_priors = [W.Prior(W.FIXED, A), W.Prior(W.FIXED, mu), W.Prior(W.GAMMA, 4.0, 0.25)]
    ll = lambda b: _log_lik_gauss(spec.y, spec.sigma, A * np.exp(-b * (spec.x - mu) ** 2 / 2))
    grid = np.linspace(0.5, 80, 800)
    lmax = max(ll(b) for b in grid)
    Z, _ = integrate.quad(lambda b: stats.gamma(4.0, scale=4.0).pdf(b) * math.exp(ll(b) - lmax),
                          0, 120, limit=400, points=[float(grid[np.argmax([ll(b) for b in grid])])],
                          epsabs=0, epsrel=1e-11)
    exact = math.log(Z) + lmax
    vals = [oracle.run_job(spec, 1, W.Options(particles=3000, sweeps=8, seed=s))["log_z"]
            for s in range(1, 6)]
    se = np.std(vals, ddof=1) / math.sqrt(len(vals))
    assert abs(np.mean(vals) - exact) < max(0.05, 4 * se)


def test_flat_likelihood_single_stage():
    spec = W.gaussian_small(1)
    spec.sigma = np.full_like(spec.x, 1e6)
    r = oracle.run_job(spec, 2, W.Options(particles=256, sweeps=2, seed=3))
    c = -np.sum(np.log(np.sqrt(2 * np.pi) * spec.sigma))
    assert r["n_stages"] == 1
    assert abs(r["log_z"] - c) < 1e-8


def test_posterior_over_k_is_softmax_of_evidence():
    p = oracle.posterior_over_k([-3.0, -1.0, -1.0 - math.log(3.0)])
    # exp(-F) weights 1 : e^2 : e^2/3 (uniform p(K), Eq. (2))
    ref = np.array([math.exp(-2.0), 1.0, 1.0 / 3.0])
    np.testing.assert_allclose(p, ref / ref.sum(), rtol=1e-14)


def test_posterior_over_k_survives_large_evidences():
    # log Z of order 1e5 (large N): the softmax must not overflow
    p = oracle.posterior_over_k([-1.0e5, -1.0e5 + 2.0, -1.0e5 + 1.0])
    ref = np.array([math.exp(-2.0), 1.0, math.exp(-1.0)])
    np.testing.assert_allclose(p, ref / ref.sum(), rtol=1e-13)


def test_sorted_summary_orders_peaks_by_centre():
    # two samples of a K = 2 Gaussian model plus a linear background, written
    # out by hand: sorting each sample's peaks by centre (R10) gives peak 1 =
    # (2, 3, 2) and (3, 1, 3), peak 2 = (1, 5, 1) and (4, 7, 4); the background
    # components are not reordered
    s = np.array([[1.0, 5.0, 1.0, 2.0, 3.0, 2.0, 10.0, 20.0],
                  [3.0, 1.0, 3.0, 4.0, 7.0, 4.0, 30.0, 40.0]])
    mean, sd = oracle.sorted_summary(s, W.GAUSS, 2)
    np.testing.assert_allclose(mean, [2.5, 2.0, 2.5, 2.5, 6.0, 2.5, 20.0, 30.0], rtol=1e-15)
    np.testing.assert_allclose(sd, [0.5, 1.0, 0.5, 1.5, 1.0, 1.5, 10.0, 10.0], rtol=1e-15)
    # pseudo-Voigt: four components a peak, the mixing ratio moves with its peak
    pv = np.array([[1.0, 5.0, 1.0, 0.1, 2.0, 3.0, 2.0, 0.2],
                   [3.0, 1.0, 3.0, 0.3, 4.0, 7.0, 4.0, 0.4]])
    mean, _ = oracle.sorted_summary(pv, W.PSEUDO_VOIGT, 2)
    np.testing.assert_allclose(mean, [2.5, 2.0, 2.5, 0.25, 2.5, 6.0, 2.5, 0.25], rtol=1e-15)
    # App. D phases are not exchangeable: no reordering
    ph = np.arange(2 * 18, dtype=np.float64).reshape(2, 18)[:, ::-1].copy()
    mean, _ = oracle.sorted_summary(ph, W.XRD_PHASE, 2)
    np.testing.assert_allclose(mean, ph.mean(axis=0), rtol=1e-15)


def test_invalid_inputs_rejected():
    spec = W.gaussian_small(1)
    spec.sigma = spec.sigma.copy()
    spec.sigma[5] = 0.0
    r = oracle.run_job(spec, 1, W.Options(particles=64, sweeps=1))
    assert r["status"] == oracle.EINVAL


def test_waste_free_particle_count():
    # S = ceil(T / n) = ceil(100 / 7) = 15 chains, n = 7 states kept per chain
    spec = W.gaussian_small(1)
    r = oracle.run_job(spec, 1, W.Options(particles=100, sweeps=7, waste_free=1, seed=2))
    assert r["status"] == 0
    assert r["n_out"] == 15 * 7 and r["samples"].shape[0] == 15 * 7
    # every kept state is a real one: its energy is the energy of its sample
    e = np.array([oracle.energy_spec(spec, 1, nat) for nat in r["samples"]])
    np.testing.assert_allclose(r["energies"], e, rtol=1e-12)


# --------------------------------------------------------------------------
# XPS model of App. E: Shirley background, variance that follows the model
# --------------------------------------------------------------------------

def test_shirley_background_endpoints_and_gaussian_closed_form():
    # one Gaussian peak on a fine grid: the background is a at the first point,
    # b at the last, and in between a + (b - a) times the normalised running
    # integral of the peak, which for a Gaussian is a difference of erf values
    x = np.linspace(0.0, 10.0, 20001)
    A, mu, w, a, b = 2.0, 4.3, 0.7, 1.5, 3.25
    f = oracle.model_vec(GAUSS, 1, W.BG_SHIRLEY, 0, [A, mu, w, a, b], x)
    peak = A * np.exp(-0.5 * ((x - mu) / w) ** 2)
    bg = f - peak
    assert bg[0] == pytest.approx(a, rel=1e-15) and bg[-1] == pytest.approx(b, rel=1e-15)
    Phi = lambda z: 0.5 * (1.0 + special.erf(z / math.sqrt(2.0)))
    frac = (Phi((x - mu) / w) - Phi((x[0] - mu) / w)) / (Phi((x[-1] - mu) / w) - Phi((x[0] - mu) / w))
    np.testing.assert_allclose(bg, a + (b - a) * frac, atol=2e-3 * (b - a))
    assert np.all(np.diff(bg) >= 0.0)
    # no peak signal: the background is the start value
    f0 = oracle.model_vec(GAUSS, 0, W.BG_SHIRLEY, 0, [a, b], x)
    np.testing.assert_array_equal(f0, np.full_like(x, a))


def test_shirley_known_sigma_run_is_exact_at_fixed_parameters():
    # Shirley background with known per-point sigma in a run: every parameter
    # fixed, so one stage and log Z = sum log N(y_i; f_i, sigma_i^2) with f the
    # peak plus its Shirley background (B = a + (b - a) C_i / C_N, C_i the
    # right-end rectangle sum of the peak from the first point), computed here
    rng = np.random.default_rng(12)
    x = np.linspace(845.0, 860.0, 61)
    A, mu, w, eta, a, b = 900.0, 851.0, 1.1, 0.4, 120.0, 260.0
    d2 = (x - mu) ** 2
    peak = A * (eta * np.exp(-math.log(2.0) * d2 / (w * w)) + (1 - eta) * w * w / (w * w + d2))
    inc = np.concatenate([[0.0], peak[1:] * np.abs(np.diff(x))])
    f = peak + a + (b - a) * np.cumsum(inc) / inc.sum()
    sig = np.full_like(x, 25.0)
    y = f + rng.normal(0.0, 25.0, x.shape)
    pri = W.Priors(amp=W.Prior(W.UNIFORM, 0, 2000), centre=W.Prior(W.UNIFORM, 845, 860),
                   width=W.Prior(W.UNIFORM, 0.2, 3), bg=[W.Prior(W.UNIFORM, 0, 500)] * 2)
    spec = W.Spectrum(x, y, sig, W.PSEUDO_VOIGT, 1, 1, W.BG_SHIRLEY, 0, pri, truth={},
                      comp_priors=[W.Prior(W.FIXED, v) for v in (A, mu, w, eta, a, b)])
    exact = float(np.sum(stats.norm.logpdf(y, loc=f, scale=sig)))
    r = oracle.run_job(spec, 1, W.Options(particles=64, sweeps=2, seed=1))
    assert r["n_stages"] == 1
    assert r["log_z"] == pytest.approx(exact, rel=1e-12)


def _mp_energy_model(K, nat, x, y, s0, s1, s2):
    """1/2 ln(2 pi v) + 1/2 (y - f)^2 / v summed, v = s0^2 f + s1^2 f^2 + s2^2,
    f = PV peaks (Eq. (E1)) + Shirley background, in 50-digit arithmetic."""
    mpmath.mp.dps = 50
    X = [mpmath.mpf(float(v)) for v in x]
    P = []
    for xi in X:
        t = mpmath.mpf(0)
        for k in range(K):
            A, mu, g, eta = [mpmath.mpf(float(v)) for v in nat[4 * k:4 * k + 4]]
            d2 = (xi - mu) ** 2
            t += A * (eta * mpmath.e ** (-mpmath.log(2) * d2 / (g * g)) + (1 - eta) * g * g / (g * g + d2))
        P.append(t)
    a, b = mpmath.mpf(float(nat[4 * K])), mpmath.mpf(float(nat[4 * K + 1]))
    inc = [mpmath.mpf(0)] + [P[i] * abs(X[i] - X[i - 1]) for i in range(1, len(X))]
    tot = sum(inc)
    run, e = mpmath.mpf(0), mpmath.mpf(0)
    for i in range(len(X)):
        run += inc[i]
        f = P[i] + a + (b - a) * run / tot
        v = mpmath.mpf(s0) ** 2 * f + mpmath.mpf(s1) ** 2 * f * f + mpmath.mpf(s2) ** 2
        e += mpmath.log(2 * mpmath.pi * v) / 2 + (mpmath.mpf(float(y[i])) - f) ** 2 / (2 * v)
    return float(e)


def test_energy_model_variance_brute_force():
    rng = np.random.default_rng(21)
    x = np.sort(rng.uniform(845.0, 860.0, 11))
    nat = [3000.0, 850.0, 1.2, 0.6, 1200.0, 854.5, 0.8, 0.3, 800.0, 1100.0]
    f = oracle.model_vec(PV, 2, W.BG_SHIRLEY, 0, nat, x)
    y = f + rng.normal(0.0, 30.0, x.shape)
    spec = W.Spectrum(x, y, np.ones_like(x), PV, 2, 2, W.BG_SHIRLEY, 0,
                      W.Priors(amp=W.Prior(W.UNIFORM, 0, 1), centre=W.Prior(W.UNIFORM, 0, 1),
                               width=W.Prior(W.UNIFORM, 0, 1)), truth={},
                      noise=W.NOISE_MODEL, noise_par=(1.7, 0.01, 0.5))
    e = oracle.energy_spec(spec, 2, nat)
    assert e == pytest.approx(_mp_energy_model(2, nat, x, y, 1.7, 0.01, 0.5), rel=1e-13)


def test_constant_model_variance_reduces_to_known_sigma():
    # variance (0, 0, s): the energy is the known-sigma energy plus N/2 ln(2 pi s^2),
    # and log Z (which carries the normaliser in the known-sigma case) is equal
    spec = W.tiny_single_peak(7, n=31)
    s = float(spec.sigma[0])
    nat = [1.1, 0.95, 0.3]
    e_known = oracle.energy_spec(spec, 1, nat)
    spec_m = W.Spectrum(spec.x, spec.y, spec.sigma, spec.family, 1, 1, spec.bg, 0, spec.priors,
                        truth={}, noise=W.NOISE_MODEL, noise_par=(0.0, 0.0, s))
    e_model = oracle.energy_spec(spec_m, 1, nat)
    assert e_model - e_known == pytest.approx(0.5 * spec.n * math.log(2 * math.pi * s * s), rel=1e-12)
    o = W.Options(particles=400, sweeps=4, seed=3)
    assert oracle.run_job(spec_m, 1, o)["log_z"] == pytest.approx(oracle.run_job(spec, 1, o)["log_z"], abs=1e-8)


def test_evidence_k1_quadrature_model_variance_shirley():
    # App. E likelihood, K = 1 pseudo-Voigt on a Shirley background with only the
    # amplitude free (uniform prior): Z = int p(A) exp(-E(A)) dA by quadrature
    x = np.linspace(850.0, 860.0, 41)
    mu, g, eta, a, b = 855.0, 1.0, 0.5, 500.0, 900.0
    truth = [2000.0, mu, g, eta, a, b]
    f = oracle.model_vec(PV, 1, W.BG_SHIRLEY, 0, truth, x)
    rng = np.random.default_rng(4)
    y = f + np.sqrt(f + (0.01 * f) ** 2) * rng.normal(size=x.shape)
    pri = W.Priors(amp=W.Prior(W.UNIFORM, 1000.0, 3000.0), centre=W.Prior(W.UNIFORM, 850, 860),
                   width=W.Prior(W.UNIFORM, 0.1, 5.0))
    spec = W.Spectrum(x, y, np.ones_like(x), PV, 1, 1, W.BG_SHIRLEY, 0, pri, truth={},
                      noise=W.NOISE_MODEL, noise_par=(1.0, 0.01, 0.0))
    spec.comp_priors = [W.Prior(W.UNIFORM, 1000.0, 3000.0), W.Prior(W.FIXED, mu), W.Prior(W.FIXED, g),
                        W.Prior(W.FIXED, eta), W.Prior(W.FIXED, a), W.Prior(W.FIXED, b)]
    E = lambda A: oracle.energy_spec(spec, 1, [A, mu, g, eta, a, b])
    grid = np.linspace(1000.0, 3000.0, 2001)
    emin = min(E(A) for A in grid)
    Z, _ = integrate.quad(lambda A: math.exp(-(E(A) - emin)) / 2000.0, 1000.0, 3000.0,
                          points=[float(grid[np.argmin([E(A) for A in grid])])], limit=400,
                          epsabs=0, epsrel=1e-11)
    exact = math.log(Z) - emin
    vals = [oracle.run_job(spec, 1, W.Options(particles=3000, sweeps=8, seed=s))["log_z"] for s in range(1, 6)]
    se = np.std(vals, ddof=1) / math.sqrt(len(vals))
    assert abs(np.mean(vals) - exact) < max(0.05, 4 * se)


# --------------------------------------------------------------------------
# XRD phase model of App. D: Caglioti widths, asymmetry, PV background, Poisson
# --------------------------------------------------------------------------

def test_xrd_phase_model_matches_independent_synthesis():
    # the oracle's model against the numpy synthesis of the data generator
    # (written separately), at the printed true parameters and at perturbed ones
    spec = W.xrd_phase(1, n=700)
    rng = np.random.default_rng(2)
    for scale in (0.0, 0.3):
        ph = [tuple(v * (1 + scale * rng.uniform(-1, 1)) for v in q) for q in W.XRD_TRUTH]
        bg = tuple(v * (1 + scale * rng.uniform(-1, 1)) for v in W.XRD_BG_TRUTH)
        nat = [v for q in ph for v in q] + list(bg)
        f = oracle.model_spec(spec, 3, nat)
        ref = W._synth_xrd(spec.x, ph, W.XRD_REFS, bg)
        np.testing.assert_allclose(f, ref, rtol=1e-12, atol=1e-12)


def test_xrd_phase_reduces_to_gaussian_peak():
    # one reflection, no asymmetry, u = v = 0 (constant Gaussian FWHM sqrt(w)),
    # no Lorentzian part: a Gaussian of sd FWHM / sqrt(8 ln 2) (Eq. (C1) form)
    fwhm, A, mu = 0.3, 5.0, 40.0
    q = [A, 0.0, 1.0, 0.0, 0.0, 0.0, fwhm ** 2, 0.0, 0.0]
    for x in (39.7, 39.9, 40.0, 40.05, 40.4):
        assert oracle.xrd_phase(q, [mu], [1.0], x) == pytest.approx(
            oracle.peak(GAUSS, x, A, mu, fwhm / math.sqrt(8 * math.log(2))), rel=1e-13, abs=1e-300)
    # asymmetry: the right side is stretched by alpha (half height at alpha FWHM / 2)
    q[2] = 1.7
    assert oracle.xrd_phase(q, [mu], [1.0], mu + 1.7 * fwhm / 2) == pytest.approx(A / 2, rel=1e-12)
    assert oracle.xrd_phase(q, [mu], [1.0], mu - fwhm / 2) == pytest.approx(A / 2, rel=1e-12)


def test_xrd_widths_at_ninety_degrees():
    # at 2 theta = 90 degrees tan(x/2) = 1 and 1/cos(x/2) = sqrt(2), so the
    # Caglioti width is S = sqrt(u - v + w) and the Lorentzian width W =
    # s sqrt(2) + t (Eqs. of App. D written out by hand); one reflection just
    # below 90 (x right of it: both widths scaled by alpha) and one just above
    A, sh, al, r, u, v, w, sw, tw = 2.5, 0.01, 1.3, 0.4, 0.3, 0.1, 0.05, 0.2, 0.07
    q = [A, sh, al, r, u, v, w, sw, tw]
    S, Wl = math.sqrt(u - v + w), sw * math.sqrt(2.0) + tw

    def pv(dx, a):
        return (1 - r) * math.exp(-4 * math.log(2) * (dx / (a * S)) ** 2) + r / (1 + 4 * (dx / (a * Wl)) ** 2)

    for ref, I in ((89.7, 0.8), (90.25, 1.7)):
        mu = ref + sh
        dx = 90.0 - mu
        expect = A * I * pv(dx, al if dx >= 0 else 1.0)
        assert oracle.xrd_phase(q, [ref], [I], 90.0) == pytest.approx(expect, rel=1e-13)
    # a radicand below zero removes the Gaussian part only; a negative
    # Lorentzian width removes the Lorentzian part only
    q2 = list(q)
    q2[5] = u + w + 0.2  # v: u - v + w < 0
    dx = 90.0 - (89.7 + sh)
    assert oracle.xrd_phase(q2, [89.7], [1.0], 90.0) == pytest.approx(
        A * r / (1 + 4 * (dx / (al * Wl)) ** 2), rel=1e-13)
    q3 = list(q)
    q3[7], q3[8] = -0.2, 0.0
    assert oracle.xrd_phase(q3, [89.7], [1.0], 90.0) == pytest.approx(
        A * (1 - r) * math.exp(-4 * math.log(2) * (dx / (al * S)) ** 2), rel=1e-13)


def test_xrd_background_closed_form():
    # a V(x; 0, s, s, r) + b with the App. D pseudo-Voigt, at a few angles
    a, sb, rb, b = 700.0, 8.0, 0.35, 40.0
    for x in (0.0, 10.0, 33.3, 80.0):
        v = (1 - rb) * math.exp(-4 * math.log(2) * (x / sb) ** 2) + rb / (1 + 4 * (x / sb) ** 2)
        assert oracle.xrd_background([a, sb, rb, b], x) == pytest.approx(a * v + b, rel=1e-14)


def test_xrd_poisson_log_z_of_fixed_background_is_exact():
    # no phase (K = 0) and every background parameter fixed: one stage, and
    # log Z = sum_i log Poisson(y_i; f_i) exactly
    spec = W.xrd_phase(3, n=150, k_min=0, k_max=0)
    bg = [500.0, 12.0, 0.3, 90.0]
    spec.comp_priors = [W.Prior(W.FIXED, v) for v in bg]
    f = np.array([oracle.xrd_background(bg, xi) for xi in spec.x])
    exact = float(np.sum(stats.poisson.logpmf(spec.y, f)))
    r = oracle.run_job(spec, 0, W.Options(particles=64, sweeps=2, seed=1))
    assert r["n_stages"] == 1
    assert r["log_z"] == pytest.approx(exact, rel=1e-12)


def test_poisson_counts_with_a_peak_family_fixed_parameters_exact():
    # Poisson likelihood on the ordinary peak families (not only the phase
    # model): one Gaussian peak on a constant, every parameter fixed, so one
    # stage and log Z = sum_i log Poisson(y_i; f_i) exactly
    rng = np.random.default_rng(8)
    x = np.linspace(0.0, 10.0, 80)
    A, mu, w, c0 = 40.0, 4.2, 0.7, 5.0
    f = A * np.exp(-(x - mu) ** 2 / (2 * w * w)) + c0
    y = rng.poisson(f).astype(np.float64)
    pri = W.Priors(amp=W.Prior(W.UNIFORM, 0, 100), centre=W.Prior(W.UNIFORM, 0, 10),
                   width=W.Prior(W.UNIFORM, 0.1, 2), bg=[W.Prior(W.UNIFORM, 0, 20)])
    spec = W.Spectrum(x, y, np.ones_like(x), W.GAUSS, 1, 1, W.BG_CONST, 0, pri, truth={},
                      noise=W.NOISE_POISSON,
                      comp_priors=[W.Prior(W.FIXED, v) for v in (A, mu, w, c0)])
    exact = float(np.sum(stats.poisson.logpmf(y, f)))
    r = oracle.run_job(spec, 1, W.Options(particles=64, sweeps=2, seed=1))
    assert r["n_stages"] == 1
    assert r["log_z"] == pytest.approx(exact, rel=1e-12)


def test_xrd_poisson_zero_counts():
    # points with y = 0 contribute log Poisson(0; f) = -f: the same exact
    # fixed-background evidence with a tenth of the counts set to zero
    spec = W.xrd_phase(7, n=120, k_min=0, k_max=0)
    spec.y = spec.y.copy()
    spec.y[::10] = 0.0
    bg = [450.0, 9.0, 0.6, 30.0]
    spec.comp_priors = [W.Prior(W.FIXED, v) for v in bg]
    f = np.array([oracle.xrd_background(bg, xi) for xi in spec.x])
    exact = float(np.sum(stats.poisson.logpmf(spec.y, f)))
    r = oracle.run_job(spec, 0, W.Options(particles=16, sweeps=1, seed=1))
    assert r["log_z"] == pytest.approx(exact, rel=1e-12)


def test_xrd_evidence_k1_quadrature_amplitude():
    # rutile only, every parameter fixed but the intensity A ~ Gamma(4, rate):
    # Z = int Ga(A) p(D | A) dA by adaptive quadrature
    spec = W.xrd_phase(5, n=200, k_min=1, k_max=1)
    q = list(W.XRD_TRUTH[0])
    bg = list(W.XRD_BG_TRUTH)
    rate = 4.0 / 10000.0
    spec.comp_priors = ([W.Prior(W.GAMMA, 4.0, rate)] + [W.Prior(W.FIXED, v) for v in q[1:]]
                        + [W.Prior(W.FIXED, v) for v in bg])
    # data from rutile alone
    f = W._synth_xrd(spec.x, [tuple(q)], W.XRD_REFS[:1], tuple(bg))
    spec.y = np.random.default_rng(6).poisson(f).astype(float)
    ll = lambda A: float(np.sum(stats.poisson.logpmf(spec.y, oracle.model_spec(spec, 1, [A] + q[1:] + bg))))
    grid = np.linspace(8000, 12000, 401)
    lmax = max(ll(A) for A in grid)
    Z, _ = integrate.quad(lambda A: stats.gamma(4.0, scale=1 / rate).pdf(A) * math.exp(ll(A) - lmax),
                          5000, 15000, points=[float(grid[np.argmax([ll(A) for A in grid])])],
                          limit=400, epsabs=0, epsrel=1e-10)
    exact = math.log(Z) + lmax
    vals = [oracle.run_job(spec, 1, W.Options(particles=2000, sweeps=6, seed=s))["log_z"] for s in range(1, 6)]
    se = np.std(vals, ddof=1) / math.sqrt(len(vals))
    assert abs(np.mean(vals) - exact) < max(0.05, 4 * se)


def test_generators_use_the_paper_true_parameters():
    # the synthetic App. C and App. D inputs are built from the paper's printed
    # true parameters (tests/golden/paper_true_parameters.txt)
    rows = load_golden("paper_true_parameters.txt")
    for K in (3, 10, 30):
        tab = [tuple(float(v) for v in r[2:]) for r in rows if r[0] == f"deconv{K}"]
        assert [int(r[1]) for r in rows if r[0] == f"deconv{K}"] == list(range(1, K + 1))
        np.testing.assert_array_equal(np.array(tab), np.array(W.DECONV_TRUTH[K]))
    ph = [tuple(float(v) for v in r[2:]) for r in rows if r[0] == "xrd_phase"]
    np.testing.assert_array_equal(np.array(ph), np.array(W.XRD_TRUTH))
    bg = [tuple(float(v) for v in r[1:]) for r in rows if r[0] == "xrd_bg"]
    np.testing.assert_array_equal(np.array(bg[0]), np.array(W.XRD_BG_TRUTH))
    for r in (r for r in rows if r[0] == "deconv_grid"):
        K, N, L, sd = int(r[1]), int(r[2]), float(r[3]), float(r[4])
        assert W.DECONV_GRID[K] == (N, L, sd)
        s = W.gaussian_deconvolution(K, 0)
        assert s.n == N and s.x[0] == 0.0 and s.x[-1] == L and np.all(s.sigma == sd)


def test_xrd_priors_are_the_paper_table():
    rows = {r[0]: r[1:] for r in load_golden("xrd_priors.txt")}
    kinds = {"normal": W.NORMAL, "gamma": W.GAMMA, "uniform": W.UNIFORM}
    spec = W.xrd_phase(2, n=500)
    ph = spec.phase_priors  # (A, d2theta, alpha, r, u, v, w, s, t)
    names = ["d2theta", "alpha", "r", "u", "v", "w", "s", "t"]
    for name, p in zip(names, ph[1:]):
        kind, p1, p2 = rows[name]
        assert (p.kind, p.p1, p.p2) == (kinds[kind], float(p1), float(p2)), name
    ymin, ymax = float(spec.y.min()), float(spec.y.max())
    assert (ph[0].kind, ph[0].p1) == (W.GAMMA, 4.0) and ph[0].p2 == pytest.approx(4.0 / (ymax - ymin), rel=1e-15)
    a, sbg, rbg, b = spec.priors.bg[:4]
    assert (a.kind, a.p1) == (W.GAMMA, 2.0) and a.p2 == pytest.approx(1.0 / ymax, rel=1e-15)
    for name, p in (("sigma_bg", sbg), ("r_bg", rbg)):
        kind, p1, p2 = rows[name]
        assert (p.kind, p.p1, p.p2) == (kinds[kind], float(p1), float(p2)), name
    assert b.kind == W.UNIFORM
    assert (b.p1, b.p2) == pytest.approx((ymin - math.sqrt(ymin), ymin + math.sqrt(ymin)), rel=1e-15)
