"""Pins of the oracle's step-size rule and of its waste-free mode.

Step sizes (Sec. II B 4; the rule itself is the reading R9, because the paper
defers to a predictor it does not print): s_j = lambda_j * max(SD_j,
1e-9 (1 + |mean_j|)), SD_j the population SD of component j under the
incremental weights of the stage (Eq. (10)), taken BEFORE resampling, and
lambda_j <- clamp(lambda_j exp(acc_j - 0.44), 0.01, 10) from the previous
stage's acceptance rate (lambda_j = 2.38 at the first stage).

Waste-free SMC (Sec. II B 3): S = ceil(T/n) chains are resampled from all
carried particles, each runs n sweeps, and the n post-sweep states of every
chain are kept (T_eff = S n), so that the next stage's weights, evidence
increment and step sizes run over all T_eff particles.

Every expected value here comes from numpy / scipy evaluations written in
this file (weighted moments by replication of rows, np.cov with analytic
weights, the closed-form evidence of the linear-Gaussian case, 1-D adaptive
quadrature), never from the oracle's own routines, and each test is chosen so
that one plausible mistake in the oracle fails it:
  - an unweighted SD                    -> test_step_sizes_weighted_sd_by_replication,
                                           test_first_stage_step_uses_pre_resample_weights
  - weights taken after resampling      -> test_first_stage_step_uses_pre_resample_weights
  - the acceptance update's sign flipped -> test_step_sizes_lambda_updates_and_clamps,
                                           test_second_stage_step_follows_acceptance
  - the start state kept (waste-free)   -> test_waste_free_keeps_every_post_sweep_state
  - reweighting over S, not T_eff       -> test_waste_free_second_stage_runs_over_all_states
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
from paper_2604_03271_b300 import workloads as W


def _weighted_moments_by_replication(u, counts):
    """Mean and population SD of each column of u with integer weights, by
    writing every row out `count` times and taking numpy's plain moments."""
    rows = np.repeat(u, counts, axis=0)
    return rows.mean(axis=0), rows.std(axis=0)


def _spec_with_fixed():
    """Two-peak Gaussian spectrum whose second peak's width is FIXED."""
    spec = W.gaussian_small(1)
    spec.comp_priors = [W.Prior(W.GAMMA, 2.0, 1.0), W.Prior(W.UNIFORM, 0.0, 10.0),
                        W.Prior(W.LOG_UNIFORM, 0.1, 3.0),
                        W.Prior(W.GAMMA, 2.0, 1.0), W.Prior(W.UNIFORM, 0.0, 10.0),
                        W.Prior(W.FIXED, 0.8)]
    return spec


# --------------------------------------------------------------------------
# the rule on given populations
# --------------------------------------------------------------------------

def test_step_sizes_weighted_sd_by_replication():
    spec = _spec_with_fixed()
    opts = W.Options(particles=64)
    rng = np.random.default_rng(31)
    T, d = 64, 6
    u = rng.normal(size=(T, d)) * np.array([0.3, 2.0, 0.5, 1.0, 0.1, 0.0]) + 1.0
    counts = rng.integers(0, 9, size=T)
    counts[0] = 25  # one heavy outlying particle: weighted and unweighted moments differ
    u[0, :5] += 3.0 * np.array([0.3, 2.0, 0.5, 1.0, 0.1])
    w = counts * 0.125  # weights need not be normalised; the scale must not matter
    lam = np.full(d, 2.38)
    step, lam_out = oracle.step_sizes(spec, 2, opts, u, w, None, lam)
    m, sd = _weighted_moments_by_replication(u, counts)
    free = [0, 1, 2, 3, 4]
    np.testing.assert_allclose(step[free], 2.38 * sd[free], rtol=1e-12)
    assert step[5] == 0.0  # FIXED component: never proposed
    np.testing.assert_array_equal(lam_out, lam)  # no acceptance rate: lambda unchanged
    # the check can tell a weighted from an unweighted SD on these rows
    assert np.all(np.abs(u[:, free].std(axis=0) / sd[free] - 1.0) > 0.02)


def test_step_sizes_floor_for_a_collapsed_component():
    spec = W.gaussian_small(1)
    opts = W.Options(particles=16)
    u = np.tile(np.array([[1.5, -4.0, 0.25]]), (16, 1))
    u[:, 0] += np.linspace(-1, 1, 16)  # only the first component has spread
    step, _ = oracle.step_sizes(spec, 1, opts, u, np.ones(16), None, np.full(3, 2.0))
    # identical values: SD = 0 is replaced by 1e-9 (1 + |mean|)
    assert step[1] == pytest.approx(2.0 * 1e-9 * (1.0 + 4.0), rel=1e-12)
    assert step[2] == pytest.approx(2.0 * 1e-9 * (1.0 + 0.25), rel=1e-12)
    assert step[0] == pytest.approx(2.0 * np.std(np.linspace(-1, 1, 16)), rel=1e-12)


def test_step_sizes_lambda_updates_and_clamps():
    # Three successive stages: rates above 0.44 must enlarge lambda, rates
    # below must shrink it, and both clamps must hold.
    spec = _spec_with_fixed()
    opts = W.Options(particles=32)
    rng = np.random.default_rng(7)
    u = rng.normal(size=(32, 6))
    w = rng.uniform(0.1, 1.0, 32)
    sd = np.sqrt(np.cov(u.T, aweights=w, ddof=0).diagonal())
    lam = np.array([2.38, 2.38, 0.0105, 9.0, 1.0, 2.38])
    rates = [np.array([0.94, 0.0, 0.0, 1.0, 0.44, 0.5]),
             np.array([0.94, 0.1, 0.2, 1.0, 0.3, 0.5]),
             np.array([0.10, 1.0, 0.9, 0.0, 0.6, 0.5])]
    for acc in rates:
        step, lam_new = oracle.step_sizes(spec, 2, opts, u, w, acc, lam)
        for j in range(5):
            grow = acc[j] > 0.44
            if acc[j] != 0.44:
                assert (lam_new[j] > lam[j]) == grow or lam_new[j] in (0.01, 10.0)
            ideal = lam[j] * math.exp(acc[j] - 0.44)
            assert lam_new[j] == pytest.approx(min(10.0, max(0.01, ideal)), rel=1e-14)
            assert step[j] == pytest.approx(lam_new[j] * sd[j], rel=1e-12)
        assert step[5] == 0.0
        lam = lam_new
    # component 2 hit the lower clamp at the first update and component 3 the
    # upper one at the second (9 e^0.56 > 10): both stayed inside [0.01, 10]
    assert 0.01 <= lam.min() and lam.max() <= 10.0


# --------------------------------------------------------------------------
# the rule inside a run: population and weights of the stage
# --------------------------------------------------------------------------

def _to_sampling(spec, K, nat):
    """Natural values -> sampling coordinates (log for log-uniform priors)."""
    pri = [spec.priors.amp, spec.priors.centre, spec.priors.width] * K
    u = np.array(nat, dtype=np.float64, copy=True)
    for j, p in enumerate(pri):
        if p.kind == W.LOG_UNIFORM:
            u[:, j] = np.log(u[:, j])
    return u


def test_first_stage_step_uses_pre_resample_weights():
    spec = W.gaussian_small(2)
    K, T = 2, 3000
    opts = W.Options(particles=T, sweeps=4, seed=13, max_stages=1)
    r = oracle.run_job(spec, K, opts)
    assert r["status"] == oracle.EMAXSTAGES and r["n_stages"] == 1
    # the stage-1 population is the prior draw, weighted by exp(-beta_1 (E - E_min))
    u0, E0 = oracle.init_particles(spec, K, opts, T)
    w = np.exp(-r["beta"][1] * (E0 - E0.min()))
    sd_w = np.sqrt(np.cov(u0.T, aweights=w, ddof=0).diagonal())
    np.testing.assert_allclose(r["step"][1], 2.38 * sd_w, rtol=1e-9)
    # discriminating power: the unweighted SD of the prior draw, and the SD of
    # a systematically resampled population (textbook form, numpy), both miss
    # the weighted SD by far more than the tolerance above
    assert np.all(np.abs(u0.std(axis=0) / sd_w - 1.0) > 1e-3)
    cdf = np.cumsum(w) / w.sum()
    anc = np.minimum(np.searchsorted(cdf, (np.arange(T) + 0.37) / T, side="right"), T - 1)
    assert np.all(np.abs(u0[anc].std(axis=0) / sd_w - 1.0) > 1e-6)
    ess = w.sum() ** 2 / (w * w).sum()
    assert ess < 0.6 * T


def test_second_stage_step_follows_acceptance():
    spec = W.gaussian_small(2)
    K, T = 1, 2000
    one = oracle.run_job(spec, K, W.Options(particles=T, sweeps=3, seed=5, max_stages=1))
    two = oracle.run_job(spec, K, W.Options(particles=T, sweeps=3, seed=5, max_stages=2))
    assert two["n_stages"] == 2
    # the stage-2 population is the stage-1 output (same seed, same trajectory)
    u1 = _to_sampling(spec, K, one["samples"])
    E1 = one["energies"]
    d2 = two["beta"][2] - two["beta"][1]
    w = np.exp(-d2 * (E1 - E1.min()))
    sd_w = np.sqrt(np.cov(u1.T, aweights=w, ddof=0).diagonal())
    acc1 = one["acc"][1]
    assert np.all((acc1 > 0.0) & (acc1 < 1.0)) and np.any(np.abs(acc1 - 0.44) > 0.05)
    lam2 = np.clip(2.38 * np.exp(acc1 - 0.44), 0.01, 10.0)
    np.testing.assert_allclose(two["step"][2], lam2 * sd_w, rtol=1e-8)
    # a flipped update would give 2.38 exp(0.44 - acc) instead
    flipped = 2.38 * np.exp(0.44 - acc1) * sd_w
    assert np.max(np.abs(flipped / two["step"][2] - 1.0)) > 0.05


# --------------------------------------------------------------------------
# waste-free mode (Sec. II B 3)
# --------------------------------------------------------------------------

def test_waste_free_keeps_every_post_sweep_state():
    # Metropolis draws are indexed by (sweep, component, chain, stage), so the
    # state after sweep t of a waste-free stage is exactly the final state of a
    # standard stage of t + 1 sweeps from the same starts.
    spec = W.gaussian_small(1)
    K, S, n = 2, 40, 5
    wf = W.Options(particles=S * n, sweeps=n, waste_free=1, seed=3)
    u0, E0 = oracle.init_particles(spec, K, wf, S)
    step = np.array([0.3, 0.4, 0.2, 0.3, 0.4, 0.2])
    u_wf, E_wf, acc, prop = oracle.mh_stage(spec, K, wf, u0, E0, step, beta=0.02, stage=1)
    assert u_wf.shape == (S * n, 6)
    for t in range(n):
        std = W.Options(particles=S, sweeps=t + 1, waste_free=0, seed=3)
        u_t, E_t, _, _ = oracle.mh_stage(spec, K, std, u0, E0, step, beta=0.02, stage=1)
        np.testing.assert_array_equal(u_wf[t::n], u_t)  # particle m n + t
        np.testing.assert_array_equal(E_wf[t::n], E_t)
    # the kept set is not the starts: most chains moved in the first sweep
    moved = np.any(u_wf[0::n] != u0, axis=1)
    assert moved.mean() > 0.5
    assert np.all(prop == S * n)


def test_waste_free_second_stage_runs_over_all_states():
    spec = W.gaussian_small(2)
    K, T, n = 1, 600, 6
    S = T // n
    one = oracle.run_job(spec, K, W.Options(particles=T, sweeps=n, waste_free=1, seed=9,
                                            max_stages=1))
    two = oracle.run_job(spec, K, W.Options(particles=T, sweeps=n, waste_free=1, seed=9,
                                            max_stages=2))
    E1 = one["energies"]
    assert E1.shape[0] == S * n
    d2 = two["beta"][2] - two["beta"][1]
    assert d2 > 0
    # evidence increment of Eq. (11) over all S n states
    inc = -d2 * E1.min() + math.log(np.mean(np.exp(-d2 * (E1 - E1.min()))))
    assert two["logz"][2] - two["logz"][1] == pytest.approx(inc, rel=1e-11, abs=1e-11)
    # over the S chain ends only it would differ
    ends = E1[n - 1::n]
    inc_s = -d2 * ends.min() + math.log(np.mean(np.exp(-d2 * (ends - ends.min()))))
    assert abs(inc_s - inc) > 1e-3
    # and the stage-2 step sizes come from the same S n states
    u1 = _to_sampling(spec, K, one["samples"])
    w = np.exp(-d2 * (E1 - E1.min()))
    sd_w = np.sqrt(np.cov(u1.T, aweights=w, ddof=0).diagonal())
    lam2 = np.clip(2.38 * np.exp(one["acc"][1] - 0.44), 0.01, 10.0)
    np.testing.assert_allclose(two["step"][2], lam2 * sd_w, rtol=1e-8)


def _lin_gauss_exact(spec):
    t = spec.truth
    Phi = np.stack([np.exp(-(spec.x - m) ** 2 / (2 * w * w)) for m, w in zip(t["mu"], t["w"])],
                   axis=1)
    cov = np.diag(spec.sigma ** 2) + t["s0"] ** 2 * Phi @ Phi.T
    return stats.multivariate_normal(mean=Phi @ np.full(2, t["m0"]), cov=cov).logpdf(spec.y)


def test_waste_free_evidence_linear_gaussian_closed_form():
    spec = W.linear_gaussian_case(3)
    exact = _lin_gauss_exact(spec)
    vals = []
    for seed in range(1, 13):
        r = oracle.run_job(spec, 2, W.Options(particles=24000, sweeps=8, waste_free=1, seed=seed))
        assert r["status"] == 0 and r["samples"].shape[0] == 24000
        vals.append(r["log_z"])
    vals = np.array(vals)
    se = vals.std(ddof=1) / math.sqrt(len(vals))
    print("waste-free log Z: mean", vals.mean(), "exact", exact, "SE", se)
    assert se < 0.015
    assert abs(vals.mean() - exact) < 0.05, (vals.mean(), exact, se)


def test_waste_free_evidence_k1_gamma_amplitude_quadrature():
    spec = W.tiny_single_peak(5)
    mu, w = 0.9, 0.25
    spec.comp_priors = [W.Prior(W.GAMMA, 2.0, 1.0), W.Prior(W.FIXED, mu), W.Prior(W.FIXED, w)]
    phi = np.exp(-(spec.x - mu) ** 2 / (2 * w * w))

    def ll(A):
        r = (spec.y - A * phi) / spec.sigma
        return float(np.sum(-0.5 * r * r - np.log(np.sqrt(2 * np.pi) * spec.sigma)))

    lmax = max(ll(A) for A in np.linspace(0.01, 5, 500))
    Z, _ = integrate.quad(lambda A: stats.gamma(2.0).pdf(A) * math.exp(ll(A) - lmax), 0, 20,
                          limit=400, points=[1.0, 1.2, 1.5], epsabs=0, epsrel=1e-11)
    exact = math.log(Z) + lmax
    vals = np.array([oracle.run_job(spec, 1, W.Options(particles=20000, sweeps=10, waste_free=1,
                                                       seed=s))["log_z"] for s in range(1, 13)])
    se = vals.std(ddof=1) / math.sqrt(len(vals))
    print("waste-free log Z: mean", vals.mean(), "exact", exact, "SE", se)
    assert se < 0.015
    assert abs(vals.mean() - exact) < 0.05, (vals.mean(), exact, se)


# --------------------------------------------------------------------------
# the history step-size predictor (step_rule 1; Sec. II B 4 names a predictor
# from the histories of beta and of the acceptance rates)
# --------------------------------------------------------------------------

def _rw_acceptance_numeric(s, sigma):
    """Acceptance rate of a Gaussian random walk of SD s on N(0, sigma^2),
    E over x ~ N(0, sigma^2), z ~ N(0, 1) of min(1, pi(x + s z) / pi(x)).
    pi(x) min(1, pi(x + d) / pi(x)) = min(pi(x), pi(x + d)) is the density of
    whichever of x, x + d lies farther from 0, so for a fixed d = s z the x
    integral is P(X + d >= d/2) + P(X < -d/2) = 2 Phi(-|d| / (2 sigma)); the z
    integral is taken by 1-D adaptive quadrature."""
    f = lambda z: 2.0 * stats.norm.pdf(z) * 2.0 * stats.norm.cdf(-s * z / (2.0 * sigma))
    val, _ = integrate.quad(f, 0.0, np.inf, epsabs=1e-13, epsrel=1e-12)
    return val


def _rw_acceptance_monte_carlo(s, sigma, n, seed):
    """The same expectation by plain Monte Carlo of the definition."""
    rng = np.random.default_rng(seed)
    x = rng.normal(0.0, sigma, n)
    xp = x + s * rng.normal(0.0, 1.0, n)
    return np.minimum(1.0, np.exp(-(xp * xp - x * x) / (2.0 * sigma * sigma))).mean()


def _rw_acceptance(s, sigma):
    return 2.0 / math.pi * math.atan(2.0 * sigma / s)


@pytest.mark.parametrize("ratio", [0.3, 1.0, 2.42, 6.0])
def test_random_walk_acceptance_closed_form(ratio):
    # the relation the predictor inverts, checked by quadrature and, straight
    # from the definition, by Monte Carlo (4e6 draws: SE below 2.5e-4)
    assert _rw_acceptance_numeric(ratio, 1.0) == pytest.approx(_rw_acceptance(ratio, 1.0), abs=1e-10)
    assert _rw_acceptance_monte_carlo(ratio, 1.3, 4_000_000, 11) == pytest.approx(
        _rw_acceptance(ratio, 1.3), abs=1.5e-3)


@pytest.mark.parametrize("gamma", [0.5, 0.3, 0.9])
def test_predictor_hits_target_rate_on_a_power_law(gamma):
    # tempered posteriors whose SD follows sigma(beta) = 2 beta^-gamma; rates
    # observed at arbitrary steps; after two or more stages the fitted slope is
    # -gamma and the predicted step gives acceptance 0.44 at the next beta
    # exactly (with one stage the slope is -1/2, exact for gamma = 1/2)
    sig = lambda b: 2.0 * b ** -gamma
    betas = [1e-4 * 3.0 ** k for k in range(8)]
    h = np.zeros(5)
    rng = np.random.default_rng(3)
    s = 0.7 * sig(betas[0])
    for k in range(len(betas) - 1):
        a = _rw_acceptance(s, sig(betas[k]))
        assert 0.02 < a < 0.98  # inside the clamp of the observed rate
        s_new, h = oracle.predict_step(h, s, a, betas[k], betas[k + 1], sd_pop=sig(betas[k + 1]))
        if k >= 1 or gamma == 0.5:
            assert _rw_acceptance(s_new, sig(betas[k + 1])) == pytest.approx(0.44, abs=1e-9)
        # the next observation is made at an unrelated step
        s = s_new * rng.uniform(0.3, 3.0)


def test_predictor_history_weights_and_bounds():
    # the regression sums: each older stage counts half as much as the next
    h = np.zeros(5)
    obs = [(1e-3, 0.5, 0.8), (1e-2, 0.3, 0.5), (1e-1, 0.6, 0.2)]
    wts, xs, ys = [], [], []
    for k, (b, a, s) in enumerate(obs):
        _, h = oracle.predict_step(h, s, a, b, 2 * b, sd_pop=1.0)
        wts = [0.5 * q for q in wts] + [1.0]
        xs.append(math.log(b))
        ys.append(math.log(s * math.tan(math.pi * a / 2) / 2))
    wts, xs, ys = np.array(wts), np.array(xs), np.array(ys)
    np.testing.assert_allclose(h, [wts.sum(), wts @ xs, wts @ ys, wts @ xs ** 2, wts @ (xs * ys)],
                               rtol=1e-13)
    # observed rates are clamped to [0.02, 0.98]: 0.999 counts as 0.98
    a1, _ = oracle.predict_step(np.zeros(5), 1.0, 0.999, 1e-3, 1e-2, sd_pop=1e9)
    a2, _ = oracle.predict_step(np.zeros(5), 1.0, 0.98, 1e-3, 1e-2, sd_pop=1e9)
    assert a1 == a2
    # the step stays within [0.01, 10] x the population SD
    st, _ = oracle.predict_step(np.zeros(5), 1.0, 0.98, 1e-3, 1e-2, sd_pop=1e-3)
    assert st == pytest.approx(1e-2, rel=1e-14)
    st, _ = oracle.predict_step(np.zeros(5), 1.0, 0.02, 1e-3, 1e-2, sd_pop=1e3)
    assert st == pytest.approx(10.0, rel=1e-14)
    # the fitted slope is clamped to [-1, 0]: SDs growing with beta (slope
    # +0.3) predict with slope 0, SDs falling as beta^-1.5 with slope -1.  At
    # rate 1/2 the SD estimate is s tan(pi/4) / 2 = s / 2
    betas, b_next = np.array([1e-3, 1e-2, 1e-1]), 0.3
    wts = np.array([0.25, 0.5, 1.0])
    xs = np.log(betas)
    for gamma, b_used in ((0.3, 0.0), (-1.5, -1.0)):
        sig = 0.5 * betas ** gamma
        xm, ym = wts @ xs / wts.sum(), wts @ np.log(sig) / wts.sum()
        expect = 2.0 * math.exp(ym + b_used * (math.log(b_next) - xm)) / math.tan(0.22 * math.pi)
        h = np.zeros(5)
        for b, sg in zip(betas, sig):
            # population SD = the expected step: the bounds [0.01, 10] x SD do not bind
            st, h = oracle.predict_step(h, 2.0 * sg, 0.5, b, b_next, sd_pop=expect)
        assert st == pytest.approx(expect, rel=1e-12)


def test_predictor_rule_in_runs_evidence_and_rates():
    # the sampler with the history predictor: closed-form evidence of the
    # linear-Gaussian case, and the amplitudes' acceptance rates near 0.44 at
    # the later stages (their tempered posteriors are Gaussian)
    spec = W.linear_gaussian_case(3)
    exact = _lin_gauss_exact(spec)
    vals, late = [], []
    for seed in range(1, 13):
        r = oracle.run_job(spec, 2, W.Options(particles=8000, sweeps=8, seed=seed, step_rule=1))
        assert r["status"] == 0
        vals.append(r["log_z"])
        late.append(r["acc"][-3:, [0, 3]].ravel())
    vals = np.array(vals)
    se = vals.std(ddof=1) / math.sqrt(len(vals))
    print("history predictor log Z: mean", vals.mean(), "exact", exact, "SE", se)
    assert se < 0.015
    assert abs(vals.mean() - exact) < 0.05
    assert abs(np.mean(late) - 0.44) < 0.08
