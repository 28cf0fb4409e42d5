"""The App. D powder-diffraction phase model on the GPU: phases with Caglioti
widths S = a sqrt(u T^2 - v T + w), W = a (s / cos(x/2) + t T), T = tan(x/2),
asymmetry a = alpha right of each reflection, pseudo-Voigt (1 - r) G + r L over
the phase's reference reflections, the PV background a_bg V(x; 0, s, s, r) + b
and the Poisson energy sum [(f - y) - y ln(f / y)] (normaliser in log Z).  The
FP32 path runs in k_mh_phase.cuh and the XRD branch of the energy kernel.

Against the FP64 oracle on the same seeded inputs: FP64 energies relative
1e-12, FP64 Metropolis replays (accept counts equal, states to 1e-9), FP64 full
runs (log Z to 1e-7); FP32 energies within 2e-5 (|E| + N); FP32 runs as an
estimator over seeds (within three combined standard errors of the FP64 path,
printed) with the same selected K, and FP32 energies of final particles within
0.05 nat of FP64 ones."""
import numpy as np
import pytest

import oracle
from paper_2604_03271_b300 import workloads as W

pytestmark = pytest.mark.gpu

TRUTH_NAT = [v for q in W.XRD_TRUTH for v in q] + list(W.XRD_BG_TRUTH)


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_03271_b300 import api
    c = api.Context(0)
    yield c
    c.close()


def _known_sigma(spec):
    """The same phases with the Gaussian known-sigma energy (sigma = sqrt(y + 1))."""
    return W.Spectrum(spec.x, spec.y, np.sqrt(spec.y + 1.0), W.XRD_PHASE, spec.k_min, spec.k_max, W.BG_XRD_PV, 0,
                      spec.priors, truth=spec.truth, name="xrd-known", noise=W.NOISE_KNOWN, refs=spec.refs,
                      phase_priors=spec.phase_priors)


def _no_bg(spec):
    """The phases alone, Poisson counts of the phase signal plus 50."""
    rng = np.random.default_rng(11)
    sig = np.array([sum(oracle.xrd_phase(W.XRD_TRUTH[k], *spec.refs[k], xv) for k in range(3)) for xv in spec.x])
    y = rng.poisson(sig + 50.0).astype(np.float64)
    return W.Spectrum(spec.x, y, np.ones_like(y), W.XRD_PHASE, spec.k_min, spec.k_max, W.BG_NONE, 0,
                      spec.priors, truth={}, name="xrd-nobg", noise=W.NOISE_POISSON, refs=spec.refs,
                      phase_priors=spec.phase_priors)


def _gauss_approx(spec):
    """App. D's Gaussian approximation to the counts (variance = f): the
    model-variance likelihood with (s0, s1, s2) = (1, 0, 0)."""
    return W.Spectrum(spec.x, spec.y, np.ones_like(spec.y), W.XRD_PHASE, spec.k_min, spec.k_max, W.BG_XRD_PV, 0,
                      spec.priors, truth=spec.truth, name="xrd-gauss-approx", noise=W.NOISE_MODEL,
                      noise_par=(1.0, 0.0, 0.0), refs=spec.refs, phase_priors=spec.phase_priors)


def _variants(n=1000, seed=1, K=3):
    full = W.xrd_phase(seed, n=n, k_min=K, k_max=K)
    return [full, _known_sigma(full), _no_bg(full), _gauss_approx(full)]


@pytest.mark.parametrize("which", range(4))
def test_energies_fp64_and_fp32(ctx, which):
    spec = _variants()[which]
    K = spec.k_min
    opts = W.Options(particles=256, seed=5)
    u, E_or = oracle.init_particles(spec, K, opts, 256)
    nat64, E64 = ctx.prior(spec, K, opts, 256, precision=1)
    np.testing.assert_allclose(nat64, u, rtol=1e-12, atol=1e-9)
    fin = np.isfinite(E_or)
    assert np.array_equal(fin, np.isfinite(E64))
    np.testing.assert_allclose(E64[fin], E_or[fin], rtol=1e-12)
    E32 = ctx.energy(spec, K, opts, u, precision=0)
    assert np.all(np.abs(E32[fin] - E_or[fin]) <= 2e-5 * (np.abs(E_or[fin]) + spec.n))
    if which == 0:  # at the truth: about N / 2
        e_or = oracle.energy_spec(spec, 3, TRUTH_NAT)
        assert 0.3 * spec.n < e_or < 0.8 * spec.n
        e_gpu = ctx.energy(spec, 3, opts, np.array([TRUTH_NAT]), precision=1)[0]
        assert e_gpu == pytest.approx(e_or, rel=1e-12)
        e32 = ctx.energy(spec, 3, opts, np.array([TRUTH_NAT]), precision=0)[0]
        assert abs(e32 - e_or) <= 2e-5 * (abs(e_or) + spec.n)


@pytest.mark.parametrize("which,beta", [(0, 1e-3), (1, 1e-2), (2, 1e-3), (3, 1e-3)])
def test_mh_stage_replay_and_tracking(ctx, which, beta):
    spec = _variants(n=300, seed=2, K=2)[which]
    K = 2
    opts = W.Options(particles=64, sweeps=3, seed=9)
    u, E = oracle.init_particles(spec, K, opts, 64)
    ok = np.isfinite(E)
    u, E = u[ok][:48], E[ok][:48]
    step = 0.2 * np.maximum(np.std(u, axis=0), 1e-3)
    u_or, E_or, acc_or, prop_or = oracle.mh_stage(spec, K, opts, u, E, step, beta, 4)
    nat_g, E_g, acc_g, prop_g = ctx.mh_stage(spec, K, opts, u, E, step, beta, 4, precision=1)
    np.testing.assert_array_equal(prop_g, prop_or)
    np.testing.assert_array_equal(acc_g, acc_or)
    np.testing.assert_allclose(nat_g, u_or, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(E_g, E_or, rtol=1e-9)
    assert acc_or.sum() > 0.05 * prop_or.sum()
    # FP32 phase kernel on the same streams
    nat32, E32, acc32, prop32 = ctx.mh_stage(spec, K, opts, u, E, step, beta, 4, precision=0)
    np.testing.assert_array_equal(prop32, prop_or)
    assert np.abs(acc32 - acc_or).sum() <= 0.03 * prop_or.sum() + 3
    E_true = oracle.energies(spec, K, opts, nat32)
    assert np.all(np.abs(E32 - E_true) <= 2e-5 * (np.abs(E_true) + spec.n))


def test_full_run_fp64_replays_oracle(ctx):
    spec = W.xrd_phase(3, n=120, k_min=1, k_max=2)
    opts = W.Options(particles=64, sweeps=3, seed=2)
    ref = oracle.run(spec, opts)
    r = ctx.run(spec, W.Options(particles=64, sweeps=3, seed=2, energy_fp64=1))
    np.testing.assert_allclose(r["log_z"], ref["log_z"], atol=1e-7, rtol=0)
    np.testing.assert_array_equal(r["n_stages"], [j["n_stages"] for j in ref["jobs"]])


def test_fp32_estimator_and_selection(ctx):
    # the three phases on 150 points, K = 2, 3 (the first K listed phases):
    # FP32 batched vs the batched FP64 path over 24 seeds at T = 1024, within
    # three combined standard errors (printed; per-seed SD 0.6-2.7 nat), the
    # same selected K, and the FP32 energies of the final particles within
    # 0.05 nat of FP64 ones (a bound on the difference of the two energy
    # landscapes' evidences)
    from conftest import diff_and_se, estimator_stats
    spec = W.xrd_phase(4, n=150, k_min=2, k_max=3)
    lz32, lz64, k32, k64 = estimator_stats(ctx, spec, range(1, 25), particles=1024, sweeps=3)
    diff, se = diff_and_se(lz32, lz64)
    print("App. D |mean log Z FP32 - FP64| per K", diff, "SE", se)
    assert np.all(diff <= 3 * se), (diff, se)
    assert np.argmax(lz32.mean(0)) == np.argmax(lz64.mean(0)) == 1
    r = ctx.run(spec, W.Options(particles=1024, sweeps=3, seed=1), keep_samples=True)
    for a, K in enumerate(r["K"]):
        nat = r["samples"][a].astype(np.float64)
        eps = ctx.energy(spec, K, W.Options(), nat, precision=0) - ctx.energy(spec, K, W.Options(), nat,
                                                                               precision=1)
        assert np.max(np.abs(eps)) <= 0.05


def test_more_phases_than_listed_is_rejected(ctx):
    from paper_2604_03271_b300 import api
    spec = W.xrd_phase(4, n=200, k_min=1, k_max=4)
    with pytest.raises(api.SmcError):
        ctx.run(spec, W.Options(particles=64, sweeps=2, seed=1))


def test_phase_posterior_means(ctx):
    """Phases keep their order (no sorting): the K = 3 posterior means of the
    amplitudes lie near the truth's on the 1000-point pattern."""
    spec = W.xrd_phase(1, n=1000, k_min=3, k_max=3)
    r = ctx.run(spec, W.Options(particles=4096, sweeps=10, seed=7))
    m = r["post_mean"][0]
    A = m[[0, 9, 18]]
    assert np.all(np.abs(A / np.array([q[0] for q in W.XRD_TRUTH]) - 1.0) < 0.2), A


def test_full_size_sampled_energies(ctx):
    """The App. D-shaped pattern (1000 points, K = 3, 31 parameters, T = 16384,
    10 sweeps): two stages of the FP32 phase kernel, sampled final energies vs
    the oracle."""
    spec = W.xrd_phase(1, k_min=3, k_max=3)
    opts = W.Options(particles=16384, sweeps=10, seed=3, max_stages=2)
    r = ctx.run(spec, opts, keep_samples=True)
    assert r["job_status"][0] == 5 and np.isfinite(r["log_z"][0])
    smp = r["samples"][0].astype(np.float64)
    idx = np.random.default_rng(3).choice(16384, 32, replace=False)
    e64 = np.array([oracle.energy_spec(spec, 3, v) for v in smp[idx]])
    e32 = ctx.energy(spec, 3, opts, smp[idx], precision=0)
    assert np.all(np.abs(e32 - e64) <= 2e-5 * (np.abs(e64) + spec.n))


def test_paper_grid_at_truth(ctx):
    """The largest App. D grid (N = 10000): FP32 and FP64 energies at the truth."""
    spec = W.xrd_phase(5, n=10000, k_min=3, k_max=3)
    opts = W.Options(particles=64, seed=1)
    e_or = oracle.energy_spec(spec, 3, TRUTH_NAT)
    e64 = ctx.energy(spec, 3, opts, np.array([TRUTH_NAT]), precision=1)[0]
    e32 = ctx.energy(spec, 3, opts, np.array([TRUTH_NAT]), precision=0)[0]
    assert e64 == pytest.approx(e_or, rel=1e-12)
    assert abs(e32 - e_or) <= 2e-5 * (abs(e_or) + spec.n)


@pytest.mark.parametrize("J,G", [(4, 24), (8, 32), (8, 128)])
def test_cluster_chains_track_the_oracle(ctx, J, G):
    """A chain spread over a thread-block cluster of G / 8 CTAs (forced on a
    1000-point grid, most CTAs holding padding only at G = 128): the same
    proposals as the oracle, accept counts within the FP32 band, final
    energies equal to the oracle's energies of the returned states."""
    spec = W.xrd_phase(2, n=1000, k_min=2, k_max=2)
    K = 2
    opts = W.Options(particles=64, sweeps=3, seed=9)
    u, E = oracle.init_particles(spec, K, opts, 64)
    ok = np.isfinite(E)
    u, E = u[ok][:40], E[ok][:40]
    step = 0.2 * np.maximum(np.std(u, axis=0), 1e-3)
    u_or, E_or, acc_or, prop_or = oracle.mh_stage(spec, K, opts, u, E, step, 1e-3, 4)
    ctx.clear_tiles()
    ctx.set_tile(W.XRD_PHASE | 16, 1 << 20, J, G)
    try:
        nat32, E32, acc32, prop32 = ctx.mh_stage(spec, K, opts, u, E, step, 1e-3, 4, precision=0)
    finally:
        ctx.clear_tiles()
    np.testing.assert_array_equal(prop32, prop_or)
    assert np.abs(acc32 - acc_or).sum() <= 0.03 * prop_or.sum() + 3
    E_true = oracle.energies(spec, K, opts, nat32)
    assert np.all(np.abs(E32 - E_true) <= 2e-5 * (np.abs(E_true) + spec.n))


def test_cluster_stage_on_a_long_grid(ctx):
    """N = 6000 (three 8-warp CTAs per chain at J = 8): one Metropolis stage
    against the oracle's on the same streams."""
    spec = W.xrd_phase(3, n=6000, k_min=2, k_max=2)
    K = 2
    opts = W.Options(particles=16, sweeps=2, seed=4)
    u, E = oracle.init_particles(spec, K, opts, 16)
    ok = np.isfinite(E)
    u, E = u[ok], E[ok]
    step = 0.2 * np.maximum(np.std(u, axis=0), 1e-3)
    u_or, E_or, acc_or, prop_or = oracle.mh_stage(spec, K, opts, u, E, step, 1e-3, 2)
    nat32, E32, acc32, prop32 = ctx.mh_stage(spec, K, opts, u, E, step, 1e-3, 2, precision=0)
    np.testing.assert_array_equal(prop32, prop_or)
    assert np.abs(acc32 - acc_or).sum() <= 0.03 * prop_or.sum() + 3
    E_true = oracle.energies(spec, K, opts, nat32)
    assert np.all(np.abs(E32 - E_true) <= 2e-5 * (np.abs(E_true) + spec.n))


@pytest.mark.parametrize("n", [5000, 10000])
def test_paper_grid_sizes_sampled(ctx, n):
    """The paper's App. D grids N = 5000 and 10000 (K = 3, T = 8192, n = 10):
    two stages of the cluster-spanning FP32 chains, sampled final energies vs
    the oracle."""
    spec = W.xrd_phase(1, n=n, k_min=3, k_max=3)
    opts = W.Options(particles=8192, sweeps=10, seed=3, max_stages=2)
    r = ctx.run(spec, opts, keep_samples=True)
    assert r["job_status"][0] == 5 and np.isfinite(r["log_z"][0])
    smp = r["samples"][0].astype(np.float64)
    idx = np.random.default_rng(3).choice(8192, 16, replace=False)
    e64 = np.array([oracle.energy_spec(spec, 3, v) for v in smp[idx]])
    e32 = ctx.energy(spec, 3, opts, smp[idx], precision=0)
    assert np.all(np.abs(e32 - e64) <= 2e-5 * (np.abs(e64) + spec.n))


def test_thirteen_phases_without_the_profile_cache(ctx):
    """13 phases (121 parameters, near the 128-component limit) of 5
    reflections each: the profile parts of 13 phases exceed the kernel's
    shared-memory cache, so every shape proposal rebuilds both parts.  One
    FP32 stage against the oracle's on the same streams."""
    rng = np.random.default_rng(21)
    base = W.xrd_phase(6, n=600, k_min=13, k_max=13)
    refs = [(sorted(rng.uniform(22.0, 78.0, 5).tolist()), rng.uniform(0.1, 1.0, 5).tolist()) for _ in range(13)]
    spec = W.Spectrum(base.x, base.y, base.sigma, W.XRD_PHASE, 13, 13, W.BG_XRD_PV, 0, base.priors,
                      truth={}, name="xrd-13", noise=W.NOISE_POISSON, refs=refs, phase_priors=base.phase_priors)
    K = 13
    opts = W.Options(particles=32, sweeps=2, seed=5)
    u, E = oracle.init_particles(spec, K, opts, 32)
    ok = np.isfinite(E)
    u, E = u[ok], E[ok]
    step = 0.2 * np.maximum(np.std(u, axis=0), 1e-3)
    u_or, E_or, acc_or, prop_or = oracle.mh_stage(spec, K, opts, u, E, step, 1e-4, 3)
    nat32, E32, acc32, prop32 = ctx.mh_stage(spec, K, opts, u, E, step, 1e-4, 3, precision=0)
    np.testing.assert_array_equal(prop32, prop_or)
    assert np.abs(acc32 - acc_or).sum() <= 0.03 * prop_or.sum() + 3
    E_true = oracle.energies(spec, K, opts, nat32)
    assert np.all(np.abs(E32 - E_true) <= 2e-5 * (np.abs(E_true) + spec.n))


def test_zero_counts(ctx):
    """Poisson points with y = 0 (term f): FP64 and FP32 energies against the
    oracle, and one FP32 Metropolis stage on the same streams."""
    spec = W.xrd_phase(8, n=400, k_min=2, k_max=2)
    spec.y = spec.y.copy()
    spec.y[::7] = 0.0
    K = 2
    opts = W.Options(particles=64, sweeps=2, seed=3)
    u, E_or = oracle.init_particles(spec, K, opts, 64)
    nat64, E64 = ctx.prior(spec, K, opts, 64, precision=1)
    np.testing.assert_allclose(E64, E_or, rtol=1e-12)
    E32 = ctx.energy(spec, K, opts, u, precision=0)
    assert np.all(np.abs(E32 - E_or) <= 2e-5 * (np.abs(E_or) + spec.n))
    step = 0.2 * np.maximum(np.std(u, axis=0), 1e-3)
    u_or, Es_or, acc_or, prop_or = oracle.mh_stage(spec, K, opts, u[:32], E_or[:32], step, 1e-3, 2)
    nat32, Es32, acc32, prop32 = ctx.mh_stage(spec, K, opts, u[:32], E_or[:32], step, 1e-3, 2, precision=0)
    np.testing.assert_array_equal(prop32, prop_or)
    assert np.abs(acc32 - acc_or).sum() <= 0.03 * prop_or.sum() + 3
    E_true = oracle.energies(spec, K, opts, nat32)
    assert np.all(np.abs(Es32 - E_true) <= 2e-5 * (np.abs(E_true) + spec.n))


@pytest.mark.parametrize("bad", ["negative_intensity", "too_many_reflections", "empty_phase", "shirley_background",
                                 "poisson_negative_count"])
def test_invalid_phase_requests_are_rejected(ctx, bad):
    from paper_2604_03271_b300 import api
    spec = W.xrd_phase(4, n=200, k_min=1, k_max=2)
    refs = [(list(p), list(i)) for p, i in spec.refs]
    if bad == "negative_intensity":
        refs[0][1][0] = -0.5
    elif bad == "too_many_reflections":
        refs[1] = (list(np.linspace(21.0, 79.0, 65)), [1.0] * 65)
    elif bad == "empty_phase":
        refs[0] = ([], [])
    elif bad == "shirley_background":
        spec.bg = W.BG_SHIRLEY
    else:
        spec.y = spec.y.copy()
        spec.y[3] = -1.0
    spec.refs = refs
    if bad == "poisson_negative_count":
        # the counts are checked on the device by the spectrum preparation:
        # the request completes with every job marked invalid
        r = ctx.run(spec, W.Options(particles=64, sweeps=2, seed=1))
        assert r["status"] != api.SMC_OK
        if r["job_status"] is not None:
            assert np.all(r["job_status"] == api.SMC_EINVAL)
        return
    with pytest.raises(api.SmcError):
        ctx.run(spec, W.Options(particles=64, sweeps=2, seed=1))
