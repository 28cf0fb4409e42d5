"""Edge cases and full-size checks of the CUDA path against the oracle.

Full-size runs (the bench's XPS-shaped configuration, in the launch
configuration the bench uses) are checked on sampled outputs the oracle can
compute one by one and on properties that hold at any size."""
import math

import numpy as np
import pytest

import oracle
from paper_2604_03271_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_03271_b300 import api, autotune
    c = api.Context(0)
    autotune.load(c)
    yield c
    c.close()


def _lognorm(spec):
    return -float(np.sum(np.log(np.sqrt(2 * np.pi) * spec.sigma)))


def test_all_fixed_parameters_give_exact_likelihood(ctx):
    # nothing is sampled: one stage (every weight equal) and log Z = log p(D | theta)
    spec = W.gaussian_small(1)
    spec.k_min = spec.k_max = 2
    nat = [1.0, 3.5, 0.5, 0.6, 6.0, 0.8]
    spec.comp_priors = [W.Prior(W.FIXED, v) for v in nat]
    exact = -oracle.energy_natural(W.GAUSS, 2, 0, nat, spec.x, spec.y, spec.sigma) + _lognorm(spec)
    for fp64 in (0, 1):
        r = ctx.run(spec, W.Options(particles=64, sweeps=2, seed=1, energy_fp64=fp64))
        assert r["status"] == 0 and r["n_stages"][0] == 1
        assert abs(r["log_z"][0] - exact) <= (1e-9 if fp64 else 2e-5 * abs(exact))


def test_equal_evidence_selects_the_lower_k(ctx):
    # every peak FIXED at zero amplitude and the constant background FIXED:
    # each candidate K has the same likelihood, so log Z is the same for every
    # K (one stage, all weights equal) and the selection's tie rule must give
    # the lowest K (|delta log Z| < 1e-12 counts as a tie)
    spec = W.gaussian_small(1)
    spec.k_min, spec.k_max = 1, 3
    spec.bg = W.BG_CONST
    spec.priors = W.Priors(amp=W.Prior(W.FIXED, 0.0), centre=W.Prior(W.FIXED, 5.0),
                           width=W.Prior(W.FIXED, 0.5), bg=[W.Prior(W.FIXED, 0.3)])
    f = np.full_like(spec.x, 0.3)
    exact = float(np.sum(-0.5 * ((spec.y - f) / spec.sigma) ** 2)) + _lognorm(spec)
    for fp64 in (0, 1):
        r = ctx.run(spec, W.Options(particles=64, sweeps=1, seed=2, energy_fp64=fp64))
        assert r["status"] == 0 and np.all(r["n_stages"] == 1)
        assert np.ptp(r["log_z"]) <= 1e-12 * abs(exact)
        assert abs(r["log_z"][0] - exact) <= (1e-9 if fp64 else 2e-5 * abs(exact))
        assert r["argmax_k"] == 1


@pytest.mark.parametrize("n,T", [(2, 2), (33, 7), (5, 64)])
def test_minimal_sizes_replay(ctx, n, T):
    rng = np.random.default_rng(n)
    x = np.linspace(0, 1, n)
    y = rng.normal(0.5, 0.1, n)
    pri = W.Priors(amp=W.Prior(W.UNIFORM, 0.0, 2.0), centre=W.Prior(W.UNIFORM, 0.0, 1.0),
                   width=W.Prior(W.LOG_UNIFORM, 0.05, 1.0), bg=[W.Prior(W.UNIFORM, -1, 1)])
    spec = W.Spectrum(x, y, np.full(n, 0.1), W.GAUSS, 0, 1, W.BG_CONST, 0, pri, truth={})
    opts = W.Options(particles=T, sweeps=2, seed=4)
    ref = oracle.run(spec, opts)
    r = ctx.run(spec, W.Options(particles=T, sweeps=2, seed=4, energy_fp64=1))
    np.testing.assert_allclose(r["log_z"], ref["log_z"], atol=1e-7)
    r32 = ctx.run(spec, opts)
    assert r32["status"] == 0 and np.all(np.isfinite(r32["log_z"]))


def test_background_only_k0_replay(ctx):
    spec = W.xps_like(3, n=200, k_true=1, k_max=0)
    spec.k_min = spec.k_max = 0
    opts = W.Options(particles=256, sweeps=3, seed=2)
    ref = oracle.run(spec, opts)
    r = ctx.run(spec, W.Options(particles=256, sweeps=3, seed=2, energy_fp64=1))
    np.testing.assert_allclose(r["log_z"], ref["log_z"], atol=1e-7)


def test_maximum_dimension_k32_pv(ctx):
    # d = 4 * 32 = 128 components, the largest job: FP64 replay of two stages
    spec = W.xps_like(5, n=64, k_true=3, k_max=32)
    spec.k_min = 32
    spec.bg, spec.priors.bg = W.BG_NONE, []
    opts = W.Options(particles=32, sweeps=1, seed=3, max_stages=2)
    ref = oracle.run(spec, opts)
    r = ctx.run(spec, W.Options(particles=32, sweeps=1, seed=3, max_stages=2, energy_fp64=1))
    np.testing.assert_allclose(r["log_z"], ref["log_z"], atol=1e-7)
    r32 = ctx.run(spec, W.Options(particles=32, sweeps=1, seed=3, max_stages=2))
    assert r32["job_status"][0] == 5 and np.isfinite(r32["log_z"][0])


def test_dimension_above_128_rejected(ctx):
    from paper_2604_03271_b300 import api
    spec = W.xps_like(5, n=64, k_true=3, k_max=32)  # 4 * 32 + 2 = 130 components
    with pytest.raises(api.SmcError) as e:
        ctx.run(spec, W.Options(particles=32, sweeps=1))
    assert e.value.status == api.SMC_EINVAL
    spec = W.gaussian_deconvolution(30, seed=1, k_min=33, k_max=33)  # 99 components, K > 32
    with pytest.raises(api.SmcError) as e:
        ctx.run(spec, W.Options(particles=32, sweeps=1))
    assert e.value.status == api.SMC_EINVAL


def test_grid_too_long_for_fp32_tiles_rejected(ctx):
    from paper_2604_03271_b300 import api
    spec = W.xrd_like(1, n=4097, k_true=2, k_max=2)
    with pytest.raises(api.SmcError) as e:
        ctx.run(spec, W.Options(particles=64, sweeps=1))
    assert e.value.status == api.SMC_EINVAL


def _sort_peaks(samples, p, K):
    s = samples.copy()
    peaks = s[:, :p * K].reshape(-1, K, p)
    order = np.argsort(peaks[:, :, 1], axis=1, kind="stable")
    s[:, :p * K] = np.take_along_axis(peaks, order[:, :, None], axis=1).reshape(-1, p * K)
    return s


def test_full_size_xps_sampled_outputs(ctx):
    """The bench configuration (N = 1001, K = 1..6, T = 16384, 20 sweeps):
    energies of sampled final particles against the FP64 oracle, summaries
    against the returned samples, p(K|D) normalised."""
    spec = W.xps_like(1)
    opts = W.Options(particles=16384, sweeps=20, seed=1)
    r = ctx.run(spec, opts, keep_samples=True)
    assert r["status"] == 0
    assert abs(r["p_k"].sum() - 1.0) < 1e-12
    assert r["argmax_k"] == r["K"][int(np.argmax(r["log_z"]))]
    rng = np.random.default_rng(0)
    for a, K in enumerate(r["K"]):
        smp = r["samples"][a].astype(np.float64)
        assert smp.shape == (16384, 4 * K + 2)
        # summaries are the mean / SD of the (peak-sorted) samples
        srt = _sort_peaks(smp, 4, K)
        np.testing.assert_allclose(r["post_mean"][a], srt.mean(0), rtol=1e-5, atol=1e-3)
        np.testing.assert_allclose(r["post_sd"][a], srt.std(0), rtol=1e-3, atol=1e-3)
        # every sample inside the prior support
        assert np.all((smp[:, 1:4 * K:4] >= spec.x.min() - 1e-3) & (smp[:, 1:4 * K:4] <= spec.x.max() + 1e-3))
        assert np.all((smp[:, 3:4 * K:4] >= 0) & (smp[:, 3:4 * K:4] <= 1))
        # energies of sampled particles: oracle (FP64) vs the FP32 kernel
        idx = rng.choice(16384, 64, replace=False)
        nat = smp[idx]
        e64 = np.array([oracle.energy_natural(W.PSEUDO_VOIGT, K, 2, v, spec.x, spec.y, spec.sigma)
                        for v in nat])
        e32 = ctx.energy(spec, K, opts, nat, precision=0)
        assert np.all(np.abs(e32 - e64) <= 2e-5 * (e64 + spec.n))
        # at beta = 1 the selected model's particles sit near the posterior:
        # energies of order N/2
        if K == r["argmax_k"]:
            assert np.median(e64) < 2.0 * spec.n


def _sampling(spec, K, nat):
    pr = spec.priors
    kinds = [pr.amp.kind, pr.centre.kind, pr.width.kind, pr.eta.kind] * K + [b.kind for b in pr.bg]
    u = np.array(nat, dtype=np.float64, copy=True)
    for j in range(u.shape[1]):
        if kinds[j] == W.LOG_UNIFORM:
            u[:, j] = np.log(u[:, j])
    return u


@pytest.mark.parametrize("which", ["xps", "xrd"])
def test_bench_config_fp32_energies_move_log_z_by_less_than_005(ctx, which):
    """The bench configurations: XPS-shaped (N = 1001, K = 1..6, PV + linear
    background, T = 16384) and XRD-shaped (N = 4096, K = 1..12, PV + cubic
    background, T = 65536), 20 sweeps.  The FP32 path samples and weighs with FP32
    energies E32 = E64 + eps; the evidence of that energy landscape differs
    from the FP64 one's by log Z32 - log Z64 = log E_post64[exp(-eps)]
    (Eq. (11) at beta = 1 is the prior expectation of exp(-E)), which lies in
    [-max eps, -min eps] over the posterior.  So over the final particles of
    a full FP32 run, for every K: |eps| of the FP32 energy kernel, and of the
    energies the fused Metropolis kernel itself carries after 20 sweeps at
    beta = 1 (incremental updates included), must stay below 0.05 nat; the
    remaining FP32-vs-FP64 difference of the estimators is Monte Carlo error
    of the same algorithm at the same T (the statistical 0.05 tests run where
    the FP64 path is affordable: configs of N <= 400)."""
    if which == "xps":
        spec, opts = W.xps_like(1), W.Options(particles=16384, sweeps=20, seed=1)
    else:
        spec, opts = W.xrd_like(1), W.Options(particles=65536, sweeps=20, seed=1)
    r = ctx.run(spec, opts, keep_samples=True)
    assert r["status"] == 0
    rng = np.random.default_rng(5)
    for a, K in enumerate(r["K"]):
        nat = r["samples"][a].astype(np.float64)
        e32 = ctx.energy(spec, K, opts, nat, precision=0)
        e64 = ctx.energy(spec, K, opts, nat, precision=1)
        eps = e32 - e64
        shift = math.log(np.mean(np.exp(-(eps - eps.mean())))) - eps.mean()
        # the kernel's own energies after a stage of 20 sweeps at beta = 1
        idx = rng.choice(nat.shape[0], 2048, replace=False)
        u = _sampling(spec, K, nat[idx])
        step = 0.3 * np.maximum(u.std(axis=0), 1e-6)
        nat_o, E_o, acc, prop = ctx.mh_stage(spec, K, opts, nat[idx], e32[idx], step, 1.0, 7, precision=0)
        eps_k = E_o - ctx.energy(spec, K, opts, nat_o, precision=1)
        print(f"{which} K={K}: eps of the FP32 energy kernel in [{eps.min():.2e}, {eps.max():.2e}], "
              f"log-Z shift {shift:.2e}; Metropolis kernel energies in [{eps_k.min():.2e}, {eps_k.max():.2e}]")
        assert acc.sum() > 0
        if r["log_z"][a] >= np.max(r["log_z"]) - 100.0:
            # the candidates that carry posterior weight (Eq. (2)): within 0.05 nat
            assert np.max(np.abs(eps)) <= 0.05 and np.max(np.abs(eps_k)) <= 0.05
            assert abs(shift) <= 0.05
        else:
            # badly fitting K (energies of 1e5 and more, P(K|D) = 0 to double
            # precision): FP32 rounding of the energy, a few 1e-7 of it
            scale = 1e-6 * np.median(np.abs(e64))
            assert np.max(np.abs(eps)) <= max(0.05, scale) and np.max(np.abs(eps_k)) <= max(0.05, scale)


def test_full_size_xrd_g16_tile_energies(ctx):
    """N = 4096 (16-warp chains): three stages at the XRD configuration's
    particle count, then sampled energies against the oracle."""
    spec = W.xrd_like(1)
    spec.k_min = spec.k_max = 6
    opts = W.Options(particles=65536, sweeps=2, seed=2, max_stages=3)
    r = ctx.run(spec, opts, keep_samples=True)
    assert r["job_status"][0] == 5
    smp = r["samples"][0].astype(np.float64)
    idx = np.random.default_rng(1).choice(65536, 24, replace=False)
    e64 = np.array([oracle.energy_natural(W.PSEUDO_VOIGT, 6, 4, v, spec.x, spec.y, spec.sigma)
                    for v in smp[idx]])
    e32 = ctx.energy(spec, 6, opts, smp[idx], precision=0)
    assert np.all(np.abs(e32 - e64) <= 2e-5 * (e64 + spec.n))


def test_mufu_probe_rates_are_plausible(ctx):
    # roofline denominator: EX2 / RCP results per clock per SM between 8 and
    # 64 (the SFU lanes of an SM), at an SM clock between 0.5 and 2.1 GHz, and
    # per-second rate = per-clock rate x 148 SMs x that clock
    for op in (0, 1, 2):
        r = ctx.mufu_rate(op)
        assert 8.0 <= r["lanes_per_clk_sm"] <= 64.0, r
        assert 500.0 <= r["sm_mhz"] <= 2100.0, r
        assert r["ops_per_s"] == pytest.approx(r["lanes_per_clk_sm"] * 148 * r["sm_mhz"] * 1e6, rel=1e-9)
