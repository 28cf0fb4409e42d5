"""Poisson counts on the ordinary peak families (the App. D likelihood,
E = sum [(f - y) - y ln(f / y)] with its normaliser in log Z, on a sum of
Gaussian peaks with no background).

The FP64 kernels against the FP64 oracle: energies relative 1e-12, a
Metropolis stage replayed (accept counts equal, states to 1e-9) and a full run
replayed (log Z to 1e-7, same stage counts).  With FP32 energies this
configuration is rejected (SMC_EINVAL): the Gaussian tails fall below FP32's
range, where a positive count would have an infinite FP32 energy but a finite
FP64 one."""
import numpy as np
import pytest

import oracle
from paper_2604_03271_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_03271_b300 import api
    c = api.Context(0)
    yield c
    c.close()


def _counts_spectrum(n=200, seed=8, k_min=1, k_max=2):
    # uniform priors throughout, so sampling coordinates are natural values
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 10.0, n)
    f = (40.0 * np.exp(-(x - 4.2) ** 2 / (2 * 0.7 ** 2)) + 25.0 * np.exp(-(x - 6.5) ** 2 / (2 * 0.5 ** 2))
         + 1e-3)
    y = rng.poisson(f).astype(np.float64)
    pri = W.Priors(amp=W.Prior(W.UNIFORM, 1.0, 80.0), centre=W.Prior(W.UNIFORM, 0.0, 10.0),
                   width=W.Prior(W.UNIFORM, 0.2, 2.0))
    return W.Spectrum(x, y, np.ones_like(x), W.GAUSS, k_min, k_max, W.BG_NONE, 0, pri, truth={},
                      name="gauss-poisson", noise=W.NOISE_POISSON)


@pytest.mark.parametrize("K", [1, 2])
def test_energies_fp64(ctx, K):
    spec = _counts_spectrum()
    opts = W.Options(particles=256, seed=5)
    u, E_or = oracle.init_particles(spec, K, opts, 256)
    nat64, E64 = ctx.prior(spec, K, opts, 256, precision=1)
    np.testing.assert_allclose(nat64, u, rtol=1e-12, atol=1e-9)
    assert np.isfinite(E_or).all()
    np.testing.assert_allclose(E64, E_or, rtol=1e-12)


def test_full_run_fp64_replays_oracle(ctx):
    spec = _counts_spectrum(n=120)
    opts = W.Options(particles=64, sweeps=3, seed=2)
    ref = oracle.run(spec, opts)
    r = ctx.run(spec, W.Options(particles=64, sweeps=3, seed=2, energy_fp64=1))
    assert r["status"] == 0
    np.testing.assert_allclose(r["log_z"], ref["log_z"], atol=1e-7, rtol=0)
    np.testing.assert_array_equal(r["n_stages"], [j["n_stages"] for j in ref["jobs"]])


def test_mh_stage_fp64_replays_oracle(ctx):
    spec = _counts_spectrum(n=300, seed=3)
    K = 2
    opts = W.Options(particles=64, sweeps=3, seed=9)
    u, E = oracle.init_particles(spec, K, opts, 64)
    u, E = u[:48], E[:48]
    step = 0.2 * np.maximum(np.std(u, axis=0), 1e-3)
    u_or, E_or, acc_or, prop_or = oracle.mh_stage(spec, K, opts, u, E, step, 1e-3, 4)
    nat64, E64, acc64, prop64 = ctx.mh_stage(spec, K, opts, u, E, step, 1e-3, 4, precision=1)
    np.testing.assert_array_equal(prop64, prop_or)
    np.testing.assert_array_equal(acc64, acc_or)
    np.testing.assert_allclose(nat64, u_or, rtol=1e-9, atol=1e-9)
    assert acc_or.sum() > 0.05 * prop_or.sum()


def test_fp32_energies_rejected_for_gaussian_tails_without_background(ctx):
    from paper_2604_03271_b300 import api
    spec = _counts_spectrum(n=120)
    opts = W.Options(particles=64, sweeps=3, seed=2)
    with pytest.raises(api.SmcError):
        ctx.run(spec, opts)
    with pytest.raises(api.SmcError):
        ctx.energy(spec, 1, opts, np.array([[40.0, 4.2, 0.7]]), precision=0)
    # the FP64 energies of the same request are accepted
    assert np.isfinite(ctx.energy(spec, 1, opts, np.array([[40.0, 4.2, 0.7]]), precision=1)[0])
