"""Host-side marshalling of the Python binding (no GPU): the one-call form's
spectrum record."""
import numpy as np

from paper_2604_03271_b300 import api
from paper_2604_03271_b300 import workloads as W


def _priors(bg=None):
    return W.Priors(amp=W.Prior(W.GAMMA, 2.0, 1.0), centre=W.Prior(W.UNIFORM, 0.0, 10.0),
                    width=W.Prior(W.LOG_UNIFORM, 0.1, 3.0), bg=list(bg or []))


def test_make_spectrum_fields():
    x = np.linspace(0.0, 10.0, 50)
    y = np.sin(x) + 2.0
    s = api.make_spectrum(x, y, 0.05, range(1, 7), W.PSEUDO_VOIGT, _priors())
    assert (s.k_min, s.k_max, s.family, s.bg, s.bg_degree) == (1, 6, W.PSEUDO_VOIGT, W.BG_NONE, 0)
    assert s.sigma.shape == x.shape and np.all(s.sigma == 0.05)
    assert s.x.dtype == np.float64 and s.x.flags.c_contiguous and s.sigma.flags.c_contiguous
    assert s.noise == W.NOISE_KNOWN and s.comp_priors is None and not s.priors.bg
    # a (k_min, k_max) pair and per-point sigma
    sig = np.full(50, 0.1)
    s2 = api.make_spectrum(x.tolist(), y, sig, (2, 5), W.GAUSS, _priors())
    assert (s2.k_min, s2.k_max) == (2, 5)
    np.testing.assert_array_equal(s2.sigma, sig)


def test_make_spectrum_background_priors():
    x = np.linspace(0.0, 10.0, 50)
    y = 3.0 + 0.1 * x
    # none given: uniform priors from the data range, one per coefficient
    s = api.make_spectrum(x, y, 0.05, (1, 2), W.GAUSS, _priors(), bg=W.BG_LINEAR)
    assert s.priors.bg == W.data_bg_priors(y, 2)
    s3 = api.make_spectrum(x, y, 0.05, (1, 2), W.GAUSS, _priors(), bg=W.BG_POLY, bg_degree=3)
    assert len(s3.priors.bg) == 4
    # given: kept as they are
    mine = [W.Prior(W.UNIFORM, -1.0, 1.0), W.Prior(W.UNIFORM, -2.0, 2.0)]
    s2 = api.make_spectrum(x, y, 0.05, (1, 2), W.GAUSS, _priors(mine), bg=W.BG_LINEAR)
    assert s2.priors.bg == mine
