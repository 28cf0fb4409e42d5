"""Seeded synthetic inputs: spectra, priors and sampler options.

This module only *makes inputs*.  It holds none of the sampler's arithmetic
(no energy, tempering, resampling or Metropolis code) and imports neither the
CUDA binding nor the oracle, so both sides can be fed from it.  The peak shapes
used to synthesise the data are written out here with numpy, independently of
the oracle and of the kernels.

Workload shapes follow the paper's experiments: a Gaussian-peak deconvolution
spectrum (Sec. III A 2, App. C), an XPS-like pseudo-Voigt spectrum on a
binding-energy axis (App. E, Eq. (E1)) and an XRD-like sparse Lorentzian /
pseudo-Voigt pattern on a 2-theta axis (App. D).  The measured spectra of the
paper are not available; these seeded generators stand in for them.

Parameter conventions (shared by the C ABI):
  family 0 GAUSS   : A exp(-(x-mu)^2 / (2 w^2)),        w = standard deviation
  family 3 GAUSS_PRECISION : A exp(-b (x-mu)^2 / 2),    b = precision (App. C Eq. (C1))
  family 1 LORENTZ : A g^2 / (g^2 + (x-mu)^2),           g = HWHM
  family 2 PV      : A [eta 2^(-(x-mu)^2/s^2) + (1-eta) s^2/(s^2+(x-mu)^2)],
                     s = shared HWHM, eta = Gaussian fraction (Eq. (E1))
  background       : sum_j c_j T_j(t), T_j Chebyshev, t = x scaled to [-1, 1],
                     or Shirley a + (b - a) C(x)/C(x_last) (App. E), C the running
                     integral of the peak signal from the first point
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

GAUSS, LORENTZ, PSEUDO_VOIGT, GAUSS_PRECISION, XRD_PHASE = 0, 1, 2, 3, 4
BG_NONE, BG_CONST, BG_LINEAR, BG_POLY, BG_SHIRLEY, BG_XRD_PV = 0, 1, 2, 3, 4, 5
NOISE_KNOWN, NOISE_MODEL, NOISE_POISSON = 0, 1, 2
UNIFORM, LOG_UNIFORM, NORMAL, GAMMA, FIXED = 0, 1, 2, 3, 4


@dataclasses.dataclass
class Prior:
    kind: int
    p1: float = 0.0
    p2: float = 0.0


@dataclasses.dataclass
class Priors:
    amp: Prior
    centre: Prior
    width: Prior
    eta: Prior = dataclasses.field(default_factory=lambda: Prior(UNIFORM, 0.0, 1.0))
    bg: List[Prior] = dataclasses.field(default_factory=list)


@dataclasses.dataclass
class Options:
    particles: int = 1024
    ess_target: float = 0.5
    sweeps: int = 10
    waste_free: int = 0
    energy_fp64: int = 0
    seed: int = 1
    max_stages: int = 10000
    step_rule: int = 0  # 0: lambda x weighted population SD; 1: history predictor


@dataclasses.dataclass
class Spectrum:
    x: np.ndarray
    y: np.ndarray
    sigma: np.ndarray
    family: int
    k_min: int
    k_max: int
    bg: int
    bg_degree: int
    priors: Priors
    truth: dict
    name: str = ""
    # Optional per-component priors (one per component, in component order);
    # only meaningful when k_min == k_max.  Overrides the shared priors.
    comp_priors: Optional[List[Prior]] = None
    # likelihood: NOISE_KNOWN (sigma per point) or NOISE_MODEL (variance
    # s0^2 f + s1^2 f^2 + s2^2 of the model value f, App. E; sigma unused)
    noise: int = 0
    noise_par: tuple = (0.0, 0.0, 0.0)
    # XRD phase model (App. D): per phase (reference positions, relative
    # intensities), and the shared priors of (A, d2theta, alpha, r, u, v, w, s, t)
    refs: Optional[list] = None
    phase_priors: Optional[List[Prior]] = None

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


# ----------------------------------------------------------------------------
# independent numpy peak synthesis (data generation only)
# ----------------------------------------------------------------------------

def _synth_gauss(x, A, mu, w):
    return A * np.exp(-0.5 * ((x - mu) / w) ** 2)


def _synth_pv(x, A, mu, hwhm, eta):
    t2 = ((x - mu) / hwhm) ** 2
    return A * (eta * np.exp(-math.log(2.0) * t2) + (1.0 - eta) / (1.0 + t2))


def _synth_cheb(x, coeffs):
    t = (2.0 * x - (x.min() + x.max())) / (x.max() - x.min())
    return np.polynomial.chebyshev.chebval(t, coeffs)


def bg_count(bg: int, bg_degree: int) -> int:
    return {BG_NONE: 0, BG_CONST: 1, BG_LINEAR: 2, BG_SHIRLEY: 2, BG_XRD_PV: 4}.get(bg, bg_degree + 1)


def data_bg_priors(y: np.ndarray, nbg: int) -> List[Prior]:
    """Uniform background-coefficient priors derived from the data range."""
    ymin, ymax = float(y.min()), float(y.max())
    dy = ymax - ymin
    out = []
    for j in range(nbg):
        if j == 0:
            out.append(Prior(UNIFORM, ymin - 0.2 * dy, ymin + 0.5 * dy))
        else:
            out.append(Prior(UNIFORM, -0.5 * dy, 0.5 * dy))
    return out


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------

# App. C: the paper's Gaussian spectral-deconvolution data.  Grid and noise per
# K (Table "experimental conditions"), the printed true (A_k, mu_k, b_k) per K
# (Tables of true parameter values) and the sweeps per stage (Sec. III A 2).
DECONV_GRID = {3: (300, 3.0, 0.1), 10: (1000, 10.0, 0.1), 30: (3000, 30.0, 0.05)}
DECONV_SWEEPS = {3: 10, 10: 10, 30: 100}
DECONV_TRUTH = {
    3: [(0.587, 1.210, 95.689), (1.522, 1.455, 146.837), (1.183, 1.703, 164.469)],
    10: [(1.049, 0.558, 114.335), (1.215, 2.082, 194.467), (1.103, 2.804, 152.185),
         (1.045, 3.549, 141.466), (0.924, 4.678, 126.456), (1.146, 5.633, 177.423),
         (0.938, 7.098, 145.615), (1.392, 7.418, 156.843), (1.464, 8.625, 101.879),
         (0.883, 9.158, 161.764)],
    30: [(0.576, 0.486, 105.313), (1.280, 1.065, 130.885), (0.938, 2.378, 159.259),
         (1.223, 2.814, 123.512), (1.478, 4.815, 196.497), (1.038, 5.375, 194.505),
         (1.001, 6.277, 184.840), (0.572, 7.822, 147.232), (0.768, 8.005, 184.148),
         (1.000, 9.661, 113.111), (1.179, 9.881, 130.873), (1.304, 11.301, 146.300),
         (0.881, 12.139, 174.185), (0.566, 13.939, 148.583), (0.788, 15.030, 113.688),
         (1.410, 15.401, 134.354), (0.713, 16.752, 132.443), (0.952, 17.446, 130.042),
         (1.431, 18.670, 116.550), (0.525, 19.274, 141.490), (1.101, 19.987, 144.812),
         (1.450, 20.959, 177.490), (0.730, 22.615, 179.639), (1.048, 24.174, 152.239),
         (1.409, 24.581, 146.063), (0.633, 25.343, 177.821), (1.023, 27.074, 188.729),
         (1.250, 27.571, 167.492), (1.169, 28.530, 180.048), (0.968, 29.576, 193.911)],
}


def deconv_priors(K: int) -> Priors:
    """App. C prior table: A ~ Ga(5, 5), b ~ Ga(5, 0.04) (shape, rate); the
    centre ~ N(1.5, variance 0.2) at K = 3, U over the x range otherwise."""
    L = DECONV_GRID[K][1]
    centre = Prior(NORMAL, 1.5, math.sqrt(0.2)) if K == 3 else Prior(UNIFORM, 0.0, L)
    return Priors(amp=Prior(GAMMA, 5.0, 5.0), centre=centre, width=Prior(GAMMA, 5.0, 0.04))


def gaussian_deconvolution(K: int = 10, seed: int = 0, k_min: Optional[int] = None,
                           k_max: Optional[int] = None, n: Optional[int] = None) -> Spectrum:
    """The paper's Gaussian-peak deconvolution spectrum with K true peaks
    (K in 3, 10, 30), precision-parameterised, on N equally spaced points of
    [0, L] with known noise sd; the noise is drawn from `seed` (the paper's
    noise draws are not given).  Candidate range defaults to K alone.  `n`
    overrides the point count (same x range) for small test cases."""
    N, L, sd = DECONV_GRID[K]
    N = n or N
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, L, N)
    f = np.zeros_like(x)
    for A, mu, b in DECONV_TRUTH[K]:
        f += _synth_gauss(x, A, mu, 1.0 / math.sqrt(b))
    y = f + rng.normal(0.0, sd, size=x.shape)
    t = DECONV_TRUTH[K]
    return Spectrum(x, y, np.full_like(x, sd), GAUSS_PRECISION, K if k_min is None else k_min,
                    K if k_max is None else k_max, BG_NONE, 0,
                    deconv_priors(K),
                    truth={"K": K, "A": [a for a, _, _ in t], "mu": [m for _, m, _ in t],
                           "b": [b for _, _, b in t]},
                    name=f"deconv-K{K}-{N}")


def gaussian_small(seed: int = 1) -> Spectrum:
    """301-point, two-Gaussian spectrum on [0, 10], noise sd 0.05, K in 1..3.

    Truth: (A, mu, sd) = (1.0, 3.5, 0.5) and (0.6, 6.0, 0.8).  Priors:
    centre ~ U[0, 10], log sd ~ U[log 0.1, log 3], amplitude ~ Gamma(2, 1)
    (shape, rate).
    """
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 10.0, 301)
    f = _synth_gauss(x, 1.0, 3.5, 0.5) + _synth_gauss(x, 0.6, 6.0, 0.8)
    y = f + rng.normal(0.0, 0.05, size=x.shape)
    pri = Priors(amp=Prior(GAMMA, 2.0, 1.0), centre=Prior(UNIFORM, 0.0, 10.0),
                 width=Prior(LOG_UNIFORM, 0.1, 3.0))
    return Spectrum(x, y, np.full_like(x, 0.05), GAUSS, 1, 3, BG_NONE, 0, pri,
                    truth={"K": 2, "A": [1.0, 0.6], "mu": [3.5, 6.0], "w": [0.5, 0.8]},
                    name="gauss-301")


def xps_like(seed: int = 1, n: int = 1001, k_true: int = 4, k_max: int = 6,
             scale: float = 1.0e4) -> Spectrum:
    """XPS-shaped pseudo-Voigt spectrum on a 20 eV binding-energy axis at 280 eV.

    k_true peaks with eta ~ U[0, 1], FWHM ~ U[0.8, 2.0] eV, amplitude
    S 10^U[-1, 0] (S = scale counts), centres ~ U[283, 297] at least 1 eV apart;
    linear background 0.1 S + 0.002 S/eV (x - 280); variance f + (0.01 S)^2
    (counting-like plus a floor).  Fitted with PV peaks + linear background,
    K = 1..k_max.
    """
    rng = np.random.default_rng(seed)
    x = 280.0 + np.linspace(0.0, 20.0, n)
    mus: List[float] = []
    while len(mus) < k_true:
        m = rng.uniform(283.0, 297.0)
        if all(abs(m - o) >= 1.0 for o in mus):
            mus.append(m)
    mus.sort()
    eta = rng.uniform(0.0, 1.0, k_true)
    fwhm = rng.uniform(0.8, 2.0, k_true)
    amp = scale * 10.0 ** rng.uniform(-1.0, 0.0, k_true)
    f = 0.1 * scale + 0.002 * scale * (x - 280.0)
    for k in range(k_true):
        f = f + _synth_pv(x, amp[k], mus[k], 0.5 * fwhm[k], eta[k])
    var = f + (0.01 * scale) ** 2
    y = f + np.sqrt(var) * rng.normal(size=x.shape)
    sig = np.sqrt(var)
    ymin, ymax = float(y.min()), float(y.max())
    pri = Priors(amp=Prior(LOG_UNIFORM, 1e-3 * (ymax - ymin), 2.0 * ymax),
                 centre=Prior(UNIFORM, float(x.min()), float(x.max())),
                 width=Prior(LOG_UNIFORM, 0.2, 3.0),
                 eta=Prior(UNIFORM, 0.0, 1.0),
                 bg=data_bg_priors(y, 2))
    return Spectrum(x, y, sig, PSEUDO_VOIGT, 1, k_max, BG_LINEAR, 1, pri,
                    truth={"K": k_true, "A": amp.tolist(), "mu": mus,
                           "hwhm": (0.5 * fwhm).tolist(), "eta": eta.tolist()},
                    name=f"xps-{n}")


def _synth_shirley(x, peaks, a, b):
    """Shirley background a + (b - a) C(x)/C(x_last), C the running integral of
    the peak signal from the first point (right-end rectangle rule)."""
    inc = np.zeros_like(x)
    inc[1:] = peaks[1:] * np.abs(np.diff(x))
    c = np.cumsum(inc)
    return a + (b - a) * c / c[-1] if c[-1] > 0 else np.full_like(x, a)


def xps_shirley(seed: int = 1, n: int = 840, k_true: int = 7, k_min: int = 5, k_max: int = 8,
                scale: float = 3.0e4) -> Spectrum:
    """XPS spectrum of the App. E kind: a Ni 2p-like core level on 840 points of
    binding energy 845-887 eV (the paper's measured grid), pseudo-Voigt peaks on
    a Shirley background, noise of variance f + (0.01 f)^2 (App. E with
    sigma_0 = 1, sigma_1 = 0.01, sigma_2 = 0), and the paper's data-derived
    uniform priors (App. E prior table).  Peaks: two spin-orbit groups 17.3 eV
    apart (main line, a second chemical state +2.7 eV, a satellite +6 eV) and
    one weak feature between them; HWHM 0.6-2.0 eV, eta ~ U[0.4, 0.9], amplitudes
    S 10^U[-0.8, 0]; Shirley start 0.3 S, end 0.9 S.  The measured spectrum is
    not available; this stands in for it."""
    rng = np.random.default_rng(seed)
    x = np.linspace(845.0, 887.0, n)
    base = [852.6, 855.3, 858.6, 869.9, 872.6, 875.9, 864.5][:k_true]
    mus = [m + rng.uniform(-0.3, 0.3) for m in base]
    hwhm = rng.uniform(0.6, 2.0, len(mus))
    eta = rng.uniform(0.4, 0.9, len(mus))
    amp = scale * 10.0 ** rng.uniform(-0.8, 0.0, len(mus))
    peaks = np.zeros_like(x)
    for k in range(len(mus)):
        peaks += _synth_pv(x, amp[k], mus[k], hwhm[k], eta[k])
    f = peaks + _synth_shirley(x, peaks, 0.3 * scale, 0.9 * scale)
    s0, s1, s2 = 1.0, 0.01, 0.0
    var = s0 ** 2 * f + s1 ** 2 * f ** 2 + s2 ** 2
    y = f + np.sqrt(var) * rng.normal(size=x.shape)
    ymin, ymax = float(y.min()), float(y.max())
    pri = Priors(amp=Prior(UNIFORM, max(0.0, 0.3 * ymin), 1.05 * ymax),
                 centre=Prior(UNIFORM, float(x.min()), float(x.max())),
                 width=Prior(UNIFORM, 0.1, 15.0),
                 eta=Prior(UNIFORM, 0.0, 1.0),
                 bg=[Prior(UNIFORM, 0.95 * float(y[0]), 1.01 * float(y[0])),
                     Prior(UNIFORM, 0.95 * float(y[-1]), 1.01 * float(y[-1]))])
    return Spectrum(x, y, np.ones_like(x), PSEUDO_VOIGT, k_min, k_max, BG_SHIRLEY, 0, pri,
                    truth={"K": len(mus), "A": amp.tolist(), "mu": mus, "hwhm": hwhm.tolist(),
                           "eta": eta.tolist(), "a": 0.3 * scale, "b": 0.9 * scale},
                    name=f"xps-shirley-{n}", noise=NOISE_MODEL, noise_par=(s0, s1, s2))


# App. D stand-in reference reflections (2 theta in degrees for Cu K-alpha,
# relative intensities) of rutile, anatase and brookite: approximate values of
# the common powder patterns, standing in for the crystallographic references
# the paper uses but does not list.
XRD_REFS = [
    ([27.45, 36.09, 39.19, 41.23, 44.05, 54.32, 56.64, 62.74, 64.04, 69.01, 69.79],
     [1.00, 0.50, 0.08, 0.25, 0.10, 0.60, 0.20, 0.10, 0.10, 0.20, 0.12]),
    ([25.28, 36.95, 37.80, 38.58, 48.05, 53.89, 55.06, 62.12, 62.69, 68.76, 70.31, 75.03],
     [1.00, 0.10, 0.20, 0.10, 0.35, 0.20, 0.20, 0.04, 0.14, 0.06, 0.06, 0.10]),
    ([25.34, 25.69, 30.81, 36.25, 37.30, 38.37, 39.21, 40.15, 42.34, 46.07, 48.01, 49.17, 52.02,
      54.20, 55.23, 57.18, 62.06, 63.65, 64.10, 65.01],
     [1.00, 0.80, 0.90, 0.25, 0.18, 0.04, 0.18, 0.18, 0.16, 0.16, 0.30, 0.18, 0.08, 0.20, 0.30,
      0.13, 0.10, 0.12, 0.10, 0.12]),
]
# App. D table of true phase parameters (A, d2theta, alpha, r, u, v, w, s, t) and background
XRD_TRUTH = [(10000.0, 0.035, 0.6, 0.50, 0.03, 0.03, 0.06, 0.06, 0.03),
             (3500.0, 0.055, 0.9, 0.65, 0.1, 0.1, 0.2, 0.2, 0.1),
             (1000.0, 0.04, 1.0, 0.75, 0.1, 0.1, 0.2, 0.2, 0.1)]
XRD_BG_TRUTH = (60000.0, 10.0, 0.0, 100.0)


def _synth_xrd(x, phases, refs, bg):
    """App. D forward model, written out with numpy for data generation."""
    th = np.radians(x / 2.0)
    tn, sc = np.tan(th), 1.0 / np.cos(th)

    def pv(dx, S, W, r):
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.where(S > 0, np.exp(-4.0 * math.log(2.0) * dx * dx / np.where(S > 0, S * S, 1.0)), 0.0)
            l = np.where(W > 0, 1.0 / (1.0 + 4.0 * dx * dx / np.where(W > 0, W * W, 1.0)), 0.0)
        return (1.0 - r) * g + r * l

    f = np.zeros_like(x)
    for q, (pos, inten) in zip(phases, refs):
        A, sh, al, r, u, v, w, s, t = q
        S0 = np.sqrt(np.maximum(u * tn * tn - v * tn + w, 0.0))
        W0 = s * sc + t * tn
        for m, I in zip(pos, inten):
            mu = m + sh
            asym = np.where(x >= mu, al, 1.0)
            f += A * I * pv(x - mu, asym * S0, asym * W0, r)
    a, sbg, rbg, b = bg
    return f + a * pv(x, np.full_like(x, sbg), np.full_like(x, sbg), rbg) + b


def xrd_phase(seed: int = 1, n: int = 1000, k_min: int = 1, k_max: int = 3) -> Spectrum:
    """The paper's XRD artificial data (App. D): rutile, anatase and brookite
    phases (stand-in reference reflections XRD_REFS) with the printed true
    parameters, on n points of 2 theta in [20, 80] degrees, Poisson counts; the
    App. D priors with y_min / y_max from the data; K = number of phases."""
    rng = np.random.default_rng(seed)
    x = np.linspace(20.0, 80.0, n)
    f = _synth_xrd(x, XRD_TRUTH, XRD_REFS, XRD_BG_TRUTH)
    y = rng.poisson(f).astype(np.float64)
    ymin, ymax = float(y.min()), float(y.max())
    phase_pri = [Prior(GAMMA, 4.0, 4.0 / (ymax - ymin)), Prior(NORMAL, 0.0, 0.05), Prior(GAMMA, 5.0, 4.0),
                 Prior(UNIFORM, 0.0, 1.0), Prior(GAMMA, 1.0, 10.0), Prior(GAMMA, 1.0, 10.0),
                 Prior(GAMMA, 2.0, 20.0), Prior(GAMMA, 2.0, 20.0), Prior(GAMMA, 1.0, 10.0)]
    bg = [Prior(GAMMA, 2.0, 1.0 / ymax), Prior(GAMMA, 2.0, 0.4), Prior(UNIFORM, 0.0, 1.0),
          Prior(UNIFORM, ymin - math.sqrt(ymin), ymin + math.sqrt(ymin))]
    pri = Priors(amp=phase_pri[0], centre=phase_pri[1], width=phase_pri[2], bg=bg)
    return Spectrum(x, y, np.ones_like(x), XRD_PHASE, k_min, k_max, BG_XRD_PV, 0, pri,
                    truth={"phases": XRD_TRUTH, "bg": XRD_BG_TRUTH, "K": 3}, name=f"xrd-phase-{n}",
                    noise=NOISE_POISSON, refs=[(list(p), list(i)) for p, i in XRD_REFS],
                    phase_priors=phase_pri)


def xrd_like(seed: int = 1, n: int = 4096, k_true: int = 10, k_max: int = 12) -> Spectrum:
    """XRD-shaped sparse pattern on 2-theta in [10, 90] degrees.

    k_true peaks, each Lorentzian (eta = 0) or pseudo-Voigt (eta ~ U[0, 1]) with
    probability 1/2, FWHM ~ U[0.05, 0.3], amplitude 1e4 10^U[-3, 0]; cubic
    Chebyshev background of amplitude 0.05 max; Gaussian noise of sd 1% of the
    maximum of the noiseless pattern.  Fitted with PV peaks + cubic background.
    """
    rng = np.random.default_rng(seed)
    x = np.linspace(10.0, 90.0, n)
    mus = np.sort(rng.uniform(12.0, 88.0, k_true))
    lor = rng.uniform(size=k_true) < 0.5
    eta = np.where(lor, 0.0, rng.uniform(0.0, 1.0, k_true))
    fwhm = rng.uniform(0.05, 0.3, k_true)
    amp = 1.0e4 * 10.0 ** rng.uniform(-3.0, 0.0, k_true)
    f = np.zeros_like(x)
    for k in range(k_true):
        f = f + _synth_pv(x, amp[k], mus[k], 0.5 * fwhm[k], eta[k])
    peak_max = float(f.max())
    cheb = 0.05 * peak_max * np.array([1.0, -0.4, 0.25, -0.1])
    f = f + _synth_cheb(x, cheb)
    sd = 0.01 * float(f.max())
    y = f + rng.normal(0.0, sd, size=x.shape)
    ymin, ymax = float(y.min()), float(y.max())
    pri = Priors(amp=Prior(LOG_UNIFORM, 1e-3 * (ymax - ymin), 2.0 * ymax),
                 centre=Prior(UNIFORM, float(x.min()), float(x.max())),
                 width=Prior(LOG_UNIFORM, 0.01, 0.5),
                 eta=Prior(UNIFORM, 0.0, 1.0),
                 bg=data_bg_priors(y, 4))
    return Spectrum(x, y, np.full_like(x, sd), PSEUDO_VOIGT, 1, k_max, BG_POLY, 3, pri,
                    truth={"K": k_true, "A": amp.tolist(), "mu": mus.tolist(),
                           "hwhm": (0.5 * fwhm).tolist(), "eta": eta.tolist()},
                    name=f"xrd-{n}")


def mixed_batch(seed: int = 1, count: int = 256) -> List[tuple]:
    """Uneven batch: N ~ U{200..4000}, true K ~ U{1..8}, Gaussian or PV peaks.

    Returns a list of (Spectrum, Options) pairs; particles per K in
    {4096, 8192, 16384, 32768}, K_max ~ U{3..10}, 10 sweeps per stage.
    """
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.integers(200, 4001))
        k_true = int(rng.integers(1, 9))
        k_max = int(rng.integers(3, 11))
        fam = GAUSS if rng.uniform() < 0.5 else PSEUDO_VOIGT
        x = np.linspace(0.0, 1.0, n) * 10.0
        mus = np.sort(rng.uniform(0.5, 9.5, k_true))
        amp = 10.0 ** rng.uniform(-1.0, 0.0, k_true)
        if fam == GAUSS:
            w = rng.uniform(0.1, 0.5, k_true)
            f = sum(_synth_gauss(x, amp[k], mus[k], w[k]) for k in range(k_true))
            sd = 0.02
            pri = Priors(amp=Prior(GAMMA, 2.0, 2.0), centre=Prior(UNIFORM, 0.0, 10.0),
                         width=Prior(LOG_UNIFORM, 0.05, 2.0))
            bgk, bgd = BG_NONE, 0
        else:
            hw = rng.uniform(0.05, 0.3, k_true)
            eta = rng.uniform(0.0, 1.0, k_true)
            f = 0.05 + sum(_synth_pv(x, amp[k], mus[k], hw[k], eta[k]) for k in range(k_true))
            sd = 0.02
            bgk, bgd = BG_LINEAR, 1
            pri = None
        y = f + rng.normal(0.0, sd, size=x.shape)
        if pri is None:
            ymin, ymax = float(y.min()), float(y.max())
            pri = Priors(amp=Prior(LOG_UNIFORM, 1e-3 * (ymax - ymin), 2.0 * ymax),
                         centre=Prior(UNIFORM, 0.0, 10.0), width=Prior(LOG_UNIFORM, 0.02, 1.0),
                         eta=Prior(UNIFORM, 0.0, 1.0), bg=data_bg_priors(y, 2))
        spec = Spectrum(x, y, np.full_like(x, sd), fam, 1, k_max, bgk, bgd, pri,
                        truth={"K": k_true}, name=f"mixed-{b}")
        opts = Options(particles=int(rng.choice([4096, 8192, 16384, 32768])), sweeps=10,
                       seed=seed * 100003 + b)
        out.append((spec, opts))
    return out


def poisson_arrivals(rate_per_s: float, count: int, seed: int = 1) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def linear_gaussian_case(seed: int = 3, n: int = 40, family: int = GAUSS) -> Spectrum:
    """Two peaks with fixed centres and widths and Normal amplitude priors.

    With every nonlinear parameter fixed the likelihood is linear-Gaussian in
    the amplitudes, so log Z and the amplitude posterior have closed forms.
    """
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 4.0, n)
    mus, ws, amps = [1.3, 2.6], [0.35, 0.5], [0.9, 0.5]
    f = sum(_synth_gauss(x, amps[k], mus[k], ws[k]) for k in range(2))
    sd = 0.1
    y = f + rng.normal(0.0, sd, size=x.shape)
    pri = Priors(amp=Prior(NORMAL, 0.5, 0.7), centre=Prior(UNIFORM, 0.0, 4.0),
                 width=Prior(LOG_UNIFORM, 0.1, 1.0))
    comp = []
    for k in range(2):
        comp += [Prior(NORMAL, 0.5, 0.7), Prior(FIXED, mus[k]), Prior(FIXED, ws[k])]
    return Spectrum(x, y, np.full_like(x, sd), family, 2, 2, BG_NONE, 0, pri,
                    truth={"mu": mus, "w": ws, "m0": 0.5, "s0": 0.7}, name="linear-gaussian",
                    comp_priors=comp)


def tiny_single_peak(seed: int = 5, n: int = 21) -> Spectrum:
    """21-point single Gaussian peak on [0, 2] for quadrature checks of log Z."""
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 2.0, n)
    f = _synth_gauss(x, 1.2, 0.9, 0.25)
    sd = 0.15
    y = f + rng.normal(0.0, sd, size=x.shape)
    pri = Priors(amp=Prior(GAMMA, 2.0, 1.0), centre=Prior(UNIFORM, 0.0, 2.0),
                 width=Prior(LOG_UNIFORM, 0.1, 1.0))
    return Spectrum(x, y, np.full_like(x, sd), GAUSS, 1, 1, BG_NONE, 0, pri,
                    truth={"A": 1.2, "mu": 0.9, "w": 0.25}, name="tiny-single")
