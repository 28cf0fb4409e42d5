"""FP64 CPU oracle of the tempered SMC sampler -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never loads it, and it
imports nothing from the CUDA binding.  The arithmetic lives in
``smc_oracle.c`` (plain sequential C in double precision); this module only
marshals numpy arrays into it and adds the cross-K post-processing of
Sec. II A (posterior over K from the free energies, Eq. (2)).

Parity pins for every function are in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

OK, EINVAL, ENOMEM, EMAXSTAGES, ENUMERIC = 0, 1, 2, 5, 8


def compile_library(src: str, out: str) -> str:
    """gcc of one C source into a shared library (strict IEEE double, no
    fast-math, no contraction into FMA)."""
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", out, src, "-lm"])
    return out


def build(force: bool = False) -> str:
    """Compile the oracle."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        compile_library(_SRC, tmp)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def source() -> str:
    """Path of the oracle's C source."""
    return _SRC


class Prior(C.Structure):
    _fields_ = [("kind", C.c_int32), ("p1", C.c_double), ("p2", C.c_double)]


class Job(C.Structure):
    _fields_ = [("x", C.POINTER(C.c_double)), ("y", C.POINTER(C.c_double)),
                ("sigma", C.POINTER(C.c_double)), ("n", C.c_int64),
                ("family", C.c_int32), ("K", C.c_int32), ("bg_kind", C.c_int32),
                ("bg_degree", C.c_int32),
                ("amp", Prior), ("centre", Prior), ("width", Prior), ("eta", Prior),
                ("bg", Prior * 8),
                ("comp_priors", C.POINTER(Prior)), ("n_comp_priors", C.c_int32),
                ("particles", C.c_int64), ("ess_target", C.c_double),
                ("sweeps", C.c_int32), ("waste_free", C.c_int32),
                ("seed", C.c_uint64), ("max_stages", C.c_int32),
                ("noise", C.c_int32), ("noise_par", C.c_double * 3),
                ("ref_pos", C.POINTER(C.c_double)), ("ref_int", C.POINTER(C.c_double)),
                ("ref_off", C.POINTER(C.c_int32)), ("n_phase", C.c_int32),
                ("phase", Prior * 9), ("step_rule", C.c_int32)]


class Out(C.Structure):
    _fields_ = [("log_z", C.c_double), ("n_stages", C.c_int32), ("status", C.c_int32),
                ("n_out", C.c_int64), ("d", C.c_int32),
                ("samples", C.POINTER(C.c_double)), ("energies", C.POINTER(C.c_double)),
                ("beta_trace", C.POINTER(C.c_double)), ("logz_trace", C.POINTER(C.c_double)),
                ("acc_trace", C.POINTER(C.c_double)), ("step_trace", C.POINTER(C.c_double))]


def lib():
    global _lib
    if _lib is None:
        _lib = bind(C.CDLL(build()))
    return _lib


def bind(handle):
    """Declare the argument and result types of every exported function on a
    loaded oracle library."""
    L = handle
    d, i64, u32, i32 = C.c_double, C.c_int64, C.c_uint32, C.c_int
    P = C.POINTER
    L.orc_philox.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
    L.orc_peak.argtypes = [i32, d, d, d, d, d]
    L.orc_peak.restype = d
    L.orc_model_at.argtypes = [i32, i32, i32, P(d), d, d, d]
    L.orc_model_at.restype = d
    L.orc_energy_nat.argtypes = [i32, i32, i32, P(d), P(d), P(d), P(d), i64]
    L.orc_energy_nat.restype = d
    L.orc_model_vec.argtypes = [i32, i32, i32, i32, P(d), P(d), i64, P(d)]
    L.orc_energy_model.argtypes = [i32, i32, i32, i32, i32, P(d), P(d), P(d), P(d), P(d), i64]
    L.orc_energy_model.restype = d
    L.orc_energy_job.argtypes = [P(Job), P(d)]
    L.orc_energy_job.restype = d
    L.orc_xrd_phase.argtypes = [P(d), P(d), P(d), i32, d]
    L.orc_xrd_phase.restype = d
    L.orc_xrd_background.argtypes = [P(d), d]
    L.orc_xrd_background.restype = d
    L.orc_model_vec_xrd.argtypes = [i32, i32, P(d), P(d), i64, P(d), P(d), P(C.c_int32), P(d)]
    L.orc_dim.argtypes = [i32, i32, i32, i32]
    L.orc_dim.restype = i32
    L.orc_prior_draw.argtypes = [Prior, C.c_uint64, u32, u32, u32]
    L.orc_prior_draw.restype = d
    L.orc_ess_frac.argtypes = [P(d), i64, d]
    L.orc_ess_frac.restype = d
    L.orc_choose_delta.argtypes = [P(d), i64, d, d, P(C.c_int), P(C.c_int)]
    L.orc_choose_delta.restype = d
    L.orc_quantise.argtypes = [P(d), i64, P(C.c_uint64)]
    L.orc_resample.argtypes = [P(C.c_uint64), i64, i64, u32, P(C.c_int32)]
    L.orc_init_particles.argtypes = [P(Job), i64, P(d), P(d)]
    L.orc_energies.argtypes = [P(Job), i64, P(d), P(d)]
    L.orc_mh_stage.argtypes = [P(Job), P(d), P(d), i64, P(d), d, u32, P(d), P(d),
                               P(C.c_int64), P(C.c_int64)]
    L.orc_step_sizes.argtypes = [P(Job), P(d), P(d), i64, P(d), P(d), P(d)]
    L.orc_predict_step.argtypes = [P(d), d, d, d, d, d]
    L.orc_predict_step.restype = d
    L.orc_run_job.argtypes = [P(Job), P(Out)]
    L.orc_run_job.restype = i32
    return L


def use_library(handle) -> None:
    """Route every wrapper in this module through another build of the oracle
    (a library returned by bind()); None goes back to the default build."""
    global _lib
    _lib = handle


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ----------------------------------------------------------------------------
# elementary functions
# ----------------------------------------------------------------------------

def philox(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().orc_philox(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def peak(family: int, x: float, A: float, mu: float, w: float, eta: float = 0.0) -> float:
    return lib().orc_peak(family, x, A, mu, w, eta)


def dim(family: int, K: int, bg: int, bg_degree: int) -> int:
    return lib().orc_dim(family, K, bg, bg_degree)


def model(family: int, K: int, nbg: int, nat: np.ndarray, x: np.ndarray) -> np.ndarray:
    nat = _f64(nat)
    x = _f64(x)
    lo, hi = float(x.min()), float(x.max())
    return np.array([lib().orc_model_at(family, K, nbg, _dp(nat), float(xi), lo, hi) for xi in x])


def energy_natural(family: int, K: int, nbg: int, nat, x, y, sigma) -> float:
    nat, x, y, sigma = _f64(nat), _f64(x), _f64(y), _f64(sigma)
    return lib().orc_energy_nat(family, K, nbg, _dp(nat), _dp(x), _dp(y), _dp(sigma), x.shape[0])


def model_vec(family: int, K: int, bg: int, bg_degree: int, nat, x) -> np.ndarray:
    """Forward model at every grid point (any background, Shirley included)."""
    nat, x = _f64(nat), _f64(x)
    f = np.zeros(x.shape[0])
    lib().orc_model_vec(family, K, bg, bg_degree, _dp(nat), _dp(x), x.shape[0], _dp(f))
    return f


def energy_spec(spec, K: int, nat) -> float:
    """Energy of natural parameters for the spectrum's model, background and noise."""
    h = _JobHolder(spec, K, _ENERGY_OPTS)
    nat = _f64(nat)
    return lib().orc_energy_job(C.byref(h.job), _dp(nat))


def xrd_phase(nat_phase, positions, intensities, x: float) -> float:
    """One phase of the App. D model at x (degrees 2 theta)."""
    q, pos, it = _f64(nat_phase), _f64(positions), _f64(intensities)
    return lib().orc_xrd_phase(_dp(q), _dp(pos), _dp(it), pos.shape[0], float(x))


def xrd_background(bg, x: float) -> float:
    b = _f64(bg)
    return lib().orc_xrd_background(_dp(b), float(x))


def model_spec(spec, K: int, nat) -> np.ndarray:
    """Forward model of natural parameters at every grid point of the spectrum."""
    nat, x = _f64(nat), _f64(spec.x)
    if spec.family != 4:
        return model_vec(spec.family, K, spec.bg, spec.bg_degree, nat, x)
    pos, it, off = _refs_arrays(spec)
    f = np.zeros(x.shape[0])
    lib().orc_model_vec_xrd(K, spec.bg, _dp(nat), _dp(x), x.shape[0], _dp(pos), _dp(it),
                            off.ctypes.data_as(C.POINTER(C.c_int32)), _dp(f))
    return f


def _refs_arrays(spec):
    refs = getattr(spec, "refs", None) or []
    pos = _f64(np.concatenate([np.asarray(r[0], float) for r in refs]) if refs else np.zeros(1))
    it = _f64(np.concatenate([np.asarray(r[1], float) for r in refs]) if refs else np.zeros(1))
    off = np.zeros(len(refs) + 1, dtype=np.int32)
    for k, r in enumerate(refs):
        off[k + 1] = off[k] + len(r[0])
    return pos, it, off


def prior_draw(kind: int, p1: float, p2: float, seed: int, comp: int, particle: int, tag: int) -> float:
    return lib().orc_prior_draw(Prior(kind, p1, p2), seed, comp, particle, tag)


def ess_frac(e: np.ndarray, delta: float) -> float:
    e = _f64(e)
    return lib().orc_ess_frac(_dp(e), e.shape[0], delta)


def choose_delta(e: np.ndarray, beta: float, rho: float):
    e = _f64(e)
    fin, it = C.c_int(), C.c_int()
    dl = lib().orc_choose_delta(_dp(e), e.shape[0], beta, rho, C.byref(fin), C.byref(it))
    return dl, bool(fin.value), it.value


def quantise(w: np.ndarray) -> np.ndarray:
    w = _f64(w)
    q = np.zeros(w.shape[0], dtype=np.uint64)
    lib().orc_quantise(_dp(w), w.shape[0], q.ctypes.data_as(C.POINTER(C.c_uint64)))
    return q


def resample(q: np.ndarray, M: int, u32: int) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.uint64)
    a = np.zeros(M, dtype=np.int32)
    lib().orc_resample(q.ctypes.data_as(C.POINTER(C.c_uint64)), q.shape[0], M, u32,
                       a.ctypes.data_as(C.POINTER(C.c_int32)))
    return a


# ----------------------------------------------------------------------------
# jobs
# ----------------------------------------------------------------------------

class _EnergyOpts:
    particles, ess_target, sweeps, waste_free, seed, max_stages = 2, 0.5, 1, 0, 1, 1


_ENERGY_OPTS = _EnergyOpts()


class _JobHolder:
    """Keeps the numpy buffers referenced by a Job structure alive."""

    def __init__(self, spec, K: int, opts, comp_priors=None):
        self.x, self.y, self.s = _f64(spec.x), _f64(spec.y), _f64(spec.sigma)
        pr = spec.priors
        j = Job()
        j.x, j.y, j.sigma, j.n = _dp(self.x), _dp(self.y), _dp(self.s), self.x.shape[0]
        j.family, j.K, j.bg_kind, j.bg_degree = spec.family, K, spec.bg, spec.bg_degree
        j.amp = Prior(pr.amp.kind, pr.amp.p1, pr.amp.p2)
        j.centre = Prior(pr.centre.kind, pr.centre.p1, pr.centre.p2)
        j.width = Prior(pr.width.kind, pr.width.p1, pr.width.p2)
        j.eta = Prior(pr.eta.kind, pr.eta.p1, pr.eta.p2)
        for i, b in enumerate(pr.bg[:8]):
            j.bg[i] = Prior(b.kind, b.p1, b.p2)
        cps = comp_priors if comp_priors is not None else getattr(spec, "comp_priors", None)
        if cps:
            self.cp = (Prior * len(cps))(*[Prior(p.kind, p.p1, p.p2) for p in cps])
            j.comp_priors = self.cp
            j.n_comp_priors = len(cps)
        j.particles, j.ess_target = opts.particles, opts.ess_target
        j.sweeps, j.waste_free = opts.sweeps, opts.waste_free
        j.seed, j.max_stages = opts.seed, opts.max_stages
        j.step_rule = int(getattr(opts, "step_rule", 0))
        j.noise = getattr(spec, "noise", 0)
        for i, v in enumerate(getattr(spec, "noise_par", (0.0, 0.0, 0.0))):
            j.noise_par[i] = v
        if getattr(spec, "refs", None):
            self.rp, self.ri, self.ro = _refs_arrays(spec)
            j.ref_pos, j.ref_int = _dp(self.rp), _dp(self.ri)
            j.ref_off = self.ro.ctypes.data_as(C.POINTER(C.c_int32))
            j.n_phase = len(spec.refs)
        for i, q in enumerate(getattr(spec, "phase_priors", None) or []):
            j.phase[i] = Prior(q.kind, q.p1, q.p2)
        self.job = j
        self.d = dim(spec.family, K, spec.bg, spec.bg_degree)


def init_particles(spec, K: int, opts, count: int):
    h = _JobHolder(spec, K, opts)
    u = np.zeros((count, max(h.d, 1)))
    E = np.zeros(count)
    lib().orc_init_particles(C.byref(h.job), count, _dp(u), _dp(E))
    return u[:, :h.d], E


def energies(spec, K: int, opts, u: np.ndarray) -> np.ndarray:
    h = _JobHolder(spec, K, opts)
    u = _f64(u).reshape(-1, h.d)
    E = np.zeros(u.shape[0])
    lib().orc_energies(C.byref(h.job), u.shape[0], _dp(u), _dp(E))
    return E


def mh_stage(spec, K: int, opts, u_start, E_start, step, beta: float, stage: int):
    h = _JobHolder(spec, K, opts)
    u_start = _f64(u_start).reshape(-1, h.d)
    E_start = _f64(E_start)
    S = u_start.shape[0]
    n_out = S * opts.sweeps if opts.waste_free else S
    u_out = np.zeros((n_out, h.d))
    E_out = np.zeros(n_out)
    acc = np.zeros(h.d, dtype=np.int64)
    prop = np.zeros(h.d, dtype=np.int64)
    step = _f64(step)
    P64 = C.POINTER(C.c_int64)
    lib().orc_mh_stage(C.byref(h.job), _dp(u_start), _dp(E_start), S, _dp(step), beta, stage,
                       _dp(u_out), _dp(E_out), acc.ctypes.data_as(P64), prop.ctypes.data_as(P64))
    return u_out, E_out, acc, prop


def step_sizes(spec, K: int, opts, u, w, acc_rate, lam):
    h = _JobHolder(spec, K, opts)
    u, w = _f64(u).reshape(-1, h.d), _f64(w)
    lam = _f64(lam).copy()
    step = np.zeros(h.d)
    rate = None if acc_rate is None else _f64(acc_rate)
    lib().orc_step_sizes(C.byref(h.job), _dp(u), _dp(w), u.shape[0],
                         None if rate is None else _dp(rate), _dp(lam), _dp(step))
    return step, lam


def predict_step(hist, s_prev: float, acc: float, beta_prev: float, beta_next: float,
                 sd_pop: float):
    """The history step-size predictor for one component: returns the new step
    and the updated history sums (W, X, Y, XX, XY)."""
    h = _f64(hist).copy()
    assert h.shape == (5,)
    st = lib().orc_predict_step(_dp(h), s_prev, acc, beta_prev, beta_next, sd_pop)
    return st, h


def run_job(spec, K: int, opts, comp_priors=None, traces: bool = True) -> dict:
    """One (spectrum, K) SMC run.  Returns log Z, the stage traces and samples."""
    h = _JobHolder(spec, K, opts, comp_priors)
    T = opts.particles
    n_out = ((T + opts.sweeps - 1) // opts.sweeps) * opts.sweeps if opts.waste_free else T
    dd = max(h.d, 1)
    samples = np.zeros((n_out, dd))
    en = np.zeros(n_out)
    ms = opts.max_stages + 1
    bt, lt = np.zeros(ms), np.zeros(ms)
    at, st = np.zeros((ms, dd)), np.zeros((ms, dd))
    o = Out()
    o.samples, o.energies = _dp(samples), _dp(en)
    if traces:
        o.beta_trace, o.logz_trace, o.acc_trace, o.step_trace = _dp(bt), _dp(lt), _dp(at), _dp(st)
    lib().orc_run_job(C.byref(h.job), C.byref(o))
    L = o.n_stages
    # the final set as the oracle reports it (n_out particles)
    m = min(int(o.n_out), n_out) if o.status in (OK, EMAXSTAGES) else n_out
    return {"status": o.status, "log_z": o.log_z, "n_stages": L, "d": h.d, "n_out": int(o.n_out),
            "samples": samples[:m, :h.d], "energies": en[:m],
            "beta": bt[:L + 1], "logz": lt[:L + 1], "acc": at[:L + 1, :h.d],
            "step": st[:L + 1, :h.d]}


def posterior_over_k(log_z: Sequence[float]) -> np.ndarray:
    """p(K|D) with a uniform p(K): exp(-F(K)) normalised over K (Sec. II A, Eq. (2))."""
    lz = np.asarray(log_z, dtype=np.float64)
    m = lz.max()
    p = np.exp(lz - m)
    return p / p.sum()


def sorted_summary(samples: np.ndarray, family: int, K: int):
    """Posterior mean and SD per component after ordering each sample's peaks by
    centre (peaks are exchangeable in Eq. (1), so labels are fixed by sorting)."""
    if family == 4:  # App. D phases: not exchangeable, not sorted
        return samples.mean(axis=0), samples.std(axis=0)
    p = 4 if family == 2 else 3
    s = np.array(samples, dtype=np.float64, copy=True)
    if K > 1:
        peaks = s[:, :p * K].reshape(-1, K, p)
        order = np.argsort(peaks[:, :, 1], axis=1, kind="stable")
        peaks = np.take_along_axis(peaks, order[:, :, None], axis=1)
        s[:, :p * K] = peaks.reshape(-1, p * K)
    return s.mean(axis=0), s.std(axis=0)


def run(spec, opts, k_range: Optional[Sequence[int]] = None, comp_priors=None) -> dict:
    """All candidate K of one spectrum; log Z per K, p(K|D), summaries."""
    ks = list(k_range) if k_range is not None else list(range(spec.k_min, spec.k_max + 1))
    res = [run_job(spec, K, opts, comp_priors=comp_priors) for K in ks]
    lz = [r["log_z"] for r in res]
    summ = [sorted_summary(r["samples"], spec.family, K) for r, K in zip(res, ks)]
    return {"K": ks, "log_z": lz, "p_k": posterior_over_k(lz), "jobs": res,
            "post_mean": [m for m, _ in summ], "post_sd": [s for _, s in summ],
            "argmax_k": ks[int(np.argmax(lz))]}
