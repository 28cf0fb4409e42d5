"""Thin ctypes binding of the C ABI in include/smc.h and include/smc_kernels.h.

Argument marshalling only: every step of the sampler runs in the CUDA library
(libsmc_b300.so, built in-tree by ``python -m paper_2604_03271_b300.build``).
Importing this module on a machine without the built library raises at once;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsmc_b300.so")

SMC_OK, SMC_EINVAL, SMC_ENOMEM, SMC_ECUDA, SMC_ETIMEOUT = 0, 1, 2, 3, 4
SMC_EMAXSTAGES, SMC_ENOTREADY, SMC_ECANCELLED, SMC_ENUMERIC = 5, 6, 7, 8


class SmcError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {_strerror(status)} (status {status})")
        self.status = status


class Prior(C.Structure):
    _fields_ = [("kind", C.c_int32), ("p1", C.c_double), ("p2", C.c_double)]


class Priors(C.Structure):
    _fields_ = [("amp", Prior), ("centre", Prior), ("width", Prior), ("eta", Prior),
                ("bg", Prior * 8), ("comp", C.POINTER(Prior)), ("n_comp", C.c_int32),
                ("phase", Prior * 9)]


GRAPH_WHILE, GRAPH_CHUNKED, GRAPH_NONE = 0, 1, 2


class CreateOpts(C.Structure):
    _fields_ = [("device", C.c_int32), ("mem_budget_bytes", C.c_size_t), ("cuda_stream", C.c_void_p),
                ("graph_mode", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("particles", C.c_int64), ("ess_target", C.c_double), ("sweeps", C.c_int32),
                ("waste_free", C.c_int32), ("energy_fp64", C.c_int32), ("seed", C.c_uint64),
                ("max_stages", C.c_int32), ("keep_samples", C.c_int32), ("step_rule", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("sigma", C.c_void_p), ("n", C.c_int64),
                ("k_min", C.c_int32), ("k_max", C.c_int32), ("family", C.c_int32),
                ("bg", C.c_int32), ("bg_degree", C.c_int32),
                ("priors", C.POINTER(Priors)), ("opts", C.POINTER(Options)),
                ("noise", C.c_int32), ("noise_par", C.c_double * 3),
                ("ref_pos", C.c_void_p), ("ref_int", C.c_void_p), ("ref_off", C.c_void_p),
                ("n_phase", C.c_int32)]


class Profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * 5), ("ms", C.c_double * 5), ("point_evals", C.c_double),
                ("sfu_ops", C.c_double), ("gather_bytes", C.c_double), ("resample_bytes", C.c_double),
                ("h2d_bytes", C.c_double), ("d2h_bytes", C.c_double),
                ("stages", C.c_int64), ("jobs", C.c_int64),
                ("ex2_ops", C.c_double), ("rcp_ops", C.c_double), ("lg2_ops", C.c_double),
                ("max_batch_requests", C.c_int64), ("peak_point_evals", C.c_double),
                ("peak_sfu_per_eval", C.c_double)]


KERNEL_CLASSES = ("reweight", "resample", "gather", "metropolis", "stage_end")


class ResultView(C.Structure):
    _fields_ = [("k_min", C.c_int32), ("k_max", C.c_int32), ("dim_max", C.c_int32),
                ("status", C.c_int32), ("log_z", C.POINTER(C.c_double)),
                ("p_k", C.POINTER(C.c_double)), ("n_stages", C.POINTER(C.c_int32)),
                ("job_status", C.POINTER(C.c_int32)), ("post_mean", C.POINTER(C.c_double)),
                ("post_sd", C.POINTER(C.c_double)), ("samples", C.POINTER(C.c_float)),
                ("n_samples", C.c_int64), ("latency_ms", C.c_double), ("selected_k", C.c_int32)]


_lib = None


def lib():
    """Load the CUDA library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing; build it with "
                           "`python -m paper_2604_03271_b300.build`")
    L = C.CDLL(LIB_PATH)
    P, i32, i64, u32, u64, dbl = C.POINTER, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
    vp = C.c_void_p
    L.smc_strerror.restype = C.c_char_p
    L.smc_strerror.argtypes = [C.c_int]
    L.smc_create.argtypes = [P(vp), P(CreateOpts)]
    L.smc_destroy.argtypes = [vp]
    L.smc_run.argtypes = [vp, vp, vp, vp, i64, i32, i32, i32, i32, i32, P(Priors), P(Options), P(u64)]
    L.smc_run_batch.argtypes = [vp, P(Request), i32, i32, P(u64)]
    L.smc_submit.argtypes = [vp, P(Request), P(u64)]
    L.smc_submit_batch.argtypes = [vp, P(Request), i32, P(u64)]
    L.smc_request_bytes.argtypes = [vp, P(Request), P(C.c_size_t)]
    L.smc_poll.argtypes = [vp, u64, P(i32)]
    L.smc_wait.argtypes = [vp, u64, dbl]
    L.smc_result.argtypes = [vp, u64, P(ResultView)]
    L.smc_release.argtypes = [vp, u64]
    L.smc_k_philox.argtypes = [vp, u64, vp, vp, i64]
    L.smc_k_energy.argtypes = [vp, P(Request), i32, vp, i64, i32, vp]
    L.smc_k_prior.argtypes = [vp, P(Request), i32, i64, i32, vp, vp]
    L.smc_k_reweight.argtypes = [vp, vp, i64, dbl, dbl, i32, P(dbl), P(dbl), P(i32), vp]
    L.smc_k_resample.argtypes = [vp, vp, i64, i64, u32, vp]
    L.smc_k_mh_stage.argtypes = [vp, P(Request), i32, vp, vp, i64, vp, dbl, u32, i32, vp, vp, vp, vp]
    L.smc_set_tile.argtypes = [vp, i32, i64, i32, i32, i32]
    L.smc_set_tile.restype = C.c_int
    L.smc_profile_reset.argtypes = [vp, i32]
    L.smc_profile_read.argtypes = [vp, P(Profile)]
    L.smc_k_mufu_rate.argtypes = [i32, P(dbl), P(dbl), P(dbl), vp]
    for f in ("smc_k_mufu_rate", "smc_profile_reset", "smc_profile_read", "smc_create", "smc_destroy", "smc_run", "smc_run_batch", "smc_submit", "smc_submit_batch",
              "smc_request_bytes", "smc_poll",
              "smc_wait", "smc_result", "smc_release", "smc_k_philox", "smc_k_energy",
              "smc_k_prior", "smc_k_reweight", "smc_k_resample", "smc_k_mh_stage"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _strerror(status: int) -> str:
    try:
        return lib().smc_strerror(status).decode()
    except Exception:  # library not loadable
        return "error"


def _check(st: int, what: str):
    if st != SMC_OK:
        raise SmcError(st, what)


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _c_prior(p: W.Prior) -> Prior:
    return Prior(int(p.kind), float(p.p1), float(p.p2))


class _Marshalled:
    """ctypes structures of one spectrum + options, with their buffers kept alive."""

    def __init__(self, spec: W.Spectrum, opts: W.Options, device_arrays=None, keep_samples=1):
        self.pri = Priors()
        pr = spec.priors
        self.pri.amp, self.pri.centre = _c_prior(pr.amp), _c_prior(pr.centre)
        self.pri.width, self.pri.eta = _c_prior(pr.width), _c_prior(pr.eta)
        for i, b in enumerate(pr.bg[:8]):
            self.pri.bg[i] = _c_prior(b)
        for i, q in enumerate((getattr(spec, "phase_priors", None) or [])[:9]):
            self.pri.phase[i] = _c_prior(q)
        if spec.comp_priors:
            self.comp = (Prior * len(spec.comp_priors))(*[_c_prior(p) for p in spec.comp_priors])
            self.pri.comp = self.comp
            self.pri.n_comp = len(spec.comp_priors)
        self.opts = Options(int(opts.particles), float(opts.ess_target), int(opts.sweeps),
                            int(opts.waste_free), int(opts.energy_fp64), int(opts.seed),
                            int(opts.max_stages), int(keep_samples), int(getattr(opts, "step_rule", 0)))
        if device_arrays is None:
            self.x, self.y, self.s = _f64(spec.x), _f64(spec.y), _f64(spec.sigma)
            xp, yp, sp = self.x.ctypes.data, self.y.ctypes.data, self.s.ctypes.data
        else:
            self.dev = device_arrays  # keep torch tensors alive
            xp, yp, sp = [int(t.data_ptr()) for t in device_arrays]
        self.req = Request(xp, yp, sp, spec.n, spec.k_min, spec.k_max, spec.family, spec.bg,
                           spec.bg_degree, C.pointer(self.pri), C.pointer(self.opts),
                           int(getattr(spec, "noise", 0)),
                           (C.c_double * 3)(*getattr(spec, "noise_par", (0.0, 0.0, 0.0))))
        refs = getattr(spec, "refs", None)
        if refs:
            self.rpos = _f64(np.concatenate([np.asarray(p, np.float64) for p, _ in refs]))
            self.rint = _f64(np.concatenate([np.asarray(i, np.float64) for _, i in refs]))
            self.roff = np.ascontiguousarray(np.cumsum([0] + [len(p) for p, _ in refs]), dtype=np.int32)
            self.req.ref_pos, self.req.ref_int = self.rpos.ctypes.data, self.rint.ctypes.data
            self.req.ref_off, self.req.n_phase = self.roff.ctypes.data, len(refs)


def _dim(family: int, K: int, bg: int, bg_degree: int) -> int:
    p = 9 if family == W.XRD_PHASE else (4 if family == W.PSEUDO_VOIGT else 3)
    return p * K + W.bg_count(bg, bg_degree)


class Context:
    """One device context (smc_create / smc_destroy)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, stream: Optional[int] = None,
                 graph_mode: int = GRAPH_WHILE):
        self._L = lib()
        h = C.c_void_p()
        o = CreateOpts(device, mem_budget_bytes, stream, graph_mode)
        _check(self._L.smc_create(C.byref(h), C.byref(o)), "smc_create")
        self.h = h

    def close(self):
        if self.h:
            self._L.smc_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- results ---------------------------------------------------------
    def result(self, job: int, spec: W.Spectrum) -> dict:
        v = ResultView()
        _check(self._L.smc_result(self.h, C.c_uint64(job), C.byref(v)), "smc_result")
        nK = v.k_max - v.k_min + 1
        ks = list(range(v.k_min, v.k_max + 1))
        out = {"K": ks, "status": v.status, "latency_ms": v.latency_ms, "n_samples": v.n_samples,
               "argmax_k": v.selected_k if v.selected_k >= 0 else None}
        if not v.log_z:  # the request failed before producing results
            out.update({"log_z": None, "p_k": None, "n_stages": None, "job_status": None,
                        "post_mean": None, "post_sd": None, "argmax_k": None})
            return out
        dm = v.dim_max
        log_z = np.ctypeslib.as_array(v.log_z, (nK,)).copy()
        out.update({"log_z": log_z,
                    "p_k": np.ctypeslib.as_array(v.p_k, (nK,)).copy(),
                    "n_stages": np.ctypeslib.as_array(v.n_stages, (nK,)).copy(),
                    "job_status": np.ctypeslib.as_array(v.job_status, (nK,)).copy()})
        mean = np.ctypeslib.as_array(v.post_mean, (nK, dm))
        sd = np.ctypeslib.as_array(v.post_sd, (nK, dm))
        dims = [_dim(spec.family, K, spec.bg, spec.bg_degree) for K in ks]
        out["post_mean"] = [mean[a, :dims[a]].copy() for a in range(nK)]
        out["post_sd"] = [sd[a, :dims[a]].copy() for a in range(nK)]
        if v.samples:
            smp = np.ctypeslib.as_array(v.samples, (nK, v.n_samples, dm))
            out["samples"] = [smp[a, :, :dims[a]].copy() for a in range(nK)]
        return out

    def release(self, job: int):
        _check(self._L.smc_release(self.h, C.c_uint64(job)), "smc_release")

    # -- blocking runs -----------------------------------------------------
    def run(self, spec: W.Spectrum, opts: W.Options, keep_samples: bool = True) -> dict:
        """One spectrum, blocking.  Known-sigma spectra go through smc_run (host
        arrays); spectra that need smc_request's extra fields (model variance,
        Poisson counts, App. D reflections) through smc_run_batch."""
        if int(getattr(spec, "noise", 0)) != 0 or getattr(spec, "refs", None):
            return self.run_batch([(spec, opts)], keep_samples=keep_samples)[0]
        m = _Marshalled(spec, opts, None, 1 if keep_samples else 0)
        job = C.c_uint64()
        _check(self._L.smc_run(self.h, _ptr(m.x), _ptr(m.y), _ptr(m.s), spec.n, spec.k_min,
                               spec.k_max, spec.family, spec.bg, spec.bg_degree, C.pointer(m.pri),
                               C.pointer(m.opts), C.byref(job)), "smc_run")
        out = self.result(int(job.value), spec)
        self.release(int(job.value))
        return out

    def run_batch(self, items: Sequence[tuple], keep_samples: bool = True,
                  device_arrays: Optional[Sequence] = None) -> List[dict]:
        """Run several (spectrum, options) pairs in one batched launch sequence.

        device_arrays: optional per-item (x, y, sigma) float64 CUDA tensors; the
        library then reads the inputs from device memory.
        """
        ms = [_Marshalled(s, o, None if device_arrays is None else device_arrays[i],
                          1 if keep_samples else 0) for i, (s, o) in enumerate(items)]
        reqs = (Request * len(ms))(*[m.req for m in ms])
        jobs = (C.c_uint64 * len(ms))()
        _check(self._L.smc_run_batch(self.h, reqs, len(ms), 0 if device_arrays is None else 1, jobs),
               "smc_run_batch")
        out = []
        for j, (s, _) in zip(jobs, items):
            out.append(self.result(int(j), s))
            self.release(int(j))
        return out

    # -- serving -----------------------------------------------------------
    def submit(self, spec: W.Spectrum, opts: W.Options, keep_samples: bool = False) -> int:
        m = _Marshalled(spec, opts, None, 1 if keep_samples else 0)
        job = C.c_uint64()
        _check(self._L.smc_submit(self.h, C.byref(m.req), C.byref(job)), "smc_submit")
        return int(job.value)

    def submit_batch(self, items: Sequence[tuple], keep_samples: bool = False) -> List[int]:
        """Enqueue several (spectrum, options) pairs at once (smc_submit_batch)."""
        ms = [_Marshalled(s, o, None, 1 if keep_samples else 0) for s, o in items]
        reqs = (Request * len(ms))(*[m.req for m in ms])
        jobs = (C.c_uint64 * len(ms))()
        _check(self._L.smc_submit_batch(self.h, reqs, len(ms), jobs), "smc_submit_batch")
        return [int(j) for j in jobs]

    def request_bytes(self, spec: W.Spectrum, opts: W.Options, keep_samples: bool = False) -> int:
        """Device bytes the request would hold while running (smc_request_bytes)."""
        m = _Marshalled(spec, opts, None, 1 if keep_samples else 0)
        b = C.c_size_t()
        _check(self._L.smc_request_bytes(self.h, C.byref(m.req), C.byref(b)), "smc_request_bytes")
        return int(b.value)

    def poll(self, job: int) -> bool:
        d = C.c_int32()
        _check(self._L.smc_poll(self.h, C.c_uint64(job), C.byref(d)), "smc_poll")
        return bool(d.value)

    def wait(self, job: int, timeout_s: float = -1.0):
        _check(self._L.smc_wait(self.h, C.c_uint64(job), float(timeout_s)), "smc_wait")

    # -- tiles -------------------------------------------------------------
    def set_tile(self, family: int, n_max: int, J: int, G: int, regs: int = 0):
        _check(self._L.smc_set_tile(self.h, family, n_max, J, G, regs), "smc_set_tile")

    def clear_tiles(self):
        _check(self._L.smc_set_tile(self.h, 0, 1, 0, 0, 0), "smc_set_tile")

    # -- profiling ---------------------------------------------------------
    def profile_reset(self, events: bool = False):
        _check(self._L.smc_profile_reset(self.h, 1 if events else 0), "smc_profile_reset")

    def profile(self) -> dict:
        p = Profile()
        _check(self._L.smc_profile_read(self.h, C.byref(p)), "smc_profile_read")
        return {"launches": dict(zip(KERNEL_CLASSES, list(p.launches))),
                "ms": dict(zip(KERNEL_CLASSES, list(p.ms))),
                "point_evals": p.point_evals, "sfu_ops": p.sfu_ops,
                "gather_bytes": p.gather_bytes, "resample_bytes": p.resample_bytes,
                "h2d_bytes": p.h2d_bytes, "d2h_bytes": p.d2h_bytes,
                "stages": p.stages, "jobs": p.jobs, "ex2_ops": p.ex2_ops, "rcp_ops": p.rcp_ops,
                "lg2_ops": p.lg2_ops, "max_batch_requests": p.max_batch_requests,
                "peak_point_evals": p.peak_point_evals, "peak_sfu_per_eval": p.peak_sfu_per_eval}

    def mufu_rate(self, op: int, stream=None) -> dict:
        """Measured SFU throughput of EX2 (op 0), RCP (op 1) or LG2 (op 2) on this
        context's device: results per second, the SM clock seen (MHz) and
        results per clock per SM at that clock."""
        rate, per_clk, mhz = C.c_double(), C.c_double(), C.c_double()
        _check(self._L.smc_k_mufu_rate(op, C.byref(rate), C.byref(per_clk), C.byref(mhz), stream),
               "smc_k_mufu_rate")
        return {"ops_per_s": rate.value, "lanes_per_clk_sm": per_clk.value, "sm_mhz": mhz.value}

    # -- step-level entry points (include/smc_kernels.h) -------------------
    def philox(self, seed: int, ctr: np.ndarray) -> np.ndarray:
        ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
        out = np.zeros_like(ctr)
        _check(self._L.smc_k_philox(self.h, seed, _ptr(ctr), _ptr(out), ctr.shape[0]), "smc_k_philox")
        return out

    def energy(self, spec, K: int, opts, nat: np.ndarray, precision: int = 0) -> np.ndarray:
        m = _Marshalled(spec, opts)
        nat = _f64(nat).reshape(-1, max(1, _dim(spec.family, K, spec.bg, spec.bg_degree)))
        E = np.zeros(nat.shape[0])
        _check(self._L.smc_k_energy(self.h, C.byref(m.req), K, _ptr(nat), nat.shape[0], precision,
                                    _ptr(E)), "smc_k_energy")
        return E

    def prior(self, spec, K: int, opts, count: int, precision: int = 0):
        m = _Marshalled(spec, opts)
        d = _dim(spec.family, K, spec.bg, spec.bg_degree)
        nat = np.zeros((count, max(d, 1)))
        E = np.zeros(count)
        _check(self._L.smc_k_prior(self.h, C.byref(m.req), K, count, precision, _ptr(nat), _ptr(E)),
               "smc_k_prior")
        return nat[:, :d], E

    def reweight(self, E: np.ndarray, beta: float, rho: float, precision: int = 1):
        E = _f64(E)
        dl, lz, fin = C.c_double(), C.c_double(), C.c_int32()
        q = np.zeros(E.shape[0], dtype=np.uint64)
        _check(self._L.smc_k_reweight(self.h, _ptr(E), E.shape[0], beta, rho, precision, C.byref(dl),
                                      C.byref(lz), C.byref(fin), _ptr(q)), "smc_k_reweight")
        return dl.value, lz.value, bool(fin.value), q

    def resample(self, q: np.ndarray, M: int, u32: int) -> np.ndarray:
        q = np.ascontiguousarray(q, dtype=np.uint64)
        a = np.zeros(M, dtype=np.int32)
        _check(self._L.smc_k_resample(self.h, _ptr(q), q.shape[0], M, u32, _ptr(a)), "smc_k_resample")
        return a

    def mh_stage(self, spec, K: int, opts, nat_start, E_start, step, beta: float, stage: int,
                 precision: int = 0):
        m = _Marshalled(spec, opts)
        d = _dim(spec.family, K, spec.bg, spec.bg_degree)
        nat_start = _f64(nat_start).reshape(-1, d)
        S = nat_start.shape[0]
        T = S * opts.sweeps if opts.waste_free else S
        E_start, step = _f64(E_start), _f64(step)
        nat_out, E_out = np.zeros((T, d)), np.zeros(T)
        acc, prop = np.zeros(d, dtype=np.int64), np.zeros(d, dtype=np.int64)
        _check(self._L.smc_k_mh_stage(self.h, C.byref(m.req), K, _ptr(nat_start), _ptr(E_start), S,
                                      _ptr(step), beta, stage, precision, _ptr(nat_out), _ptr(E_out),
                                      _ptr(acc), _ptr(prop)), "smc_k_mh_stage")
        return nat_out, E_out, acc, prop


# ---------------------------------------------------------------------------
# one-call form: one known-sigma spectrum, every candidate K (smc_run)
# ---------------------------------------------------------------------------
def make_spectrum(x, y, sigma, k_range, family: int, priors: W.Priors, bg: int = W.BG_NONE,
                  bg_degree: int = 0) -> W.Spectrum:
    """The spectrum record smc_run takes: grid x, data y, per-point sigma (a
    scalar is broadcast to every point), candidate peak counts k_range (a range
    or a (k_min, k_max) pair: every K from its smallest to its largest value),
    peak family, priors of the peak components and the background kind.  An
    empty list of background priors is filled with uniform priors derived from
    the data range (workloads.data_bg_priors)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    s = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma, dtype=np.float64), x.shape))
    ks = [int(k) for k in k_range]
    nbg = W.bg_count(int(bg), int(bg_degree))
    if nbg and not priors.bg:
        priors = W.Priors(amp=priors.amp, centre=priors.centre, width=priors.width, eta=priors.eta,
                          bg=W.data_bg_priors(y, nbg))
    return W.Spectrum(x, y, s, int(family), min(ks), max(ks), int(bg), int(bg_degree), priors, truth={})


def run(x, y, sigma, k_range, family: int, priors: W.Priors, bg: int = W.BG_NONE, bg_degree: int = 0,
        particles: int = 1024, ess: float = 0.5, sweeps: int = 10, waste_free: int = 0,
        energy_fp64: int = 0, seed: int = 1, max_stages: int = 10000, step_rule: int = 0,
        device: int = 0, keep_samples: bool = True) -> dict:
    """Run the sampler on one spectrum for every candidate K and return log Z
    per K, P(K|D), the selected K, posterior summaries and (optionally) the
    samples: smc_create, smc_run, smc_result, smc_release, smc_destroy.  The
    arguments are those of make_spectrum and of smc_options (ess: the ESS
    target of the tempering bisection)."""
    spec = make_spectrum(x, y, sigma, k_range, family, priors, bg, bg_degree)
    opts = W.Options(particles=int(particles), ess_target=float(ess), sweeps=int(sweeps),
                     waste_free=int(waste_free), energy_fp64=int(energy_fp64), seed=int(seed),
                     max_stages=int(max_stages), step_rule=int(step_rule))
    with Context(device) as ctx:
        return ctx.run(spec, opts, keep_samples=keep_samples)
