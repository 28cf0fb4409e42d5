#!/usr/bin/env python
"""Throughput benchmark of the batched FP32-energy SMC sampler.

Workload (default): one XRD-shaped spectrum per step -- N = 4096 points on
2 theta in [10, 90] degrees, 10 sparse Lorentzian / pseudo-Voigt peaks with
amplitudes over three decades on a cubic background, Gaussian noise of 1 % of
the maximum -- fitted with pseudo-Voigt peaks + cubic Chebyshev background for
every K = 1..12 at once, 65536 particles per K, 20 Metropolis sweeps per stage,
ESS target 0.5 (seeded synthetic data, see paper_2604_03271_b300/workloads.py).
`--workload xps` is the XPS-shaped one (N = 1001, K = 1..6, 16384 particles
per K, two spectra per step).  One step = one full SMC run (prior to beta = 1,
every K) over a batch of B spectra.  Metric: spectra/s (higher is better).
The timed region runs the shipped launch path (one CUDA graph launch per
run); per-kernel event times (kernel shares, the Metropolis kernel's roofline)
come from a separate untimed pass right after it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 the driver launches one rank per GPU with torchrun; spectra are
sharded across ranks (independent jobs, no collective on the data path).
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_03271_b300 import workloads as W  # noqa: E402
from paper_2604_03271_b300.sharding import max_over_ranks, shard_seeds  # noqa: E402

METRIC = "spectra/s (all candidate K per spectrum, |dlogZ|<=0.05 vs FP64)"
SM_COUNT = 148
# DRAM bytes (read + write) of one k_mh launch per spectrum, from ncu captures
# of one spectrum per step, per workload; valid only for the kernel source
# (k_mh_impl.cuh, by sha1) they were taken on; scaled by the spectra a launch
# processes (the particle state of each spectrum's jobs is its own)
MH_TRAFFIC = {"xps": {"sha1": "6bb139c702a2", "bytes_per_spectrum": 6.608e6 + 0.529e6},
              "xrd": {"sha1": "6bb139c702a2", "bytes_per_spectrum": 105.22e6 + 58.61e6}}
SFU_PER_SM_CLK = 16  # MUFU results per SM per clock (EX2, RCP)


_MIXED = None


def workload(name: str, seed: int):
    global _MIXED
    if name == "mixed":
        if _MIXED is None:
            _MIXED = W.mixed_batch(1, count=256)
        return _MIXED[(seed - 1) % len(_MIXED)]
    if name == "xps":
        return W.xps_like(seed), W.Options(particles=16384, sweeps=20, seed=seed)
    if name == "xps_wf":
        # waste-free SMC (Sec. II B 3): 16384 chains per K resampled from
        # 20 x 16384 carried particles, every sweep's state kept
        return W.xps_like(seed), W.Options(particles=16384 * 20, sweeps=20, waste_free=1, seed=seed)
    if name == "xrd":
        return W.xrd_like(seed), W.Options(particles=65536, sweeps=20, seed=seed)
    if name == "gauss":
        return W.gaussian_small(seed), W.Options(particles=1024, sweeps=10, seed=seed)
    if name == "xps_shirley":
        # App. E: PV peaks on a Shirley background, model-dependent variance,
        # the paper's data-derived priors, K = 5..8 (the paper compares 6, 7, 8)
        return W.xps_shirley(seed), W.Options(particles=16384, sweeps=20, seed=seed)
    if name.startswith("xrd_phase"):
        # App. D: three TiO2-like phases (31 parameters) on N = 1000 / 5000 /
        # 10000 points of 2 theta, Poisson counts, the paper's n = 10 sweeps; T
        # from the paper's range (100 x {1 .. 10000}): 10^5 / 3 10^4 / 10^4
        n = {"xrd_phase": 1000, "xrd_phase_5000": 5000, "xrd_phase_10000": 10000}[name]
        T = {1000: 100000, 5000: 30000, 10000: 10000}[n]
        return W.xrd_phase(seed, n=n, k_min=3, k_max=3), W.Options(particles=T, sweeps=10, seed=seed)
    if name.startswith("deconv"):
        # App. C Gaussian deconvolution at the true K, the paper's sweeps per
        # stage; particles from the paper's range (100 x {3 .. 10000})
        K = int(name[6:])
        T = {3: 100000, 10: 100000, 30: 30000}[K]
        return (W.gaussian_deconvolution(K, seed),
                W.Options(particles=T, sweeps=W.DECONV_SWEEPS[K], seed=seed))
    raise ValueError(name)


def config_of(name: str, batch: int) -> dict:
    s, o = workload(name, 1)
    return {"workload": {"xps": "xps-pv-1001", "xps_wf": "xps-pv-1001-waste-free", "xrd": "xrd-pv-4096",
                         "gauss": "gauss-301",
                         "mixed": "mixed-256", "xps_shirley": "xps-shirley-model-variance-840",
                         "xrd_phase": "xrd-phase-poisson-K3-1000", "xrd_phase_5000": "xrd-phase-poisson-K3-5000",
                         "xrd_phase_10000": "xrd-phase-poisson-K3-10000",
                         "deconv3": "deconv-gauss-K3-300",
                         "deconv10": "deconv-gauss-K10-1000", "deconv30": "deconv-gauss-K30-3000"}[name],
            "n_points": s.n, "k_range": [s.k_min, s.k_max], "particles_per_k": o.particles,
            "sweeps": o.sweeps, "ess_target": o.ess_target, "spectra_per_step": batch,
            "waste_free": bool(o.waste_free),
            "family": {W.GAUSS: "gauss", W.LORENTZ: "lorentz", W.PSEUDO_VOIGT: "pseudo-voigt",
                       W.GAUSS_PRECISION: "gauss-precision", W.XRD_PHASE: "xrd-phase"}[s.family],
            "l2": "flushed between steps (256 MiB write)"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [t.strip() for t in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# the oracle, timed on a bounded sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_rate(name: str, seconds: float = 12.0) -> dict:
    """Particle-point evaluations per second of the FP64 oracle on a bounded
    sample of the workload: one Metropolis stage (beta = 1e-3) of a few chains
    for every candidate K, from prior draws."""
    import oracle

    spec, opts = workload(name, 1)
    t0 = time.perf_counter()
    units = 0.0
    chains = 0
    ks = list(range(spec.k_min, spec.k_max + 1))
    o = W.Options(particles=4, sweeps=1, seed=3)
    while time.perf_counter() - t0 < seconds:
        for K in ks:
            u, E = oracle.init_particles(spec, K, o, 4)
            d = u.shape[1]
            step = 0.05 * np.maximum(np.abs(u).mean(0), 1e-3)
            _, _, acc, prop = oracle.mh_stage(spec, K, o, u, E, step, 1e-3, 1)
            units += float(prop.sum()) * spec.n
            chains += 4
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return {"units_per_s": units / dt, "seconds": dt,
            "sample": f"{chains} chains x 1 sweep over K={ks[0]}..{ks[-1]} (FP64 oracle, full energy "
                      f"per proposal), scaled by the GPU run's particle-point evaluations per spectrum"}


def _oracle_worker(a):
    name, seconds = a
    return oracle_rate(name, seconds)


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_pool():
    """One process per host core, started with spawn (no CUDA state inherited)."""
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(os.cpu_count() or 1)


def oracle_rate_all_cores(name: str, seconds: float, pool=None) -> dict:
    """oracle_rate on every host core at once: one process per core, each
    timing its own bounded sample for `seconds`; the rates add up."""
    procs = os.cpu_count() or 1
    own = pool is None
    if own:
        pool = oracle_pool()
    try:
        res = pool.map(_oracle_worker, [(name, seconds)] * procs)
    finally:
        if own:
            pool.close()
            pool.join()
    rate = sum(r["units_per_s"] for r in res)
    chains = res[0]["sample"].split(" chains")[0]
    return {"units_per_s": rate, "seconds": max(r["seconds"] for r in res), "cores": procs,
            "cpu": cpu_model(),
            "sample": f"{procs} processes x ({res[0]['sample']}); process 0 ran {chains} chains"}


def reference_arm(args, world: int, rank: int):
    if rank != 0:
        return
    name = args.workload
    # particle-point evaluations per spectrum of this workload (measured on the
    # GPU arm; stated constant so the reference arm needs no GPU)
    per_spec = UNITS_PER_SPECTRUM.get(name)
    if per_spec is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no measured particle-point evaluations per "
                                                              f"spectrum for workload {name}"}), flush=True)
        return
    step_s = []
    rates = []
    pool = oracle_pool()
    for k in range(args.warmup + args.steps):
        r = oracle_rate_all_cores(name, seconds=max(2.0, 60.0 / (args.warmup + args.steps)), pool=pool)
        if k >= args.warmup:
            step_s.append(r["seconds"])
            rates.append(r["units_per_s"])
    pool.close()
    pool.join()
    rate = float(np.mean(rates))
    value = rate / per_spec
    line = {"metric": METRIC, "value": value, "unit": "spectra/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.mean(step_s)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(name, args.batch), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "spectra/s", "cores": r["cores"], "cpu": r["cpu"],
                             "kind": "oracle", "sample": r["sample"], "units_per_s": rate},
            "e2e": {"value": value, "unit": "spectra/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# particle-point evaluations per spectrum (prior energies + every evaluated
# proposal x N), from the GPU arm's own counters on the same seeds
UNITS_PER_SPECTRUM = {"xps": 7.70e11, "xps_wf": 7.73e11, "xrd": 5.73e13, "gauss": 8.0e8, "mixed": 8.64e11,
                      "xps_shirley": 1.10e12, "xrd_phase": 9.63e11, "xrd_phase_5000": 2.2e12,
                      "xrd_phase_10000": 1.7e12, "deconv3": 3.6e10, "deconv10": 8.24e11, "deconv30": 4.8e13}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="xrd", choices=["xps", "xps_wf", "xrd", "gauss", "mixed", "xps_shirley", "xrd_phase", "xrd_phase_5000",
                                                       "xrd_phase_10000", "deconv3", "deconv10",
                                                       "deconv30"])
    ap.add_argument("--batch", type=int, default=None,
                    help="spectra per step per GPU (default: 1 for xrd, 2 otherwise)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-sample", type=int, default=None,
                    help="time the plain FP64 path on a sample (default: on, except for xrd, where one "
                         "plain stage of K = 12 takes minutes)")
    ap.add_argument("--serve-rate", type=float, default=None,
                    help="Poisson arrivals per s (0: skip; default 1.0, 0 for xrd: its serving is the "
                         "separate --serving-sweep)")
    ap.add_argument("--serve-requests", type=int, default=12)
    ap.add_argument("--event-steps", type=int, default=1,
                    help="steps of the untimed per-kernel event pass (kernel shares, roofline)")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="steps of the end-to-end pass (default 3, 1 for xrd)")
    ap.add_argument("--particles", type=int, default=0,
                    help="particles per K instead of the workload's (smaller cases for profilers)")
    ap.add_argument("--serving-sweep", action="store_true",
                    help="only the serving sweep (Poisson mix of XPS- and XRD-shaped requests)")
    ap.add_argument("--serve-rates", default="0.5,1.0,3.0")
    ap.add_argument("--serve-saturate", type=float, default=2.0,
                    help="rates at or above this are saturation probes (half the requests)")
    ap.add_argument("--serve-particles", type=int, default=2048)
    ap.add_argument("--plain-requests", type=int, default=0)
    args = ap.parse_args()

    if args.serving_sweep:
        serving_sweep(args)
        return
    big = args.workload == "xrd"
    if args.batch is None:
        args.batch = 1 if big else 2
    if args.plain_sample is None:
        args.plain_sample = 0 if big else 1
    if args.serve_rate is None:
        args.serve_rate = 0.0 if big else 1.0
    if args.e2e_steps is None:
        args.e2e_steps = 1 if big else 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        reference_arm(args, world, rank)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2604_03271_b300 import api

    stream = torch.cuda.current_stream(dev)
    ctx = api.Context(local, stream=stream.cuda_stream)
    from paper_2604_03271_b300 import autotune
    n_tiles = autotune.load(ctx)  # tuned Metropolis tiles, if a table is present
    # SFU throughput of this device (roofline denominator), before any timing
    mufu = {"ex2": ctx.mufu_rate(0, stream.cuda_stream), "rcp": ctx.mufu_rate(1, stream.cuda_stream),
            "lg2": ctx.mufu_rate(2, stream.cuda_stream)}
    B = args.batch
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def batch_for(step: int):
        items = [workload(args.workload, seed) for seed in shard_seeds(step, world, rank, B)]
        if args.particles:
            import dataclasses
            items = [(s, dataclasses.replace(o, particles=args.particles)) for s, o in items]
        return items

    def to_dev(items):
        out = []
        for s, _ in items:
            out.append(tuple(torch.tensor(a, dtype=torch.float64, device=dev) for a in (s.x, s.y, s.sigma)))
        return out

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---- warm-up (untimed)
    for k in range(args.warmup):
        items = batch_for(k)
        ctx.run_batch(items, keep_samples=False, device_arrays=to_dev(items))

    # ---- timed: inputs resident in HBM, the shipped launch path (each run is
    # one CUDA graph launch: a conditional while node over the stages)
    steps = [batch_for(args.warmup + k) for k in range(args.steps)]
    dev_in = [to_dev(it) for it in steps]
    ctx.profile_reset(events=False)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in steps]
    results = []
    t_wall = time.perf_counter()
    for k, items in enumerate(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        results.append(ctx.run_batch(items, keep_samples=False, device_arrays=dev_in[k]))
        ev[k][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    prof = ctx.profile()
    total_ms = max_over_ranks(float(sum(step_ms)), dist, dev)
    spectra = args.steps * B * world
    value = spectra / (total_ms / 1000.0)

    # ---- per-kernel CUDA events: a separate, untimed pass over the first
    # steps with host-replayed four-stage graphs (the same kernels in the same
    # order, with event nodes between kernel classes; a conditional graph
    # node's body takes no event nodes)
    n_ev = max(1, min(args.steps, args.event_steps))
    ctx.profile_reset(events=True)
    barrier()
    for k in range(n_ev):
        flush.fill_(float(k))
        ctx.run_batch(steps[k], keep_samples=False, device_arrays=dev_in[k])
    barrier()
    prof_ev = ctx.profile()
    launches_per_stage = sum(prof_ev["launches"].values()) / max(1, prof_ev["stages"])

    # ---- end to end through the public API: host inputs, results to host
    n_e2e = max(1, min(args.steps, args.e2e_steps))
    ctx.profile_reset(events=False)
    barrier()
    e2e_ms = 0.0
    for k in range(n_e2e):
        flush.fill_(float(k))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.run_batch(steps[k], keep_samples=False)
        e2e_ms += 1000.0 * (time.perf_counter() - t0)
    prof_e2e = ctx.profile()
    e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    # the device-timed rate of the same steps (same spectra and seeds), for a
    # like-for-like comparison when the end-to-end pass covers fewer steps
    dev_same_ms = max_over_ranks(float(sum(step_ms[:n_e2e])), dist, dev)
    e2e = {"value": n_e2e * B * world / (e2e_ms / 1000.0), "unit": "spectra/s",
           "h2d_bytes_per_step": prof_e2e["h2d_bytes"] / n_e2e,
           "d2h_bytes_per_step": prof_e2e["d2h_bytes"] / n_e2e, "steps": n_e2e,
           "device_value_same_steps": n_e2e * B * world / (dev_same_ms / 1000.0)}

    # ---- roofline of the dominant kernel (fused Metropolis, SFU-issue bound),
    # from the event pass: algorithmic SFU operations per launch over the
    # launch's average event-timed duration
    mh_ms = prof_ev["ms"]["metropolis"]
    mh_n = max(1, prof_ev["launches"]["metropolis"])
    launch_s = mh_ms / mh_n / 1000.0
    # the kernel's own count: SFU operations of the centre / width proposals
    # (the current shape's re-evaluation per block not counted)
    sfu_kernel = (prof_ev["sfu_ops"] + 2.0 * prof_ev["lg2_ops"]) / mh_n
    achieved_kernel = sfu_kernel / launch_s / 1e9 if mh_ms > 0 else 0.0
    # the method's count per unit (one new peak evaluation per peak-component
    # point evaluation: EX2 for a Gaussian, RCP for a Lorentzian, both for a
    # pseudo-Voigt; none for background components) x the units of a launch
    if prof_ev.get("peak_point_evals", 0.0) > 0:
        units_launch = prof_ev["peak_point_evals"] / mh_n
        sfu_per_launch = units_launch * prof_ev["peak_sfu_per_eval"]
        count = "method count: %.0f SFU op per peak-component point evaluation" % prof_ev["peak_sfu_per_eval"]
    else:
        units_launch = None
        sfu_per_launch = sfu_kernel
        count = "kernel count: SFU ops of evaluated shape proposals"
    achieved = sfu_per_launch / launch_s / 1e9 if mh_ms > 0 else 0.0
    # denominator: the SFU rate measured on this device for the workload's mix
    # of EX2, RCP and LG2 (time-weighted harmonic combination of the rates);
    # algorithmic units: the shape operations plus the model variance's LG2/RCP
    rx, rr, rl = mufu["ex2"]["ops_per_s"], mufu["rcp"]["ops_per_s"], mufu["lg2"]["ops_per_s"]
    n_ex2, n_rcp, n_lg2 = prof_ev["ex2_ops"], prof_ev["rcp_ops"], prof_ev["lg2_ops"]
    n_all = n_ex2 + n_rcp + n_lg2
    peak = (n_all / (n_ex2 / rx + n_rcp / rr + n_lg2 / rl) if n_all > 0 else rx) / 1e9
    nominal = SM_COUNT * SFU_PER_SM_CLK * 2032e6 / 1e9
    import hashlib
    src = open(os.path.join(ROOT, "paper_2604_03271_b300", "csrc", "k_mh_impl.cuh"), "rb").read()
    tr = MH_TRAFFIC.get(args.workload)
    same_kernel = tr is not None and hashlib.sha1(src).hexdigest()[:12] == tr["sha1"]
    # per launch: the bytes of the spectra one launch processes (a launch
    # advances every spectrum of the step by one stage)
    traffic = tr["bytes_per_spectrum"] * B if same_kernel else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s (SFU)",
                "frac": achieved / peak, "traffic": traffic, "count": count,
                "units_per_launch": units_launch, "sfu_ops_per_launch": sfu_per_launch,
                "achieved_kernel_count": achieved_kernel, "frac_kernel_count": achieved_kernel / peak,
                "kernel": "k_mh (fused Metropolis)", "avg_launch_ms": mh_ms / mh_n,
                "peak_note": ("measured EX2 %.1f / RCP %.1f / LG2 %.1f results per clock per SM at %.0f MHz "
                              "(smc_k_mufu_rate), mix %.0f%% EX2 %.0f%% RCP %.0f%% LG2; a 16/clk/SM SFU x "
                              "148 x 2032 MHz would be %.0f Gop/s (frac %.3f)"
                              % (mufu["ex2"]["lanes_per_clk_sm"], mufu["rcp"]["lanes_per_clk_sm"],
                                 mufu["lg2"]["lanes_per_clk_sm"], mufu["ex2"]["sm_mhz"],
                                 100.0 * n_ex2 / max(n_all, 1.0), 100.0 * n_rcp / max(n_all, 1.0),
                                 100.0 * n_lg2 / max(n_all, 1.0), nominal, achieved / nominal)),
                "peak_measured": {k: v for k, v in mufu.items()}}
    shares = {k: prof_ev["ms"][k] for k in prof_ev["ms"]}
    tot = sum(shares.values()) or 1.0
    gather_gbs = (prof_ev["gather_bytes"] / (prof_ev["ms"]["gather"] / 1000.0) / 1e9
                  if prof_ev["ms"]["gather"] else None)
    resample_gbs = (prof_ev["resample_bytes"] / (prof_ev["ms"]["resample"] / 1000.0) / 1e9
                    if prof_ev["ms"]["resample"] else None)
    units_per_spec = prof["point_evals"] / (args.steps * B)

    # ---- parity spot check against the plain FP64 path and the oracle is in
    # the tests; here: model selection summary
    lz = [list(map(float, r["log_z"])) for res in results for r in res]
    sel = [int(r["argmax_k"]) if r["argmax_k"] is not None else None for res in results for r in res]

    line = {"metric": METRIC, "value": value, "unit": "spectra/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 energies, Metropolis and ESS-search weights (Kahan); f64 evidence, beta and moment totals",
            "data": "synthetic", "config": dict(config_of(args.workload, B),
                                                **({"particles_per_k": args.particles} if args.particles else {})),
            "impl": "ours",
            "e2e": e2e,
            # kernels of the timed runs: every stage's kernels (counted in the
            # event pass) times the stages run, plus six set-up and result
            # kernels per spectrum
            "gpu_launches": int(round(prof["stages"] * launches_per_stage)) + 6 * args.steps * B,
            "clocks": clk, "roofline": roofline,
            "particle_point_evals_per_s": prof["point_evals"] / (total_ms / 1000.0) * world,
            "kernel_ms_share": {k: v / tot for k, v in shares.items()},
            "gather_gbs": gather_gbs, "resample_gbs": resample_gbs,
            "stages": prof["stages"], "jobs": prof["jobs"], "selected_k": sel,
            "units_per_spectrum": units_per_spec, "wall_s": t_wall, "tuned_tiles": n_tiles}

    if rank == 0 and args.serve_rate > 0:
        line["serving"] = serve_sample(api, local, args.workload, args.serve_rate, args.serve_requests)
    if rank == 0 and args.plain_sample:
        line["plain_fp64"] = plain_sample(ctx, args.workload, units_per_spec)
    if rank == 0 and not args.no_cpu_baseline:
        r = oracle_rate_all_cores(args.workload, seconds=12.0)
        line["cpu_baseline"] = {"value": r["units_per_s"] / units_per_spec, "unit": "spectra/s",
                                "cores": r["cores"], "cpu": r["cpu"], "kind": "oracle",
                                "sample": r["sample"], "units_per_s": r["units_per_s"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def serve_sample(api, device: int, name: str, rate: float, count: int) -> dict:
    """Continuous-batching serving loop: requests arrive as a Poisson stream,
    are submitted on arrival (smc_submit) and waited for; latency is the
    library's submit-to-result time."""
    import threading

    from paper_2604_03271_b300 import autotune
    ctx = api.Context(device)
    autotune.load(ctx)
    items = [workload(name, 1000 + i) for i in range(count)]
    arrivals = W.poisson_arrivals(rate, count, seed=7)
    jobs = [None] * count
    t0 = time.perf_counter()

    def submitter():
        for i, (s, o) in enumerate(items):
            delay = arrivals[i] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            jobs[i] = ctx.submit(s, o)

    th = threading.Thread(target=submitter)
    th.start()
    lat = []
    t_done = 0.0
    for i in range(count):
        while jobs[i] is None:
            time.sleep(0.001)
        ctx.wait(jobs[i], 600.0)
        r = ctx.result(jobs[i], items[i][0])
        lat.append(r["latency_ms"])
        t_done = time.perf_counter() - t0
        ctx.release(jobs[i])
    th.join()
    ctx.close()
    lat = np.array(lat)
    return {"offered_per_s": rate, "requests": count, "achieved_per_s": count / max(t_done, 1e-9),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "note": "FP32 batched path; arrivals from t = 0"}


def serve_stream(api, device: int, items, rate: float, seed: int = 7) -> dict:
    """Submit `items` on a Poisson arrival stream of `rate` requests/s to one
    context (continuous batching); per-request latency is the library's
    submit-to-result time.  Returns offered and achieved load and the latency
    percentiles."""
    import threading

    from paper_2604_03271_b300 import autotune
    ctx = api.Context(device)
    autotune.load(ctx)
    count = len(items)
    arrivals = W.poisson_arrivals(rate, count, seed=seed)
    jobs = [None] * count
    t0 = time.perf_counter()

    def submitter():
        for i, (s, o) in enumerate(items):
            delay = arrivals[i] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            jobs[i] = ctx.submit(s, o)

    th = threading.Thread(target=submitter)
    th.start()
    lat = np.zeros(count)
    ok = 0
    for i in range(count):
        while jobs[i] is None:
            time.sleep(0.0005)
        ctx.wait(jobs[i], 3600.0)
        r = ctx.result(jobs[i], items[i][0])
        lat[i] = r["latency_ms"]
        ok += int(r["status"] == 0)
        ctx.release(jobs[i])
    t_done = time.perf_counter() - t0
    th.join()
    prof = ctx.profile()
    ctx.close()
    span = max(t_done - arrivals[0], 1e-9)
    return {"offered_per_s": rate, "requests": count, "ok": ok,
            "achieved_per_s": count / span, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "max_ms": float(lat.max()), "max_batch_requests": prof["max_batch_requests"]}


def serving_sweep(args):
    """Serving: a Poisson stream mixing XPS-shaped (N = 1001, K = 1..6) and
    XRD-shaped (N = 4096, K = 1..12) spectra 50/50, served by the FP32 batched
    path with continuous batching at several offered rates, and the plain FP64
    one-spectrum-per-launch path on the same kind of requests one at a time."""
    import torch

    from paper_2604_03271_b300 import api
    torch.cuda.set_device(0)
    T = args.serve_particles

    def mix(n, seed0):
        out = []
        for i in range(n):
            if i % 2 == 0:
                out.append((W.xps_like(seed0 + i), W.Options(particles=T, sweeps=20, seed=seed0 + i)))
            else:
                out.append((W.xrd_like(seed0 + i), W.Options(particles=T, sweeps=20, seed=seed0 + i)))
        return out

    rates = [float(r) for r in args.serve_rates.split(",")]
    res = {"workload": "poisson mix: 50% xps-pv-1001 (K=1..6), 50% xrd-pv-4096 (K=1..12)",
           "particles_per_k": T, "sweeps": 20, "rates": []}
    for k, rate in enumerate(rates):
        n = args.serve_requests if rate < args.serve_saturate else max(args.serve_requests // 2, 20)
        res["rates"].append(serve_stream(api, 0, mix(n, 10000 * (k + 1)), rate, seed=11 + k))
        print(json.dumps(res["rates"][-1]), flush=True)
    res["saturation_per_s"] = max(r["achieved_per_s"] for r in res["rates"])
    if args.plain_requests > 0:
        ctx = api.Context(0)
        lat = []
        for i in range(args.plain_requests):
            s = W.xps_like(50000 + i)
            t0 = time.perf_counter()
            r = ctx.run(s, W.Options(particles=T, sweeps=20, seed=50000 + i, energy_fp64=1), keep_samples=False)
            lat.append(1000.0 * (time.perf_counter() - t0))
            assert r["status"] == 0
        ctx.close()
        res["plain_fp64_xps"] = {"requests": len(lat), "p50_ms": float(np.percentile(lat, 50)),
                                 "max_ms": float(np.max(lat)), "note": "one request at a time, XPS-shaped only"}
    print(json.dumps({"serving_sweep": res}), flush=True)


def plain_sample(ctx, name: str, units_per_spec: float) -> dict:
    """The plain one-spectrum-per-launch FP64 path on a bounded sample: the
    first tempering stage of one spectrum, every K, at the workload's full
    particle count.  Its particle-point evaluation rate, scaled by the
    workload's evaluations per spectrum, gives its spectra/s."""
    spec, o = workload(name, 1)
    # the App. D model costs ~40 FP64 pseudo-Voigts per particle-point: a fifth
    # of its particles keeps the sample near ten seconds (the rate per
    # particle-point is what is scaled; 20000 threads fill the device)
    T = min(o.particles, 20000 * 1000 // spec.n) if name.startswith("xrd_phase") else o.particles
    opts = W.Options(particles=T, sweeps=o.sweeps, seed=1, energy_fp64=1, max_stages=1)
    ctx.profile_reset(events=False)
    t0 = time.perf_counter()
    ctx.run(spec, opts, keep_samples=False)
    dt = time.perf_counter() - t0
    p = ctx.profile()
    rate = p["point_evals"] / dt
    return {"units_per_s": rate, "spectra_per_s": rate / units_per_spec, "seconds": dt,
            "sample": f"1 stage, T={opts.particles}, K={spec.k_min}..{spec.k_max}, FP64 thread-per-chain"}


if __name__ == "__main__":
    main()
