"""Autotuner for the fused Metropolis kernel's tile.

The tile (J grid points per lane, G warps per chain, 32 G J >= N, and a
register budget R per thread) decides the kernel's occupancy, spills and
per-proposal reduction cost.  For each peak family and grid-length bucket this
times every admissible tile -- and, for four- and eight-warp chains, every
compiled register budget -- on a short run of a synthetic spectrum (same
spectrum, seed and stages for all) and keeps the fastest Metropolis time.  The
table is stored next to this file (tiles_b300.json) and applied with
`load(ctx)`; the library itself falls back to a padding-minimising default for
buckets the table does not cover.

    python -m paper_2604_03271_b300.autotune      # on a B300: tune and write
"""
from __future__ import annotations

import json
import os
import time
from typing import Dict, List, Optional, Tuple

from . import workloads as W

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiles_b300.json")
BUCKETS = (256, 512, 1024, 2048, 4096)
J_SET = {W.PSEUDO_VOIGT: (4, 8, 12, 16), W.GAUSS: (4, 8, 12, 16, 24, 32), W.LORENTZ: (4, 8, 12, 16, 24, 32)}
COUPLED = 16  # family flag of the coupled-grid kernel (Shirley background, model variance)
J_SET_COUPLED = (4, 8)
G_SET = (1, 2, 4, 8, 16)
# the phase kernel also spreads a chain over a cluster of 8-warp CTAs (G = 8 C)
G_SET_CLUSTER = tuple(8 * c for c in range(3, 17))
BUCKETS_XRD = (512, 1024, 2048, 4096, 5120, 10240)


R_SET = (64, 80, 96, 128)  # register budgets of four- and eight-warp chains with J = 4, 8, 16


def variants(family: int, J: int, G: int) -> List[int]:
    """Register budgets to try for a tile: 0 (the tile's default) and, for the
    fused kernel's four- and eight-warp chains with J = 4, 8, 16, R_SET."""
    if family & COUPLED or G not in (4, 8) or J not in (4, 8, 16):
        return [0]
    return [0] + list(R_SET)


def candidates(family: int, n: int, slack: float = 1.5) -> List[Tuple[int, int]]:
    """Admissible tiles for an n-point grid whose padding is within `slack` of
    the smallest one."""
    tiles = []
    gs = G_SET + (G_SET_CLUSTER if family == W.XRD_PHASE | COUPLED else ())
    for J in (J_SET_COUPLED if family & COUPLED else J_SET[family]):
        for G in gs:
            if G == 16 and J > 8:
                continue
            if J > 16 and G > 1:
                continue
            if 32 * G * J >= n:
                tiles.append((J, G, 32 * G * J))
                break
    best = min(p for _, _, p in tiles)
    return [(J, G) for J, G, p in tiles if p <= slack * best]


def tuning_spectrum(family: int, n: int) -> W.Spectrum:
    if family == W.XRD_PHASE | COUPLED:
        # App. D: three phases (31 parameters), Poisson counts
        return W.xrd_phase(11, n=n, k_min=3, k_max=3)
    if family & COUPLED:
        s = W.xps_shirley(11, n=n, k_true=7, k_min=5, k_max=8)
        fam = family & (COUPLED - 1)
        if fam != W.PSEUDO_VOIGT:
            s.family = fam
            s.priors = W.Priors(amp=s.priors.amp, centre=s.priors.centre, width=s.priors.width,
                                bg=s.priors.bg)
        return s
    s = W.xps_like(11, n=n, k_true=3, k_max=4)
    if family != W.PSEUDO_VOIGT:
        s.family = family
        s.priors = W.Priors(amp=s.priors.amp, centre=s.priors.centre, width=s.priors.width,
                            bg=s.priors.bg)
    return s


def tune(ctx, families=(W.PSEUDO_VOIGT, W.GAUSS, W.LORENTZ, W.PSEUDO_VOIGT | COUPLED, W.XRD_PHASE | COUPLED),
         buckets=BUCKETS,
         particles: int = 8192, sweeps: int = 4, stages: int = 6, verbose: bool = True,
         registers: bool = True) -> List[Dict]:
    table = []
    for fam in families:
        for n in (BUCKETS_XRD if fam == W.XRD_PHASE | COUPLED else buckets):
            spec = tuning_spectrum(fam, n)
            opts = W.Options(particles=particles, sweeps=sweeps, seed=5, max_stages=stages)
            results = []
            for J, G in candidates(fam, n):
                for R in (variants(fam, J, G) if registers else [0]):
                    ctx.clear_tiles()
                    ctx.set_tile(fam, n, J, G, R)
                    ctx.run(spec, W.Options(particles=1024, sweeps=1, seed=1, max_stages=1), keep_samples=False)
                    ctx.profile_reset(events=True)
                    ctx.run(spec, opts, keep_samples=False)
                    p = ctx.profile()
                    ms = p["ms"]["metropolis"]
                    results.append((ms, J, G, R, p["sfu_ops"] / max(ms, 1e-9) / 1e6))
            ms, J, G, R, gops = min(results)
            row = {"family": fam, "n_max": n, "J": J, "G": G, "R": R, "mh_ms": ms, "sfu_gops": gops,
                   "tried": [{"J": j, "G": g, "R": rr, "mh_ms": m} for m, j, g, rr, _ in results]}
            if verbose:
                print(json.dumps(row), flush=True)
            table.append(row)
    ctx.clear_tiles()
    return table


def load(ctx, path: Optional[str] = None) -> int:
    """Apply a tuned table to a context; returns the number of entries."""
    path = path or TABLE
    if not os.path.exists(path):
        return 0
    with open(path) as fh:
        rows = json.load(fh)["tiles"]
    ctx.clear_tiles()
    for r in sorted(rows, key=lambda r: (r["family"], r["n_max"])):
        ctx.set_tile(int(r["family"]), int(r["n_max"]), int(r["J"]), int(r["G"]), int(r.get("R", 0)))
    return len(rows)


def main(argv=None):
    """Tune every family, or only the families given as arguments (their rows
    replace those of the same family in the stored table)."""
    import sys
    from . import api
    fams = [int(a) for a in (sys.argv[1:] if argv is None else argv)]
    ctx = api.Context(0)
    t0 = time.time()
    rows = tune(ctx, families=tuple(fams)) if fams else tune(ctx)
    if fams and os.path.exists(TABLE):
        with open(TABLE) as fh:
            old = [r for r in json.load(fh)["tiles"] if r["family"] not in fams]
        rows = old + rows
    with open(TABLE, "w") as fh:
        json.dump({"device": "B300", "seconds": time.time() - t0, "tiles": rows}, fh, indent=1)
    print("wrote", TABLE)


if __name__ == "__main__":
    main()
