import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running statistical check")


def load_golden(name):
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def estimator_stats(ctx, spec, seeds, **kw):
    """log Z per K of the FP32 batched path and of the batched FP64 path (the
    plain FP64 kernels, which replay the oracle) over the same seeds, each in
    one batched call: arrays [seed][K] and the selected K of every run."""
    import numpy as np

    from paper_2604_03271_b300 import workloads as W
    a = ctx.run_batch([(spec, W.Options(seed=s, **kw)) for s in seeds], keep_samples=False)
    b = ctx.run_batch([(spec, W.Options(seed=s, energy_fp64=2, **kw)) for s in seeds], keep_samples=False)
    assert all(r["status"] == 0 for r in a + b)
    return (np.array([r["log_z"] for r in a]), np.array([r["log_z"] for r in b]),
            [r["argmax_k"] for r in a], [r["argmax_k"] for r in b])


def diff_and_se(lz32, lz64):
    """|difference of the means| per K and the combined standard error."""
    import numpy as np
    se = np.sqrt(lz32.var(axis=0, ddof=1) / lz32.shape[0] + lz64.var(axis=0, ddof=1) / lz64.shape[0])
    return np.abs(lz32.mean(0) - lz64.mean(0)), se
