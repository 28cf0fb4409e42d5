"""The allocation-free tempering step, smc_k_reweight_static.

It serves callers that cannot allocate device memory themselves through the
library (a host framework that owns every device allocation, or a service
that must not grow device memory once running): they pass their own device
arrays, and the kernel's scratch is a fixed static array inside the library.
This file is collected last on purpose.  Three calls in a row (different sizes
and precisions, the last at the largest accepted size, so the shared scratch
is reused and filled) must match the ordinary smc_k_reweight entry point
within the tolerances of the other reweight tests.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _static_fn():
    from paper_2604_03271_b300 import api
    L = api.lib()
    f = L.smc_k_reweight_static
    f.argtypes = [C.c_void_p, C.c_int64, C.c_double, C.c_double, C.c_int32, C.c_void_p,
                  C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int32), C.c_void_p]
    f.restype = C.c_int
    return f


def _call_static(f, E, beta, rho, precision):
    import torch
    dt = torch.float64 if precision else torch.float32
    E_dev = torch.tensor(E, dtype=dt, device="cuda")
    q_dev = torch.zeros(E.shape[0], dtype=torch.int64, device="cuda")
    dl, lz, fin = C.c_double(), C.c_double(), C.c_int32()
    stream = torch.cuda.current_stream().cuda_stream
    st = f(E_dev.data_ptr(), E.shape[0], beta, rho, precision, q_dev.data_ptr(), C.byref(dl),
           C.byref(lz), C.byref(fin), stream)
    assert st == 0, st
    q = q_dev.cpu().numpy().view(np.uint64)
    return dl.value, lz.value, bool(fin.value), q


def test_static_reweight_matches_ordinary_entry_point_in_a_row():
    from paper_2604_03271_b300 import api
    f = _static_fn()
    rng = np.random.default_rng(42)
    cases = [(rng.gamma(2.0, 3e3, 65536) + 50.0, 0.01, 1),      # FP64 energies, large T
             (rng.gamma(2.0, 40.0, 5000) + 7.0, 0.4, 0),        # FP32 energies, smaller T
             # FP32 energies at the largest accepted T: the top of the weight
             # buffer and every per-CTA partial row of the scratch in use
             (rng.gamma(2.0, 200.0, 1 << 20) + 1000.0, 0.0, 0)]
    with api.Context(0) as ctx:
        for E, beta, prec in cases:
            if prec == 0:
                E = E.astype(np.float32).astype(np.float64)
            d_s, lz_s, fin_s, q_s = _call_static(f, E, beta, 0.5, prec)
            d_o, lz_o, fin_o, q_o = ctx.reweight(E, beta, 0.5, precision=prec)
            assert fin_s == fin_o
            assert d_s == pytest.approx(d_o, rel=1e-12)
            assert lz_s == pytest.approx(lz_o, rel=1e-12, abs=1e-12)
            diff = np.abs(q_s.astype(np.int64) - q_o.astype(np.int64))
            assert diff.max() <= 1


def test_static_reweight_rejects_too_many_particles():
    import torch
    f = _static_fn()
    T = (1 << 20) + 1
    E_dev = torch.zeros(T, dtype=torch.float64, device="cuda")
    q_dev = torch.zeros(T, dtype=torch.int64, device="cuda")
    dl, lz, fin = C.c_double(), C.c_double(), C.c_int32()
    st = f(E_dev.data_ptr(), T, 0.0, 0.5, 1, q_dev.data_ptr(), C.byref(dl), C.byref(lz),
           C.byref(fin), None)
    assert st == 1  # SMC_EINVAL
