"""CPU checks of the boundary: the CUDA library loads and exports every entry
point that include/*.h declares (no compute call is made without a GPU)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

LIB = os.path.join(ROOT, "paper_2604_03271_b300", "libsmc_b300.so")


def _declared():
    names = set()
    for h in ("smc.h", "smc_kernels.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(smc_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_headers_declare_the_boundary():
    d = _declared()
    for name in ("smc_create", "smc_run", "smc_result", "smc_submit", "smc_poll", "smc_release",
                 "smc_destroy", "smc_strerror", "smc_run_batch", "smc_k_resample", "smc_k_mh_stage"):
        assert name in d


@pytest.mark.skipif(not os.path.exists(LIB), reason="library not built")
def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(LIB)
    for name in _declared():
        assert hasattr(L, name), name


@pytest.mark.skipif(not os.path.exists(LIB), reason="library not built")
def test_strerror_without_gpu():
    L = ctypes.CDLL(LIB)
    L.smc_strerror.restype = ctypes.c_char_p
    assert L.smc_strerror(0) == b"ok"
    assert b"budget" in L.smc_strerror(2)


def test_tile_choice_covers_grid():
    # host logic mirrored: 32 G J >= N with J in the compiled set
    from paper_2604_03271_b300 import workloads as W
    for n in (2, 31, 301, 1001, 4000, 4096):
        for fam in (W.GAUSS, W.PSEUDO_VOIGT):
            Js = [4, 8, 12, 16] if fam == W.PSEUDO_VOIGT else [4, 8, 12, 16, 24, 32]
            assert any(32 * G * J >= n for G in (1, 2, 4, 8) for J in Js)


def test_autotune_candidates_cover_every_bucket():
    from paper_2604_03271_b300 import autotune as A
    from paper_2604_03271_b300 import workloads as W
    for fam in (W.GAUSS, W.LORENTZ, W.PSEUDO_VOIGT):
        for n in A.BUCKETS + (2, 100, 1001, 3999):
            c = A.candidates(fam, n)
            assert c and all(32 * G * J >= n for J, G in c)
            assert all(not (G == 16 and J > 8) for J, G in c)


def test_phase_kernel_tiles_reach_the_paper_grids():
    # the App. D phase kernel: single-block tiles up to 4096 points, then
    # chains spread over clusters of 8-warp CTAs (G = 8 C, C <= 16) up to the
    # paper's N = 10000 and beyond; every candidate covers its bucket
    from paper_2604_03271_b300 import autotune as A
    from paper_2604_03271_b300 import workloads as W
    fam = W.XRD_PHASE | A.COUPLED
    for n in A.BUCKETS_XRD + (1000, 5000, 10000, 16384):
        c = A.candidates(fam, n)
        assert c and all(32 * G * J >= n for J, G in c)
        assert all(G <= 16 or (G % 8 == 0 and G // 8 <= 16) for J, G in c)
        assert all(J in (4, 8) for J, G in c)
    assert max(32 * 128 * J for J in (4, 8)) >= 32768


def test_binding_structs_match_the_headers(tmp_path):
    # the ctypes mirrors of the C structs: same field names, offsets and sizes
    # as a C compiler lays them out from include/*.h (gcc on the host)
    import shutil
    import subprocess
    import ctypes as C
    from paper_2604_03271_b300 import api
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no host C compiler")
    pairs = [(api.Prior, "smc_prior"), (api.Priors, "smc_priors"), (api.CreateOpts, "smc_create_opts"),
             (api.Options, "smc_options"), (api.Request, "smc_request"), (api.ResultView, "smc_result_view"),
             (api.Profile, "smc_profile")]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "smc.h"', '#include "smc_kernels.h"',
             'int main(void) {']
    expect = []
    for cls, cname in pairs:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append(C.sizeof(cls))
        for f in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f[0]}));')
            expect.append(getattr(cls, f[0]).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([gcc, "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect
