"""Host-side pieces of bench.py (no GPU): every selectable workload builds its
synthetic spectrum and names its configuration, and the reference arm has the
per-spectrum work it scales the oracle's rate by (or says it has none)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_2604_03271_b300 import api  # noqa: E402

WORKLOADS = ["xps", "xrd", "gauss", "mixed", "xps_shirley", "xrd_phase", "xrd_phase_5000", "xrd_phase_10000",
             "deconv3", "deconv10", "deconv30"]


def test_every_workload_has_a_config():
    names = set()
    for w in WORKLOADS:
        c = bench.config_of(w, 1)
        assert c["n_points"] >= 2 and c["particles_per_k"] >= 2
        assert c["k_range"][0] <= c["k_range"][1]
        names.add(c["workload"])
    assert len(names) == len(WORKLOADS)


def test_app_d_workloads_are_the_paper_sizes():
    for w, n in (("xrd_phase", 1000), ("xrd_phase_5000", 5000), ("xrd_phase_10000", 10000)):
        s, o = bench.workload(w, 1)
        assert s.n == n and s.k_min == s.k_max == 3 and o.sweeps == 10
        assert api._dim(s.family, 3, s.bg, s.bg_degree) == 31  # the paper's 3 x 9 + 4
        assert w in bench.UNITS_PER_SPECTRUM
