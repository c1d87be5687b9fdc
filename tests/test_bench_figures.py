"""The bench's roofline figures recomputed by hand: algorithmic bytes of one fused subset
gradient (counts and background per TOF bin, factors m per LOR, one image read and one
gradient write), the windowed TOF kernel's window and name, the issue peak, and the
whole-job rate of independent replicas."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2506_04976_gb300 import synth  # noqa: E402


def _geom(name):
    return synth._setup(name, 0)["geom"]


def _c5():
    return {"geom": _geom("c5"), "nsub": 25}


def test_algorithmic_bytes_c5_and_c2():
    # c5: 224 views x 1293 planes x 357 radial bins / 25 subsets = 4,135,944.96 LORs on
    # average; per LOR 13 x (2 + 4) + 4 = 82 B; image 215 x 215 x 71 = 3,281,975 voxels
    p = _c5()
    assert bench.algorithmic_bytes_per_grad(p, 2) == pytest.approx(4135944.96 * 82 + 8 * 3281975, rel=1e-12)
    # c2: 168 x 109 x 250 / 21 = 218,000 LORs; uint16 counts: 2 + 4 + 4 = 10 B per LOR;
    # 128 x 128 x 47 = 770,048 voxels
    p2 = {"geom": _geom("c2"), "nsub": 21}
    assert bench.algorithmic_bytes_per_grad(p2, 2) == 218000 * 10 + 8 * 770048 == 8340384


def test_tof_window_and_kernel_name():
    g = _geom("c5")
    # 13 bins of 31 mm, sigma 24.83 mm: reach 3 sigma + w/2 = 90.0 mm on each side, a span
    # of 5.8 bin widths, so a sample meets at most 6 bins
    assert bench.tof_window(g) == 6
    assert bench.kernel_name(g, (2, 1)) == "k_grad_tofp<2,6,512>"
    assert bench.kernel_name(g, (4, 2)) == "k_grad_tofk<4,6,2,256>"
    assert bench.kernel_name(_geom("c2"), (2, 8)) == "k_grad_mp<2,8>"


def test_issue_peak_and_replica_rate():
    mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(mp):
        assert bench.issue_peak() == 152 * 4 * 2070e6
    else:
        assert bench.issue_peak() > 1e12
    assert bench.whole_job_rate(74 * 20, 4, 5.0) == 74 * 20 * 4 / 5.0
