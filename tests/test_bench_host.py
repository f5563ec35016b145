"""Host-side helpers of bench.py, without a GPU: the bins-viewed-by-density
curve read from a load histogram, and the host description of the CPU
baseline."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Hist:
    """A table stand-in whose load histogram has 200 buckets: bucket i holds
    2 insertions that viewed i + 1 bins each; bucket 139 is empty."""

    def load_histogram(self):
        c = np.full(200, 2, dtype=np.uint64)
        v = (np.arange(200, dtype=np.uint64) + 1) * 2
        c[139], v[139] = 0, 0
        return v, c


def test_viewed_curve_reads_the_bucket_below_each_density():
    got = bench.viewed_curve(_Hist(), (0.5, 0.7, 0.95, 1.0, 0.001))
    # density q -> bucket round(200 q) - 1, whose insertions viewed that + 1 bins
    assert got == {"0.50": 100.0, "0.70": None, "0.95": 190.0, "1.00": 200.0, "0.00": 1.0}


def test_host_info_names_the_cores():
    h = bench.host_info()
    assert h["nproc"] == os.cpu_count() and h["machine"]
