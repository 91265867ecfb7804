"""CPU pins of constant tables in the device Hankel code (csrc/hankel.cuh), read from the source:
the ascending series' stopping thresholds against their definition, and the zone radii against
the host table's reach (no GPU needed)."""
import math
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2512_14193_gb300", "csrc")


def _text(name):
    return open(os.path.join(SRC, name)).read()


def test_series_thresholds_match_their_definition():
    # THR[m-1] is the largest |w| = |z|^2/4 with |w|^m / (m!)^2 <= 1e-17: the series stops at the
    # first m with |w| <= THR[m-1]
    m = re.search(r"constexpr float THR\[(\d+)\]\s*=\s*\{([^}]*)\}", _text("hankel.cuh"))
    assert m, "threshold table not found"
    n = int(m.group(1))
    vals = [float(v.strip().rstrip("f")) for v in m.group(2).split(",") if v.strip()]
    assert len(vals) == n == 15
    for k, v in enumerate(vals, start=1):
        exact = (1e-17 * math.factorial(k) ** 2) ** (1.0 / k)
        assert abs(v - exact) <= 2e-5 * exact, (k, v, exact)
    assert all(a < b for a, b in zip(vals, vals[1:]))          # the stop test is monotone in m
    # at the zone edge |z| = 3 (|w| = 2.25) terms 1 .. 14 are summed and the stop comes at m = 15,
    # inside the loop's 15 steps
    assert vals[-1] > 2.25 and vals[-2] < 2.25


def test_zone_radii_fit_the_anchor_table():
    h = _text("hankel.cuh")
    rs = float(re.search(r"constexpr double R_SERIES = ([0-9.]+);", h).group(1))
    ra = float(re.search(r"constexpr double R_ASYM = ([0-9.]+);", h).group(1))
    t = _text("hankel_table.cu")
    r_tab = float(re.search(r"constexpr double R_TAB = ([0-9.]+);", t).group(1))
    step = float(re.search(r"g_step = ([0-9.]+)", t).group(1))
    # every z of the Taylor zone has its nearest anchor within the filled annulus 2.5 <= |z0| <= R_TAB
    reach = step / np.sqrt(2.0)
    assert rs - reach >= 2.5 and ra + reach <= r_tab
    # the coefficient layout: FP64 a_0 .. a_8 and FP32 a_9 .. a_18, two FP32 per 16-byte slot
    c = _text("common.cuh")
    k64 = int(re.search(r"HT_K64 = (\d+)", c).group(1))
    k32 = int(re.search(r"HT_K32 = (\d+)", c).group(1))
    assert re.search(r"HT_SLOTS = HT_K64 \+ HT_K32 / 2;", c)
    assert k64 == 9 and k32 == 10
