"""Host-side logic of the benchmark, without a GPU: the closed-form sample
count behind the projector's L1 roofline, the clock-record summary, and the
traffic ratios taken from the ncu captures."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2202_08627_gb300 import inputs  # noqa: E402

TWO32 = 1 << 32


def samples_by_enumeration(n, n_theta, n_det):
    """Samples of the ray-driven projector (Eq. 1 with linear interpolation)
    counted ray by ray the way the kernel decides them: the ray of pixel j
    crosses outer row o (rows when |cos| >= |sin|, else columns) at inner
    position (j - hd) inv_dom + k0 + o p1, held in 32.32 fixed point (start
    rounded to nearest, step p1 rounded to nearest), and takes a sample there
    when the position lies in [-1, n)."""
    hn, hd = 0.5 * (n - 1), 0.5 * (n_det - 1)
    total = 0
    o = np.arange(n, dtype=np.int64)
    for th in inputs.angles(n_theta):
        c, s = np.cos(th), np.sin(th)
        if abs(s) > abs(c):
            inv_dom, p1 = -1.0 / s, c / s
        else:
            inv_dom, p1 = 1.0 / c, s / c
        p1_fx = int(np.rint(p1 * TWO32))
        if p1_fx == 0:
            p1 = 0.0
        k0 = hn - hn * p1
        for j in range(n_det):
            base = int(np.rint(((j - hd) * inv_dom + k0) * TWO32))
            q = base + o * p1_fx
            total += int(np.count_nonzero((q >= -TWO32) & (q < n * TWO32)))
    return total


@pytest.mark.parametrize("shape", [(64, 90, 96), (40, 37, 57), (33, 64, 33), (65, 181, 90)])
def test_projector_samples_match_the_kernels_rule(shape):
    """The closed form decides the boundaries in floating point, the kernel in
    fixed point; on these shapes (odd and even sizes, detector narrower than
    the slice, an odd angle count) no position falls within rounding of -1 or
    n, and the counts are equal."""
    assert float(bench.projector_samples([shape])[0]) == samples_by_enumeration(*shape)


def test_projector_samples_at_normal_incidence():
    """At theta = 0 every row is crossed by the n + 1 rays whose position lies
    in [-1, n): n (n + 1) samples when the detector is wide enough."""
    n, n_det = 64, 96
    hn, hd = 0.5 * (n - 1), 0.5 * (n_det - 1)
    rays = sum(1 for j in range(n_det) if -1.0 <= hn + (j - hd) < n)
    assert rays == n + 1
    assert samples_by_enumeration(n, 1, n_det) == n * (n + 1)
    assert float(bench.projector_samples([(n, 1, n_det)])[0]) == n * (n + 1)


def test_projector_samples_follow_the_ray_spacing_along_a_row():
    """Within one outer row neighbouring rays cross 1 / max(|cos|, |sin|)
    apart, so with a detector wider than the slice's diagonal about
    (n + 1) max(|cos|, |sin|) rays cross each of the n rows inside [-1, n):
    n (n + 1) max(|cos|, |sin|) samples per angle, up to the rounding of
    where the first ray falls (under one sample per row)."""
    n, n_theta, n_det = 128, 180, 192
    th = inputs.angles(n_theta)
    dom = np.maximum(np.abs(np.cos(th)), np.abs(np.sin(th)))
    expect = n * (n + 1) * dom.sum()
    got = float(bench.projector_samples([(n, n_theta, n_det)])[0])
    assert abs(got - expect) <= n * n_theta, (got, expect)


def _summary(tmp_path, rows, max_default=2070.0):
    clk = bench.ClockSampler(None)
    clk.path = str(tmp_path / "clocks.csv")
    with open(clk.path, "w") as f:
        for r in rows:
            f.write(", ".join(r) + "\n")
    clk.proc = object()          # a sampler that ran
    return clk.summary(max_default)


def _row(sm, reasons=("Not Active",) * 4):
    return ["0", "GPU-x", str(sm), "2070", "900.0", "0x0000000000000000"] + list(reasons)


def test_clock_summary_median_and_no_reason(tmp_path):
    s = _summary(tmp_path, [_row(1965), _row(1980), _row(1950), ["garbage"], _row(2010)])
    assert s["samples"] == 4
    assert s["sm_mhz"] == pytest.approx(1972.5)
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == []


def test_clock_summary_names_active_reasons(tmp_path):
    rows = [_row(1800, ("Not Active", "Not Active", "Not Active", "Active")),
            _row(1500, ("Active", "Not Active", "Not Active", "Not Active")),
            _row(1900)]
    s = _summary(tmp_path, rows)
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert s["sm_mhz"] == 1800.0


def test_clock_summary_without_sampler(tmp_path):
    clk = bench.ClockSampler(None)
    s = clk.summary(2070.0)
    assert s["sm_mhz"] is None and s["reasons"] == ["nvidia-smi unavailable"]
    assert _summary(tmp_path, [])["reasons"] == ["no samples"]


def test_profiled_traffic_ratios_are_plausible():
    """DRAM bytes over algorithmic bytes per launch: at least the algorithmic
    bytes (every input is read once), and well under 2.5 times them (the
    staged projector's blocks re-read their windows through L2, 2.08x)."""
    for key, ratio in bench.PROFILED_TRAFFIC.items():
        assert key[0] in ("project", "backproject")
        assert 1.0 <= ratio < 2.5, (key, ratio)
