"""Host-side helpers of bench.py that turn recorded series into the errors
the benchmark line reports (FP32 against FP64 decay rates and their
summary), on the CPU with synthetic amplitude series of known decay."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _series(t, a):
    return [{"time": float(x), "amp": float(y)} for x, y in zip(t, a)]


def test_decay_rates_recover_known_rates():
    """Exact exponentials: the fitted rates are the generating ones, and the
    reported ln(A0/A_end) is that of the FP64 series over the kept window."""
    t = np.linspace(0.0, 10.0, 41)
    g64, g32 = 0.3, 0.3 * (1 + 2e-5)
    r32, r64, lnd = bench._decay_rates(_series(t, np.exp(-g32 * t)), _series(t, np.exp(-g64 * t)))
    assert abs(r64 - g64) < 1e-12 * g64
    assert abs(r32 / r64 - 1 - 2e-5) < 1e-9
    assert abs(lnd - g64 * 10.0) < 1e-12


def test_decay_rates_stop_where_the_fp64_amplitude_falls_below_the_floor():
    """Past 1e-3 of its start the FP64 amplitude is no longer compared: an
    FP32 series that sits on a rounding floor there does not bias the rate."""
    t = np.linspace(0.0, 20.0, 81)
    g = 1.0
    a64 = np.exp(-g * t)
    a32 = np.maximum(np.exp(-g * t), 1e-4)          # stalls below 1e-4 (t > 9.2)
    cut = int(np.argmin(a64 >= 1e-3))                 # first sample under the floor (t = 7)
    r32, r64, lnd = bench._decay_rates(_series(t, a32), _series(t, a64))
    assert abs(r32 / r64 - 1) < 1e-9
    assert abs(lnd - g * t[cut - 1]) < 1e-12


def test_error_summary_separates_resolved_decays():
    """The decay-rate error is reported over all lattices and over those
    whose amplitude decayed by at least the resolved amount."""
    s = bench._error_summary([1e-5, 3e-5, 2e-5], [1e-3, 2e-5, 4e-5], [0.001, 0.2, 1.5], "synthetic")
    assert s["max_rel_velocity_error"] == 3e-5
    assert s["rel_decay_rate_error"]["max"] == 1e-3
    assert s["rel_decay_rate_error"]["median"] == 4e-5
    assert s["rel_decay_rate_error"]["max_where_decay_ln_ge_0.05"] == 4e-5
    assert s["rel_decay_rate_error"]["lattices_where_decay_ln_ge_0.05"] == 2
    assert s["lattices"] == 3 and s["amplitude_decay_ln_range"] == [0.001, 1.5]
    s = bench._error_summary([1e-5], [1e-3], [0.01], "none resolved")
    assert s["rel_decay_rate_error"]["max_where_decay_ln_ge_0.05"] is None


@pytest.mark.parametrize("report,height", [
    ("[g0 CS q3 fp32 tile=256x32 grid=8192 0.7 ms/step] [g1 FD q4 fp32 tile=32x8 grid=65536 3.3 ms/step]", "8"),
    ("[g1 FD q4 fp32 cached tile=2 grid=152]", "16"),
    ("[g0 CS q3 fp32 tile=256x32 grid=8 0.1 ms/step]", "*"),
])
def test_fd_tile_height_from_the_tuner_report(report, height):
    assert bench.fd_tile_height(report, 1 if "g1" in report else 0) == height


def test_alone_seconds():
    """A run's time alone at its kind's single-lattice rate (the served
    stream's service-time estimate, slowdowns and FP64 one-at-a-time
    baseline are built from it)."""
    reqs = [{"model": "cs", "n": 64, "steps": 1000}, {"model": "fd", "n": 128, "steps": 2000}]
    got = bench.alone_seconds(reqs, {("cs", 64): 4.096e7, ("fd", 128): 1.6384e7})
    assert got == pytest.approx([0.1, 2.0], rel=1e-15)
    with pytest.raises(KeyError):
        bench.alone_seconds([{"model": "fd", "n": 256, "steps": 1}], {("fd", 128): 1.0})
