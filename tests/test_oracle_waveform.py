"""Oracle waveforms against their closed forms (CPU).

The tabulated waveform (periodic linear interpolation of samples spaced
period / n apart, times `mean`) is pinned at sample points, midpoints, the
wrap-around interval and one period later; the cosine form against its
formula; a constant table against the constant waveform through a whole run
(bit-identical trajectories).
"""
import math

import numpy as np

import oracle
from paper_2202_11770_gb300 import geometry as geo
from paper_2202_11770_gb300 import validation


def _oracle_with(wave):
    lat = geo.pipe(3.0, 8)
    o = oracle.Oracle(lat, tau=0.8)
    o.set_velocity(0, [1.0], wave)
    o.set_pressure(1, 1.0)
    return lat, o


def test_table_interpolation_closed_form():
    s = np.array([0.2, 1.0, 0.5, -0.3, 0.7])
    period, mean = 40.0, 0.03
    _, o = _oracle_with({"kind": "table", "mean": mean, "period": period, "samples": s})
    h = period / s.size
    for j in range(s.size):
        assert abs(o.wave_value(0, j * h) - mean * s[j]) < 1e-15
        mid = mean * 0.5 * (s[j] + s[(j + 1) % s.size])
        assert abs(o.wave_value(0, (j + 0.5) * h) - mid) < 1e-15
        assert abs(o.wave_value(0, (j + 0.25) * h + 3 * period) - mean * (0.75 * s[j] + 0.25 * s[(j + 1) % s.size])) < 1e-15


def test_cosine_closed_form():
    w = {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 30.0, "phase": 0.4}
    _, o = _oracle_with(w)
    for t in (0.0, 7.0, 29.0, 31.5):
        assert abs(o.wave_value(0, t) - 0.02 * (1 + 0.5 * math.cos(2 * math.pi * t / 30.0 + 0.4))) < 1e-16


def test_constant_table_equals_constant_waveform():
    _, a = _oracle_with({"kind": "table", "mean": 0.01, "period": 17.0, "samples": np.ones(6)})
    _, b = _oracle_with(0.01)
    a.init_equilibrium()
    b.init_equilibrium()
    a.step(60)
    b.step(60)
    assert np.array_equal(a.state(), b.state())


def test_cardiac_waveform_shape():
    w = validation.cardiac_waveform(period=1000.0, peak=0.02)
    s = np.asarray(w["samples"])
    assert w["kind"] == "table" and s.size == 200
    assert s.max() == 1.0 and s.min() > 0.1
    assert 0.1 <= np.argmax(s) / s.size <= 0.2     # systolic peak in the first fifth of the beat


def test_load_waveform_resamples_periodically(tmp_path):
    p = tmp_path / "wave.txt"
    np.savetxt(p, np.array([[0.5, 3.0], [0.0, 1.0], [0.25, 2.0], [0.75, 2.0]]))
    w = validation.load_waveform(p, period=100.0, scale=2.0)
    assert w["mean"] == 2.0 and w["period"] == 100.0
    assert np.allclose(w["samples"], [1.0, 2.0, 3.0, 2.0])
