"""Iolet time series of a pulsatile pipe run (the paper's Section 6 check).

The paper drives a straight pipe with a 60-beats-per-minute inlet profile
(maximum velocity over one beat, each inlet point scaled by its cross-section
weight) against a constant outlet pressure, and compares the flow rate and
the maximum velocity and pressure at the inlet and the outlet between its CPU
and GPU codes.  This module supplies the pieces of that run for this solver:

* ``cardiac_waveform``: one beat of a synthetic maximum-velocity profile
  (a systolic peak and a smaller diastolic wave over a baseline), as a
  tabulated waveform.  The paper's own profile is printed only as a figure,
  so its samples are not reproduced; this shape stands in for it.
* ``load_waveform``: a tabulated waveform read from a two-column text file
  (phase in [0, 1), value), for measured profiles.
* ``iolet_series``: steps a solver and records, every ``every`` steps, the
  per-iolet flow (mass per step through the iolet), maximum |u| and pressure
  (rho / 3) from ``hlb_iolet_monitor``.

No LB arithmetic happens here: the monitor values come from the library.
"""
from __future__ import annotations

import numpy as np


def cardiac_waveform(period: float, peak: float, n_samples: int = 200, baseline: float = 0.15) -> dict:
    """One beat of a synthetic inlet maximum-velocity profile as a TABLE waveform.

    period: steps per beat (60 beats per minute maps one second to `period`
    steps); peak: the largest sample.  Shape: baseline + systolic Gaussian at
    phase 0.15 (width 0.06) + diastolic Gaussian at phase 0.45 (width 0.08,
    30 % of the systolic height), normalised to a maximum of 1 and periodic."""
    phase = np.arange(n_samples) / n_samples
    def bump(c, w):
        d = (phase - c + 0.5) % 1.0 - 0.5  # periodic distance
        return np.exp(-0.5 * (d / w) ** 2)
    shape = baseline + bump(0.15, 0.06) + 0.3 * bump(0.45, 0.08)
    shape /= shape.max()
    return {"kind": "table", "mean": float(peak), "period": float(period), "samples": shape}


def load_waveform(path, period: float, scale: float = 1.0) -> dict:
    """A TABLE waveform from a text file of `phase value` rows (phase in [0, 1)).

    The rows are resampled onto an even grid of as many points (linear,
    periodic), which is the form the solver interpolates."""
    data = np.loadtxt(path, dtype=np.float64, ndmin=2)
    ph, val = data[:, 0] % 1.0, data[:, 1]
    order = np.argsort(ph)
    ph, val = ph[order], val[order]
    grid = np.arange(len(ph)) / len(ph)
    samples = np.interp(grid, ph, val, period=1.0)
    return {"kind": "table", "mean": float(scale), "period": float(period), "samples": samples}


def iolet_series(solver, steps: int, every: int) -> dict:
    """Step `solver` `steps` times, sampling the iolet monitor every `every` steps.

    Returns {"t": [m], "flux": [m, K], "u_max": [m, K], "pressure": [m, K]}."""
    if steps % every:
        raise ValueError("steps must be a multiple of every")
    ts, fl, um, pr = [], [], [], []
    for _ in range(steps // every):
        solver.step(every)
        f, u, r = solver.iolet_monitor()
        ts.append(solver.t)
        fl.append(f)
        um.append(u)
        pr.append(r / 3.0)
    return {"t": np.array(ts), "flux": np.array(fl), "u_max": np.array(um), "pressure": np.array(pr)}
