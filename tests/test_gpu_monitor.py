"""Iolet monitor and tabulated inlet waveform on the GPU against the oracle.

The paper's pipe check (Section 6): a pulsatile inlet profile (one beat,
tabulated) drives the 12,352-site pipe against a constant outlet pressure;
flow rate, maximum velocity and pressure at the inlet and the outlet are
recorded over time.  Here the GPU series (FP32, both streaming schemes, read
through hlb_iolet_monitor) must match the same quantities taken from the
FP64 oracle's state at every sample: flux and max |u| to 1e-5 of their
range, mean density to 1e-6.
"""
import numpy as np
import pytest

import oracle
from paper_2202_11770_gb300 import geometry as geo
from paper_2202_11770_gb300 import validation

pytestmark = pytest.mark.gpu

hemegb = pytest.importorskip("paper_2202_11770_gb300.hemegb")


def _iolet_sites(lat):
    """Sites with a link to each iolet (ascending)."""
    src = lat.src
    return [np.nonzero((src == -(2 + k)).any(axis=0))[0] for k in range(len(lat.iolets))]


def _oracle_monitor(o, sites):
    rho, u, _ = o.macros()
    speed = np.sqrt((u ** 2).sum(axis=1))
    return (o.flux(), np.array([speed[s].max() for s in sites]), np.array([rho[s].mean() for s in sites]))


@pytest.mark.parametrize("scheme", ["ab", "aa"])
def test_pulsatile_pipe_iolet_series_vs_oracle(scheme):
    lat = geo.pipe(8.0, 64)
    wave = validation.cardiac_waveform(period=400.0, peak=0.02)
    s = hemegb.Solver(lat, tau=0.8, precision="fp32", scheme=scheme)
    o = oracle.Oracle(lat, tau=0.8)
    for x in (s, o):
        x.set_velocity(0, [1.0], wave)
        x.set_pressure(1, 1.0)
        x.init_equilibrium()
    sites = _iolet_sites(lat)
    assert all(len(q) > 0 for q in sites)
    gpu = validation.iolet_series(s, 800, 40)
    ref = {"flux": [], "u_max": [], "pressure": []}
    for _ in range(20):
        o.step(40)
        f, um, r = _oracle_monitor(o, sites)
        ref["flux"].append(f)
        ref["u_max"].append(um)
        ref["pressure"].append(r / 3.0)
    for key in ref:
        ref[key] = np.array(ref[key])
    assert np.array_equal(gpu["t"], np.arange(40, 801, 40))
    for key, tol in (("flux", 1e-5), ("u_max", 1e-5)):
        span = np.abs(ref[key]).max()
        err = np.abs(gpu[key] - ref[key]).max()
        print(f"{scheme} {key}: max |gpu - oracle| = {err:.2e} of {span:.2e}")
        assert err <= tol * span
    assert np.abs(gpu["pressure"] - ref["pressure"]).max() <= 1e-6 / 3
    # the pulse is visible: inlet flow over the beat varies by more than 2x
    q_in = gpu["flux"][:, 0]
    assert q_in.max() > 2 * q_in[q_in > 0].min()


def test_monitor_matches_macros_on_tree():
    """Every iolet of a 7-outlet tree: monitor values against the solver's
    own read-back (same state, both FP32-rounded moments, FP64 reductions)."""
    lat = geo.tree(2, 2202, target_sites=50_000, length_ratio=5.0)
    s = hemegb.Solver(lat, tau=0.6, precision="fp32", scheme="aa")
    s.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 200.0})
    for k in range(1, len(lat.iolets)):
        s.set_pressure(k, 1.0 + 0.001 * k)
    s.init_equilibrium()
    s.step(151)
    flux, umax, rho_mean = s.iolet_monitor()
    _, fl = s.reduce()
    rho, u, _ = s.macros()
    speed = np.sqrt((u.astype(np.float64) ** 2).sum(axis=1))  # u [n, 3]
    for k, q in enumerate(_iolet_sites(lat)):
        assert abs(umax[k] - speed[q].max()) <= 1e-7 * max(speed[q].max(), 1e-12)
        assert abs(rho_mean[k] - rho[q].astype(np.float64).mean()) <= 1e-7
    assert np.array_equal(flux, fl)
