"""Windkessel outlets in the oracle, pinned by what the model must satisfy.

The model (oracle.c, wk_t): the outlet's ghost density for the next step is
rho_c + Rp q (q: outflow of the last step), and the compliance density
follows C d(rho_c)/dt = q - (rho_c - rho_d)/Rd, explicit in time; C = 0 is a
pure resistance rho_d + (Rp + Rd) q.  Pins:

* a resistance outlet at steady state is a pressure outlet at its own
  steady ghost density: both runs reach the same velocity field;
* the RCR fixed point: rho_c -> rho_d + Rd q, ghost density -> rho_d +
  (Rp + Rd) q, with q the steady inflow;
* mass budget: mass(t) - mass(t-1) = sum of the iolet fluxes, exactly;
* an outlet switched back to a pressure waveform behaves as before.
"""
import numpy as np
import pytest

import oracle
from paper_2202_11770_gb300 import geometry as geo


def _pipe(tau=0.8):
    lat = geo.pipe(4.0, 24)
    o = oracle.Oracle(lat, tau=tau)
    o.set_velocity(0, [1.0], 0.01)
    return lat, o


def test_resistance_outlet_equals_pressure_outlet_at_steady_state():
    R = 0.02
    _, a = _pipe()
    a.set_windkessel(1, R, 0.0, 0.0, rho_d=1.0)
    a.init_equilibrium()
    a.step(4000)
    q = -a.flux()[1]
    rho_out = a.windkessel_rho(1)
    assert q > 0 and abs(rho_out - (1.0 + R * q)) < 1e-6 * R * q + 1e-15  # steady: q changes by < 1e-6
    _, b = _pipe()
    b.set_pressure(1, rho_out)
    b.init_equilibrium()
    b.step(4000)
    _, ua, _ = a.macros()
    _, ub, _ = b.macros()
    assert np.linalg.norm(ua - ub) <= 1e-6 * np.linalg.norm(ub)


def test_rcr_fixed_point():
    Rp, C, Rd = 0.01, 40.0, 0.03
    _, o = _pipe()
    o.set_windkessel(1, Rp, C, Rd, rho_d=1.0, rho_c0=1.0)
    o.init_equilibrium()
    o.step(12000)  # rho_c relaxes by 1/(Rd C) = 0.83 of its distance per step, the pipe flow slower
    q_in = o.flux()[0]
    q = -o.flux()[1]
    assert q == pytest.approx(q_in, rel=1e-4)        # steady: outflow = inflow
    assert o.windkessel_rho_c(1) == pytest.approx(1.0 + Rd * q, rel=0, abs=1e-7)
    assert o.windkessel_rho(1) == pytest.approx(1.0 + (Rp + Rd) * q, rel=0, abs=1e-7)


def test_mass_budget_with_windkessel_outlet():
    _, o = _pipe()
    o.set_windkessel(1, 0.01, 500.0, 0.05, rho_d=1.0, rho_c0=1.002)
    o.init_equilibrium()
    m_prev = o.mass()
    for _ in range(50):
        o.step(1)
        m = o.mass()
        assert abs((m - m_prev) - o.flux().sum()) < 1e-12 * m
        m_prev = m


def test_switch_back_to_pressure_waveform():
    _, a = _pipe()
    a.set_windkessel(1, 0.02, 0.0, 0.0)
    a.set_pressure(1, 1.0)
    _, b = _pipe()
    b.set_pressure(1, 1.0)
    for x in (a, b):
        x.init_equilibrium()
        x.step(30)
    assert np.array_equal(a.state(), b.state())


def test_windkessel_rejects_bad_parameters():
    _, o = _pipe()
    with pytest.raises(ValueError):
        o.set_windkessel(0, 0.01, 0.0, 0.0)          # iolet 0 is the velocity inlet
    with pytest.raises(ValueError):
        o.set_windkessel(1, 0.01, 5.0, 0.0)          # compliance needs a distal resistance
    with pytest.raises(ValueError):
        o.set_windkessel(1, 0.01, 5.0, 0.1)          # Rd C < 1: the explicit update would overshoot
    with pytest.raises(ValueError):
        o.set_windkessel(1, -0.01, 0.0, 0.0)
