"""Oracle pins: analytic pipe flows and wall shear stress.

Pins (paper Eqs. 3-8, Section 2.3, Section 6 pipe):
  * steady flow obeys the Navier-Stokes momentum balance: the fitted
    parabola's curvature U/R^2 equals G/(4 nu), G the body-force equivalent of
    the measured density gradient (Eq. 7) and nu = (tau - 1/2)/3 (Eq. 8);
  * the velocity-driven profile is parabolic (interior sites) and the
    staircase-wall residual shrinks under refinement;
  * steady mass flux is continuous: inlet flux = - outlet flux = mid-plane
    sum of rho u_z;
  * pressure-driven flux is linear in the density difference;
  * the steady inlet mass flux approaches the integral rho A pi R^2 / 2 of the
    imposed Ladd profile A (1 - r^2/R^2) (Section 2.3.2, Section 6), closer at
    R = 12 than at R = 8, and the velocity on the first fluid plane is that
    profile;
  * WSS cross-section mean matches rho nu |du/dr| of the Poiseuille fit at
    the wall sites' radii within 10 %, closer at higher resolution;
  * oscillating pressure drive reproduces the Womersley profile (alpha = 2).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2202_11770_gb300 import geometry as geo
from helpers import CS2, density_gradient, fit_parabola, womersley_profile

TAU = 0.8
NU = (TAU - 0.5) / 3.0
A_IN = 0.01            # inlet amplitude of the velocity-driven pipes


def _velocity_driven(R, L, steps):
    lat = geo.pipe(R, L)
    o = oracle.Oracle(lat, tau=TAU)
    o.set_velocity(0, [1.0], A_IN)
    o.set_pressure(1, 1.0)
    o.init_equilibrium()
    o.step(steps)
    return lat, o


@pytest.fixture(scope="module")
def pipe8():
    lat, o = _velocity_driven(8.0, 64, 5000)
    rho, u, wss = o.macros(lat.wall_normal)
    return lat, o, rho, u, wss


@pytest.fixture(scope="module")
def pipe12():
    lat, o = _velocity_driven(12.0, 24, 9000)
    rho, u, wss = o.macros(lat.wall_normal)
    return lat, o, rho, u, wss


def _midplane(lat, z0, interior=False):
    sel = lat.xyz[:, 2] == z0
    if interior:
        sel &= lat.type == geo.INNER
    return sel


def test_poiseuille_momentum_balance(pipe8):
    lat, o, rho, u, _ = pipe8
    sel = _midplane(lat, 32, interior=True)
    r = np.hypot(lat.xyz[sel, 0], lat.xyz[sel, 1])
    U, R_eff, curv, resid = fit_parabola(r, u[sel, 2])
    G = density_gradient(lat, rho, 16, 48)
    assert U > 0 and G > 0
    assert abs(curv / (G / (4 * NU)) - 1) < 0.01
    assert resid < 0.02
    assert 7.0 < R_eff < 8.5


def test_poiseuille_refinement(pipe8, pipe12):
    res = []
    for (lat, o, rho, u, _), z0 in ((pipe8, 32), (pipe12, 12)):
        sel = _midplane(lat, z0)
        r = np.hypot(lat.xyz[sel, 0], lat.xyz[sel, 1])
        res.append(fit_parabola(r, u[sel, 2])[3])
    assert res[0] < 0.05
    assert res[1] < 0.6 * res[0]


def test_steady_flux_continuity(pipe8):
    lat, o, rho, u, _ = pipe8
    fl = o.flux()
    assert abs(fl[0] + fl[1]) < 1e-4 * fl[0]
    sel = _midplane(lat, 32)
    assert abs((rho[sel] * u[sel, 2]).sum() / fl[0] - 1) < 0.005


def test_ladd_inlet_flux_matches_profile_integral(pipe8, pipe12):
    dev = []
    for lat, o, rho, u, _ in (pipe8, pipe12):
        R = lat.info["radius"]
        first = lat.xyz[:, 2] == 0
        dev.append(o.flux()[0] / (rho[first].mean() * A_IN * math.pi * R * R / 2) - 1)
    assert abs(dev[0]) < 0.01
    assert abs(dev[1]) < 0.7 * abs(dev[0])


def test_ladd_near_inlet_profile(pipe8, pipe12):
    for (lat, o, rho, u, _), tol in ((pipe8, 0.015), (pipe12, 0.008)):
        R = lat.info["radius"]
        first = lat.xyz[:, 2] == 0
        r = np.hypot(lat.xyz[first, 0], lat.xyz[first, 1])
        imposed = A_IN * np.clip(1 - r ** 2 / R ** 2, 0, None)
        assert np.linalg.norm(u[first, 2] - imposed) / np.linalg.norm(imposed) < tol
        U, R_fit, _, _ = fit_parabola(r, u[first, 2])
        assert abs(U / A_IN - 1) < 0.005 and abs(R_fit / R - 1) < 0.005


def test_pressure_driven_linear():
    fluxes = []
    for d in (0.003, 0.006):
        lat = geo.pipe(8.0, 32, geo.PRESSURE, geo.PRESSURE)
        o = oracle.Oracle(lat, tau=TAU)
        o.set_pressure(0, 1.0 + d)
        o.set_pressure(1, 1.0)
        o.init_equilibrium()
        o.step(4000)
        rho, u, _ = o.macros()
        sel = _midplane(lat, 16, interior=True)
        r = np.hypot(lat.xyz[sel, 0], lat.xyz[sel, 1])
        _, _, curv, _ = fit_parabola(r, u[sel, 2])
        G = density_gradient(lat, rho, 6, 26)
        assert abs(curv / (G / (4 * NU)) - 1) < 0.01
        fluxes.append(o.flux()[0])
    assert fluxes[0] > 0
    assert abs(fluxes[1] / fluxes[0] - 2) < 0.01


def _wss_ratio(lat, rho, u, wss, z0):
    sel = _midplane(lat, z0, interior=True)
    r = np.hypot(lat.xyz[sel, 0], lat.xyz[sel, 1])
    _, _, curv, _ = fit_parabola(r, u[sel, 2])
    w = (lat.xyz[:, 2] == z0) & ~np.isnan(wss)
    rw = np.hypot(lat.xyz[w, 0], lat.xyz[w, 1])
    analytic = rho[w] * NU * 2 * curv * rw        # rho nu |du_z/dr| at the site radius
    return wss[w].mean() / analytic.mean()


def test_wss_poiseuille(pipe8, pipe12):
    lat, _, rho, u, wss = pipe8
    wall = (lat.src == -1).any(axis=0)
    assert np.isnan(wss[~wall]).all() and not np.isnan(wss[wall]).any()
    r8 = _wss_ratio(lat, rho, u, wss, 32)
    lat, _, rho, u, wss = pipe12
    r12 = _wss_ratio(lat, rho, u, wss, 12)
    assert abs(r8 - 1) < 0.10
    assert abs(r12 - 1) < abs(r8 - 1)


def test_womersley():
    R, L, T = 8.0, 32, 1000
    omega = 2 * math.pi / T
    assert abs(R * math.sqrt(omega / NU) - 2.0) < 0.01        # Womersley number
    lat = geo.pipe(R, L, geo.PRESSURE, geo.PRESSURE)
    # effective radius from a steady pressure-driven run of the same pipe
    o = oracle.Oracle(lat, tau=TAU)
    o.set_pressure(0, 1.003)
    o.set_pressure(1, 1.0)
    o.init_equilibrium()
    o.step(4000)
    rho, u, _ = o.macros()
    sel = _midplane(lat, 16, interior=True)
    _, R_eff, _, _ = fit_parabola(np.hypot(lat.xyz[sel, 0], lat.xyz[sel, 1]), u[sel, 2])

    o = oracle.Oracle(lat, tau=TAU)
    o.set_pressure(0, {"kind": "cosine", "mean": 1.0, "rel": 0.003, "period": T})
    o.set_pressure(1, 1.0)
    o.init_equilibrium()
    o.step(3 * T)
    mid = lat.xyz[:, 2] == 16
    rm = np.hypot(lat.xyz[mid, 0], lat.xyz[mid, 1])
    ts, Gs, prof = [], [], []
    for _ in range(20):
        rho, u, _ = o.macros()
        ts.append(o.t)
        Gs.append(density_gradient(lat, rho, 6, 26))
        prof.append(u[mid, 2].copy())
        o.step(T // 20)
    ts = np.array(ts, float)
    A = np.stack([np.cos(omega * ts), -np.sin(omega * ts)], 1)
    gc, *_ = np.linalg.lstsq(A, np.array(Gs), rcond=None)
    assert np.linalg.norm(A @ gc - Gs) / np.linalg.norm(Gs) < 0.01   # drive is sinusoidal
    shape = womersley_profile(gc[0] + 1j * gc[1], omega, NU, rm, R_eff)
    inner = lat.type[mid] == geo.INNER
    num = den = num_i = den_i = 0.0
    for t, p in zip(ts, prof):
        ana = np.real(shape * np.exp(1j * omega * t))
        num += ((p - ana) ** 2).sum()
        den += (ana ** 2).sum()
        num_i += ((p - ana)[inner] ** 2).sum()
        den_i += (ana[inner] ** 2).sum()
    assert math.sqrt(num / den) < 0.05
    assert math.sqrt(num_i / den_i) < 0.025
