"""Oracle pins: streaming, bounce-back, relaxation and conservation.

Pins (paper Eqs. 3a-3b, Section 2.3.1, Section 3.1):
  * streaming + bounce-back is the permutation enumerated here by brute force
    from the coordinates (collision is the identity on an equilibrium state);
  * an isolated site (all links walls) keeps its density, reverses its
    momentum every step and relaxes its non-equilibrium second moment by the
    factor (1 - 1/tau) per step;
  * rest state invariance with zero-amplitude velocity inlet and rho = 1
    pressure outlet;
  * exact mass conservation in a closed pipe;
  * mass budget with open iolets: M(t+1) - M(t) equals the summed iolet flux.
"""
import numpy as np
import pytest

import oracle
from paper_2202_11770_gb300 import geometry as geo
from helpers import CS2, hand_lattice, opposite_table


def _random_equilibrium_state(n, rng, du=0.05):
    rho = rng.uniform(0.9, 1.1, n)
    u = rng.uniform(-du, du, (n, 3))
    return np.stack([oracle.feq(rho[k], u[k]) for k in range(n)])


def test_streaming_permutation_bruteforce(d3q19):
    c, _ = d3q19
    opp = opposite_table(c)
    rng = np.random.default_rng(3)
    # a 4x3x3 block with some sites removed: many fluid and wall links
    pts = [(x, y, z) for x in range(4) for y in range(3) for z in range(3)
           if not (x == 1 and y == 1) and not (x == 3 and z == 2)]
    lat = hand_lattice(pts, c)
    o = oracle.Oracle(lat, tau=0.7)
    f0 = _random_equilibrium_state(lat.n, rng)
    o.set_state(f0, 0)
    o.step(1)
    got = o.state()
    index = {tuple(p): k for k, p in enumerate(lat.xyz.tolist())}
    expect = np.full_like(f0, np.nan)
    for k, p in enumerate(lat.xyz):
        for i in range(19):
            q = tuple((p + c[i]).tolist())
            if q in index:
                expect[index[q], i] = f0[k, i]
            else:
                expect[k, opp[i]] = f0[k, i]
    assert not np.isnan(expect).any()
    assert np.allclose(got, expect, rtol=0, atol=2e-15)


def test_isolated_site_relaxation(d3q19):
    c, _ = d3q19
    tau = 0.65
    lat = hand_lattice([(0, 0, 0)], c)
    o = oracle.Oracle(lat, tau=tau)
    rng = np.random.default_rng(11)
    f = oracle.feq(1.02, [0.03, -0.01, 0.02]) + rng.uniform(-2e-3, 2e-3, 19)
    o.set_state(f[None, :], 0)

    def moments(f):
        rho = f.sum()
        j = f @ c
        pi = np.einsum("i,ia,ib->ab", f, c, c)
        return rho, j, pi

    rho0, j0, pi0 = moments(f)
    for _ in range(20):
        o.step(1)
        g = o.state()[0]
        rho1, j1, pi1 = moments(g)
        u = j0 / rho0
        pi_eq = rho0 * CS2 * np.eye(3) + rho0 * np.outer(u, u)
        assert abs(rho1 - rho0) < 1e-15
        assert np.allclose(j1, -j0, atol=1e-16)
        assert np.allclose(pi1 - pi_eq, (1 - 1 / tau) * (pi0 - pi_eq), atol=1e-16)
        rho0, j0, pi0 = rho1, j1, pi1


def test_rest_state_invariance():
    lat = geo.pipe(8.0, 64)
    o = oracle.Oracle(lat, tau=0.8)
    o.set_velocity(0, [1.0], 0.0)
    o.set_pressure(1, 1.0)
    o.init_equilibrium()
    f0 = o.state()
    o.step(1000)
    assert np.abs(o.state() - f0).max() < 1e-14


def test_closed_pipe_mass_conservation():
    lat = geo.pipe(5.0, 20, geo.WALL, geo.WALL)
    o = oracle.Oracle(lat, tau=0.6)
    rng = np.random.default_rng(5)
    o.set_state(_random_equilibrium_state(lat.n, rng, du=0.02), 0)
    m0 = o.mass()
    for _ in range(10):
        o.step(50)
        assert abs(o.mass() - m0) / m0 < 1e-13
    assert (o.flux() == 0).all()


def test_mass_budget_identity_open_pipe():
    lat = geo.pipe(6.0, 24)
    o = oracle.Oracle(lat, tau=0.7)
    o.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 40.0})
    o.set_pressure(1, {"kind": "cosine", "mean": 1.0, "rel": 0.002, "period": 25.0})
    o.init_equilibrium()
    m = o.mass()
    for _ in range(60):
        o.step(1)
        m1 = o.mass()
        fl = o.flux()
        assert abs((m1 - m) - fl.sum()) < 1e-12 * m1
        m = m1
    # inflow through the velocity inlet, outflow through the pressure outlet
    o.step(400)
    fl = o.flux()
    assert fl[0] > 0 and fl[1] < 0


def test_threaded_step_gives_the_serial_state():
    """Sites split over host threads: every slot of the next state has one
    writer, so the state is bit-identical to the serial step; the iolet fluxes
    differ only in summation order."""
    lat = geo.tree(2, 2202, target_sites=30_000, length_ratio=5.0)
    runs = []
    for threads in (1, 4):
        o = oracle.Oracle(lat, tau=0.6, threads=threads)
        o.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 50.0})
        for k in range(1, len(lat.iolets)):
            o.set_pressure(k, 1.0 - 0.0005 * k)
        o.init_equilibrium()
        o.step(40)
        runs.append((o.state(), o.flux()))
    (f1, q1), (f4, q4) = runs
    assert f1.tobytes() == f4.tobytes()
    assert np.allclose(q1, q4, rtol=1e-12, atol=1e-15)
