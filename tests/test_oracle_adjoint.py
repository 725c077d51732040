"""Oracle pin: the FP64 discrete adjoint equals central finite differences.

The objective averages the squared deviation of the axial velocity at probe
sites from a target over N steps; gradients w.r.t. tau and the per-group
inlet amplitudes are compared with central differences of the oracle's own
forward map (the definition of the derivative of the discrete step), for
both readings of the Ladd density and of the ghost velocity.
"""
import numpy as np
import pytest

import oracle
from paper_2202_11770_gb300 import geometry as geo


@pytest.fixture(scope="module")
def small_tree():
    return geo.tree(1, 7, root_radius=4.0, length_ratio=5.0, n_sectors=2, n_rings=2)


def _make(lat, tau, amps, opts):
    o = oracle.Oracle(lat, tau, *opts)
    o.set_velocity(0, amps, {"kind": "cosine", "mean": 0.03, "rel": 0.5, "period": 50.0})
    for k in range(1, len(lat.iolets)):
        o.set_pressure(k, {"kind": "cosine", "mean": 1.0, "rel": 0.001 * k, "period": 30.0})
    o.init_equilibrium()
    return o


@pytest.mark.parametrize("opts", [(False, False), (True, True)])
def test_adjoint_matches_central_differences(small_tree, opts):
    lat = small_tree
    N, tau = 40, 0.7
    probe = np.nonzero(lat.xyz[:, 2] == int(lat.info["root_length"] // 2))[0]
    rng = np.random.default_rng(1)
    target = 0.02 * (1 + 0.1 * rng.uniform(-1, 1, probe.size))
    axis = [0.0, 0.0, 1.0]
    amps = np.array([1.0, 0.9, 1.1, 0.95])
    J, dtau, damp = _make(lat, tau, amps, opts).adjoint(N, probe, target, axis)
    assert J == pytest.approx(_make(lat, tau, amps, opts).objective(N, probe, target, axis), rel=1e-14)
    h = 1e-5
    fd = (_make(lat, tau + h, amps, opts).objective(N, probe, target, axis)
          - _make(lat, tau - h, amps, opts).objective(N, probe, target, axis)) / (2 * h)
    assert abs(dtau - fd) < 1e-7 * abs(fd)
    for g in range(4):
        e = np.zeros(4)
        e[g] = h
        fd = (_make(lat, tau, amps + e, opts).objective(N, probe, target, axis)
              - _make(lat, tau, amps - e, opts).objective(N, probe, target, axis)) / (2 * h)
        assert abs(damp[g] - fd) < 1e-7 * abs(fd)
    # a random direction of the amplitude vector
    d = rng.normal(size=4)
    fd = (_make(lat, tau, amps + h * d, opts).objective(N, probe, target, axis)
          - _make(lat, tau, amps - h * d, opts).objective(N, probe, target, axis)) / (2 * h)
    assert abs(damp @ d - fd) < 1e-7 * abs(fd)
