"""Windkessel outlets on the GPU against the FP64 oracle.

The outlet model (hlb_set_windkessel, oracle.c wk_t) couples the ghost
density to the outflow with one step of lag; both sides run the same
discrete model, so the velocity field, the model state (rho_c, q) and the
mass budget must agree like any other boundary: FP64 to rounding, FP32 to
the tolerances of the plain pressure outlet.
"""
import numpy as np
import pytest

import oracle
from paper_2202_11770_gb300 import geometry as geo

pytestmark = pytest.mark.gpu

hemegb = pytest.importorskip("paper_2202_11770_gb300.hemegb")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _setup(x, lat, models):
    x.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 150.0})
    for k in range(1, len(lat.iolets)):
        if k in models:
            x.set_windkessel(k, *models[k])
        else:
            x.set_pressure(k, 1.0)
    x.init_equilibrium()


@pytest.mark.parametrize("scheme", ["ab", "aa"])
def test_pipe_rcr_fp32(scheme):
    lat = geo.pipe(8.0, 64)
    models = {1: (0.01, 200.0, 0.03, 1.0, 1.001)}
    s = hemegb.Solver(lat, tau=0.8, precision="fp32", scheme=scheme)
    o = oracle.Oracle(lat, tau=0.8)
    _setup(s, lat, models)
    _setup(o, lat, models)
    s.step(600)
    o.step(600)
    _, u, _ = s.macros()
    _, u_o, _ = o.macros()
    assert rel_l2(u, u_o) <= 1e-5
    ghost, rho_c, q = s.windkessel_state(1)
    q_o, rho_c_o = -o.flux()[1], o.windkessel_rho_c(1)
    # FP32 populations: q to 1e-4; rho_c integrates q / C, to 1e-4 of its excursion
    assert abs(q - q_o) <= 1e-4 * abs(q_o)
    assert abs(rho_c - rho_c_o) <= 1e-4 * abs(rho_c_o - 1.0)
    assert abs(ghost - (rho_c_o + 0.01 * q_o)) <= 1e-4 * abs(rho_c_o + 0.01 * q_o - 1.0)
    assert rho_c > 1.0          # the compliance charged


@pytest.mark.parametrize("scheme", ["ab", "aa"])
def test_tree_mixed_outlets_fp64(scheme):
    """Depth-2 tree, 4 outlets: two RCR, one pure resistance, one fixed."""
    lat = geo.tree(2, 2202, target_sites=50_000, length_ratio=5.0)
    assert len(lat.iolets) == 5
    models = {1: (0.02, 50.0, 0.05, 1.0, 1.0), 2: (0.0, 0.0, 0.04, 1.0, 1.0), 3: (0.01, 100.0, 0.02, 0.999, 1.002)}
    s = hemegb.Solver(lat, tau=0.6, precision="fp64", scheme=scheme)
    o = oracle.Oracle(lat, tau=0.6)
    _setup(s, lat, models)
    _setup(o, lat, models)
    for _ in range(3):
        s.step(67)
        o.step(67)
        f, t = s.state()
        assert t == o.t
        ref = o.state().T - oracle.feq(1.0, [0, 0, 0])[:, None]
        assert np.abs(f - ref).max() < 1e-11
    for k, (Rp, C, Rd, rho_d, _) in models.items():
        ghost, rho_c, q = s.windkessel_state(k)
        q_o = -o.flux()[k]
        assert abs(q - q_o) <= 1e-11
        if C > 0:
            assert abs(rho_c - o.windkessel_rho_c(k)) <= 1e-13
            assert abs(ghost - (o.windkessel_rho_c(k) + Rp * q_o)) <= 1e-13
        else:
            assert abs(ghost - (rho_d + (Rp + Rd) * q_o)) <= 1e-13
    # mass budget across one more step, Windkessel outlets included
    m5, _ = s.reduce()
    s.step(1)
    m6, fl = s.reduce()
    assert abs((m6 - m5) - fl.sum()) < 1e-12 * m6


def test_windkessel_validation_and_adjoint_refusal():
    lat = geo.pipe(4.0, 12)
    s = hemegb.Solver(lat, tau=0.8, precision="fp32")
    with pytest.raises(hemegb.HlbError):
        s.set_windkessel(0, 0.01, 0.0, 0.0)        # a velocity iolet
    with pytest.raises(hemegb.HlbError):
        s.set_windkessel(1, 0.01, 5.0, 0.1)        # Rd C < 1
    with pytest.raises(hemegb.HlbError):
        s.windkessel_state(1)                      # not a Windkessel outlet yet
    s.set_windkessel(1, 0.01, 0.0, 0.0)
    s.init_equilibrium()
    with pytest.raises(hemegb.HlbError):
        s.adjoint(10, [1], [0.0], [0, 0, 1])
    s.set_pressure(1, 1.0)                         # back to a waveform outlet
    with pytest.raises(hemegb.HlbError):
        s.windkessel_state(1)
