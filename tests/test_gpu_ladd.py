"""GPU Ladd velocity iolets and the wall-shear-stress fallback normal vs the
FP64 oracle, through the C ABI.

* A uniform flow whose every boundary link is a Ladd link moving with it is
  an exact steady state (paper Section 2.3.2): the corrected bounce-back of
  f^eq_i(rho, u) is f^eq_ibar(rho, u).  The solver keeps it to FP64 rounding
  in FP64 storage and to FP32 rounding in FP32 storage, in both schemes.
* Without caller wall normals the solver and the oracle take the normalised
  sum of the wall links' directions as the normal; their wall shear stress
  agrees to the FP32 tolerance of the other parity tests.
"""
import numpy as np
import pytest

import oracle
from paper_2202_11770_gb300 import geometry as geo
from helpers import hand_lattice

pytestmark = pytest.mark.gpu
hemegb = pytest.importorskip("paper_2202_11770_gb300.hemegb")


def _box_all_ladd(c, normal):
    n_hat = np.asarray(normal, np.float64) / np.linalg.norm(normal)
    io = geo.Iolet(kind=geo.VELOCITY, role=0, centre=np.array([3.5, 2.5, 4.0]), normal=n_hat,
                   radius=1e9, n_groups=1)
    pts = [(x, y, z) for z in range(9) for y in range(6) for x in range(8)]   # 432 sites: two tiles, ragged
    return hand_lattice(pts, c, iolets=[io], classify=lambda p, i: 0), n_hat


@pytest.mark.parametrize("scheme", ["ab", "aa"])
@pytest.mark.parametrize("prec,normal,tol", [("fp64", (0.0, 0.0, 1.0), 1e-14), ("fp32", (1.0, 2.0, 2.0), 1e-7)])
def test_uniform_ladd_flow_is_steady(d3q19, prec, normal, tol, scheme):
    """FP64 takes an axis normal so that the caller's float32 initial velocity
    equals the wall velocity exactly; FP32 a tilted one."""
    c, w = d3q19
    lat, n_hat = _box_all_ladd(c, normal)
    speed, rho0 = 0.0390625, 1.03
    s = hemegb.Solver(lat, tau=0.7, precision=prec, scheme=scheme)
    s.set_velocity(0, [speed], 1.0)
    u0 = np.tile((speed * n_hat).astype(np.float32)[:, None], (1, lat.n))
    s.init_equilibrium(rho0, u0)
    f0, _ = s.state()
    s.step(21)                                          # odd: ends mid AA cycle
    f1, _ = s.state()
    assert np.abs(f1.astype(np.float64) - f0.astype(np.float64)).max() < tol
    feq = oracle.feq(rho0, speed * n_hat.astype(np.float32).astype(np.float64)) - w
    assert np.abs(f1.astype(np.float64) - feq[:, None]).max() < tol


@pytest.mark.parametrize("scheme", ["ab", "aa"])
def test_wss_fallback_normal_vs_oracle(scheme):
    lat = geo.pipe(8.0, 64)
    s = hemegb.Solver(lat, tau=0.8, precision="fp32", scheme=scheme, use_normals=False)
    o = oracle.Oracle(lat, tau=0.8)
    for x in (s, o):
        x.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.01, "rel": 0.5, "period": 80.0})
        x.set_pressure(1, 1.0)
        x.init_equilibrium()
        x.step(301)
    _, _, wss = s.macros()
    _, _, wss_o = o.macros(None)
    wall = ~np.isnan(wss_o)
    assert np.array_equal(np.isnan(wss), ~wall)
    assert np.linalg.norm(wss[wall] - wss_o[wall]) / np.linalg.norm(wss_o[wall]) < 1e-4
    # the fallback is not the analytic normal: the two readbacks differ
    _, _, wss_n = o.macros(lat.wall_normal)
    assert np.linalg.norm(wss_n[wall] - wss_o[wall]) / np.linalg.norm(wss_o[wall]) > 1e-3
