"""Oracle pins: the Ladd velocity iolet and the wall-shear-stress fallback normal.

Pins (paper Section 2.3.1: mid-link bounce-back puts the wall half way along
each boundary link; Section 2.3.2: the Ladd moving-wall correction
-2 w_i rho (c_i . u_w) / cs2; Section 6: every inlet point carries a weight
from its position in the cross-section):

  * a uniform flow is an exact steady state when every boundary link is a
    Ladd link moving with the flow: the corrected bounce-back of f^eq_i(rho, u)
    is f^eq_ibar(rho, u) exactly, which fixes the factor 2, the 1/cs2 and the
    use of the site's own density (rho != 1 here);
  * one step from rest on a tiny lattice, against an enumeration written here
    from the coordinates: every inlet link receives 6 w_i A W at the link
    midpoint x + c_i/2 (not at the site);
  * the steady inlet mass flux of the R = 8 and R = 12 pipes tends to the
    integral rho A pi R^2 / 2 of the imposed parabola (see test_oracle_flow);
  * the wall shear stress without caller normals uses the normalised sum of
    -c_i over the wall links: on a flat face that is the face normal, on an
    edge of a box the bisector of the two face normals.
"""
import numpy as np

import oracle
from paper_2202_11770_gb300 import geometry as geo
from helpers import hand_lattice


def _box(nx, ny, nz, x0=0, y0=0):
    return [(x0 + x, y0 + y, z) for z in range(nz) for y in range(ny) for x in range(nx)]


def _uniform_flow_case(c, normal, rho0=1.03, speed=0.04):
    """A 4x4x5 box whose every boundary link belongs to velocity iolet 0 with
    normal `normal` and a radius so large that W = 1 to 1e-14."""
    n_hat = np.asarray(normal, np.float64) / np.linalg.norm(normal)
    io = geo.Iolet(kind=geo.VELOCITY, role=0, centre=np.array([1.5, 1.5, 2.0]), normal=n_hat,
                   radius=1e7, n_groups=1)
    lat = hand_lattice(_box(4, 4, 5), c, iolets=[io], classify=lambda p, i: 0)
    u = speed * n_hat
    o = oracle.Oracle(lat, tau=0.7)
    o.set_velocity(0, [speed], 1.0)
    f0 = np.tile(oracle.feq(rho0, u), (lat.n, 1))
    o.set_state(f0, 0)
    return o, f0


def test_ladd_uniform_flow_is_steady(d3q19):
    c, _ = d3q19
    for normal in ((0, 0, 1), (1, 2, 2), (-2, 1, 0.5)):
        o, f0 = _uniform_flow_case(c, normal)
        o.step(20)
        assert np.abs(o.state() - f0).max() < 1e-14, normal
        assert abs(o.mass() - f0.sum()) < 1e-12


def test_ladd_uniform_flow_needs_the_sites_density(d3q19):
    """With rho = 1 in the correction (the ladd_rho_one reading) the same flow
    at rho = 1.03 is no longer steady: the default reading is the one for
    which the moving wall reproduces the equilibrium."""
    c, _ = d3q19
    o, f0 = _uniform_flow_case(c, (0, 0, 1))
    lat_o = oracle.Oracle(hand_lattice(_box(4, 4, 5), c, iolets=o.iolets, classify=lambda p, i: 0),
                          tau=0.7, ladd_rho_one=True)
    lat_o.set_velocity(0, [0.04], 1.0)
    lat_o.set_state(f0, 0)
    lat_o.step(1)
    assert np.abs(lat_o.state() - f0).max() > 1e-5


def test_ladd_one_step_midpoint_weights(d3q19):
    """From rest, one step: only the inlet links change, each by 6 w_i A W(m)
    (c_i . n < 0 out through the inlet plane), m = x + c_i/2 the midpoint of
    the link, W = max(0, 1 - r_m^2/R^2) with r_m the distance of m from the
    iolet axis.  The axis is off the lattice points so that the midpoints of
    the diagonal links sit at radii different from their sites."""
    c, w = d3q19
    pts = [(x, y, z) for z in range(3) for y in range(-3, 4) for x in range(-3, 4) if x * x + y * y < 10]
    centre = np.array([0.25, -0.4, -0.5])
    n_hat = np.array([0.0, 0.0, 1.0])
    R, A = 3.2, 0.05
    io = geo.Iolet(kind=geo.VELOCITY, role=0, centre=centre, normal=n_hat, radius=R, n_groups=1)

    def classify(p, i):       # the link from p along c_i leaves the fluid
        return 0 if p[2] + c[i][2] < 0 else None

    lat = hand_lattice(pts, c, iolets=[io], classify=classify)
    o = oracle.Oracle(lat, tau=0.9)
    o.set_velocity(0, [A], 1.0)
    o.init_equilibrium()
    o.step(1)
    expect = np.tile(w, (lat.n, 1))
    opp = [int(np.nonzero((c == -c[i]).all(axis=1))[0][0]) for i in range(19)]
    moved = 0
    for k, p in enumerate(lat.xyz):
        for i in range(1, 19):
            if p[2] + c[i][2] >= 0:
                continue
            m = p + 0.5 * c[i]
            v = m - centre
            r2 = float(v @ v - (v @ n_hat) ** 2)
            W = max(0.0, 1.0 - r2 / (R * R))
            expect[k, opp[i]] += 6.0 * w[i] * A * W * float(-(c[i] @ n_hat))
            moved += W > 0
    assert moved > 50
    assert np.abs(o.state() - expect).max() < 1e-15


def _random_nonequilibrium(n, rng):
    f = np.stack([oracle.feq(1.0 + 0.02 * rng.uniform(-1, 1), 0.03 * rng.uniform(-1, 1, 3)) for _ in range(n)])
    return f + 1e-3 * rng.uniform(-1, 1, f.shape)


def test_wss_fallback_normal_face_and_edge(d3q19):
    c, _ = d3q19
    lat = hand_lattice(_box(6, 5, 4), c)            # every out-link is a wall
    o = oracle.Oracle(lat, tau=0.6)
    o.set_state(_random_nonequilibrium(lat.n, np.random.default_rng(5)), 0)
    _, _, wss_fb = o.macros(None)
    x, y, z = lat.xyz.T
    normal = np.zeros((3, lat.n), np.float32)
    face = (z == 0) & (x > 0) & (x < 5) & (y > 0) & (y < 4)          # bottom face only
    normal[2, face] = 1.0
    edge = (z == 0) & (x == 0) & (y > 0) & (y < 4)                    # bottom-left edge
    normal[0, edge] = normal[2, edge] = np.float32(np.sqrt(0.5))
    top = (z == 3) & (x > 0) & (x < 5) & (y > 0) & (y < 4)            # top face, normal -z
    normal[2, top] = -1.0
    _, _, wss_n = o.macros(normal)
    sel = face | top
    assert sel.sum() == 24 and np.all(wss_fb[sel] > 0)
    assert np.allclose(wss_fb[sel], wss_n[sel], rtol=1e-14, atol=0)
    # float32 sqrt(1/2) in the caller's normal: agreement to its rounding
    assert np.allclose(wss_fb[edge], wss_n[edge], rtol=1e-6, atol=0)
    # interior sites have no wall link
    assert np.isnan(wss_fb[(x > 0) & (x < 5) & (y > 0) & (y < 4) & (z > 0) & (z < 3)]).all()
