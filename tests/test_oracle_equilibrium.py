"""Oracle pins: the equilibrium and the velocity set.

Pins (paper Section 2.2, Eq. 4, Eqs. 5-6):
  * feq(1, 0) equals the printed weights (golden fixture).
  * the directions recovered from the linear response of feq to u match the
    printed velocity set in the fixture's order;
  * zeroth, first and second moments of feq are rho, rho u and
    rho cs2 I + rho u u exactly.  The second-moment identity fails for the
    equilibrium exactly as printed (without the factors 1/2), so it pins the
    reading of the garbled Eq. 4.
"""
import numpy as np

import oracle

CS2 = 1.0 / 3.0


def test_rest_equilibrium_is_weights(d3q19):
    _, w = d3q19
    assert np.allclose(oracle.feq(1.0, [0, 0, 0]), w, rtol=0, atol=1e-16)
    assert abs(w.sum() - 1.0) < 1e-15


def test_direction_order_matches_fixture(d3q19):
    c, w = d3q19
    eps = 1e-4
    for a in range(3):
        e = np.zeros(3)
        e[a] = eps
        lin = (oracle.feq(1.0, e) - oracle.feq(1.0, -e)) / (2 * eps)  # = w_i c_ia / cs2
        assert np.allclose(lin * CS2 / w, c[:, a], atol=1e-9)


def test_moments_exact(d3q19):
    c, _ = d3q19
    rng = np.random.default_rng(7)
    for _ in range(50):
        rho = rng.uniform(0.5, 1.5)
        u = rng.uniform(-0.2, 0.2, 3)
        f = oracle.feq(rho, u)
        assert abs(f.sum() - rho) < 1e-14
        assert np.allclose(f @ c, rho * u, atol=1e-15)
        second = np.einsum("i,ia,ib->ab", f, c, c)
        assert np.allclose(second, rho * CS2 * np.eye(3) + rho * np.outer(u, u), atol=1e-15)


def test_printed_form_would_fail_second_moment(d3q19):
    """Equilibrium exactly as printed (no 1/2 factors) gives 2 rho u u."""
    c, w = d3q19
    rho, u = 1.0, np.array([0.05, -0.02, 0.03])
    cu = c @ u
    printed = w * rho * (1 + cu / CS2 + cu ** 2 / CS2 ** 2 - u @ u / CS2)
    second = np.einsum("i,ia,ib->ab", printed, c, c)
    expect = rho * CS2 * np.eye(3) + rho * np.outer(u, u)
    assert not np.allclose(second, expect, atol=1e-6)
    assert np.allclose(second, rho * CS2 * np.eye(3) + 2 * rho * np.outer(u, u), atol=1e-12)
