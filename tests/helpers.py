"""Test-side helpers: hand-made lattices, profile fits and closed forms.

Nothing here is imported by the solver; the formulas are the textbook closed
forms the oracle is pinned to (Poiseuille, Womersley) and brute-force
enumerations written from the velocity set in ``tests/golden/d3q19.txt``.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2202_11770_gb300 import geometry as geo

CS2 = 1.0 / 3.0


def opposite_table(c):
    return np.array([int(np.nonzero((c == -c[i]).all(axis=1))[0][0]) for i in range(19)])


def hand_lattice(points, c, iolets=(), classify=None):
    """Lattice from explicit site coordinates; links leaving the point set are
    walls unless ``classify(point, i)`` returns an iolet index."""
    pts = np.asarray(points, dtype=np.int32).reshape(-1, 3)
    index = {tuple(p): k for k, p in enumerate(pts.tolist())}
    n = len(pts)
    src = np.empty((18, n), np.int32)
    opp = opposite_table(c)
    for k, p in enumerate(pts):
        for i in range(1, 19):
            q = tuple((p - c[i]).tolist())
            if q in index:
                src[i - 1, k] = index[q]
            else:
                code = -1
                if classify is not None:
                    kk = classify(p, opp[i])  # link from p along c_opp leaves the fluid
                    if kk is not None:
                        code = -(2 + kk)
                src[i - 1, k] = code
    return geo.from_arrays(pts, src, iolets=iolets)


def fit_parabola(r, u):
    """Least squares u = U (1 - r^2/R^2) -> (U, R, curvature U/R^2, relL2 residual)."""
    A = np.stack([np.ones_like(r), -r ** 2], 1)
    coef, *_ = np.linalg.lstsq(A, u, rcond=None)
    U, k = coef
    fit = A @ coef
    return U, math.sqrt(U / k), k, float(np.linalg.norm(u - fit) / np.linalg.norm(u))


def density_gradient(lat, rho, z0, z1):
    """Body-force equivalent G = -cs2 d(rho)/dz / rho_mean from cross-section means."""
    zs = np.arange(z0, z1)
    means = np.array([rho[lat.xyz[:, 2] == z].mean() for z in zs])
    slope = np.polyfit(zs, means, 1)[0]
    return -CS2 * slope / means.mean()


def bessel_j0(z):
    """J0 of a complex argument by its power series sum (-z^2/4)^m/(m!)^2."""
    z = np.asarray(z, dtype=np.complex128)
    total = np.zeros_like(z)
    term = np.ones_like(z)
    for m in range(80):
        if m:
            term = term * (-(z * z) / 4.0) / (m * m)
        total = total + term
    return total


def womersley_profile(G_hat, omega, nu, r, R):
    """Complex amplitude U(r) of u = Re{U(r) e^{i omega t}} for a body force
    Re{G_hat e^{i omega t}} in a pipe of radius R (no-slip at R):
    i omega U = G + nu (U'' + U'/r)  =>  U = G/(i omega) (1 - J0(k r)/J0(k R)),
    k^2 = -i omega / nu."""
    k = np.sqrt(-1j * omega / nu)
    return G_hat / (1j * omega) * (1.0 - bessel_j0(k * r) / bessel_j0(k * R))
