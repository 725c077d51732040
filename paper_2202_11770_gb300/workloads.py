"""Seeded synthetic workloads (input generation only, no LB arithmetic).

The paper's patient geometries (Circle of Willis, leg arteries, veins) are
not available; these stand in for them:

* ``pipe_poiseuille``  straight pipe R = 8, L = 64 (12,352 sites), tau 0.8,
  steady parabolic Ladd inlet of peak 0.01, rho = 1 pressure outlet.
* ``tree_pulsatile``   seeded depth-6 bifurcating tree (seed 2202, ~20M
  sites, 64 pressure outlets), tau 0.55, inlet 0.02 (1 + 0.5 cos(2 pi t/2000)).
* ``adjoint_case``     seeded depth-4 tree (seed 11770, ~2M sites) whose
  inlet sites form 8 angular sectors x 8 equal-area rings (64 amplitude
  groups); probe sites on the mid-plane of the root segment and a seeded
  target: the Poiseuille profile 0.02 (1 - r^2/R^2) of that plane scaled by
  (1 + 0.1 xi), xi ~ U(-1, 1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import geometry

PULSATILE = {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 2000.0}


def tree_lattice(target_sites=20_000_000, depth=6, seed=2202, **kw):
    return geometry.tree(depth, seed, target_sites=target_sites, length_ratio=5.0, **kw)


def apply_tree_bc(solver, lattice, wave=PULSATILE, amps=None):
    """Velocity inlet (iolet 0) with per-group amplitudes (default 1) times
    `wave`; rho = 1 at every pressure outlet."""
    io0 = lattice.iolets[0]
    a = np.ones(io0.n_groups) if amps is None else np.asarray(amps, dtype=np.float64)
    solver.set_velocity(0, a, wave)
    for k in range(1, len(lattice.iolets)):
        solver.set_pressure(k, 1.0)


@dataclass
class Objective:
    sites: np.ndarray   # int64 probe sites
    target: np.ndarray  # float64 target axial velocity
    axis: np.ndarray    # unit axis


def root_midplane_objective(lattice, seed=11770, peak=0.02, spread=0.1) -> Objective:
    """Probe plane at the middle of the root segment (axis +z through x=y=0)."""
    R = float(lattice.iolets[0].radius)
    zmid = int(round(lattice.info["root_length"] / 2.0 - 0.5))
    xyz = lattice.xyz
    r2 = xyz[:, 0].astype(np.float64) ** 2 + xyz[:, 1].astype(np.float64) ** 2
    sel = np.nonzero((xyz[:, 2] == zmid) & (r2 < R * R))[0].astype(np.int64)
    rng = np.random.default_rng(seed)
    xi = rng.uniform(-1.0, 1.0, sel.size)
    target = peak * (1.0 - r2[sel] / (R * R)) * (1.0 + spread * xi)
    return Objective(sites=sel, target=target, axis=np.array([0.0, 0.0, 1.0]))


def adjoint_case(target_sites=2_000_000, depth=4, seed=11770, n_sectors=8, n_rings=8):
    lat = tree_lattice(target_sites, depth=depth, seed=seed, n_sectors=n_sectors, n_rings=n_rings)
    return lat, root_midplane_objective(lat, seed=seed)


def type_sorted(lattice):
    """The same lattice with its sites reordered by site type (inner, wall,
    inlet, outlet, inlet + wall, outlet + wall; (z, y, x) order within a type):
    the layout of the paper's six collision-streaming kernels over type ranges
    (Section 3.2.2).  Returns (lattice, [(type, first site, end)])."""
    typ = np.asarray(lattice.type)
    perm = np.argsort(typ, kind="stable")
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    src = lattice.src[:, perm]
    src = np.where(src >= 0, inv[np.maximum(src, 0)], src).astype(np.int32)
    out = geometry.from_arrays(lattice.xyz[perm], src, iolets=lattice.iolets, type=typ[perm],
                               wall_normal=lattice.wall_normal[:, perm], amp_group=lattice.amp_group[perm])
    ranges = []
    for t in np.unique(typ):
        idx = np.nonzero(typ[perm] == t)[0]
        ranges.append((int(t), int(idx[0]), int(idx[-1]) + 1))
    return out, ranges

