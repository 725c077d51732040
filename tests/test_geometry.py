"""Seeded input generator: site counts, table consistency, determinism.

The generator is shared input of the oracle and the GPU solver; these checks
make sure its tables describe the geometry it claims (no LB arithmetic here).
"""
import numpy as np
import pytest

from paper_2202_11770_gb300 import geometry as geo


def _check_table(lat, c):
    n = lat.n
    key = {tuple(p): k for k, p in enumerate(lat.xyz.tolist())} if n < 200_000 else None
    for i in range(1, 19):
        s = lat.src[i - 1]
        fluid = s >= 0
        # fluid entries point at the site x - c_i
        assert np.array_equal(lat.xyz[s[fluid]], lat.xyz[fluid] - c[i])
        if key is not None:
            # non-fluid entries really have no site at x - c_i
            for k in np.nonzero(~fluid)[0][:2000]:
                assert tuple((lat.xyz[k] - c[i]).tolist()) not in key
        assert (s >= -(2 + len(lat.iolets) - 1)).all()


def test_pipe_counts_and_table(d3q19):
    c, _ = d3q19
    lat = geo.pipe(8.0, 64)
    assert lat.n == 12352                       # 193 sites per cross-section x 64
    assert (np.bincount(lat.xyz[:, 2]) == 193).all()
    _check_table(lat, c)
    # ordering by (z, y, x)
    k = (lat.xyz[:, 2].astype(np.int64) << 40) + (lat.xyz[:, 1].astype(np.int64) + 1000 << 20) + lat.xyz[:, 0] + 1000
    assert (np.diff(k) > 0).all()
    # every z = 0 site links to the inlet along -z, every z = 63 site to the outlet along +z
    z = lat.xyz[:, 2]
    assert (lat.src[5 - 1][z == 0] == -2).all()      # direction 5 = +z pulls from z-1
    assert (lat.src[6 - 1][z == 63] == -3).all()     # direction 6 = -z pulls from z+1
    # no iolet links away from the end layers
    iol = (lat.src <= -2).any(axis=0)
    assert not iol[(z > 0) & (z < 63)].any()
    # wall normals point inwards at wall sites
    wall = (lat.src == -1).any(axis=0)
    r = lat.xyz[:, :2].astype(float)
    dots = (lat.wall_normal[:2].T * r).sum(1)
    assert (dots[wall] < 0).all()
    assert np.allclose(np.linalg.norm(lat.wall_normal[:, wall], axis=0), 1.0, atol=1e-6)


def test_closed_pipe_has_no_iolets():
    lat = geo.pipe(4.0, 6, geo.WALL, geo.WALL)
    assert len(lat.iolets) == 0
    assert (lat.src >= -1).all()


def test_tree_deterministic_and_sized(d3q19):
    c, _ = d3q19
    a = geo.tree(2, 2202, target_sites=50_000, length_ratio=5.0)
    b = geo.tree(2, 2202, target_sites=50_000, length_ratio=5.0)
    assert np.array_equal(a.xyz, b.xyz) and np.array_equal(a.src, b.src)
    assert abs(a.n - 50_000) <= 0.02 * 50_000
    assert len(a.iolets) == 1 + 4
    assert a.iolets[0].kind == geo.VELOCITY and all(io.kind == geo.PRESSURE for io in a.iolets[1:])
    _check_table(a, c)
    # every iolet has links
    for k in range(len(a.iolets)):
        assert (a.src == -(2 + k)).sum() > 0
    other = geo.tree(2, 2203, target_sites=50_000, length_ratio=5.0)
    assert other.n != a.n or not np.array_equal(other.xyz, a.xyz)


def test_tree_amplitude_groups():
    lat = geo.tree(2, 11770, target_sites=60_000, length_ratio=5.0, n_sectors=8, n_rings=8)
    inlet_sites = (lat.src == -2).any(axis=0)
    g = lat.amp_group[inlet_sites]
    assert g.min() == 0 and g.max() == 63
    counts = np.bincount(g, minlength=64)
    assert (counts > 0).all()


@pytest.mark.parametrize("depth,seed,sites", [(2, 2202, 50_000), (4, 11770, 300_000)])
def test_tile_sources_increase_and_fit_16_bits(depth, seed, sites):
    """The step kernels' compact index table rests on two properties of the
    (z, y, x) site order: over a 256-site tile the fluid sources of one
    direction increase with the site index, and they span fewer than 65,534
    sites (here a few hundred), so 16-bit offsets from a per-tile base
    reach them all."""
    lat = geo.tree(depth, seed, target_sites=sites, length_ratio=5.0)
    n, T = lat.n, 256
    order = np.lexsort((lat.xyz[:, 0], lat.xyz[:, 1], lat.xyz[:, 2]))
    assert np.array_equal(order, np.arange(n))          # sites sorted by (z, y, x)
    tile = np.arange(n) // T
    worst = 0
    for i in range(18):
        s = lat.src[i].astype(np.int64)
        x = np.nonzero(s >= 0)[0]
        same = tile[x[1:]] == tile[x[:-1]]
        assert (s[x[1:]][same] > s[x[:-1]][same]).all()  # increasing within a tile
        lo = np.full(tile[-1] + 1, np.iinfo(np.int64).max)
        hi = np.full(tile[-1] + 1, -1)
        np.minimum.at(lo, tile[x], s[x])
        np.maximum.at(hi, tile[x], s[x])
        has = hi >= 0
        worst = max(worst, int((hi[has] - lo[has]).max()))
    assert worst <= 65533
    assert worst < 4 * T


def test_type_sorted_lattice_is_a_relabelling():
    """The site permutation of the per-type layout keeps every source at
    x - c_i and every wall / iolet code, and groups the types in ranges."""
    from paper_2202_11770_gb300 import workloads
    lat = geo.tree(2, 2202, target_sites=30_000, length_ratio=5.0)
    s, ranges = workloads.type_sorted(lat)
    assert s.n == lat.n and sorted(map(tuple, s.xyz.tolist())) == sorted(map(tuple, lat.xyz.tolist()))
    assert [b for _, b, _ in ranges][0] == 0 and ranges[-1][2] == lat.n
    assert all(e == b2 for (_, _, e), (_, b2, _) in zip(ranges[:-1], ranges[1:]))
    for t, b, e in ranges:
        assert (s.type[b:e] == t).all()
    for i in range(18):
        m = s.src[i] >= 0
        assert np.array_equal(s.xyz[s.src[i][m]], s.xyz[m] - geo.CI[i + 1])
    assert np.array_equal(np.sort(s.src[s.src < 0]), np.sort(lat.src[lat.src < 0]))
