"""Compact index table (16-bit offsets from per-tile, per-direction bases).

The step and adjoint kernels read the streaming index through either form;
the gathered sources are the same, so every result must be bit-identical to
the run on the int32 table (which the other GPU tests pin to the oracle).
A tile whose sources of one direction span more than 65,533 sites cannot be
encoded: the library then uses the int32 table.

With an even number of sites the pull step on the compact table takes two
sites a thread (paired index loads, stores and collisions); the collisions
are the per-thread operations in paired instructions, so it too gives the
bits of the int32-table kernel.
"""
import numpy as np
import pytest

from paper_2202_11770_gb300 import geometry as geo, workloads

pytestmark = pytest.mark.gpu
hemegb = pytest.importorskip("paper_2202_11770_gb300.hemegb")

SCHEMES = ["ab", "aa"]


@pytest.fixture(scope="module")
def tree():
    lat = geo.tree(2, 2202, target_sites=50_000, length_ratio=5.0)
    assert lat.n % 256   # ragged last tile
    return lat


def _bc(x, lat):
    x.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.03, "rel": 0.5, "period": 40.0})
    for k in range(1, len(lat.iolets)):
        x.set_pressure(k, {"kind": "cosine", "mean": 1.0, "rel": 0.002, "period": 25.0})


@pytest.mark.parametrize("wide", [False, True], ids=["off32", "off64"])
@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16", "fp64"])
def test_steps_bit_identical_to_int32_table(tree, prec, scheme, wide):
    out = []
    for full in (False, True):
        s = hemegb.Solver(tree, tau=0.55, precision=prec, scheme=scheme, wide_offsets=wide, full_index=full)
        assert s.compact_index == (not full)
        _bc(s, tree)
        s.init_equilibrium()
        s.step(9)                       # both AA parities, gathers from step 2 on
        f, t = s.state()
        mass, flux = s.reduce()
        out.append((f, t, mass, flux))
    (fa, ta, ma, qa), (fb, tb, mb, qb) = out
    assert ta == tb == 9
    assert fa.tobytes() == fb.tobytes()
    assert ma == mb and np.array_equal(qa, qb)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_adjoint_bit_identical_to_int32_table(tree, prec):
    obj = workloads.root_midplane_objective(tree, seed=2202)
    amps = 1.0 + 0.05 * np.random.default_rng(5).uniform(-1, 1, tree.iolets[0].n_groups)
    res = []
    for full in (False, True):
        s = hemegb.Solver(tree, tau=0.6, precision=prec, full_index=full)
        assert s.compact_index == (not full)
        s.set_velocity(0, amps, {"kind": "cosine", "mean": 0.03, "rel": 0.5, "period": 40.0})
        for k in range(1, len(tree.iolets)):
            s.set_pressure(k, 1.0)
        s.init_equilibrium()
        res.append(s.adjoint(60, obj.sites, obj.target, obj.axis))
    (Ja, da, ga), (Jb, db, gb) = res
    assert Ja == Jb and da == db
    assert np.array_equal(ga, gb)


def _span_lattice(span):
    """Sites on a line (geometry irrelevant here) with two reciprocal link
    pairs: site 0 pulls direction 1 from site 10 and site 1 from site
    10 + span, so tile 0's direction-1 sources span exactly `span`; the
    sources pull direction 2 back.  Every other link is a wall."""
    n = 10 + span + 300
    xyz = np.zeros((n, 3), np.int32)
    xyz[:, 0] = np.arange(n)
    src = np.full((18, n), -1, np.int32)
    src[0, 0], src[1, 10] = 10, 0
    src[0, 1], src[1, 10 + span] = 10 + span, 1
    return geo.from_arrays(xyz, src)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("span,compact", [(65533, True), (65534, False)])
def test_largest_encodable_span(scheme, span, compact):
    lat = _span_lattice(span)
    rng = np.random.default_rng(span)
    h0 = rng.uniform(-0.01, 0.01, (19, lat.n))
    out = []
    for full in (False, True):
        s = hemegb.Solver(lat, tau=0.7, precision="fp64", scheme=scheme, full_index=full)
        assert s.compact_index == (compact and not full)
        s.set_state(h0.copy(), 0)
        s.step(4)
        out.append(s.state()[0])
    assert out[0].tobytes() == out[1].tobytes()


@pytest.mark.parametrize("prec,scheme", [("fp32", "ab"), ("bf16", "ab"), ("fp16", "ab"), ("bf16", "aa"),
                                         ("fp16", "aa")])
def test_two_site_kernels_bit_identical(prec, scheme):
    """Even site count (49,986, ragged last tile pair): the two-site pull
    kernel on the compact table against the one-site kernels (int32 table,
    and the large-lattice offsets), including pairs that hold one iolet
    site; and the AA kernels at an even site count (two-site even step)."""
    lat = geo.tree(2, 2202, target_sites=50_009, length_ratio=5.0)
    assert lat.n % 2 == 0 and lat.n % 512
    isite = (lat.src <= -2).any(axis=0)
    assert (isite[0::2] != isite[1::2]).any()
    out = []
    for full, wide in ((False, False), (True, False), (False, True)):
        s = hemegb.Solver(lat, tau=0.55, precision=prec, scheme=scheme, full_index=full, wide_offsets=wide)
        _bc(s, lat)
        s.init_equilibrium()
        s.step(9)
        out.append((s.state()[0], s.reduce()))
    for f, (m, q) in out[1:]:
        assert f.tobytes() == out[0][0].tobytes()
        assert m == out[0][1][0] and np.array_equal(q, out[0][1][1])
