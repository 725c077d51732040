"""Partitioned pull A-B runs on one GPU (include/hlb_partition.h) against the
undivided solver, through the C ABI.

Every part is an ordinary lattice for the solver (owned sites plus ghost
copies of the remote sources); after each step the owners' post-collision
values are packed and unpacked into the ghosts' slots on the device.  The
owned sites then see exactly the undivided inputs, so states and macroscopic
fields are bit-identical; mass and iolet fluxes are sums over parts, equal to
rounding.  Part counts span a split inside the root vessel, through the
bifurcations and across the outlets; precisions include 16-bit storage.
"""
import numpy as np
import pytest

from paper_2202_11770_gb300 import geometry as geo

pytestmark = pytest.mark.gpu
hemegb = pytest.importorskip("paper_2202_11770_gb300.hemegb")
partition = pytest.importorskip("paper_2202_11770_gb300.partition")


def _bc(x, lat):
    x.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 40.0})
    for k in range(1, len(lat.iolets)):
        x.set_pressure(k, 1.0 - 0.0005 * k)


@pytest.fixture(scope="module")
def tree():
    return geo.tree(2, 2202, target_sites=50_000, length_ratio=5.0)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp64"])
@pytest.mark.parametrize("n_parts", [2, 3, 7])
def test_partitioned_run_is_bit_identical(tree, n_parts, prec):
    lat = tree
    ref = hemegb.Solver(lat, tau=0.6, precision=prec, scheme="ab")
    ps = partition.PartitionedSolver(lat, n_parts, tau=0.6, precision=prec)
    for x in (ref, ps):
        _bc(x, lat)
        x.init_equilibrium()
        x.step(41)
    assert all(s.compact_index for s in ps.parts)      # local lattices keep the global order
    f_ref, t_ref = ref.state()
    f, t = ps.state()
    assert t == t_ref == 41
    assert f.tobytes() == f_ref.tobytes()
    for a, b in zip(ps.macros(), ref.macros()):
        assert np.array_equal(a, b, equal_nan=True)
    m, fl = ps.reduce()
    m_ref, fl_ref = ref.reduce()
    assert abs(m - m_ref) <= 1e-12 * m_ref
    assert np.allclose(fl, fl_ref, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("n_parts", [2, 5])
def test_edge_first_overlapped_steps_are_bit_identical(tree, n_parts):
    """The edge-first order: edge tiles, then the halo exchange on a second
    stream while the interior tiles run (hlb_step_range)."""
    lat = tree
    ref = hemegb.Solver(lat, tau=0.6, precision="fp32", scheme="ab")
    ps = partition.PartitionedSolver(lat, n_parts, tau=0.6, precision="fp32")
    _bc(ref, lat)
    _bc(ps, lat)
    ref.init_equilibrium()
    ps.init_equilibrium()
    ref.step(37)
    ps.step(37, overlap=True)
    assert all(len(e) and len(i) for e, i in zip(ps._edge, ps._interior))
    assert ps.state()[0].tobytes() == ref.state()[0].tobytes()
    m, fl = ps.reduce()
    m_ref, fl_ref = ref.reduce()
    assert abs(m - m_ref) <= 1e-12 * m_ref and np.allclose(fl, fl_ref, rtol=1e-12, atol=1e-15)


def test_partitioned_pipe_inlet_and_outlet_in_different_parts():
    lat = geo.pipe(8.0, 64)
    ref = hemegb.Solver(lat, tau=0.8, precision="fp32", scheme="ab")
    ps = partition.PartitionedSolver(lat, 2, tau=0.8, precision="fp32")
    for x in (ref, ps):
        x.set_velocity(0, [1.0], 0.01)
        x.set_pressure(1, 1.0)
        x.init_equilibrium()
        x.step(200)
    assert ps.state()[0].tobytes() == ref.state()[0].tobytes()
    fl, fl_ref = ps.reduce()[1], ref.reduce()[1]
    assert np.allclose(fl, fl_ref, rtol=1e-12, atol=1e-15)
