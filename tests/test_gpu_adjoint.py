"""GPU discrete adjoint vs the oracle's FP64 adjoint and central differences.

* FP64 storage: the GPU adjoint (pull-form transpose, gathers) equals the
  oracle's explicit-Jacobian push-form adjoint to rounding.
* FP32 storage on a ~50k-site depth-2 tree: within 1e-4 relative of the
  oracle's FP64 adjoint.
* Full size (seeded depth-4 tree, ~2M sites, 64 inlet amplitude groups,
  N = 2000 steps, sqrt(N) checkpoints): the FP32 adjoint agrees within 1e-3
  with central differences (h = 1e-4) of the GPU FP64 forward on dJ/dtau,
  four single amplitudes and four random amplitude directions.
"""
import numpy as np
import pytest

import oracle
from paper_2202_11770_gb300 import geometry as geo, workloads

pytestmark = pytest.mark.gpu
hemegb = pytest.importorskip("paper_2202_11770_gb300.hemegb")


def _setup(x, lat, amps):
    x.set_velocity(0, amps, {"kind": "cosine", "mean": 0.03, "rel": 0.5, "period": 50.0})
    for k in range(1, len(lat.iolets)):
        x.set_pressure(k, {"kind": "cosine", "mean": 1.0, "rel": 0.001 * k, "period": 30.0})
    x.init_equilibrium()


@pytest.mark.parametrize("opts,wide,scheme", [((False, False), False, "ab"), ((True, True), False, "aa"),
                                             ((False, False), True, "aa"), ((True, True), True, "ab")])
def test_fp64_adjoint_equals_oracle(opts, wide, scheme):
    """The solver's own scheme only decides how the final state is handed back."""
    lat = geo.tree(1, 7, root_radius=4.0, length_ratio=5.0, n_sectors=2, n_rings=2)
    N, tau = 40, 0.7
    probe = np.nonzero(lat.xyz[:, 2] == int(lat.info["root_length"] // 2))[0]
    rng = np.random.default_rng(1)
    target = 0.02 * (1 + 0.1 * rng.uniform(-1, 1, probe.size))
    amps = np.array([1.0, 0.9, 1.1, 0.95])
    o = oracle.Oracle(lat, tau, *opts)
    _setup(o, lat, amps)
    J_o, dtau_o, damp_o = o.adjoint(N, probe, target, [0, 0, 1])
    s = hemegb.Solver(lat, tau=tau, precision="fp64", ladd_rho_one=opts[0], ghost_full_u=opts[1],
                      wide_offsets=wide, scheme=scheme)
    _setup(s, lat, amps)
    J, dtau, damp = s.adjoint(N, probe, target, [0, 0, 1])
    assert s.t == N
    assert J == pytest.approx(J_o, rel=1e-12)
    assert dtau == pytest.approx(dtau_o, rel=1e-9)
    assert np.allclose(damp, damp_o, rtol=1e-9, atol=0)


def test_fp32_adjoint_vs_oracle_depth2_tree():
    lat = geo.tree(2, 2202, target_sites=50_000, length_ratio=5.0, n_sectors=8, n_rings=8)
    obj = workloads.root_midplane_objective(lat, seed=2202)
    N, tau = 100, 0.6
    amps = 1.0 + 0.05 * np.random.default_rng(2).uniform(-1, 1, 64)
    o = oracle.Oracle(lat, tau)
    _setup(o, lat, amps)
    J_o, dtau_o, damp_o = o.adjoint(N, obj.sites, obj.target, obj.axis)
    s = hemegb.Solver(lat, tau=tau, precision="fp32")
    _setup(s, lat, amps)
    J, dtau, damp = s.adjoint(N, obj.sites, obj.target, obj.axis)
    assert J == pytest.approx(J_o, rel=1e-4)
    assert dtau == pytest.approx(dtau_o, rel=1e-4)
    assert np.linalg.norm(damp - damp_o) <= 1e-4 * np.linalg.norm(damp_o)


def test_adjoint_validation():
    lat = geo.pipe(4.0, 8)
    s = hemegb.Solver(lat, tau=0.7, precision="bf16")
    with pytest.raises(hemegb.HlbError):
        s.adjoint(10, [1, 2], [0.0, 0.0], [0, 0, 1])     # 16-bit storage has no adjoint
    s = hemegb.Solver(lat, tau=0.7, precision="fp32")
    with pytest.raises(hemegb.HlbError):
        s.adjoint(10, [1, 1], [0.0, 0.0], [0, 0, 1])     # duplicate probes
    with pytest.raises(hemegb.HlbError):
        s.adjoint(10, [lat.n], [0.0], [0, 0, 1])         # out of range
    with pytest.raises(hemegb.HlbError):
        s.adjoint(0, [1], [0.0], [0, 0, 1])


def test_full_size_adjoint_vs_central_differences():
    lat, obj = workloads.adjoint_case()
    assert abs(lat.n - 2_000_000) < 0.02 * 2_000_000
    assert lat.iolets[0].n_groups == 64
    N, tau, h = 2000, 0.55, 1e-4
    amps = np.ones(64)

    def run(precision, tau_, amps_):
        s = hemegb.Solver(lat, tau=tau_, precision=precision)
        workloads.apply_tree_bc(s, lat, amps=amps_)
        s.init_equilibrium()
        out = s.adjoint(N, obj.sites, obj.target, obj.axis)
        del s
        return out

    J, dtau, damp = run("fp32", tau, amps)
    assert damp.shape == (64,) and np.isfinite(damp).all()
    Jp = run("fp64", tau + h, amps)[0]
    Jm = run("fp64", tau - h, amps)[0]
    fd = (Jp - Jm) / (2 * h)
    assert abs(dtau - fd) <= 1e-3 * abs(fd), (dtau, fd)
    rng = np.random.default_rng(11770)
    dirs = [np.eye(64)[g] for g in (0, 21, 42, 63)] + [rng.normal(size=64) for _ in range(4)]
    for d in dirs:
        fd = (run("fp64", tau, amps + h * d)[0] - run("fp64", tau, amps - h * d)[0]) / (2 * h)
        assert abs(damp @ d - fd) <= 1e-3 * abs(fd), (damp @ d, fd)


@pytest.mark.parametrize("scheme", ["ab", "aa"])
def test_adjoint_leaves_the_forward_state(scheme):
    """The forward sweep runs the solver's own step kernels: afterwards the
    solver holds, bit for bit, the state of N plain steps, and stepping on
    from there matches too."""
    lat = geo.tree(1, 7, root_radius=4.0, length_ratio=5.0, n_sectors=2, n_rings=2)
    N = 23                                   # odd: ends mid AA cycle; > one checkpoint interval
    probe = np.nonzero(lat.xyz[:, 2] == int(lat.info["root_length"] // 2))[0]
    target = np.full(probe.size, 0.02)
    amps = np.array([1.0, 0.9, 1.1, 0.95])
    runs = []
    for adj in (True, False):
        s = hemegb.Solver(lat, tau=0.7, precision="fp32", scheme=scheme)
        _setup(s, lat, amps)
        if adj:
            s.adjoint(N, probe, target, [0, 0, 1])
        else:
            s.step(N)
        f, t = s.state()
        m, q = s.reduce()
        s.step(5)
        runs.append((f, t, m, q, s.state()[0]))
    (fa, ta, ma, qa, ga), (fb, tb, mb, qb, gb) = runs
    assert ta == tb == N
    assert fa.tobytes() == fb.tobytes() and ga.tobytes() == gb.tobytes()
    assert ma == mb and np.array_equal(qa, qb)


@pytest.mark.parametrize("precision,scheme", [("fp32", "aa"), ("fp32", "ab"), ("fp64", "aa")])
def test_kept_segments_give_identical_results(precision, scheme):
    """A larger workspace keeps whole segments of post-collision states from
    the forward sweep instead of recomputing them: the gradients, J and the
    final state are bit-identical to the sqrt(N)-memory run, whether none,
    some or all but the last segment are kept."""
    lat = geo.tree(1, 7, root_radius=4.0, length_ratio=5.0, n_sectors=2, n_rings=2)
    N = 41                                   # K = 8, six segments, the last one short and odd
    probe = np.nonzero(lat.xyz[:, 2] == int(lat.info["root_length"] // 2))[0]
    target = np.full(probe.size, 0.02)
    amps = np.array([1.0, 0.9, 1.1, 0.95])
    s = hemegb.Solver(lat, tau=0.7, precision=precision, scheme=scheme)
    base = hemegb.hlb_adjoint_workspace_bytes(s._h, N, probe.size)
    K, kept_all, rec_all, used_all = s.adjoint_plan(N, probe.size, 1 << 40)
    assert K == 8 and kept_all == 5 and rec_all == N - 5 * K
    per_seg = (used_all - base) // kept_all
    assert per_seg * kept_all == used_all - base and per_seg >= 19 * lat.n * K * (4 if precision == "fp32" else 8)
    assert s.adjoint_plan(N, probe.size, base)[1:] == (0, N, base)
    with pytest.raises(hemegb.HlbError):
        s.adjoint_plan(N, probe.size, base - 1)
    runs = []
    for n_keep in (0, 2, 5):
        s = hemegb.Solver(lat, tau=0.7, precision=precision, scheme=scheme)
        _setup(s, lat, amps)
        s.step(3)                            # start mid AA cycle
        ws = s.adjoint_workspace(N, probe.size, extra_bytes=n_keep * per_seg + per_seg // 2)
        assert s.adjoint_plan(N, probe.size, ws[2])[1] == n_keep
        J, dtau, damp = s.adjoint(N, probe, target, [0, 0, 1], workspace=ws)
        f, t = s.state()
        s.step(4)
        runs.append((J, dtau, np.asarray(damp), f, t, s.state()[0]))
    for r in runs[1:]:
        assert r[0] == runs[0][0] and r[1] == runs[0][1] and r[2].tobytes() == runs[0][2].tobytes()
        assert r[3].tobytes() == runs[0][3].tobytes() and r[4] == runs[0][4] == N + 3
        assert r[5].tobytes() == runs[0][5].tobytes()
