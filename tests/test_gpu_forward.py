"""GPU forward path vs the FP64 oracle, through the C ABI.

Tolerances: FP32 storage and arithmetic must reach relative L2 velocity
error <= 1e-5 after 1000 steps on the 12,352-site pipe; FP64 agrees to
rounding (1e-11); integer-like behaviour (rest state, permutations) is exact.
Sizes span many 256-site tiles with ragged tails; the full-size case runs the
seeded 20M-site tree in the benchmark's launch configuration and checks one
step against the oracle at every site.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2202_11770_gb300 import geometry as geo
from helpers import hand_lattice

pytestmark = pytest.mark.gpu

hemegb = pytest.importorskip("paper_2202_11770_gb300.hemegb")


SCHEMES = ["ab", "aa"]


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _both(lat, tau, setup, precision="fp32", scheme="ab", **kw):
    s = hemegb.Solver(lat, tau=tau, precision=precision, scheme=scheme, **kw)
    o = oracle.Oracle(lat, tau=tau, ladd_rho_one=kw.get("ladd_rho_one", False),
                      ghost_full_u=kw.get("ghost_full_u", False))
    setup(s)
    setup(o)
    s.init_equilibrium()
    o.init_equilibrium()
    return s, o


def _pipe_bc(x):
    x.set_velocity(0, [1.0], 0.01)
    x.set_pressure(1, 1.0)


@pytest.fixture(scope="module")
def pipe():
    return geo.pipe(8.0, 64)


@pytest.mark.parametrize("wide", [False, True], ids=["off32", "off64"])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_pipe_fp32_1000_steps(pipe, scheme, wide):
    """wide: the 64-bit-offset kernels, which lattices above ~226M sites use."""
    s, o = _both(pipe, 0.8, _pipe_bc, scheme=scheme, wide_offsets=wide)
    s.step(1000)
    o.step(1000)
    rho, u, wss = s.macros()
    rho_o, u_o, wss_o = o.macros(pipe.wall_normal)
    err_u = rel_l2(u, u_o)
    assert err_u <= 1e-5, err_u
    assert np.abs(rho - rho_o).max() < 1e-6
    wall = ~np.isnan(wss_o)
    assert np.array_equal(np.isnan(wss), ~wall)
    assert rel_l2(wss[wall], wss_o[wall]) < 1e-4
    mass, flux = s.reduce()
    # FP32 storage rounds every stored population: mass drifts at roundoff level
    print(f"{scheme}/{'wide' if wide else 'off32'}: FP32 mass - oracle mass = {mass - o.mass():.3e} "
          f"({(mass - o.mass()) / mass:.3e} relative)")
    assert abs(mass - o.mass()) < 1e-7 * mass
    assert np.allclose(flux, o.flux(), rtol=1e-4, atol=1e-9)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_pipe_fp64_matches_to_rounding(pipe, scheme):
    def bc(x):
        x.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.01, "rel": 0.5, "period": 60.0})
        x.set_pressure(1, {"kind": "cosine", "mean": 1.0, "rel": 0.001, "period": 45.0})
    s, o = _both(pipe, 0.7, bc, precision="fp64", scheme=scheme)
    s.step(300)
    o.step(300)
    f, t = s.state()
    assert t == 300
    from conftest import load_d3q19
    _, w = load_d3q19()
    f_o = o.state().T - w[:, None]
    assert np.abs(f - f_o).max() < 1e-13
    rho, u, wss = s.macros()
    _, u_o, _ = o.macros(pipe.wall_normal)
    assert rel_l2(u, u_o) < 2e-7          # macros are returned as float32
    mass, flux = s.reduce()
    assert abs(mass - o.mass()) < 1e-12 * mass
    assert np.allclose(flux, o.flux(), rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16", "fp64"])
def test_rest_state_exact(pipe, prec, scheme):
    def bc(x):
        x.set_velocity(0, [1.0], 0.0)
        x.set_pressure(1, 1.0)
    s = hemegb.Solver(pipe, tau=0.8, precision=prec, scheme=scheme)
    bc(s)
    s.init_equilibrium()
    s.step(1001)
    f, _ = s.state()
    assert not f.view(np.uint8).any()         # shifted state stays exactly zero


@pytest.mark.parametrize("scheme", SCHEMES)
def test_streaming_permutation_bruteforce(d3q19, scheme):
    c, w = d3q19
    from helpers import opposite_table
    opp = opposite_table(c)
    rng = np.random.default_rng(3)
    pts = [(x, y, z) for x in range(9) for y in range(7) for z in range(6) if (x * 7 + y * 3 + z) % 5]
    lat = hand_lattice(pts, c)
    assert lat.n > 256 and lat.n % 256   # several tiles, ragged tail
    n = lat.n
    rho0 = rng.uniform(0.9, 1.1, n)
    u0 = rng.uniform(-0.05, 0.05, (n, 3))
    f0 = np.stack([oracle.feq(rho0[k], u0[k]) for k in range(n)])     # equilibrium: collision is identity
    s = hemegb.Solver(lat, tau=0.7, precision="fp64", scheme=scheme)
    s.set_state((f0 - w).T.copy(), 0)
    s.step(1)          # collision is the identity on an equilibrium state
    got, t = s.state()  # gathered through the index table (post-collision buffer)
    assert t == 1
    index = {tuple(p): k for k, p in enumerate(lat.xyz.tolist())}
    exp = np.full_like(f0, np.nan)
    for k, p in enumerate(lat.xyz):
        for i in range(19):
            q = tuple((p + c[i]).tolist())
            if q in index:
                exp[index[q], i] = f0[k, i]
            else:
                exp[k, opp[i]] = f0[k, i]
    assert not np.isnan(exp).any()
    assert np.abs(got.T + w - exp).max() < 1e-14


@pytest.mark.parametrize("scheme", SCHEMES)
def test_isolated_site_and_small_lattices(d3q19, scheme):
    c, _ = d3q19
    for pts in ([(0, 0, 0)], [(0, 0, 0), (1, 0, 0)], [(0, 0, 0), (1, 1, 0), (1, 1, 1)]):
        lat = hand_lattice(pts, c)
        s = hemegb.Solver(lat, tau=0.6, precision="fp32", scheme=scheme)
        o = oracle.Oracle(lat, tau=0.6)
        rng = np.random.default_rng(len(pts))
        u0 = rng.uniform(-0.05, 0.05, (lat.n, 3))
        s.init_equilibrium(1.0, u0.T.astype(np.float32).copy())
        o.init_equilibrium(1.0, u0.astype(np.float32).astype(np.float64))
        s.step(7)
        o.step(7)
        rho, u, _ = s.macros()
        rho_o, u_o, _ = o.macros()
        assert np.abs(u - u_o).max() < 1e-7
        assert np.abs(rho - rho_o).max() < 1e-6


@pytest.mark.parametrize("wide", [False, True], ids=["off32", "off64"])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_tree_several_tiles_fp32(scheme, wide):
    lat = geo.tree(2, 2202, target_sites=50_000, length_ratio=5.0)
    assert lat.n % 256

    def bc(x):
        x.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 200.0})
        for k in range(1, len(lat.iolets)):
            x.set_pressure(k, 1.0)
    s, o = _both(lat, 0.55, bc, scheme=scheme, wide_offsets=wide)
    s.step(301)
    o.step(301)
    _, u, wss = s.macros()
    _, u_o, wss_o = o.macros(lat.wall_normal)
    assert rel_l2(u, u_o) <= 1e-5
    wall = ~np.isnan(wss_o)
    assert rel_l2(wss[wall], wss_o[wall]) < 1e-4


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("opts", [dict(ladd_rho_one=True), dict(ghost_full_u=True)])
def test_boundary_options(opts, scheme):
    lat = geo.tree(1, 5, root_radius=5.0, length_ratio=5.0)

    def bc(x):
        x.set_velocity(0, [1.0], 0.02)
        for k in range(1, len(lat.iolets)):
            x.set_pressure(k, 1.0 - 0.001 * k)
    s, o = _both(lat, 0.6, bc, precision="fp64", scheme=scheme, **opts)
    s.step(100)
    o.step(100)
    _, u, _ = s.macros()
    _, u_o, _ = o.macros()
    assert rel_l2(u, u_o) < 2e-7


@pytest.mark.parametrize("scheme", SCHEMES)
def test_mass_budget_and_closed_conservation(scheme):
    lat = geo.pipe(5.0, 20, geo.WALL, geo.WALL)
    s = hemegb.Solver(lat, tau=0.6, precision="fp64", scheme=scheme)
    rng = np.random.default_rng(5)
    s.init_equilibrium(1.0, rng.uniform(-0.02, 0.02, (3, lat.n)).astype(np.float32))
    m0, _ = s.reduce()
    s.step(500)
    m1, _ = s.reduce()
    assert abs(m1 - m0) < 1e-13 * m0

    lat = geo.pipe(6.0, 24)
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-12)):
        s = hemegb.Solver(lat, tau=0.7, precision=prec, scheme=scheme)
        s.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 40.0})
        s.set_pressure(1, {"kind": "cosine", "mean": 1.0, "rel": 0.002, "period": 25.0})
        s.init_equilibrium()
        m, _ = s.reduce()
        for _ in range(30):
            s.step(1)
            m1, fl = s.reduce()
            # the FP64 reduction sees exactly the stored values: the budget is exact to FP64 rounding
            assert abs((m1 - m) - fl.sum()) < tol * m1 + (2e-6 if prec == "fp32" else 0)
            m = m1


@pytest.mark.parametrize("scheme", SCHEMES)
def test_divergence_detected(pipe, scheme):
    """A non-finite population (planted on the host in the state handed to the
    solver) makes the FP64 mass non-finite: reduce() reports HLB_ERR_DIVERGED
    instead of a number, and keeps doing so as the NaN spreads."""
    s, _ = _both(pipe, 0.8, _pipe_bc, scheme=scheme)
    s.step(10)
    f, t = s.state()
    f[3, pipe.n // 2] = np.nan
    s.set_state(f, t)
    for steps in (0, 3):
        s.step(steps)
        with pytest.raises(hemegb.HlbError) as err:
            s.reduce()
        assert err.value.code == hemegb.HLB_ERR_DIVERGED


@pytest.mark.parametrize("scheme", SCHEMES)
def test_state_roundtrip_resumes_bit_identical(pipe, scheme):
    s, _ = _both(pipe, 0.8, _pipe_bc, scheme=scheme)
    s.step(37)
    f, t = s.state()
    s.step(20)
    ref, _ = s.state()
    s2 = hemegb.Solver(pipe, tau=0.8, precision="fp32", scheme=scheme)
    _pipe_bc(s2)
    s2.set_state(f, t)
    s2.step(20)
    got, t2 = s2.state()
    assert t2 == t + 20
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("prec,bound", [("bf16", 0.1), ("fp16", 0.02)])
def test_16bit_storage_error_reported(pipe, prec, bound, scheme):
    s, o = _both(pipe, 0.8, _pipe_bc, precision=prec, scheme=scheme)
    s.step(1000)
    o.step(1000)
    _, u, _ = s.macros()
    _, u_o, _ = o.macros(pipe.wall_normal)
    err = rel_l2(u, u_o)
    print(f"{prec}: rel L2(u) after 1000 steps = {err:.3e}")
    assert err < bound


def _stored_to_f64(a, prec):
    if prec == "bf16":
        return hemegb.bf16_to_float(a).astype(np.float64)
    return a.astype(np.float64)


def _half_ulp(v, prec):
    """Half a unit in the last place of the 16-bit format at magnitude |v|."""
    mant, emin = (7, -126) if prec == "bf16" else (10, -14)
    e = np.floor(np.log2(np.maximum(np.abs(v), 2.0 ** emin)))
    return 0.5 * 2.0 ** (e - mant)


def _one_step_within_rounding(lat, tau, bc, prec, scheme, w, warm=5, wide=False, checks=2):
    """Step the 16-bit solver `warm` steps, then compare each of the next
    `checks` steps with the oracle's FP64 step from the same (exactly
    representable) state; two checks cover both AA parities.

    Tight entries: a stored value is the FP64 result rounded to the 16-bit
    format, up to the FP32 collision arithmetic (delta) before the rounding.
    Loose entries (iolet links, and values copied from an iolet site): the
    solver computes boundary values in FP32 from its rounded stored state
    and collides with them unrounded, while the state handed to the oracle
    carries them rounded.  Each such input is off by at most half an ulp of
    the site's largest value; through the moments (d u / d s'_j = (c_j - u)/rho,
    sum |c_j| < 24) and the equilibrium's sensitivity (w_i rho |d feq/d u|
    < 0.3, and < 7 w_i per unit of input in the collision) that is below 16
    such half-ulps on the result."""
    s = hemegb.Solver(lat, tau=tau, precision=prec, scheme=scheme, wide_offsets=wide)
    bc(s)
    s.init_equilibrium()
    s.step(warm)
    o = oracle.Oracle(lat, tau=tau)
    bc(o)
    n = lat.n
    src = lat.src
    iolet_site = (src <= -2).any(axis=0)
    y = np.where(src >= 0, src, np.arange(n)[None, :])  # site whose s'(t) f_i(x) copies
    loose = np.empty((19, n), bool)
    loose[0] = iolet_site
    loose[1:] = iolet_site[y] | (src <= -2)
    assert loose.mean() < 0.05
    delta = 5e-8
    h_prev, t_prev = s.state()
    for _ in range(checks):
        s.step(1)
        h_next, _ = s.state()
        o.set_state((_stored_to_f64(h_prev, prec) + w[:, None]).T, t_prev)
        o.step(1)
        ref = o.state().T - w[:, None]
        got = _stored_to_f64(h_next, prec)
        bound = _half_ulp(np.abs(ref) + delta, prec) + delta
        site_max = np.abs(ref).max(axis=0)
        mag = np.maximum(site_max[None, :], np.concatenate([site_max[None, :], site_max[y]]))
        bound = np.where(loose, bound + 16 * _half_ulp(mag, prec), bound)
        excess = np.abs(got - ref) - bound
        k = np.unravel_index(excess.argmax(), excess.shape)
        assert excess.max() <= 0.0, f"t={t_prev}: worst excess {excess.max():.3e} at {k} (loose={loose[k]})"
        tight = ~loose
        print(f"{prec}/{scheme} t={t_prev}: max |err|/half-ulp on tight entries "
              f"{(np.abs(got - ref)[tight] / _half_ulp(np.abs(ref[tight]) + delta, prec)).max():.3f}, "
              f"loose entries {loose.mean():.2%}")
        h_prev, t_prev = h_next, t_prev + 1
    return o


@pytest.mark.parametrize("wide", [False, True], ids=["off32", "off64"])
@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_16bit_one_step_within_storage_rounding(d3q19, prec, scheme, wide):
    """Ragged tree of many 256-site blocks (pulsatile inlet, 4 pressure outlets)."""
    _, w = d3q19
    lat = geo.tree(2, 2202, target_sites=50_000, length_ratio=5.0)
    assert lat.n % 256

    def bc(x):
        x.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 200.0})
        for k in range(1, len(lat.iolets)):
            x.set_pressure(k, 1.0)
    _one_step_within_rounding(lat, 0.55, bc, prec, scheme, w, wide=wide)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_16bit_two_site_even_step_within_storage_rounding(d3q19, pipe, prec):
    """Even n (the 12,352-site pipe): the AA even step takes two sites per
    thread and runs their collisions in paired FP32 instructions; both AA
    parities stay within storage rounding of the oracle's step."""
    _, w = d3q19
    assert pipe.n % 2 == 0 and pipe.n % 256

    def bc(x):
        x.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 200.0})
        x.set_pressure(1, 1.0)
    _one_step_within_rounding(pipe, 0.55, bc, prec, "aa", w)


def test_invalid_arguments(pipe):
    s = hemegb.Solver(pipe, tau=0.8)
    with pytest.raises(hemegb.HlbError):
        s.set_tau(0.5)
    with pytest.raises(hemegb.HlbError):
        s.set_pressure(0, 1.0)              # iolet 0 is a velocity iolet
    with pytest.raises(hemegb.HlbError):
        s.set_velocity(0, [1.0, 2.0], 0.01)  # one group only
    with pytest.raises(hemegb.HlbError):
        s.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.01, "rel": 0.5, "period": 0.0})
    s.step(0)
    assert s.t == 0


@pytest.fixture(scope="module")
def tree20m():
    return geo.tree(6, 2202, target_sites=20_000_000, length_ratio=5.0)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_full_size_tree_one_step_vs_oracle(d3q19, scheme, tree20m):
    """Seeded 20M-site depth-6 tree (the benchmark workload), FP32 solver in
    the benchmark's launch configuration: after 5 pulsatile steps, each of the
    next two steps is compared with the oracle's step from the same state, at
    every site (for AA: the odd and the even kernel, each with its iolet
    fix-up); mass budget checked at full size."""
    _, w = d3q19
    lat = tree20m
    assert abs(lat.n - 20_000_000) < 0.02 * 20_000_000
    wave = {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 2000.0}
    s = hemegb.Solver(lat, tau=0.55, precision="fp32", scheme=scheme)
    s.set_velocity(0, [1.0], wave)
    for k in range(1, len(lat.iolets)):
        s.set_pressure(k, 1.0)
    s.init_equilibrium()
    s.step(5)
    m_prev, _ = s.reduce()
    f_prev, t_prev = s.state()
    o = oracle.Oracle(lat, tau=0.55, threads=os.cpu_count() or 1)
    o.set_velocity(0, [1.0], wave)
    for k in range(1, len(lat.iolets)):
        o.set_pressure(k, 1.0)
    for _ in range(2):
        s.step(1)
        m, fl = s.reduce()
        assert abs((m - m_prev) - fl.sum()) < 1e-9 * m
        f, t = s.state()
        o.set_state((f_prev.astype(np.float64) + w[:, None]).T, t_prev)
        o.step(1)
        diff = np.abs(f.T.astype(np.float64) + w[None, :] - o.state())
        assert diff.max() < 2e-8, (t_prev, diff.max())
        assert abs(o.mass() - m) < 1e-9 * m
        f_prev, t_prev, m_prev = f, t, m


def test_full_size_tree_one_step_bf16_aa(d3q19, tree20m):
    """Full-size 20M-site tree with BF16 storage in the benchmark's default
    scheme: one step within storage rounding of the oracle at every site."""
    _, w = d3q19
    lat = tree20m

    def bc(x):
        x.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 2000.0})
        for k in range(1, len(lat.iolets)):
            x.set_pressure(k, 1.0)
    _one_step_within_rounding(lat, 0.55, bc, "bf16", "aa", w)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("opts", [dict(), dict(ladd_rho_one=True), dict(ghost_full_u=True),
                                  dict(wide_offsets=True)], ids=["default", "rho1", "fullu", "wide"])
def test_aa_and_ab_give_the_same_bits(precision, opts):
    """FP32 and FP64 storage: the AA pattern and pull A-B compute the same
    operations in the same order at every site, boundary values included, so
    their states agree bit for bit at every time (16-bit storage rounds the
    AA boundary values to storage, which A-B never stores)."""
    lat = geo.tree(2, 2202, target_sites=30_000, length_ratio=5.0)

    def bc(x):
        x.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.03, "rel": 0.5, "period": 40.0})
        for k in range(1, len(lat.iolets)):
            x.set_pressure(k, {"kind": "cosine", "mean": 1.0, "rel": 0.002 * k, "period": 30.0})
    out = {}
    for scheme in SCHEMES:
        s = hemegb.Solver(lat, tau=0.58, precision=precision, scheme=scheme, **opts)
        bc(s)
        s.init_equilibrium()
        got = []
        for n in (1, 36, 40):                # odd and even times
            s.step(n)
            got.append(s.state())
        out[scheme] = got
    for (fa, ta), (fb, tb) in zip(out["aa"], out["ab"]):
        assert ta == tb and fa.tobytes() == fb.tobytes()
