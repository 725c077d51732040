"""Slab decomposition and halo exchange (include/hlb_partition.h), on the CPU.

* The plan's local lattices and exchange lists are checked against the
  global lattice: the owned ranges tile the site list, every owned site keeps
  its global sources and link codes, and every exchange entry pairs the same
  global site and direction on both sides.
* Two gloo ranks run the FP64 oracle on one part each, exchanging the ghosts'
  pre-collision states through the product's HaloExchange before every step
  (the oracle streams by push, so a ghost must hold its owner's state before
  it collides); their owned states equal a serial oracle run on the whole
  lattice bit for bit (paper Section 3.1: per-domain steps with an exchange
  of the populations crossing domain edges).
* A rank that stops exchanging makes its neighbour's exchange end with
  ExchangeTimeout within the time limit instead of hanging.
"""
import os
import socket
import time

import numpy as np
import pytest

import oracle
from paper_2202_11770_gb300 import geometry as geo
from paper_2202_11770_gb300 import partition

torch = pytest.importorskip("torch")


def _tree():
    return geo.tree(2, 2202, target_sites=30_000, length_ratio=5.0)


def _bc(x, lat):
    x.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 40.0})
    for k in range(1, len(lat.iolets)):
        x.set_pressure(k, 1.0 - 0.0005 * k)


@pytest.mark.parametrize("n_parts", [1, 2, 3, 5])
def test_plan_matches_the_global_lattice(n_parts):
    lat = _tree()
    plan = partition.Plan(lat, n_parts)
    owned = []
    for p in range(n_parts):
        local, lo, hi, g = plan.local(p)
        assert (np.diff(g) > 0).all()                      # global order
        owned.append(g[lo:hi])
        assert np.array_equal(local.xyz, lat.xyz[g])
        for i in range(18):
            s_glob = lat.src[i, g[lo:hi]]
            s_loc = local.src[i, lo:hi]
            fluid = s_glob >= 0
            assert np.array_equal(g[s_loc[fluid]], s_glob[fluid])       # same sources
            assert np.array_equal(s_loc[~fluid], s_glob[~fluid])        # same wall / iolet codes
        ghost = np.r_[0:lo, hi:local.n]
        assert (local.src[:, ghost] >= -1).all()           # ghosts carry no iolet link
    assert np.array_equal(np.concatenate(owned), np.arange(lat.n))
    locals_ = [plan.local(p) for p in range(n_parts)]
    needed = 0
    for p in range(n_parts):
        _, lo, hi, g = locals_[p]
        gp = g[lo:hi]
        needed += int(((lat.src[:, gp] >= 0) & ((lat.src[:, gp] < gp[0]) | (lat.src[:, gp] > gp[-1]))).sum())
        for q in range(n_parts):
            if q == p:
                continue
            a, b = plan.halo(q, p)
            mq, mp_ = locals_[q][0].n, locals_[p][0].n
            assert np.array_equal(a // mq, b // mp_)                             # same direction
            assert np.array_equal(locals_[q][3][a % mq], locals_[p][3][b % mp_])  # same global site
            qlo, qhi = locals_[q][1], locals_[q][2]
            assert ((a % mq >= qlo) & (a % mq < qhi)).all()                      # sent from owned sites
            sa, sb = plan.ghosts(q, p)
            assert np.array_equal(locals_[q][3][sa], locals_[p][3][sb])
    assert needed == sum(plan.halo(q, p)[0].size for p in range(n_parts) for q in range(n_parts) if q != p)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_run(rank, world, port, steps, stop_after, timeout, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lat = _tree()
    plan = partition.Plan(lat, world)
    local, lo, hi, g = plan.local(rank)
    o = oracle.Oracle(local, tau=0.6)
    _bc(o, local)
    o.init_equilibrium()
    hx = partition.HaloExchange(plan, rank, dist, kind="ghosts", timeout=timeout)
    status, t0 = "ok", time.monotonic()
    try:
        for step in range(steps):
            if rank == 1 and step == stop_after:
                break                          # this rank stops exchanging
            f = o.state()
            hx.exchange(lambda q, idx: torch.from_numpy(np.ascontiguousarray(f[idx])),
                        lambda q, idx, buf: f.__setitem__(idx, buf.numpy()),
                        lambda q, k: torch.empty((k, 19), dtype=torch.float64))
            o.set_state(f, o.t)
            o.step(1)
    except partition.ExchangeTimeout:
        status = "timeout"
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), f=o.state()[lo:hi], g=g[lo:hi], flux=o.flux(),
             status=status, elapsed=time.monotonic() - t0)
    if rank == 1 and stop_after < steps:
        time.sleep(timeout + 3)                # stay alive: the neighbour must time out, not see a reset
    if status == "ok":
        dist.destroy_process_group()


def _spawn(steps, stop_after, timeout, tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_run, args=(2, _free_port(), steps, stop_after, timeout, str(tmp_path)), nprocs=2,
                       join=True, start_method="spawn")
    return [dict(np.load(tmp_path / f"rank{r}.npz")) for r in range(2)]


def test_two_gloo_ranks_match_the_serial_oracle(tmp_path):
    steps = 30
    res = _spawn(steps, steps, 60.0, tmp_path)
    assert all(str(r["status"]) == "ok" for r in res)
    lat = _tree()
    o = oracle.Oracle(lat, tau=0.6)
    _bc(o, lat)
    o.init_equilibrium()
    o.step(steps)
    ref = o.state()
    got = np.empty_like(ref)
    for r in res:
        got[r["g"]] = r["f"]
    assert got.tobytes() == ref.tobytes()
    assert np.allclose(res[0]["flux"] + res[1]["flux"], o.flux(), rtol=1e-12, atol=1e-16)


def test_stopped_neighbour_times_out(tmp_path):
    res = _spawn(steps=10, stop_after=3, timeout=3.0, tmp_path=tmp_path)
    assert str(res[0]["status"]) == "timeout"
    assert float(res[0]["elapsed"]) < 3.0 + 10.0
