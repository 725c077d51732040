"""Benchmark: fluid-site MLUPS and HBM GB/s of the fused D3Q19 step on GB300.

Workload (one GPU): the seeded depth-6 bifurcating vessel tree, ~20M fluid
sites (seed 2202, Murray radii, 30-70 degree bifurcations, 64 pressure
outlets), tau = 0.55, pulsatile inlet u(t) = 0.02 (1 + 0.5 cos(2 pi t/2000))
with a parabolic cross-section weight, rho = 1 at every outlet.  Inputs are
synthetic and seeded; the paper's patient geometries are not available.

One benchmark step = one LB time step over the whole lattice: one launch of
the fused stream-collide-boundary kernel (pull A-B: k_step, iolet sites
included), or for the AA pattern k_aa_odd / k_aa_even (alternating) plus
the k_aa_fix pass over the iolet sites (0.3 % of the sites).  ``value`` is MLUPS (Eq. 9 of arXiv
2202.11770) with the lattice resident in HBM, timed with one CUDA event pair
around all timed steps; the state (~3.4 GB touched per step) is far larger
than L2, so no flush is needed between steps.

``--gpus N`` (under torchrun) runs N independent replicas, one per GPU
(the single-GPU solver does not shard); ``value`` sums the ranks' site
updates over the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle (test infrastructure, plain C,
sites split over all host cores) for the same --warmup and --steps, on the
same lattice, or on a smaller tree of the same generator when the full one
would not finish within --ref-budget seconds.  The default run also reports the oracle at one thread,
and checks every storage form's velocity and wall shear stress against the
oracle on a 1M-site tree after 1,000 steps (``precision_vs_oracle``).
"""
from __future__ import annotations

import argparse
import ctypes as C
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "fluid-site MLUPS and HBM GB/s (% of peak), FP32 vs 16-bit store; adjoint/fwd"
WORKLOAD = "seeded depth-6 vessel tree, 20M fluid sites, D3Q19 LBGK tau=0.55, pulsatile Ladd inlet, 64 pressure outlets"


def workload_name(n, tau):
    return (f"seeded depth-6 vessel tree, {n / 1e6:.0f}M fluid sites, D3Q19 LBGK tau={tau:g}, "
            "pulsatile Ladd inlet, 64 pressure outlets")

# Index bytes per site: the int32 streaming-index table (18 x 4 B), or its
# compact form (18 x 2 B of offsets plus 20 int32 tile bases per 256 sites).
INDEX_BYTES = {False: 18 * 4, True: 18 * 2 + 20 * 4 / 256}


# Algorithmic bytes per site update (storage element size e): 19 populations
# read + 19 written, plus the index table when the kernel gathers through
# it.  Pull A-B gathers every step; the AA pattern only on odd steps.
# Boundary-link records are O(boundary sites), not counted.
def bytes_per_site(elem: int, kernel: str = "ab", compact: bool = False) -> float:
    local = 19 * elem * 2
    idx = INDEX_BYTES[bool(compact)]
    if kernel in ("ab", "aa_odd"):
        return local + idx
    if kernel == "aa_even":
        return local
    if kernel == "aa":
        return local + idx / 2
    raise ValueError(kernel)


ELEM = {"fp32": 4, "bf16": 2, "fp16": 2, "fp64": 8}
CTYPE = {"fp32": "float", "bf16": "__nv_bfloat16", "fp16": "__half", "fp64": "double"}

# DRAM traffic per site update from one ncu capture (profiles/), valid only
# while the kernel sources hash to the recorded value.
TRAFFIC_FILES = ["paper_2202_11770_gb300/csrc/hlb_common.cuh", "paper_2202_11770_gb300/csrc/hlb_forward.cu"]
TRAFFIC = {"sha": "67b390820d1752e1",
           # ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch (mean of two), 20,000,864-site
           # tree, kernels on the compact index table with the L2 prefetch
           "index": "compact",
           "bytes_per_site": {"k_aa_odd": ((2265953280 + 1483422208) + (2266168576 + 1480823808)) / 2 / 20000864,
                              "k_step2": ((2373115392 + 1484953600) + (2366690304 + 1480613632)) / 2 / 20000864}}


def kernel_sha() -> str:
    """Hash of the kernel sources with comments and blank space removed, so
    that only a change of the code itself invalidates the recorded traffic."""
    h = hashlib.sha256()
    for f in TRAFFIC_FILES:
        text = (ROOT / f).read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in Path(self.path).read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, flags in rows for k, v in enumerate(flags) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
def tree_lattice(target):
    from paper_2202_11770_gb300 import workloads
    return workloads.tree_lattice(target)


def set_bc(x, lat):
    from paper_2202_11770_gb300 import workloads
    workloads.apply_tree_bc(x, lat)


def aggregate_ranks(ms_local, updates_local, dist=None, device="cpu"):
    """Whole-job timing over replicas: the slowest rank's time and the sum of
    all ranks' site updates (weak scaling; no data-path collective)."""
    if dist is None:
        return ms_local, updates_local
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(updates_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def time_form(lat, precision, scheme, steps, warmup, torch, dist=None, tau=0.55, wide=False, full_index=False):
    """Time `steps` steps on the solver stream, twice after `warmup` steps.

    The first pass has one CUDA event on each side of all steps (an event
    recorded between steps costs ~5 us a step); it gives the total time.  The
    second pass records an event after every step; it gives the duration of
    each step kernel (AA: odd and even steps) for the roofline.  Returns
    (total_ms, per-step durations in ms, solver time before the first
    instrumented step, whether the kernels read the compact index table)."""
    from paper_2202_11770_gb300 import hemegb
    s = hemegb.Solver(lat, tau=tau, precision=precision, scheme=scheme, wide_offsets=wide, full_index=full_index)
    compact = s.compact_index
    set_bc(s, lat)
    s.init_equilibrium()
    s.step(warmup)
    stream = s.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    total = e0.elapsed_time(e1)
    t_first = s.t
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for k in range(steps):
        s.step(1)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    durs = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    mass, _ = s.reduce()
    assert math.isfinite(mass)
    del s
    torch.cuda.empty_cache()
    return total, durs, t_first, compact


def kernel_names(n, compact=True, wide=False):
    """Names of the step kernels the library launches (pull A-B, AA odd step):
    the pull step takes two sites a thread (k_step2) on the compact table
    with 32-bit offsets when the site count is even."""
    return ("k_step2" if compact and not wide and n % 2 == 0 else "k_step", "k_aa_odd")


def form_stats(lat, precision, scheme, total, durs, t_first, steps, peak, compact):
    """MLUPS, algorithmic GB/s and per-kernel rooflines of one timed form
    (CUDA events around every step: each step is one kernel launch)."""
    n = lat.n
    k_ab, k_odd = kernel_names(n, compact)
    e = ELEM[precision]
    out = {"scheme": scheme, "mlups": n * steps / (total * 1e-3) / 1e6, "ms_per_step": total / steps,
           "index": "compact" if compact else "int32"}
    if scheme == "ab":
        b = bytes_per_site(e, "ab", compact)
        gbs = b * n / (total / steps * 1e-3) / 1e9
        out.update(gbs=gbs, frac_of_measured_peak=gbs / peak, bytes_per_site=b,
                   kernels={k_ab: {"launches": steps, "mean_us": total / steps * 1e3, "gbs": gbs,
                                   "frac": gbs / peak, "bytes_per_site": b}})
    else:
        odd = [d for k, d in enumerate(durs) if (t_first + k) % 2 == 1]
        even = [d for k, d in enumerate(durs) if (t_first + k) % 2 == 0]
        b = bytes_per_site(e, "aa", compact)
        gbs = b * n / (total / steps * 1e-3) / 1e9
        kern = {}
        for name, ds, kb in ((k_odd, odd, bytes_per_site(e, "aa_odd", compact)),
                             ("k_aa_even", even, bytes_per_site(e, "aa_even"))):
            m = sum(ds) / len(ds)
            g = kb * n / (m * 1e-3) / 1e9
            kern[name] = {"launches": len(ds), "mean_us": m * 1e3, "gbs": g, "frac": g / peak, "bytes_per_site": kb}
        out.update(gbs=gbs, frac_of_measured_peak=gbs / peak, bytes_per_site=b, kernels=kern)
    return out


def e2e_job(lat, steps, torch):
    """Whole job through the public API from host buffers: create (lattice
    tables uploaded from pinned host memory), init, `steps` steps with the
    density and velocity read back to host every 100 steps (the paper's
    property-cache interval) and a final FP64 reduction."""
    from paper_2202_11770_gb300 import hemegb
    from paper_2202_11770_gb300.geometry import Lattice
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    lat_p = Lattice(xyz=pin(lat.xyz), src=pin(lat.src), type=lat.type, wall_normal=pin(lat.wall_normal),
                    amp_group=pin(lat.amp_group), iolets=lat.iolets, info=lat.info)
    n = lat.n
    rho_h = torch.empty(n, dtype=torch.float32).pin_memory().numpy()
    u_h = torch.empty(3 * n, dtype=torch.float32).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = hemegb.Solver(lat_p, tau=0.55, precision="fp32")
    set_bc(s, lat_p)
    s.init_equilibrium()
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    reads = 0
    for k in range(steps // 100):
        s.step(100)
        hemegb.hlb_read_macros(s.handle, rho_h.ctypes.data, u_h.ctypes.data, None, hemegb.HLB_HOST)
        reads += 1
    s.step(steps % 100)
    mass, flux = s.reduce()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h2d = lat.xyz.nbytes + lat.src.nbytes + lat.wall_normal.nbytes + lat.amp_group.nbytes
    h2d_step = h2d / steps + 2096          # lattice upload amortised + per-launch boundary parameters
    d2h_step = reads * (rho_h.nbytes + u_h.nbytes) / steps + 8 * (1 + len(lat.iolets)) / steps
    del s
    torch.cuda.empty_cache()
    return n * steps / dt / 1e6, h2d_step, d2h_step, t_create, dt


def adjoint_ratio(steps, torch, sites=2_000_000, full_index=False, memory=True):
    """Adjoint (forward with sqrt(N) checkpoints + recompute + reverse) vs
    forward-only time over the same N steps: seeded depth-4 tree, ~2M sites,
    64 inlet amplitude groups, FP32."""
    from paper_2202_11770_gb300 import hemegb, workloads
    lat, obj = workloads.adjoint_case(target_sites=sites)
    fwd = {}
    for sch in ("ab", "aa"):
        s = hemegb.Solver(lat, tau=0.55, precision="fp32", scheme=sch, full_index=full_index)
        workloads.apply_tree_bc(s, lat)
        s.init_equilibrium()
        s.step(10)
        s.init_equilibrium()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
        torch.cuda.synchronize()
        fwd[sch] = e0.elapsed_time(e1)
        del s
    s = hemegb.Solver(lat, tau=0.55, precision="fp32", scheme="auto", full_index=full_index)
    workloads.apply_tree_bc(s, lat)
    ws = s.adjoint_workspace(steps, obj.sites.size)
    s.init_equilibrium()
    s.adjoint(min(steps, 50), obj.sites, obj.target, obj.axis, workspace=ws)   # warm-up
    s.init_equilibrium()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    J, dtau, damp = s.adjoint(steps, obj.sites, obj.target, obj.axis, workspace=ws)
    e1.record(s.stream)
    torch.cuda.synchronize()
    adj = e0.elapsed_time(e1)
    K = s.adjoint_plan(steps, obj.sites.size, ws[2])[0]
    out = {"workload": "seeded depth-4 tree, 64 inlet amplitude groups, FP32", "n_sites": lat.n, "steps": steps,
           "checkpoint_interval": K, "forward_ms": fwd, "adjoint_ms": adj,
           "ratio": adj / min(fwd.values()), "ratio_vs_pull_ab": adj / fwd["ab"],
           "J": J, "dJ_dtau": dtau, "probe_sites": int(obj.sites.size),
           "adjoint_workspace_gb": ws[2] / 1e9, "index": "compact" if s.compact_index else "int32"}
    del ws
    torch.cuda.empty_cache()
    # the same run with most of the free device memory as workspace: whole
    # segments of states are kept from the forward sweep, not recomputed
    free = torch.cuda.mem_get_info()[0]
    base = hemegb.hlb_adjoint_workspace_bytes(s._h, steps, obj.sites.size)
    extra = max(0, int(0.6 * free) - base)
    _, kept, rec, used = s.adjoint_plan(steps, obj.sites.size, base + extra)
    if memory and kept > 0:
        ws = s.adjoint_workspace(steps, obj.sites.size, extra_bytes=used - base)
        s.init_equilibrium()
        torch.cuda.synchronize()
        e0.record(s.stream)
        J2, dtau2, damp2 = s.adjoint(steps, obj.sites, obj.target, obj.axis, workspace=ws)
        e1.record(s.stream)
        torch.cuda.synchronize()
        adj2 = e0.elapsed_time(e1)
        out["memory"] = {"adjoint_ms": adj2, "ratio": adj2 / min(fwd.values()), "workspace_gb": used / 1e9,
                         "kept_segments": kept, "recomputed_steps": rec,
                         "identical": bool(J2 == J and dtau2 == dtau and np.array_equal(damp2, damp))}
        del ws
    del s
    torch.cuda.empty_cache()
    return out


def precision_study(lat, checkpoints, torch):
    """Velocity and wall-shear-stress error of FP32, BF16 and FP16 storage
    against FP64 on the same lattice and boundary conditions, at the given
    step counts.  The FP64 reference is the GPU FP64 path, which matches the
    FP64 oracle to rounding in the parity tests (the oracle itself would need
    hours for this size)."""
    from paper_2202_11770_gb300 import hemegb
    solvers = {}
    for prec in ("fp64", "fp32", "bf16", "fp16"):
        s = hemegb.Solver(lat, tau=0.55, precision=prec)
        set_bc(s, lat)
        s.init_equilibrium()
        solvers[prec] = s
    out = {}
    done = 0
    for k in checkpoints:
        for s in solvers.values():
            s.step(k - done)
        done = k
        ref = solvers["fp64"].macros_device()
        wall = ~torch.isnan(ref[2])
        row = {}
        for prec in ("fp32", "bf16", "fp16"):
            r, u, w = solvers[prec].macros_device()
            row[prec] = {
                "u_rel_l2": float(torch.linalg.norm(u - ref[1]) / torch.linalg.norm(ref[1])),
                "wss_rel_l2": float(torch.linalg.norm(w[wall] - ref[2][wall]) / torch.linalg.norm(ref[2][wall])),
                "rho_max_abs": float((r - ref[0]).abs().max()),
            }
        out[str(k)] = row
    del solvers
    torch.cuda.empty_cache()
    return out


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_mlups(lat, steps, threads, tau=0.55, bc=None):
    """FP64 oracle MLUPS over `steps` full-lattice steps after one warm-up step."""
    import oracle
    o = oracle.Oracle(lat, tau=tau, threads=threads)
    if bc is None:
        set_bc(o, lat)
    else:
        bc(o)
    o.init_equilibrium()
    o.step(1)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return lat.n * steps / dt / 1e6, dt


def cpu_baseline(lat, steps_1, steps_all, pipe_steps):
    """The FP64 oracle (test infrastructure, plain C) on the host cores: the
    bench's tree at one thread and at all cores, and the 12,352-site pipe."""
    from paper_2202_11770_gb300 import geometry
    cores = host_cores()
    v1, d1 = oracle_mlups(lat, steps_1, 1)
    vn, dn = oracle_mlups(lat, steps_all, cores)
    pipe = geometry.pipe(8.0, 64)

    def pipe_bc(o):
        o.set_velocity(0, [1.0], 0.01)
        o.set_pressure(1, 1.0)
    p1, pd1 = oracle_mlups(pipe, pipe_steps, 1, tau=0.8, bc=pipe_bc)
    pn, pdn = oracle_mlups(pipe, pipe_steps, cores, tau=0.8, bc=pipe_bc)
    return {"value": vn, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": (f"{steps_all} full-lattice steps of the {lat.n}-site tree on {cores} threads ({dn:.1f} s); "
                       f"FP64 oracle, sites split over threads"),
            "single_thread": {"value": v1, "sample": f"{steps_1} steps of the same tree ({d1:.1f} s)"},
            "pipe_12352": {"threads_1": p1, f"threads_{cores}": pn, "steps": pipe_steps,
                           "seconds": [round(pd1, 2), round(pdn, 2)]}}


def split_kernels(lat, steps, torch):
    """The paper's per-site-type kernels on streams (Section 3.2.2) against
    the fused kernel, FP32 pull A-B: the fused kernel on the (z, y, x) site
    order; the fused kernel on the sites sorted by type (the order the
    per-type kernels need); one launch per type range, each on its own
    stream (hlb_step_range over the 256-site tiles of the range)."""
    from paper_2202_11770_gb300 import hemegb, partition, workloads
    lib = partition.library()
    sorted_lat, ranges = workloads.type_sorted(lat)
    out = {"types": {str(t): e - b for t, b, e in ranges}}

    def run(lattice, label, per_type=None, full_index=False):
        s = hemegb.Solver(lattice, tau=0.55, precision="fp32", scheme="ab", full_index=full_index)
        set_bc(s, lattice)
        s.init_equilibrium()
        s.step(5)
        main = s.stream
        streams = [torch.cuda.Stream() for _ in (per_type or [])]
        tiles = (lattice.n + 255) // 256
        cuts = sorted({0, tiles} | {min(tiles, b // 256) for _, b, _ in (per_type or [])})
        chunks = [(a, b - a) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for _ in range(steps):
            if per_type is None:
                s.step(1)
                continue
            start = torch.cuda.Event()
            start.record(main)
            done = []
            for k, (a, cnt) in enumerate(chunks):
                st = streams[k % len(streams)]
                st.wait_event(start)
                lib.hlb_set_stream(s.handle, C.c_void_p(st.cuda_stream))
                rc = lib.hlb_step_range(s.handle, a, cnt, int(k == 0), int(k == len(chunks) - 1))
                assert rc == 0, lib.hlb_last_error()
                ev = torch.cuda.Event()
                ev.record(st)
                done.append(ev)
            for ev in done:
                main.wait_event(ev)
            lib.hlb_set_stream(s.handle, C.c_void_p(main.cuda_stream))
        e1.record(main)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) / steps * 1e3
        out[label] = {"us_per_step": us, "index": "compact" if s.compact_index else "int32",
                      "launches_per_step": 1 if per_type is None else len(chunks)}
        del s
        torch.cuda.empty_cache()

    run(lat, "fused_zyx")
    run(lat, "fused_zyx_int32", full_index=True)
    run(sorted_lat, "fused_type_sorted")
    run(sorted_lat, "per_type_streams", per_type=ranges)
    return out


def precision_vs_oracle(sites, steps, torch, forms=(("fp32", "ab"), ("fp32", "aa"), ("bf16", "ab"), ("bf16", "aa"),
                                                     ("fp16", "ab"), ("fp16", "aa"))):
    """Velocity and wall-shear-stress error of each storage form against the
    FP64 oracle: the seeded depth-6 tree at `sites` sites with the bench's
    boundary conditions (pulsatile Ladd inlet, rho = 1 outlets, tau 0.55),
    `steps` steps from rest, relative L2 over all sites (WSS over wall sites)."""
    import oracle
    from paper_2202_11770_gb300 import hemegb
    lat = tree_lattice(sites)
    cores = host_cores()
    o = oracle.Oracle(lat, tau=0.55, threads=cores)
    set_bc(o, lat)
    o.init_equilibrium()
    t0 = time.perf_counter()
    o.step(steps)
    t_oracle = time.perf_counter() - t0
    _, u_o, wss_o = o.macros(lat.wall_normal)
    del o
    wall = ~np.isnan(wss_o)
    out = {}
    for prec, sch in forms:
        s = hemegb.Solver(lat, tau=0.55, precision=prec, scheme=sch)
        set_bc(s, lat)
        s.init_equilibrium()
        s.step(steps)
        _, u, wss = s.macros()
        out[f"{prec}_{sch}"] = {
            "u_rel_l2": float(np.linalg.norm(u - u_o) / np.linalg.norm(u_o)),
            "wss_rel_l2": float(np.linalg.norm(wss[wall] - wss_o[wall]) / np.linalg.norm(wss_o[wall]))}
        del s
    torch.cuda.empty_cache()
    info = {"reference": "FP64 oracle", "workload": f"seeded depth-6 tree, {lat.n} sites, tau 0.55, pulsatile "
            "Ladd inlet, 64 pressure outlets", "steps": steps, "oracle_threads": cores,
            "oracle_s": round(t_oracle, 1)}
    return out, info


# ---------------------------------------------------------------------------
def run_reference(args):
    """The oracle arm: exactly `--warmup` W untimed and `--steps` K timed
    oracle steps, sites split over all host cores.  One full-lattice step is
    timed first (it counts as the first warm-up step); when W + K full steps
    would take longer than --ref-budget seconds, every step instead runs on a
    smaller tree from the same seeded generator, sized to fit that budget
    (the sample is named in the line)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    cores = host_cores()
    lat = tree_lattice(args.sites)
    n_full = lat.n
    w, k = max(args.warmup, 1), max(args.steps, 1)

    def oracle_on(lattice):
        o = oracle.Oracle(lattice, tau=0.55, threads=cores)
        set_bc(o, lattice)
        o.init_equilibrium()
        return o

    o = oracle_on(lat)
    t0 = time.perf_counter()
    o.step(1)
    t_full = time.perf_counter() - t0
    done = 1
    full = (w + k) * t_full <= args.ref_budget
    if not full:
        target = max(1_000_000, int(lat.n * args.ref_budget / ((w + k) * t_full)))
        del o
        lat = tree_lattice(target)
        o = oracle_on(lat)
        done = 0
    o.step(w - done)
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    v = lat.n * k / dt / 1e6
    sample = (f"{k} steps after {w} warm-up step(s) of the {lat.n}-site seeded tree"
              + ("" if full else f" (a smaller tree of the same generator: {w + k} full steps of the "
                                 f"{args.sites // 1_000_000}M-site tree would take {(w + k) * t_full:.0f} s)")
              + f", FP64 oracle on {cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": k, "warmup": w, "ms_per_step": dt / k * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(n_full, 0.55), "n_sites": n_full, "tau": 0.55},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        torch.cuda.set_device(local)
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    else:
        torch.cuda.set_device(0)
    from paper_2202_11770_gb300 import hemegb
    hemegb.library()

    lat = tree_lattice(args.sites)
    n = lat.n
    peak, peak_kind = measured_peaks()

    scheme = args.scheme
    clocks = ClockSampler(local)
    clocks.start()
    prec0 = args.precision if args.quick else "fp32"
    ms, durs, t_first, compact = time_form(lat, prec0, scheme, args.steps, args.warmup, torch, dist, tau=args.tau,
                                           wide=args.wide_offsets, full_index=args.full_index)
    clk = clocks.stop()
    ms, total_updates = aggregate_ranks(ms, n * args.steps, dist, "cuda")
    value = total_updates / (ms * 1e-3) / 1e6
    head = form_stats(lat, prec0, scheme, ms, durs, t_first, args.steps, peak, compact)
    kname = kernel_names(n, compact, args.wide_offsets)[0 if scheme == "ab" else 1]
    kst = head["kernels"][kname]
    traffic = None
    # the recorded bytes belong to the 32-bit-offset kernels (lattices below
    # ~226M sites without --wide-offsets); larger lattices run the wide form
    off32 = not args.wide_offsets and 19 * ((n + 3) // 4 * 4) <= 0xFFFFFFFF
    if (TRAFFIC["sha"] == kernel_sha() and TRAFFIC["index"] == ("compact" if compact else "int32") and off32
            and kname in TRAFFIC["bytes_per_site"]):
        traffic = TRAFFIC["bytes_per_site"][kname] * n

    forms = {f"{prec0}_{scheme}": head}
    if not args.quick:
        for prec in ("fp32", "bf16", "fp16"):
            for sch in ("ab", "aa"):
                if f"{prec}_{sch}" in forms:
                    continue
                tot, d, tf, ct = time_form(lat, prec, sch, args.steps, args.warmup, torch, dist,
                                           full_index=args.full_index)
                forms[f"{prec}_{sch}"] = form_stats(lat, prec, sch, tot, d, tf, args.steps, peak, ct)

    adjoint = None
    if not args.quick and args.adjoint_steps > 0:
        adjoint = adjoint_ratio(args.adjoint_steps, torch, full_index=args.full_index)

    e2e = None
    if not args.quick:
        v, h2d, d2h, t_create, t_all = e2e_job(lat, args.e2e_steps, torch)
        e2e = {"value": v * world, "unit": "MLUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "job": f"create + init + {args.e2e_steps} steps + host readback of rho,u every 100 steps",
               "create_s": round(t_create, 3), "total_s": round(t_all, 3)}

    precision = None
    if not args.quick and args.precision_sites > 0 and rank == 0:
        errs, info = precision_vs_oracle(args.precision_sites, args.precision_steps, torch)
        for key, e in errs.items():
            if key in forms:
                forms[key]["vs_oracle"] = e
        precision = dict(info, forms=errs)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(lat, args.cpu_steps, args.cpu_steps_all, args.cpu_pipe_steps)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16 storage, f32 math", "fp16": "f16 storage, f32 math", "fp64": "f64"}[prec0], "data": "synthetic",
            "config": {"workload": workload_name(n, args.tau), "n_sites": n, "tau": args.tau,
                       "scheme": {"ab": "pull A-B", "aa": "AA pattern"}[scheme],
                       "index": ("compact: 16-bit offsets from per-tile bases" if compact else "int32 table"),
                       "parallelism": f"replicas x{world}", "l2": f"working set {n * head['bytes_per_site'] / 1e9:.1f} GB/step >> 129 MB L2, no flush",
                       "fill": round(lat.info["fill"], 4)},
            "roofline": {"bound": "hbm", "achieved": kst["gbs"], "peak": peak, "unit": "GB/s",
                         "frac": kst["gbs"] / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": f"{kname}<{CTYPE[prec0]}>", "launches": kst["launches"], "mean_us": kst["mean_us"],
                         "timed": "CUDA events around each step" + (
                             " (odd step = k_aa_odd + the k_aa_fix pass)" if scheme == "aa" else ""),
                         "algorithmic_bytes_per_site": kst["bytes_per_site"],
                         "step_gbs": head["gbs"], "step_bytes_per_site": head["bytes_per_site"]},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            # per step: the fused kernel, plus the iolet fix-up pass for AA
            "gpu_launches": args.steps * (2 if scheme == "aa" and bool((lat.src <= -2).any()) else 1),
            "forms": forms,
            "precision_vs_oracle": precision,
            "adjoint": adjoint,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sites", type=int, default=20_000_000)
    ap.add_argument("--e2e-steps", type=int, default=2000)
    ap.add_argument("--cpu-steps", type=int, default=2, help="oracle steps of the one-thread CPU baseline")
    ap.add_argument("--cpu-steps-all", type=int, default=6, help="oracle steps of the all-cores CPU baseline")
    ap.add_argument("--cpu-pipe-steps", type=int, default=200, help="oracle steps on the 12,352-site pipe")
    ap.add_argument("--precision-sites", type=int, default=1_000_000,
                    help="tree size of the storage-precision check against the oracle (0: skip)")
    ap.add_argument("--precision-steps", type=int, default=1000)
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--adjoint-sites", type=int, default=2_000_000)
    ap.add_argument("--adjoint-only", action="store_true", help="only the adjoint/forward timing")
    ap.add_argument("--no-adjoint-memory", action="store_true",
                    help="skip the adjoint run that keeps whole segments in most of the free device memory")
    ap.add_argument("--split-kernels", action="store_true",
                    help="the paper's per-site-type kernels on streams against the fused kernel (FP32 pull A-B)")
    ap.add_argument("--precision-only", action="store_true",
                    help="only the storage forms' u and WSS error against the FP64 oracle "
                         "(--precision-sites, --precision-steps)")
    ap.add_argument("--precision-study", action="store_true",
                    help="u and WSS error of FP32/BF16/FP16 storage vs FP64 at 1k, 5k, 10k steps")
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="seconds the oracle arm may spend on its warm-up and timed steps")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--quick", action="store_true", help="one form only, no e2e (profiling runs)")
    ap.add_argument("--tau", type=float, default=0.55, help="relaxation time of the timed headline form")
    ap.add_argument("--full-index", action="store_true",
                    help="time the kernels on the int32 index table instead of its compact form")
    ap.add_argument("--wide-offsets", action="store_true",
                    help="time the large-lattice (direction-pair offset) kernels at this size")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16", "fp64"],
                    help="storage precision of the one form timed by --quick")
    ap.add_argument("--scheme", default="aa", choices=["ab", "aa"],
                    help="streaming scheme of the headline FP32 form (the solver's AUTO choice is aa)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.precision_study:
        import torch
        torch.cuda.set_device(0)
        lat = tree_lattice(args.sites)
        res = precision_study(lat, [1000, 5000, 10000], torch)
        print(json.dumps({"precision_study": res, "n_sites": lat.n, "workload": WORKLOAD,
                          "reference": "GPU FP64 storage and arithmetic (equal to the FP64 oracle to rounding "
                                       "in the parity tests)"}))
    elif args.precision_only:
        import torch
        torch.cuda.set_device(0)
        errs, info = precision_vs_oracle(args.precision_sites, args.precision_steps, torch)
        print(json.dumps({"precision_vs_oracle": dict(info, forms=errs)}))
    elif args.split_kernels:
        import torch
        torch.cuda.set_device(0)
        lat = tree_lattice(args.sites)
        print(json.dumps({"split_kernels": split_kernels(lat, args.steps, torch), "n_sites": lat.n,
                          "workload": workload_name(lat.n, 0.55)}))
    elif args.adjoint_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"adjoint": adjoint_ratio(args.adjoint_steps, torch, args.adjoint_sites,
                                                   full_index=args.full_index,
                                                   memory=not args.no_adjoint_memory)}))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
