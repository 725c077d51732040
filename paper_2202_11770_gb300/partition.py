"""Domain decomposition and halo exchange (``include/hlb_partition.h``).

The paper runs one MPI rank per GPU over a split lattice and exchanges, every
step, the populations that stream across domain edges (arXiv 2202.11770,
Section 3.1; Section 3.2.2 for the GPU's scatter of received populations).
Here:

* :class:`Plan` wraps the library's slab decomposition: each part is a local
  lattice of its own ("owned") sites plus ghost copies of the remote sites
  they pull from, with the exchange lists between parts.
* :class:`HaloExchange` is the exchange protocol of one part: for every
  neighbouring part, gather what it needs (``pack``), send it, receive what
  this part needs, scatter it (``unpack``).  The transport is either a
  direct hand-over between parts in one process, or point-to-point messages
  over ``torch.distributed`` (NCCL with device buffers; gloo through host
  buffers), with a time limit on every wait.
* :class:`PartitionedSolver` runs all parts of a plan on one GPU in one
  process: a pull A-B step of every part, then the exchange of the
  post-collision halo values, device to device.  Its owned states are
  bit-identical to the undivided solver's.

Argument marshalling only: the decomposition runs in the library's C++ code
and the pack / unpack in its kernels.
"""
from __future__ import annotations

import ctypes as C
import time
from datetime import timedelta

import numpy as np

from . import geometry, hemegb

_P = C.c_void_p
_I64P = C.POINTER(C.c_int64)
_PROTOS = {
    "hlb_part_create": (C.c_int, [C.POINTER(hemegb.hlb_lattice), C.c_int32, C.POINTER(_P)]),
    "hlb_part_destroy": (C.c_int, [_P]),
    "hlb_part_count": (C.c_int32, [_P]),
    "hlb_part_local": (C.c_int, [_P, C.c_int32, C.POINTER(hemegb.hlb_lattice), _I64P, _I64P,
                                 C.POINTER(_I64P)]),
    "hlb_part_halo": (C.c_int, [_P, C.c_int32, C.c_int32, _I64P, C.POINTER(_I64P), C.POINTER(_I64P)]),
    "hlb_part_ghosts": (C.c_int, [_P, C.c_int32, C.c_int32, _I64P, C.POINTER(_I64P), C.POINTER(_I64P)]),
    "hlb_halo_pack": (C.c_int, [_P, _P, C.c_int64, _P]),
    "hlb_halo_unpack": (C.c_int, [_P, _P, C.c_int64, _P]),
    "hlb_set_owned_range": (C.c_int, [_P, C.c_int64, C.c_int64]),
    "hlb_step_range": (C.c_int, [_P, C.c_int64, C.c_int64, C.c_int32, C.c_int32]),
}
_bound = False


def library():
    global _bound
    lib = hemegb.library()
    if not _bound:
        for name, (res, args) in _PROTOS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _bound = True
    return lib


def exported_symbols():
    return sorted(_PROTOS)


def _check(rc):
    if rc != hemegb.HLB_OK:
        raise hemegb.HlbError(rc, library().hlb_last_error().decode())


def _array(ptr, n, dtype):
    out = np.empty(n, dtype=dtype)
    if n:
        C.memmove(out.ctypes.data, ptr, out.nbytes)
    return out


class Plan:
    """Slab decomposition of ``lattice`` into ``n_parts`` parts of equal site
    counts (contiguous ranges of the (z, y, x)-ordered site list)."""

    def __init__(self, lattice, n_parts: int):
        lib = library()
        self._keep = [np.ascontiguousarray(lattice.xyz, np.int32), np.ascontiguousarray(lattice.src, np.int32),
                      np.ascontiguousarray(lattice.wall_normal, np.float32),
                      np.ascontiguousarray(lattice.amp_group, np.int32)]
        xyz, src, nrm, grp = self._keep
        ios = (hemegb.hlb_iolet * max(1, len(lattice.iolets)))()
        for k, io in enumerate(lattice.iolets):
            ios[k].kind = int(io.kind)
            ios[k].centre = tuple(float(v) for v in io.centre)
            ios[k].normal = tuple(float(v) for v in io.normal)
            ios[k].radius = float(io.radius)
            ios[k].n_groups = int(io.n_groups)
        lat = hemegb.hlb_lattice(n_sites=lattice.n, xyz=xyz.ctypes.data_as(C.POINTER(C.c_int32)),
                                 src=src.ctypes.data_as(C.POINTER(C.c_int32)),
                                 wall_normal=nrm.ctypes.data_as(C.POINTER(C.c_float)),
                                 amp_group=grp.ctypes.data_as(C.POINTER(C.c_int32)),
                                 n_iolets=len(lattice.iolets), iolets=ios)
        h = _P()
        _check(lib.hlb_part_create(C.byref(lat), int(n_parts), C.byref(h)))
        self._h = h
        self._lib = lib
        self.n = lattice.n
        self.n_parts = int(n_parts)
        self.iolets = list(lattice.iolets)
        self._keep = None  # the plan copied what it needs

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.hlb_part_destroy(h)
            self._h = None

    def local(self, p: int):
        """(local Lattice, owned_lo, owned_hi, global index of each local site)."""
        lat = hemegb.hlb_lattice()
        lo, hi = C.c_int64(), C.c_int64()
        glob = _I64P()
        _check(self._lib.hlb_part_local(self._h, int(p), C.byref(lat), C.byref(lo), C.byref(hi), C.byref(glob)))
        m = int(lat.n_sites)
        xyz = _array(lat.xyz, 3 * m, np.int32).reshape(m, 3)
        src = _array(lat.src, 18 * m, np.int32).reshape(18, m)
        nrm = _array(lat.wall_normal, 3 * m, np.float32).reshape(3, m)
        grp = _array(lat.amp_group, m, np.int32)
        g = _array(glob, m, np.int64)
        local = geometry.from_arrays(xyz, src, iolets=self.iolets, wall_normal=nrm, amp_group=grp)
        return local, int(lo.value), int(hi.value), g

    def _pairs(self, fn, q, p):
        n = C.c_int64()
        a, b = _I64P(), _I64P()
        _check(fn(self._h, int(q), int(p), C.byref(n), C.byref(a), C.byref(b)))
        k = int(n.value)
        return _array(a, k, np.int64), _array(b, k, np.int64)

    def halo(self, q: int, p: int):
        """(slots of q's population array, matching slots of p's): the
        post-collision values p's owned sites pull from q."""
        return self._pairs(self._lib.hlb_part_halo, q, p)

    def ghosts(self, q: int, p: int):
        """(local sites of q, matching ghost sites of p)."""
        return self._pairs(self._lib.hlb_part_ghosts, q, p)

    def neighbours(self, p: int):
        """Parts that exchange with part p (either direction)."""
        out = []
        for q in range(self.n_parts):
            if q != p and (self.halo(q, p)[0].size or self.halo(p, q)[0].size):
                out.append(q)
        return out


class ExchangeTimeout(RuntimeError):
    """A neighbour's message did not arrive within the time limit."""


class HaloExchange:
    """Exchange protocol of part ``part`` of ``plan`` over ``torch.distributed``
    (one part per rank; rank r owns part r).

    ``exchange(pack, unpack)`` gathers, for every neighbour q, the values q
    needs (``pack(q, idx)`` with this part's index list, returning a tensor),
    sends it to q, receives q's values for this part and hands them to
    ``unpack(q, idx, tensor)`` with this part's index list.  ``kind`` picks the
    lists: "halo" (post-collision population slots, pull A-B solvers) or
    "ghosts" (whole sites, solvers that exchange pre-collision states).  All
    sends and receives of one exchange are posted together; every wait gives
    up after ``timeout`` seconds with :class:`ExchangeTimeout`.
    """

    def __init__(self, plan: Plan, part: int, dist, kind: str = "halo", timeout: float = 30.0):
        self.plan, self.part, self.dist, self.kind, self.timeout = plan, int(part), dist, kind, float(timeout)
        lists = plan.halo if kind == "halo" else plan.ghosts
        self.peers = plan.neighbours(self.part)
        self.send_idx = {q: lists(self.part, q)[0] for q in self.peers}   # my slots q pulls
        self.recv_idx = {q: lists(q, self.part)[1] for q in self.peers}   # my slots filled by q

    def exchange(self, pack, unpack, recv_like):
        """recv_like(q, n): an empty tensor for n incoming values from q."""
        ops, recv = [], {}
        for q in self.peers:
            recv[q] = recv_like(q, self.recv_idx[q].size)
            ops.append(self.dist.irecv(recv[q], src=q))
        for q in self.peers:
            buf = pack(q, self.send_idx[q])
            ops.append(self.dist.isend(buf, dst=q))
        deadline = time.monotonic() + self.timeout
        for op in ops:
            left = deadline - time.monotonic()
            try:
                ok = op.wait(timeout=timedelta(seconds=max(left, 0.001)))
            except RuntimeError as e:
                raise ExchangeTimeout(f"part {self.part}: halo exchange did not complete: {e}") from e
            if ok is False:
                raise ExchangeTimeout(f"part {self.part}: halo exchange did not complete in {self.timeout} s")
        for q in self.peers:
            unpack(q, self.recv_idx[q], recv[q])


def _runs(tiles):
    """Sorted tile numbers -> [(first, count)] of consecutive runs."""
    out = []
    for t in tiles:
        if out and out[-1][0] + out[-1][1] == t:
            out[-1][1] += 1
        else:
            out.append([int(t), 1])
    return [tuple(r) for r in out]


class PartitionedSolver:
    """All parts of an ``n_parts`` slab decomposition on the current GPU, one
    process: every step runs a pull A-B step of each part, then copies the
    post-collision halo values from their owners into the ghosts, device to
    device (hlb_halo_pack / hlb_halo_unpack).  The owned states, and so the
    macroscopic fields, mass and iolet fluxes, equal the undivided solver's
    bit for bit.

    With ``overlap`` (the paper's edge-first order, Section 3.2.3), a step
    first runs each part's edge tiles (the 256-site tiles holding the sites
    whose values other parts pull, or ghosts, and the iolet sites), then packs
    and unpacks the halo on a second stream while the interior tiles run on
    the solver stream; the next step waits for both."""

    def __init__(self, lattice, n_parts: int, tau=1.0, precision="fp32", **kw):
        import torch
        self._torch = torch
        lib = library()
        self._lib = lib
        self.plan = Plan(lattice, n_parts)
        self.n = lattice.n
        self.n_parts = int(n_parts)
        self.iolets = list(lattice.iolets)
        self.parts, self.owned, self.glob = [], [], []
        for p in range(self.n_parts):
            local, lo, hi, g = self.plan.local(p)
            s = hemegb.Solver(local, tau=tau, precision=precision, scheme="ab", **kw)
            _check(lib.hlb_set_owned_range(s.handle, lo, hi))
            self.parts.append(s)
            self.owned.append((lo, hi))
            self.glob.append(g)
        self.precision = self.parts[0].precision
        elem = {hemegb.HLB_FP32: torch.float32, hemegb.HLB_FP64: torch.float64, hemegb.HLB_BF16: torch.bfloat16,
                hemegb.HLB_FP16: torch.float16}[self.precision]
        self._links = []  # (q, p, src slots, dst slots, buffer) on the device
        send_sites = [set() for _ in range(self.n_parts)]
        for p in range(self.n_parts):
            for q in range(self.n_parts):
                if q == p:
                    continue
                a, b = self.plan.halo(q, p)
                if a.size:
                    self._links.append((q, p, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(),
                                        torch.empty(a.size, dtype=elem, device="cuda")))
                    send_sites[q].update((a % self.parts[q].n).tolist())
        # tile runs of each part: edge (holding sites others pull, or ghosts,
        # whose slots the exchange writes and the step must not overwrite
        # after it) and interior
        self._edge, self._interior = [], []
        for p, s in enumerate(self.parts):
            tiles = (s.n + 255) // 256
            lo, hi = self.owned[p]
            ghost_tiles = set(range(0, (lo + 255) // 256)) | set(range(hi // 256, tiles))
            edge = sorted({x // 256 for x in send_sites[p]} | ghost_tiles)
            eset = set(edge)
            self._edge.append(_runs(edge))
            self._interior.append(_runs([t for t in range(tiles) if t not in eset]))
        self._side = torch.cuda.Stream()
        self._fresh = True   # the next step is the first after init / set_state (a plain step)

    # ---- parameters, forwarded to every part ----
    def set_tau(self, tau):
        for s in self.parts:
            s.set_tau(tau)

    def set_velocity(self, k, amps, wave):
        for s in self.parts:
            s.set_velocity(k, amps, wave)

    def set_pressure(self, k, wave):
        for s in self.parts:
            s.set_pressure(k, wave)

    def init_equilibrium(self, rho0=1.0, u0=None):
        for p, s in enumerate(self.parts):
            s.init_equilibrium(rho0, None if u0 is None else np.ascontiguousarray(np.asarray(u0)[:, self.glob[p]]))
        self._fresh = True

    # ---- stepping ----
    def exchange(self):
        for q, p, a, b, buf in self._links:
            _check(self._lib.hlb_halo_pack(self.parts[q].handle, _P(a.data_ptr()), a.numel(), _P(buf.data_ptr())))
            _check(self._lib.hlb_halo_unpack(self.parts[p].handle, _P(b.data_ptr()), b.numel(), _P(buf.data_ptr())))

    def step(self, n=1, overlap=False):
        for _ in range(int(n)):
            if overlap and not self._fresh:
                self._step_overlapped()
            else:
                for s in self.parts:
                    s.step(1)
                self.exchange()
            self._fresh = False

    def _step_overlapped(self):
        torch, lib = self._torch, self._lib
        main = self.parts[0].stream
        for p, s in enumerate(self.parts):
            for k, (a, cnt) in enumerate(self._edge[p]):
                last = k == len(self._edge[p]) - 1 and not self._interior[p]
                _check(lib.hlb_step_range(s.handle, a, cnt, int(k == 0), int(last)))
            if not self._edge[p] and not self._interior[p]:
                raise RuntimeError("empty part")
        edges_done = torch.cuda.Event()
        edges_done.record(main)
        self._side.wait_event(edges_done)
        for s in self.parts:
            _check(lib.hlb_set_stream(s.handle, _P(self._side.cuda_stream)))
        self.exchange()
        for s in self.parts:
            _check(lib.hlb_set_stream(s.handle, _P(main.cuda_stream)))
        halo_done = torch.cuda.Event()
        halo_done.record(self._side)
        for p, s in enumerate(self.parts):
            runs = self._interior[p]
            for k, (a, cnt) in enumerate(runs):
                _check(lib.hlb_step_range(s.handle, a, cnt, int(not self._edge[p] and k == 0),
                                          int(k == len(runs) - 1)))
        main.wait_event(halo_done)

    @property
    def t(self):
        return self.parts[0].t

    # ---- read-back of the owned sites, in global order ----
    def state(self):
        out = None
        for p, s in enumerate(self.parts):
            f, t = s.state()
            lo, hi = self.owned[p]
            if out is None:
                out = np.empty((19, self.n), dtype=f.dtype)
            out[:, self.glob[p][lo:hi]] = f[:, lo:hi]
        return out, t

    def macros(self):
        rho = np.empty(self.n, np.float32)
        u = np.empty((self.n, 3), np.float32)
        wss = np.empty(self.n, np.float32)
        for p, s in enumerate(self.parts):
            r, v, w = s.macros()
            lo, hi = self.owned[p]
            idx = self.glob[p][lo:hi]
            rho[idx], u[idx], wss[idx] = r[lo:hi], v[lo:hi], w[lo:hi]
        return rho, u, wss

    def reduce(self):
        """(mass, per-iolet flux) summed over the parts' owned sites."""
        mass, flux = 0.0, np.zeros(len(self.iolets))
        for s in self.parts:
            m, fl = s.reduce()
            mass += m
            flux += fl
        return mass, flux
