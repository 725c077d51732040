"""ctypes binding of ``libhemegb`` (``include/hemegb.h``).

Argument marshalling only: every computation runs in the library's sm_103a
kernels.  PyTorch provides device memory (the workspaces are ``uint8``
tensors) and the CUDA stream.  The module raises ``ImportError`` when the
compiled library is absent; there is no fallback path.

Functions keep the C names (``hlb_create``, ``hlb_step``, ...);
:class:`Solver` bundles them with workspace ownership for convenience.

Method: arXiv 2202.11770, D3Q19 LBGK (Section 2.2, Eqs. 3-6), bounce-back
walls and Ladd / ghost-density iolets (Section 2.3), the GPU solver of
Section 3.2 with pull streaming over a compact site list.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libhemegb.so"

HLB_OK, HLB_ERR_ARG, HLB_ERR_WS, HLB_ERR_CUDA, HLB_ERR_STATE, HLB_ERR_DIVERGED, HLB_ERR_NOMEM = 0, -1, -2, -3, -4, -5, -6
HLB_FP32, HLB_BF16, HLB_FP16, HLB_FP64 = 0, 1, 2, 3
HLB_SCHEME_AUTO, HLB_PULL_AB, HLB_AA = 0, 1, 2
HLB_VELOCITY, HLB_PRESSURE = 0, 1
HLB_WAVE_CONST, HLB_WAVE_COSINE, HLB_WAVE_TABLE = 0, 1, 2
HLB_HOST, HLB_DEVICE = 0, 1

PRECISIONS = {"fp32": HLB_FP32, "bf16": HLB_BF16, "fp16": HLB_FP16, "fp64": HLB_FP64}
SCHEMES = {"auto": HLB_SCHEME_AUTO, "ab": HLB_PULL_AB, "aa": HLB_AA}
_ELEM = {HLB_FP32: 4, HLB_BF16: 2, HLB_FP16: 2, HLB_FP64: 8}


class HlbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hemegb error {code}: {msg}")
        self.code = code


class hlb_iolet(C.Structure):
    _fields_ = [("kind", C.c_int32), ("centre", C.c_double * 3), ("normal", C.c_double * 3),
                ("radius", C.c_double), ("n_groups", C.c_int32)]


class hlb_lattice(C.Structure):
    _fields_ = [("n_sites", C.c_int64), ("xyz", C.POINTER(C.c_int32)), ("src", C.POINTER(C.c_int32)),
                ("wall_normal", C.POINTER(C.c_float)), ("amp_group", C.POINTER(C.c_int32)),
                ("n_iolets", C.c_int32), ("iolets", C.POINTER(hlb_iolet))]


class hlb_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("scheme", C.c_int32), ("ladd_rho_one", C.c_int32),
                ("ghost_full_u", C.c_int32), ("wide_offsets", C.c_int32), ("full_index", C.c_int32)]


class hlb_waveform(C.Structure):
    _fields_ = [("kind", C.c_int32), ("mean", C.c_double), ("rel_amp", C.c_double), ("period", C.c_double),
                ("phase", C.c_double), ("n_samples", C.c_int32), ("samples", C.POINTER(C.c_double))]


class hlb_objective(C.Structure):
    _fields_ = [("n_probe", C.c_int64), ("sites", C.POINTER(C.c_int64)), ("target", C.POINTER(C.c_double)),
                ("axis", C.c_double * 3)]


_P = C.c_void_p
_PROTOS = {
    "hlb_last_error": (C.c_char_p, []),
    "hlb_version": (C.c_int, []),
    "hlb_workspace_bytes": (C.c_int, [C.POINTER(hlb_lattice), C.POINTER(hlb_options), C.POINTER(C.c_size_t)]),
    "hlb_create": (C.c_int, [C.POINTER(hlb_lattice), C.POINTER(hlb_options), _P, C.c_size_t, _P, C.POINTER(_P)]),
    "hlb_destroy": (C.c_int, [_P]),
    "hlb_set_stream": (C.c_int, [_P, _P]),
    "hlb_n_sites": (C.c_int64, [_P]),
    "hlb_n_amp_groups": (C.c_int, [_P]),
    "hlb_compact_index": (C.c_int, [_P]),
    "hlb_set_tau": (C.c_int, [_P, C.c_double]),
    "hlb_set_velocity_waveform": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_double), C.c_int32,
                                            C.POINTER(hlb_waveform)]),
    "hlb_set_pressure": (C.c_int, [_P, C.c_int32, C.POINTER(hlb_waveform)]),
    "hlb_init_equilibrium": (C.c_int, [_P, C.c_double, _P, C.c_int32]),
    "hlb_step": (C.c_int, [_P, C.c_int64]),
    "hlb_time": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "hlb_read_macros": (C.c_int, [_P, _P, _P, _P, C.c_int32]),
    "hlb_reduce": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "hlb_iolet_monitor": (C.c_int, [_P, _P, _P, _P]),
    "hlb_set_windkessel": (C.c_int, [_P, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]),
    "hlb_windkessel_state": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]),
    "hlb_get_state": (C.c_int, [_P, _P, C.c_int32, C.POINTER(C.c_int64)]),
    "hlb_set_state": (C.c_int, [_P, _P, C.c_int32, C.c_int64]),
    "hlb_adjoint_workspace_bytes": (C.c_int, [_P, C.c_int64, C.c_int64, C.POINTER(C.c_size_t)]),
    "hlb_adjoint_plan": (C.c_int, [_P, C.c_int64, C.c_int64, C.c_size_t, C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_size_t)]),
    "hlb_adjoint_run": (C.c_int, [_P, C.c_int64, C.POINTER(hlb_objective), _P, C.c_size_t,
                                  C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "hlb_mass_static": (C.c_int, [_P, C.c_int32, C.c_int64, _P, _P]),
}

_lib = None


def library():
    """Load libhemegb (raises ImportError if it has not been built)."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise ImportError(f"{_LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "(nvcc, sm_103a); there is no CPU fallback")
        lib = C.CDLL(str(_LIB_PATH))
        for name, (res, args) in _PROTOS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return sorted(_PROTOS)


def _check(rc):
    if rc != HLB_OK:
        raise HlbError(rc, library().hlb_last_error().decode())
    return rc


# ---------------------------------------------------------------------------
# thin wrappers with the C names
# ---------------------------------------------------------------------------
def hlb_workspace_bytes(lat, opt) -> int:
    out = C.c_size_t()
    _check(library().hlb_workspace_bytes(C.byref(lat), C.byref(opt), C.byref(out)))
    return out.value


def hlb_create(lat, opt, ws_ptr: int, ws_bytes: int, stream: int):
    h = _P()
    _check(library().hlb_create(C.byref(lat), C.byref(opt), _P(ws_ptr), ws_bytes, _P(stream), C.byref(h)))
    return h


def hlb_destroy(h):
    _check(library().hlb_destroy(h))


def hlb_set_tau(h, tau):
    _check(library().hlb_set_tau(h, float(tau)))


def hlb_step(h, n):
    _check(library().hlb_step(h, int(n)))


def hlb_read_macros(h, rho, u, wss, where):
    _check(library().hlb_read_macros(h, _P(rho), _P(u), _P(wss), where))


def hlb_reduce(h, n_iolets):
    mass = C.c_double()
    flux = (C.c_double * max(1, n_iolets))()
    rc = library().hlb_reduce(h, C.byref(mass), flux)
    if rc not in (HLB_OK, HLB_ERR_DIVERGED):
        _check(rc)
    return mass.value, np.array(flux[:n_iolets], dtype=np.float64), rc


def make_objective(sites, target, axis):
    """(hlb_objective, keep-alive arrays) from probe sites, targets and axis."""
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    target = np.ascontiguousarray(target, dtype=np.float64)
    obj = hlb_objective(n_probe=sites.size, sites=sites.ctypes.data_as(C.POINTER(C.c_int64)),
                        target=target.ctypes.data_as(C.POINTER(C.c_double)),
                        axis=tuple(float(a) for a in axis))
    return obj, (sites, target)


def hlb_adjoint_workspace_bytes(h, nsteps, n_probe) -> int:
    nb = C.c_size_t()
    _check(library().hlb_adjoint_workspace_bytes(h, int(nsteps), int(n_probe), C.byref(nb)))
    return nb.value


def hlb_adjoint_run(h, nsteps, obj, ws_ptr, ws_bytes, n_groups):
    J = C.c_double()
    dtau = C.c_double()
    damp = (C.c_double * max(1, n_groups))()
    _check(library().hlb_adjoint_run(h, int(nsteps), C.byref(obj), _P(ws_ptr), ws_bytes, C.byref(J),
                                     C.byref(dtau), damp))
    return J.value, dtau.value, np.array(damp[:n_groups])


def make_waveform(w):
    """dict (or number) -> (hlb_waveform, keep-alive buffer).

    {"kind": "const", "mean"}, {"kind": "cosine", "mean", "rel", "period",
    "phase"}, {"kind": "table", "mean", "period", "samples"}."""
    if isinstance(w, (int, float)):
        w = {"kind": "const", "mean": float(w)}
    kind = {"const": HLB_WAVE_CONST, "cosine": HLB_WAVE_COSINE, "table": HLB_WAVE_TABLE}[w.get("kind", "const")]
    buf = None
    wf = hlb_waveform(kind=kind, mean=float(w.get("mean", 1.0)), rel_amp=float(w.get("rel", 0.0)),
                      period=float(w.get("period", 1.0)), phase=float(w.get("phase", 0.0)), n_samples=0)
    if kind == HLB_WAVE_TABLE:
        buf = np.ascontiguousarray(w["samples"], dtype=np.float64)
        wf.n_samples = buf.size
        wf.samples = buf.ctypes.data_as(C.POINTER(C.c_double))
    return wf, buf


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("hemegb needs a CUDA device")
    return torch


class Solver:
    """D3Q19 LBGK solver over a sparse lattice on the current CUDA device.

    ``lattice`` is a :class:`paper_2202_11770_gb300.geometry.Lattice` (or any
    object with ``xyz``, ``src``, ``iolets``, ``wall_normal``, ``amp_group``).
    """

    def __init__(self, lattice, tau=1.0, precision="fp32", scheme="auto", ladd_rho_one=False,
                 ghost_full_u=False, use_normals=True, stream=None, wide_offsets=False, full_index=False):
        torch = _torch()
        lib = library()
        self._torch = torch
        self.n = int(lattice.n)
        self.iolets = list(lattice.iolets)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._xyz = np.ascontiguousarray(lattice.xyz, dtype=np.int32)
        self._src = np.ascontiguousarray(lattice.src, dtype=np.int32)
        self._nrm = np.ascontiguousarray(lattice.wall_normal, dtype=np.float32) if use_normals else None
        self._grp = np.ascontiguousarray(lattice.amp_group, dtype=np.int32)
        ios = (hlb_iolet * max(1, len(self.iolets)))()
        for k, io in enumerate(self.iolets):
            ios[k].kind = int(io.kind)
            ios[k].centre = tuple(float(v) for v in io.centre)
            ios[k].normal = tuple(float(v) for v in io.normal)
            ios[k].radius = float(io.radius)
            ios[k].n_groups = int(io.n_groups)
        self._lat = hlb_lattice(
            n_sites=self.n, xyz=self._xyz.ctypes.data_as(C.POINTER(C.c_int32)),
            src=self._src.ctypes.data_as(C.POINTER(C.c_int32)),
            wall_normal=self._nrm.ctypes.data_as(C.POINTER(C.c_float)) if self._nrm is not None else None,
            amp_group=self._grp.ctypes.data_as(C.POINTER(C.c_int32)),
            n_iolets=len(self.iolets), iolets=ios)
        self._ios = ios
        scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        self._opt = hlb_options(precision=self.precision, scheme=scheme, ladd_rho_one=int(ladd_rho_one),
                                ghost_full_u=int(ghost_full_u), wide_offsets=int(wide_offsets),
                                full_index=int(full_index))
        nbytes = hlb_workspace_bytes(self._lat, self._opt)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = hlb_create(self._lat, self._opt, self._ws_ptr, nbytes, self.stream.cuda_stream)
        self.ws_bytes = nbytes
        self._lib = lib
        self.set_tau(tau)
        # the solver copied what it needs; drop the host tables
        self._xyz = self._src = self._nrm = self._grp = None
        self._lat = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.hlb_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    @property
    def compact_index(self) -> bool:
        """True if the step and adjoint kernels read the compact index table."""
        r = int(self._lib.hlb_compact_index(self._h))
        _check(min(r, 0))
        return bool(r)

    @property
    def n_groups(self) -> int:
        return int(self._lib.hlb_n_amp_groups(self._h))

    @property
    def t(self) -> int:
        t = C.c_int64()
        _check(self._lib.hlb_time(self._h, C.byref(t)))
        return t.value

    def set_tau(self, tau):
        self.tau = float(tau)
        hlb_set_tau(self._h, tau)

    def set_velocity(self, k, amps, wave):
        amps = np.ascontiguousarray(np.atleast_1d(amps), dtype=np.float64)
        wf, keep = make_waveform(wave)
        _check(self._lib.hlb_set_velocity_waveform(self._h, int(k), amps.ctypes.data_as(C.POINTER(C.c_double)),
                                                   amps.size, C.byref(wf)))

    def set_pressure(self, k, wave):
        wf, keep = make_waveform(wave)
        _check(self._lib.hlb_set_pressure(self._h, int(k), C.byref(wf)))

    def init_equilibrium(self, rho0=1.0, u0=None):
        """u0: None, numpy float32 [3, n] (host) or torch float32 [3, n] (device)."""
        if u0 is None:
            _check(self._lib.hlb_init_equilibrium(self._h, float(rho0), None, HLB_HOST))
        elif isinstance(u0, np.ndarray):
            a = np.ascontiguousarray(u0, dtype=np.float32).reshape(3, self.n)
            _check(self._lib.hlb_init_equilibrium(self._h, float(rho0), _P(a.ctypes.data), HLB_HOST))
        else:
            a = u0.contiguous().float().reshape(3, self.n)
            _check(self._lib.hlb_init_equilibrium(self._h, float(rho0), _P(a.data_ptr()), HLB_DEVICE))

    def step(self, n=1):
        hlb_step(self._h, n)

    def macros_device(self, rho=True, u=True, wss=True):
        """Device tensors (rho [n], u [3, n], wss [n]), asynchronous."""
        torch = self._torch
        r = torch.empty(self.n, dtype=torch.float32, device="cuda") if rho else None
        v = torch.empty((3, self.n), dtype=torch.float32, device="cuda") if u else None
        w = torch.empty(self.n, dtype=torch.float32, device="cuda") if wss else None
        hlb_read_macros(self._h, r.data_ptr() if r is not None else None, v.data_ptr() if v is not None else None,
                        w.data_ptr() if w is not None else None, HLB_DEVICE)
        return r, v, w

    def macros(self):
        """Host numpy arrays (rho [n], u [n, 3], wss [n]); synchronises."""
        rho = np.empty(self.n, np.float32)
        u = np.empty((3, self.n), np.float32)
        wss = np.empty(self.n, np.float32)
        hlb_read_macros(self._h, rho.ctypes.data, u.ctypes.data, wss.ctypes.data, HLB_HOST)
        return rho, u.T.copy(), wss

    def reduce(self):
        """(mass, per-iolet flux) in FP64; raises on divergence."""
        mass, flux, rc = hlb_reduce(self._h, len(self.iolets))
        if rc == HLB_ERR_DIVERGED:
            raise HlbError(rc, library().hlb_last_error().decode())
        return mass, flux

    def set_windkessel(self, k, Rp, C, Rd, rho_d=1.0, rho_c0=None):
        """Pressure iolet k as a three-element Windkessel outlet (hlb_set_windkessel)."""
        _check(self._lib.hlb_set_windkessel(self._h, int(k), float(Rp), float(C), float(Rd), float(rho_d),
                                            float(rho_d if rho_c0 is None else rho_c0)))

    def windkessel_state(self, k):
        """(ghost density of the next step, rho_c, last outflow q) of outlet k."""
        g, r, q = C.c_double(), C.c_double(), C.c_double()
        _check(self._lib.hlb_windkessel_state(self._h, int(k), C.byref(g), C.byref(r), C.byref(q)))
        return g.value, r.value, q.value

    def iolet_monitor(self):
        """Per iolet: (mass flux of the last step, max |u|, mean rho) over the
        sites linked to it, FP64 arrays [n_iolets] (pressure = rho / 3)."""
        k = len(self.iolets)
        flux, umax, rho = (np.zeros(k), np.zeros(k), np.zeros(k))
        _check(self._lib.hlb_iolet_monitor(self._h, _P(flux.ctypes.data), _P(umax.ctypes.data), _P(rho.ctypes.data)))
        return flux, umax, rho

    def state(self):
        """Host copy of the shifted pre-collision state [19, n] (storage dtype) and t."""
        dt = {HLB_FP32: np.float32, HLB_FP64: np.float64, HLB_FP16: np.float16, HLB_BF16: np.uint16}[self.precision]
        out = np.empty((19, self.n), dtype=dt)
        t = C.c_int64()
        _check(self._lib.hlb_get_state(self._h, _P(out.ctypes.data), HLB_HOST, C.byref(t)))
        return out, t.value

    def set_state(self, f, t=0):
        f = np.ascontiguousarray(f)
        assert f.nbytes == 19 * self.n * _ELEM[self.precision]
        _check(self._lib.hlb_set_state(self._h, _P(f.ctypes.data), HLB_HOST, int(t)))

    def adjoint_workspace(self, nsteps, n_probe, extra_bytes=0):
        """A device workspace (uint8 tensor, 256-byte aligned pointer, size) for
        adjoint(): the sqrt(N)-checkpoint minimum, plus ``extra_bytes`` in which
        the run keeps whole segments of states instead of recomputing them."""
        nb = hlb_adjoint_workspace_bytes(self._h, nsteps, n_probe) + int(extra_bytes)
        ws = self._torch.empty(nb + 256, dtype=self._torch.uint8, device="cuda")
        return ws, (ws.data_ptr() + 255) & ~255, nb

    def adjoint_plan(self, nsteps, n_probe, ws_bytes):
        """(checkpoint interval K, kept segments, recomputed steps, bytes used)
        of an adjoint run with a workspace of ``ws_bytes``."""
        k, kept, rec, used = C.c_int64(), C.c_int64(), C.c_int64(), C.c_size_t()
        _check(self._lib.hlb_adjoint_plan(self._h, int(nsteps), int(n_probe), int(ws_bytes), C.byref(k),
                                          C.byref(kept), C.byref(rec), C.byref(used)))
        return k.value, kept.value, rec.value, used.value

    def adjoint(self, nsteps, sites, target, axis, workspace=None):
        """(J, dJ/dtau, dJ/da[groups]) over nsteps from the current state.

        ``workspace`` may be a tuple from adjoint_workspace(); otherwise one
        is allocated for the call."""
        obj, keep = make_objective(sites, target, axis)
        ws = workspace if workspace is not None else self.adjoint_workspace(nsteps, obj.n_probe)
        return hlb_adjoint_run(self._h, nsteps, obj, ws[1], ws[2], self.n_groups)


def bf16_to_float(a: np.ndarray) -> np.ndarray:
    """Host conversion of raw bfloat16 bits (uint16) to float32."""
    return (a.astype(np.uint32) << 16).view(np.float32)
