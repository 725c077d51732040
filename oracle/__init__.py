"""FP64 CPU oracle of the D3Q19 LBGK sparse-lattice step — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain C, FP64,
array-of-structures populations, push streaming) through ctypes and shares no
code with the GPU solver.  Inputs come as a lattice object with attributes
``xyz``, ``src``, ``iolets`` (kind, centre, normal, radius, n_groups) and
``amp_group`` — the output of the seeded input generator.

Paper references (arXiv 2202.11770): Eqs. 3a-3b (collide, stream), Eq. 4
(equilibrium, with the factors 1/2 the printed form lacks), Eqs. 5-6
(moments), Eq. 7 (p = cs2 rho), Section 2.3 (bounce-back walls, Ladd velocity
iolets, ghost-density pressure iolets), Section 3.1 (the step loop).

Every function here is pinned by the tests in ``tests/test_oracle_*.py``
against closed forms and invariants (moment identities, rest state, exact
mass conservation, Poiseuille and Womersley flow, the Poiseuille wall shear
stress, hand-enumerated streaming, central finite differences for the
adjoint).  The Ladd velocity iolet is pinned by the uniform flow it must keep
exactly, by a one-step enumeration of its link-midpoint weights, and by the
steady inlet flux and near-inlet profile against the imposed parabola; the
wall-shear-stress fallback normal by flat faces and box edges
(``tests/test_oracle_ladd.py``, ``tests/test_oracle_flow.py``).
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)


def _load():
    global _lib
    if _lib is None:
        # HLB_ORACLE_LIB lets the mutation test load a deliberately broken copy
        path = os.environ.get("HLB_ORACLE_LIB") or str(_build.build())
        lib = C.CDLL(path)
        lib.ora_create.argtypes = [C.c_int64, _I32, _I32, C.c_int, _I32, _D, _D, _D, _I32, _I32,
                                   C.POINTER(_P)]
        lib.ora_free.argtypes = [_P]
        lib.ora_set_tau.argtypes = [_P, C.c_double]
        lib.ora_set_options.argtypes = [_P, C.c_int, C.c_int]
        lib.ora_set_threads.argtypes = [_P, C.c_int]
        lib.ora_set_velocity.argtypes = [_P, C.c_int, _D, C.c_int, C.c_int, C.c_double, C.c_double,
                                         C.c_double, C.c_double, C.c_int, _D]
        lib.ora_set_pressure.argtypes = [_P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_int, _D]
        lib.ora_feq.argtypes = [C.c_double, _D, _D]
        lib.ora_init_equilibrium.argtypes = [_P, C.c_double, _D]
        lib.ora_step.argtypes = [_P, C.c_int64]
        lib.ora_time.argtypes = [_P]
        lib.ora_time.restype = C.c_int64
        lib.ora_get_state.argtypes = [_P, _D]
        lib.ora_set_state.argtypes = [_P, _D, C.c_int64]
        lib.ora_mass.argtypes = [_P]
        lib.ora_mass.restype = C.c_double
        lib.ora_flux.argtypes = [_P, _D]
        lib.ora_wave_value.argtypes = [_P, C.c_int, C.c_double]
        lib.ora_wave_value.restype = C.c_double
        lib.ora_set_windkessel.argtypes = [_P, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                           C.c_double]
        lib.ora_windkessel_rho.argtypes = [_P, C.c_int]
        lib.ora_windkessel_rho.restype = C.c_double
        lib.ora_windkessel_rho_c.argtypes = [_P, C.c_int]
        lib.ora_windkessel_rho_c.restype = C.c_double
        lib.ora_macros.argtypes = [_P, _D, _D, _D, C.POINTER(C.c_float)]
        lib.ora_objective.argtypes = [_P, C.c_int64, C.c_int64, _I64, _D, _D]
        lib.ora_objective.restype = C.c_double
        lib.ora_adjoint.argtypes = [_P, C.c_int64, C.c_int64, _I64, _D, _D, _D, _D, _D]
        lib.ora_n_groups.argtypes = [_P]
        lib.ora_last_error.restype = C.c_char_p
        _lib = lib
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def _wave_args(w):
    """Waveform dict -> (kind, mean, rel, period, phase, nsamp, samples).

    {"kind": "const", "mean": m}                       w(t) = m
    {"kind": "cosine", "mean", "rel", "period", "phase"=0}
                                      w(t) = m (1 + rel cos(2 pi t / period + phase))
    {"kind": "table", "mean"=1, "period", "samples"}   periodic linear interpolation
                                      of samples spaced period/len(samples), times mean
    """
    if isinstance(w, (int, float)):
        w = {"kind": "const", "mean": float(w)}
    kind = w.get("kind", "const")
    if kind == "const":
        return 0, float(w["mean"]), 0.0, 1.0, 0.0, 0, None
    if kind == "cosine":
        return 1, float(w["mean"]), float(w["rel"]), float(w["period"]), float(w.get("phase", 0.0)), 0, None
    if kind == "table":
        s = np.ascontiguousarray(w["samples"], dtype=np.float64)
        return 2, float(w.get("mean", 1.0)), 0.0, float(w["period"]), 0.0, int(s.size), s
    raise ValueError(f"unknown waveform kind {kind!r}")


def feq(rho: float, u) -> np.ndarray:
    """Equilibrium populations for density rho and velocity u (Eq. 4, with 1/2)."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(19, np.float64)
    lib.ora_feq(float(rho), _ptr(u, C.c_double), _ptr(out, C.c_double))
    return out


class Oracle:
    """Plain FP64 LBGK solver on a sparse lattice (push streaming, AoS)."""

    def __init__(self, lattice, tau: float, ladd_rho_one: bool = False, ghost_full_u: bool = False,
                 threads: int = 1):
        lib = _load()
        self._lib = lib
        xyz = np.ascontiguousarray(lattice.xyz, dtype=np.int32)
        src = np.ascontiguousarray(lattice.src, dtype=np.int32)
        n = xyz.shape[0]
        io = list(lattice.iolets)
        nio = len(io)
        kind = np.array([i.kind for i in io] or [0], np.int32)
        centre = np.array([i.centre for i in io] or [[0, 0, 0]], np.float64).reshape(-1)
        normal = np.array([i.normal for i in io] or [[0, 0, 0]], np.float64).reshape(-1)
        radius = np.array([i.radius for i in io] or [0], np.float64)
        ngroups = np.array([i.n_groups for i in io] or [1], np.int32)
        group = np.ascontiguousarray(lattice.amp_group, dtype=np.int32)
        h = _P()
        rc = lib.ora_create(n, _ptr(xyz, C.c_int32), _ptr(src, C.c_int32), nio, _ptr(kind, C.c_int32),
                            _ptr(centre, C.c_double), _ptr(normal, C.c_double), _ptr(radius, C.c_double),
                            _ptr(ngroups, C.c_int32), _ptr(group, C.c_int32), C.byref(h))
        if rc != 0:
            raise ValueError(lib.ora_last_error().decode())
        self._h = h
        self.n = n
        self.nio = nio
        self.iolets = io
        self.tau = tau
        lib.ora_set_tau(h, float(tau))
        lib.ora_set_options(h, int(ladd_rho_one), int(ghost_full_u))
        lib.ora_set_threads(h, int(threads))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.ora_free(h)
            self._h = None

    # ---- parameters ----
    def set_threads(self, threads: int):
        """Host threads of a step (sites split into contiguous blocks).  The
        state does not depend on the count; iolet fluxes are summed per block
        and then in block order."""
        self._lib.ora_set_threads(self._h, int(threads))

    def set_tau(self, tau: float):
        self.tau = tau
        self._lib.ora_set_tau(self._h, float(tau))

    def set_velocity(self, k: int, amps, wave):
        amps = np.ascontiguousarray(np.atleast_1d(amps), dtype=np.float64)
        kind, mean, rel, period, phase, ns, s = _wave_args(wave)
        rc = self._lib.ora_set_velocity(self._h, k, _ptr(amps, C.c_double), amps.size, kind, mean, rel,
                                        period, phase, ns, _ptr(s, C.c_double))
        if rc != 0:
            raise ValueError(self._lib.ora_last_error().decode())

    def set_pressure(self, k: int, wave):
        kind, mean, rel, period, phase, ns, s = _wave_args(wave)
        rc = self._lib.ora_set_pressure(self._h, k, kind, mean, rel, period, phase, ns, _ptr(s, C.c_double))
        if rc != 0:
            raise ValueError(self._lib.ora_last_error().decode())

    # ---- state ----
    def init_equilibrium(self, rho0: float = 1.0, u0=None):
        u = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64).reshape(self.n, 3)
        self._lib.ora_init_equilibrium(self._h, float(rho0), _ptr(u, C.c_double))

    def step(self, nsteps: int = 1):
        self._lib.ora_step(self._h, int(nsteps))

    @property
    def t(self) -> int:
        return int(self._lib.ora_time(self._h))

    def state(self) -> np.ndarray:
        f = np.empty((self.n, 19), np.float64)
        self._lib.ora_get_state(self._h, _ptr(f, C.c_double))
        return f

    def set_state(self, f, t: int = 0):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.n, 19)
        self._lib.ora_set_state(self._h, _ptr(f, C.c_double), int(t))

    # ---- outputs ----
    def macros(self, wall_normal=None):
        """(rho[n], u[n,3], wss[n]) of the current state; wss NaN off the wall."""
        rho = np.empty(self.n, np.float64)
        u = np.empty((self.n, 3), np.float64)
        wss = np.empty(self.n, np.float64)
        wn = None if wall_normal is None else np.ascontiguousarray(wall_normal, dtype=np.float32)
        self._lib.ora_macros(self._h, _ptr(rho, C.c_double), _ptr(u, C.c_double), _ptr(wss, C.c_double),
                             _ptr(wn, C.c_float))
        return rho, u, wss

    def mass(self) -> float:
        return float(self._lib.ora_mass(self._h))

    def flux(self) -> np.ndarray:
        out = np.zeros(max(self.nio, 1), np.float64)
        self._lib.ora_flux(self._h, _ptr(out, C.c_double))
        return out[: self.nio]

    def set_windkessel(self, k: int, Rp: float, C: float, Rd: float, rho_d: float = 1.0, rho_c0=None):
        """Pressure iolet k as a three-element Windkessel outlet (see oracle.c)."""
        rc = self._lib.ora_set_windkessel(self._h, int(k), float(Rp), float(C), float(Rd), float(rho_d),
                                          float(rho_d if rho_c0 is None else rho_c0))
        if rc:
            raise ValueError(self._lib.ora_last_error().decode())

    def windkessel_rho(self, k: int) -> float:
        """Ghost density outlet k used in the last step."""
        return float(self._lib.ora_windkessel_rho(self._h, int(k)))

    def windkessel_rho_c(self, k: int) -> float:
        return float(self._lib.ora_windkessel_rho_c(self._h, int(k)))

    def wave_value(self, k: int, t: float) -> float:
        """Waveform of iolet k at time t (velocity: the w(t) multiplying the
        amplitudes; pressure: the ghost density)."""
        return float(self._lib.ora_wave_value(self._h, int(k), float(t)))

    # ---- objective / adjoint ----
    def objective(self, nsteps, sites, target, axis) -> float:
        sites = np.ascontiguousarray(sites, dtype=np.int64)
        target = np.ascontiguousarray(target, dtype=np.float64)
        axis = np.ascontiguousarray(axis, dtype=np.float64)
        return float(self._lib.ora_objective(self._h, int(nsteps), sites.size, _ptr(sites, C.c_int64),
                                             _ptr(target, C.c_double), _ptr(axis, C.c_double)))

    def adjoint(self, nsteps, sites, target, axis):
        """(J, dJ/dtau, dJ/da[groups]) over nsteps from the current state."""
        sites = np.ascontiguousarray(sites, dtype=np.int64)
        target = np.ascontiguousarray(target, dtype=np.float64)
        axis = np.ascontiguousarray(axis, dtype=np.float64)
        ng = self._lib.ora_n_groups(self._h)
        damp = np.zeros(max(ng, 1), np.float64)
        J = C.c_double()
        dtau = C.c_double()
        rc = self._lib.ora_adjoint(self._h, int(nsteps), sites.size, _ptr(sites, C.c_int64),
                                   _ptr(target, C.c_double), _ptr(axis, C.c_double), C.byref(J),
                                   C.byref(dtau), _ptr(damp, C.c_double))
        if rc != 0:
            raise MemoryError(self._lib.ora_last_error().decode())
        return J.value, dtau.value, damp[:ng]


def mlups(n_sites: int, n_steps: int, seconds: float) -> float:
    """Million lattice-site updates per second (Eq. 9)."""
    return n_sites * n_steps / (seconds * 1e6) if seconds > 0 else math.inf
