"""Seeded synthetic sparse lattices (input generator).

Thin ctypes binding of ``libhlbgeom`` (``include/hlb_geometry.h``).  The
returned :class:`Lattice` holds numpy copies of the generator's arrays; it is
the common input of the GPU solver and of the FP64 oracle.  Nothing here
computes lattice Boltzmann quantities.

Paper context (arXiv 2202.11770): Section 3.2.1 lists the per-site inputs of
the GPU solver (streaming indices, wall/iolet link information, iolet ranges
and normals); Section 3.2.2 the six site types; Section 6 the straight pipe
used to compare CPU and GPU results.  The seeded vessel tree stands in for
the paper's patient geometries, which are not available.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import _build

# D3Q19 directions, order of Section 2.2 with opposite pairs adjacent.
CI = np.array(
    [[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
     [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1],
     [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]],
    dtype=np.int32)

VELOCITY, PRESSURE, WALL = 0, 1, 2
INNER, WALLSITE, INLET, OUTLET, INLET_WALL, OUTLET_WALL = range(6)


class _Iolet(C.Structure):
    _fields_ = [("kind", C.c_int32), ("role", C.c_int32), ("centre", C.c_double * 3),
                ("normal", C.c_double * 3), ("radius", C.c_double), ("n_groups", C.c_int32)]


@dataclass
class Iolet:
    kind: int              # VELOCITY or PRESSURE
    role: int              # 0 inlet, 1 outlet
    centre: np.ndarray     # point on the plane, on the vessel axis
    normal: np.ndarray     # unit normal into the fluid
    radius: float
    n_groups: int = 1


@dataclass
class Lattice:
    """A sparse D3Q19 lattice.

    ``src`` is the SoA pull-source table ``int32[18, n]``: row ``i-1`` holds,
    for every site, the index of the fluid site at ``x - c_i`` or a link code
    (-1 wall, -(2+k) iolet k).  Sites are ordered by (z, y, x)."""
    xyz: np.ndarray            # int32 [n, 3]
    src: np.ndarray            # int32 [18, n]
    type: np.ndarray           # uint8 [n]
    wall_normal: np.ndarray    # float32 [3, n]
    amp_group: np.ndarray      # int32 [n]
    iolets: List[Iolet] = field(default_factory=list)
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_geometry()
        lib = C.CDLL(str(path))
        P = C.c_void_p
        lib.hlbg_pipe.argtypes = [C.c_double, C.c_int32, C.c_int32, C.c_int32, C.POINTER(P)]
        lib.hlbg_tree.argtypes = [C.c_int32, C.c_uint64, C.c_int64, C.c_double, C.c_double,
                                  C.c_int32, C.c_int32, C.POINTER(P)]
        lib.hlbg_n_sites.argtypes = [P]
        lib.hlbg_n_sites.restype = C.c_int64
        for name, rt in (("hlbg_xyz", C.POINTER(C.c_int32)), ("hlbg_src", C.POINTER(C.c_int32)),
                         ("hlbg_type", C.POINTER(C.c_uint8)),
                         ("hlbg_wall_normal", C.POINTER(C.c_float)),
                         ("hlbg_amp_group", C.POINTER(C.c_int32)),
                         ("hlbg_iolets", C.POINTER(_Iolet))):
            getattr(lib, name).argtypes = [P]
            getattr(lib, name).restype = rt
        lib.hlbg_n_iolets.argtypes = [P]
        lib.hlbg_n_iolets.restype = C.c_int32
        lib.hlbg_info.argtypes = [P, C.POINTER(C.c_double)]
        lib.hlbg_free.argtypes = [P]
        lib.hlbg_last_error.restype = C.c_char_p
        _lib = lib
    return _lib


def _copy(ptr, count, dtype):
    out = np.empty(count, dtype=dtype)
    if count:
        C.memmove(out.ctypes.data, ptr, out.nbytes)
    return out


def _wrap(handle) -> Lattice:
    lib = _load()
    try:
        n = lib.hlbg_n_sites(handle)
        xyz = _copy(lib.hlbg_xyz(handle), 3 * n, np.int32).reshape(n, 3)
        src = _copy(lib.hlbg_src(handle), 18 * n, np.int32).reshape(18, n)
        typ = _copy(lib.hlbg_type(handle), n, np.uint8)
        wn = _copy(lib.hlbg_wall_normal(handle), 3 * n, np.float32).reshape(3, n)
        grp = _copy(lib.hlbg_amp_group(handle), n, np.int32)
        nio = lib.hlbg_n_iolets(handle)
        raw = lib.hlbg_iolets(handle)
        iolets = [Iolet(kind=raw[k].kind, role=raw[k].role,
                        centre=np.array(raw[k].centre[:], dtype=np.float64),
                        normal=np.array(raw[k].normal[:], dtype=np.float64),
                        radius=float(raw[k].radius), n_groups=int(raw[k].n_groups))
                  for k in range(nio)]
        info = (C.c_double * 8)()
        lib.hlbg_info(handle, info)
        meta = {"root_radius": info[0], "fill": info[1],
                "bbox": (int(info[2]), int(info[3]), int(info[4])),
                "n_segments": int(info[5]), "rejected_shapes": int(info[6]),
                "root_length": info[7]}
    finally:
        lib.hlbg_free(handle)
    return Lattice(xyz=xyz, src=src, type=typ, wall_normal=wn, amp_group=grp,
                   iolets=iolets, info=meta)


def _check(rc):
    if rc != 0:
        raise ValueError(_load().hlbg_last_error().decode())


def pipe(radius: float = 8.0, length: int = 64, inlet: int = VELOCITY,
         outlet: int = PRESSURE) -> Lattice:
    """Straight pipe along +z (sites with x^2+y^2 < radius^2, z = 0..length-1).

    The ends at z = -1/2 and z = length-1/2 are velocity iolets, pressure
    iolets or walls.  radius 8, length 64 gives 12,352 sites."""
    lib = _load()
    h = C.c_void_p()
    _check(lib.hlbg_pipe(radius, length, inlet, outlet, C.byref(h)))
    lat = _wrap(h)
    lat.info.update(kind="pipe", radius=radius, length=length)
    return lat


def tree(depth: int, seed: int, target_sites: int = 0, root_radius: float = 0.0,
         length_ratio: float = 8.0, n_sectors: int = 1, n_rings: int = 1) -> Lattice:
    """Seeded bifurcating vessel tree (2^depth pressure outlets, one velocity
    inlet at the root).  Radii follow Murray's law r_child = r_parent/2^(1/3);
    bifurcation angles are uniform in 30-70 degrees.  With target_sites > 0
    the root radius is tuned to reach that count within 2 %."""
    lib = _load()
    h = C.c_void_p()
    _check(lib.hlbg_tree(depth, seed, target_sites, root_radius, length_ratio,
                         n_sectors, n_rings, C.byref(h)))
    lat = _wrap(h)
    lat.info.update(kind="tree", depth=depth, seed=seed, length_ratio=length_ratio)
    return lat


def from_arrays(xyz, src, iolets=(), type=None, wall_normal=None, amp_group=None) -> Lattice:
    """Build a Lattice from caller arrays (hand-made test lattices)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    n = xyz.shape[0]
    src = np.ascontiguousarray(src, dtype=np.int32).reshape(18, n)
    typ = np.zeros(n, np.uint8) if type is None else np.asarray(type, np.uint8)
    wn = np.zeros((3, n), np.float32) if wall_normal is None else np.asarray(wall_normal, np.float32)
    grp = np.zeros(n, np.int32) if amp_group is None else np.asarray(amp_group, np.int32)
    return Lattice(xyz=xyz, src=src, type=typ, wall_normal=wn, amp_group=grp,
                   iolets=list(iolets), info={"kind": "custom"})
