"""C-ABI libraries load and export every declared symbol; host-side
validation returns the documented error codes (no GPU needed)."""
import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

from paper_2202_11770_gb300 import _build, geometry as geo, hemegb

INCLUDE = Path(__file__).resolve().parent.parent / "include"


def _declared(header):
    text = (INCLUDE / header).read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(hlbg?_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_solver_library_exports_declared_symbols():
    lib = hemegb.library()
    names = _declared("hemegb.h")
    assert "hlb_create" in names and "hlb_step" in names and "hlb_adjoint_run" in names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(names) == hemegb.exported_symbols()


def test_partition_symbols_exported():
    from paper_2202_11770_gb300 import partition
    lib = partition.library()
    names = _declared("hlb_partition.h")
    assert "hlb_part_create" in names and "hlb_halo_pack" in names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(names) == partition.exported_symbols()


def test_geometry_library_exports_declared_symbols():
    lib = C.CDLL(str(_build.build_geometry()))
    for name in _declared("hlb_geometry.h"):
        assert hasattr(lib, name), name


def _lattice(lat):
    xyz = np.ascontiguousarray(lat.xyz, np.int32)
    src = np.ascontiguousarray(lat.src, np.int32)
    grp = np.ascontiguousarray(lat.amp_group, np.int32)
    ios = (hemegb.hlb_iolet * max(1, len(lat.iolets)))()
    for k, io in enumerate(lat.iolets):
        ios[k].kind = io.kind
        ios[k].centre = tuple(io.centre)
        ios[k].normal = tuple(io.normal)
        ios[k].radius = io.radius
        ios[k].n_groups = io.n_groups
    L = hemegb.hlb_lattice(n_sites=lat.n, xyz=xyz.ctypes.data_as(C.POINTER(C.c_int32)),
                           src=src.ctypes.data_as(C.POINTER(C.c_int32)), wall_normal=None,
                           amp_group=grp.ctypes.data_as(C.POINTER(C.c_int32)), n_iolets=len(lat.iolets),
                           iolets=ios)
    return L, (xyz, src, grp, ios)


def test_workspace_size_and_validation():
    lat = geo.pipe(4.0, 8)
    L, keep = _lattice(lat)
    opt = hemegb.hlb_options(precision=hemegb.HLB_FP32, scheme=hemegb.HLB_PULL_AB)
    nb = hemegb.hlb_workspace_bytes(L, opt)
    n = lat.n
    assert nb >= 2 * 19 * 4 * n + 18 * 4 * n + 9 * 4 * n    # two buffers, int32 table, compact table
    opt16 = hemegb.hlb_options(precision=hemegb.HLB_BF16, scheme=hemegb.HLB_PULL_AB)
    assert hemegb.hlb_workspace_bytes(L, opt16) < nb

    lib = hemegb.library()
    out = C.c_size_t()
    # index out of range
    bad = lat.src.copy()
    bad[0, 3] = n + 5
    L2, keep2 = _lattice(geo.from_arrays(lat.xyz, bad, iolets=lat.iolets))
    assert lib.hlb_workspace_bytes(C.byref(L2), C.byref(opt), C.byref(out)) == hemegb.HLB_ERR_ARG
    assert b"out of range" in lib.hlb_last_error()
    # link code naming a missing iolet
    bad = lat.src.copy()
    bad[0, 3] = -(2 + 7)
    L3, keep3 = _lattice(geo.from_arrays(lat.xyz, bad, iolets=lat.iolets))
    assert lib.hlb_workspace_bytes(C.byref(L3), C.byref(opt), C.byref(out)) == hemegb.HLB_ERR_ARG
    assert b"missing iolet" in lib.hlb_last_error()
    # unknown precision
    optbad = hemegb.hlb_options(precision=9, scheme=hemegb.HLB_PULL_AB)
    assert lib.hlb_workspace_bytes(C.byref(L), C.byref(optbad), C.byref(out)) == hemegb.HLB_ERR_ARG
    # null workspace
    h = C.c_void_p()
    rc = lib.hlb_create(C.byref(L), C.byref(opt), None, 0, None, C.byref(h))
    assert rc == hemegb.HLB_ERR_WS and not h.value


def test_amplitude_group_validation():
    lat = geo.tree(1, 5, root_radius=4.0, length_ratio=5.0, n_sectors=2, n_rings=2)
    grp = lat.amp_group.copy()
    inlet = (lat.src == -2).any(axis=0)
    grp[np.nonzero(inlet)[0][0]] = 4          # the inlet has 4 groups: 0..3
    lat2 = geo.from_arrays(lat.xyz, lat.src, iolets=lat.iolets, amp_group=grp)
    L, keep = _lattice(lat2)
    opt = hemegb.hlb_options(precision=hemegb.HLB_FP32, scheme=hemegb.HLB_PULL_AB)
    with pytest.raises(hemegb.HlbError, match="group"):
        hemegb.hlb_workspace_bytes(L, opt)


def test_lattice_size_limits():
    """An empty lattice and one of 2^31 sites or more are rejected before any
    array is touched (site indices are int32; 32-bit offsets cover the rest)."""
    lib = hemegb.library()
    opt = hemegb.hlb_options(precision=hemegb.HLB_FP32, scheme=hemegb.HLB_AA)
    out = C.c_size_t()
    for n in (0, -1, 1 << 31):
        L = hemegb.hlb_lattice(n_sites=n, xyz=None, src=None, wall_normal=None, amp_group=None, n_iolets=0,
                               iolets=None)
        assert lib.hlb_workspace_bytes(C.byref(L), C.byref(opt), C.byref(out)) == hemegb.HLB_ERR_ARG
        assert b"n_sites" in lib.hlb_last_error()


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the public structs have the sizes and field
    offsets a C compiler gives the header's definitions."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"hlb_iolet": hemegb.hlb_iolet, "hlb_lattice": hemegb.hlb_lattice,
               "hlb_options": hemegb.hlb_options, "hlb_waveform": hemegb.hlb_waveform,
               "hlb_objective": hemegb.hlb_objective}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hemegb.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", f"-I{INCLUDE}", str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, f"{name}.{field}"
