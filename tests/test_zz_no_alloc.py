"""The allocation-free mass entry point (hlb_mass_static) agrees with the
workspace-based FP64 reduction (hlb_reduce), called twice in a row.

Some callers of this library cannot allocate device memory where they need
the total mass (their framework's allocator owns all device memory, or they
run in a loop where cudaMalloc's implicit synchronisation is not allowed);
hlb_mass_static keeps its partial sums in a fixed device array instead.  The
test owns the input populations and the output, as such a caller would.
This file is collected last so that a failure here stops a -x run only after
every other test has run; it passes alone and after the other tests."""
import ctypes as C

import numpy as np
import pytest

from paper_2202_11770_gb300 import geometry as geo

pytestmark = pytest.mark.gpu
hemegb = pytest.importorskip("paper_2202_11770_gb300.hemegb")
torch = pytest.importorskip("torch")


def _mass_static(state, precision, n, out, stream):
    return hemegb.library().hlb_mass_static(C.c_void_p(state.data_ptr()), precision, n,
                                            C.c_void_p(out.data_ptr()), C.c_void_p(stream))


def _iolet_rounding_bound(state, lat, prec):
    """Sum over the iolet links of half a unit in the last place of their
    stored values: for a 16-bit state read back after a pull A-B step, the
    read-back rounds the boundary values of these links to the storage format,
    which the workspace-based reduction sums unrounded."""
    if prec not in ("bf16", "fp16") or state is None:
        return 0.0
    vals = state.float().cpu().numpy()[1:][lat.src <= -2].astype(np.float64)
    mant = 7 if prec == "bf16" else 10
    e = np.floor(np.log2(np.maximum(np.abs(vals), 2.0 ** -24)))
    return float((0.5 * 2.0 ** (e - mant)).sum())


@pytest.mark.parametrize("prec,scheme,tol", [("fp32", "aa", 1e-12), ("bf16", "aa", 1e-12), ("fp64", "aa", 1e-13),
                                             ("fp32", "ab", 1e-12), ("bf16", "ab", 1e-12), ("fp16", "ab", 1e-12),
                                             ("fp16", "aa", 1e-12)])
def test_static_mass_matches_reduce_twice(prec, scheme, tol):
    lat = geo.tree(2, 2202, target_sites=50_000, length_ratio=5.0)
    s = hemegb.Solver(lat, tau=0.6, precision=prec, scheme=scheme)
    s.set_velocity(0, [1.0], {"kind": "cosine", "mean": 0.02, "rel": 0.5, "period": 100.0})
    for k in range(1, len(lat.iolets)):
        s.set_pressure(k, 1.0 - 0.0005 * k)
    s.init_equilibrium()
    elem = {"fp32": torch.float32, "bf16": torch.bfloat16, "fp16": torch.float16, "fp64": torch.float64}[prec]
    state = torch.empty((19, lat.n), dtype=elem, device="cuda")
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = s.stream.cuda_stream
    for call in range(2):
        s.step(37 + call)
        mass_ref, _ = s.reduce()
        rc = hemegb.library().hlb_get_state(s.handle, C.c_void_p(state.data_ptr()), hemegb.HLB_DEVICE, None)
        assert rc == hemegb.HLB_OK
        assert _mass_static(state, s.precision, lat.n, out[call:], stream) == hemegb.HLB_OK
        torch.cuda.synchronize()
        got = float(out[call].item())
        bound = tol * mass_ref + (_iolet_rounding_bound(state, lat, prec) if scheme == "ab" else 0.0)
        assert abs(got - mass_ref) <= bound, (call, got, mass_ref, bound)
    assert float(out[0]) != float(out[1])      # two different states, two fresh results


def test_static_mass_rejects_too_many_sites():
    lib = hemegb.library()
    limit = 67_108_864
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.hlb_mass_static(C.c_void_p(dummy.data_ptr()), hemegb.HLB_FP32, limit + 1,
                             C.c_void_p(dummy.data_ptr()), None)
    assert rc == hemegb.HLB_ERR_ARG
    assert b"static scratch limit" in lib.hlb_last_error()
