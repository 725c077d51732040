"""GB300-native D3Q19 LBGK solver over sparse vascular lattices (arXiv 2202.11770).

Submodules:
  geometry  — seeded synthetic lattices (pipe, bifurcating tree); input only.
  hemegb    — ctypes binding of the C-ABI solver library ``libhemegb``
              (sm_103a CUDA kernels) plus the ``Solver`` convenience class.
  adjoint   — ``torch.autograd.Function`` over the solver's discrete adjoint.

Submodules are imported lazily so that the input generator can be used
without loading the CUDA library.
"""
import importlib

__all__ = ["geometry", "hemegb", "adjoint"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
