"""B300-native HPR-LP hot path: CUDA kernels for sm_103a behind a C ABI.

Submodules:
  ``hpr``    -- ctypes binding of the C ABI declared in ``include/hpr.h`` (same names)
  ``lpgen``  -- seeded synthetic LP generators (problem data only)
  ``build``  -- nvcc build step for the shared library

The binding is imported lazily so that the generators can be used without the CUDA
library; calling into the binding without the built library raises.
"""

__all__ = ["hpr", "lpgen", "build"]


def __getattr__(name):
    if name in __all__:
        import importlib

        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
