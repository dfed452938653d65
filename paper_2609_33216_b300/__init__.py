"""B300 (sm_103a) symmetric HSS direct solver for 2-D Helmholtz transmission scattering.

The compute path is the CUDA library ``libsymhss.so`` (C ABI: ``include/symhss.h``).
``paper_2609_33216_b300.symhss`` is its ctypes binding and
``paper_2609_33216_b300.solver`` a small torch-facing wrapper.  Importing either
raises if the library has not been built (``python -m paper_2609_33216_b300.build``);
there is no CPU fallback.
"""

__all__ = ["symhss", "solver", "build"]


def __getattr__(name):
    if name in __all__:
        import importlib

        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
