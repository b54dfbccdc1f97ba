"""GB300-native lensed-image simulation: ray-trace, Sersic source, bin-down, PSF.

The compute path is the CUDA library ``liblenssim.so`` behind the C ABI declared in
``include/lens_sim.h``; ``paper_2606_01547_gb300.lenssim`` is the thin ctypes binding
(torch tensors for device memory and streams).  ``workloads`` draws seeded inputs.
The binding is imported lazily so that the input generators can be used without
torch or a GPU.
"""
import importlib

__all__ = ["lenssim", "workloads"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
