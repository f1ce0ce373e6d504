"""GB300-native p-multigrid compact gas-kinetic scheme (CGKS).

``meshgen`` builds the synthetic input meshes; ``cgks`` is the thin ctypes
binding of the CUDA library ``libcgks.so`` (imported lazily so the mesh
generators work without a GPU or a built library).
"""
import importlib

__all__ = ["meshgen", "cgks"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
