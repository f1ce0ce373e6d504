"""GB300-native p-multigrid compact gas-kinetic scheme (CGKS).

``meshgen`` builds the synthetic input meshes; ``cgks`` is the thin ctypes
binding of the CUDA library ``libcgks.so`` (imported lazily so the mesh
generators work without a GPU or a built library).
"""
__all__ = ["meshgen", "cgks"]


def __getattr__(name):
    if name == "cgks":
        from . import cgks
        return cgks
    if name == "meshgen":
        from . import meshgen
        return meshgen
    raise AttributeError(name)
