"""GB300-native exact 2D convex hull: the data-parallel hot path of Mei's
gScan method (arXiv 1508.05931) as hand-written sm_103a CUDA behind a C ABI.

``paper_1508_05931_gb300.hull`` is the Python binding of that C ABI; it is
imported lazily so that the input generators in ``workloads`` stay usable
without the compiled library.
"""
__all__ = ["hull", "workloads"]


def __getattr__(name):
    if name == "hull":
        import importlib
        return importlib.import_module(__name__ + ".hull")
    raise AttributeError(name)
