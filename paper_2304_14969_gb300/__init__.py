"""GB300-native state-vector simulation of arXiv 2304.14969's hot path.

``workloads`` holds the seeded circuit and state generators. ``qsim`` is the
thin ctypes binding over the C-ABI library ``libqsim.so`` (built from
``csrc/`` by ``build.build()``); it is imported on first use so that the
generators stay importable on a machine without the compiled library.
"""
__all__ = ["workloads", "qsim", "build"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
