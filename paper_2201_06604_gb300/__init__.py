"""GB300-native multi-stream MRG32k3a (arXiv 2201.06604, "clrng").

The CUDA library is loaded on first use of a binding name, so that
``paper_2201_06604_gb300.workloads`` and ``paper_2201_06604_gb300.build`` can
be imported on a machine where it is not built yet.  Every compute call goes
through libmrg32k3a's kernels; there is no CPU path.
"""
__all__ = ["mrg", "build", "workloads", "grf"]


def __getattr__(name):
    import importlib

    if name in ("mrg", "build", "workloads", "serve", "batch", "tune", "grf"):
        return importlib.import_module(f".{name}", __name__)
    mod = importlib.import_module(".mrg", __name__)
    try:
        return getattr(mod, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None
