"""GB300-native finite-volume hot path of Manapy (arXiv 2203.00925).

The compute lives in ``libfvgb.so`` (CUDA, sm_103a) behind the C ABI of
``include/fvgb.h``; ``capi`` binds it with ctypes and ``device`` adds a small
convenience layer over torch CUDA tensors. Both are imported lazily so that
``python -m paper_2203_00925_gb300.build`` works before the library exists.
"""

__all__ = ["capi", "device", "build"]


def __getattr__(name):
    if name in ("capi", "device", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
