"""GB300-native GridPull step library (Chen, Liu, Han, ICCV 2023).

The hot path - band build, query sampling, nearest surface point, the fused
loss forward + hand-written backward of Eq. 8, and Adam - runs in the CUDA
kernels of ``libgridpull.so`` behind the C ABI of ``include/gridpull.h``.
``binding`` exposes that ABI to Python under the same names (torch supplies
device memory and the stream); ``fit`` strings the calls into a fitting step.
The library is built with ``build.build()``; nothing here falls back to a CPU
path when it is missing.
"""
__all__ = ["autograd", "binding", "build", "fit", "synth", "torch_reference"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
