"""GB300-native batched log-likelihood of the disc-galaxy model of Rigamonti et al. (2022).

The compute path is libbang.so (hand-written sm_103a CUDA behind the C ABI of
include/bang.h); ``Model``/``LogLike`` are thin PyTorch-facing wrappers and ``synth``
draws seeded synthetic inputs.
"""
import importlib

__all__ = ["Model", "Galaxy", "LogLike", "synth", "build"]


def __getattr__(name):
    if name in ("Model", "Galaxy", "LogLike"):
        return getattr(importlib.import_module(__name__ + ".model"), name)
    if name in ("synth", "build", "model"):
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
