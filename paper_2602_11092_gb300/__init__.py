"""GB300-native batched strong simulation of linear-optical layers.

C ABI: include/slos.h (libslos.so, built by ``build_library()``).
Python: ``binding`` (ctypes marshalling), ``functions`` (autograd Functions
and QuantumLayer), ``workloads`` (seeded synthetic inputs).

Importing the package does not load the CUDA library; ``load()`` does and
raises if it is missing (there is no CPU fallback).
"""


def load():
    """Load libslos.so and return the ``binding`` module."""
    from . import binding as _b
    _b.load()
    return _b


def build_library(force: bool = False) -> str:
    from .buildlib import build as _build
    return _build(force=force)
