"""GB300-native short-range TreePM tree-force library (OpenGadget3 gravity path).

The compute path is the CUDA shared library built from ``csrc/`` for sm_103a
and reached through the C-ABI of ``include/og.h``; ``og`` is its ctypes
binding.  Importing the package does not load the library; the first call
does, and fails loudly when it has not been built.
"""
import importlib

from . import build  # noqa: F401

__all__ = ["build", "og"]


def __getattr__(name):
    if name == "og":
        return importlib.import_module(__name__ + ".og")
    raise AttributeError(name)
