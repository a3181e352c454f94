"""GB300-native finite-volume solidification solver (arXiv:1810.08572).

The compute path is the CUDA library ``libfvs.so`` (built from csrc/ for
sm_103a); ``fvs`` is its ctypes binding.  Importing ``fvs`` fails loudly if
the library is missing; there is no CPU fallback.
"""
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfvs.so")


def build(verbose=False):
    from .build import build as _build
    return _build(verbose=verbose)


def load():
    from . import fvs
    return fvs
