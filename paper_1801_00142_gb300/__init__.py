"""GB300-native XTRG beta-doubling engine (arXiv:1801.00142).

The compute path is ``libxtrg.so`` (hand-written CUDA for sm_103a) behind the
C ABI of include/xtrg.h; ``_lib`` is its ctypes binding and ``engine.XTRG`` a
convenience handle that takes device memory and the stream from PyTorch.
"""
import os

LIB_DIR = os.path.dirname(os.path.abspath(__file__))


def build(force=False):
    from .build import build as _b
    return _b(force=force)
