"""GB300-native matrix-free wedge Stokes operator (TERRA-NG, arxiv 2609.21633).

The compute path is the in-tree shared library ``lib/libterra_wedge.so``
(hand-written sm_103a CUDA behind the C ABI of ``include/terra_wedge.h``);
``_lib`` is its ctypes binding and ``layout`` holds the node-layout helpers.
"""
from . import _lib
from ._lib import *  # noqa: F401,F403  (entry points under their C names)
