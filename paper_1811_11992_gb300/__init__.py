"""GB300 (sm_103a) implementation of the Newton linearise-and-solve step of the
in-situ-combustion simulator of arXiv 1811.11992.

The compute path is libisc (CUDA, built in-tree by ``build.build()``) behind
the C ABI of ``include/isc.h``; ``isc`` is its Python binding.
"""
from .isc import Simulator, default_options, load_library  # noqa: F401
