"""Column-generation direct aperture optimisation (arXiv:1003.5402) on one GB300.

The product is libdao.so (CUDA kernels for sm_103a behind the C ABI of
include/dao.h); ``binding`` is its ctypes marshalling layer and ``build``
compiles it in-tree.  Importing this package does not load the library; the
first binding call does, and fails loudly if it has not been built.
"""
from . import binding  # noqa: F401
from .binding import Plan, Server, DaoError, load, release_cached_memory  # noqa: F401

__all__ = ["Plan", "Server", "DaoError", "load", "release_cached_memory", "binding"]
