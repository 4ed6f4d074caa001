"""GB300 (sm_103a) pattern-count engine with the method of GraphPi.

The C ABI lives in ``include/graphpi.h``; ``_native`` binds it with ctypes
under the same names. Importing this package does not load the library;
the first call into ``_native`` does (building it in-tree if needed), and
fails loudly when it cannot.
"""

__all__ = ["native"]


def native():
    from . import _native
    _native.load()
    return _native
