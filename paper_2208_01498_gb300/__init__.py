"""GB300 tensor-network amplitude executor (separator-tree contraction of
quantum circuits, arXiv 2208.01498).  The C ABI is ``include/tnc.h``; this
package holds its sources (``csrc/``), the in-tree build and the ctypes
binding (``tnc``)."""

__all__ = ["tnc", "build"]
