"""GB300 (sm_103a) domain wall fermion multigrid hot path (arXiv:2103.05034).

The compute path is the CUDA library libdwfmg.so behind the C ABI in
include/dwfmg.h; `ops` is its Python binding.  Importing `ops` without the
built library raises: there is no CPU fallback.
"""
from . import _lib  # noqa: F401

__all__ = ["ops", "layout"]
