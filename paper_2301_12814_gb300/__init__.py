"""GB300 (sm_103a) U(1)-symmetric MPO simulation of a lossy Gaussian-boson-sampling
beam-splitter mesh (Liu et al., arXiv:2301.12814, App. D), behind the C ABI of
include/gbs_mpo.h.

`MPO` and `Plan` (in `mpo.py`) marshal arguments to libgbsmpo.so; `build.py`
compiles the library in-tree for sm_103a.  There is no CPU path.
"""
from .mpo import MPO, MPOError, Plan, EXPORTS, LIB_PATH, load_library  # noqa: F401

__all__ = ["MPO", "MPOError", "Plan", "EXPORTS", "LIB_PATH", "load_library"]
