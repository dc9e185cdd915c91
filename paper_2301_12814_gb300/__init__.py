"""GB300 (sm_103a) U(1)-symmetric MPO simulation of a lossy Gaussian-boson-sampling
beam-splitter mesh (Liu et al., arXiv:2301.12814, App. D), behind the C ABI of
include/gbs_mpo.h.

`MPO` and `Plan` (in `mpo.py`) marshal arguments to libgbsmpo.so; `build.py`
compiles the library in-tree for sm_103a.  There is no CPU path.  `experiments.py`
drives the paper's run protocols (App. A: the choice of d, the bond-dimension search,
the depth rule, Fig. 4(b)) and the App. C estimates (Fig. 1) over the same ABI.
"""
from .mpo import MPO, MPOError, Plan, EXPORTS, LIB_PATH, load_library  # noqa: F401

__all__ = ["MPO", "MPOError", "Plan", "EXPORTS", "LIB_PATH", "load_library"]
