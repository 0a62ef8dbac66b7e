"""FP64 CPU oracle of the coarse-grained CFD-DEM step (arXiv 2211.06142).

Test infrastructure only: tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use it.  The CUDA library never imports it.
"""
from .oracle import *  # noqa: F401,F403
