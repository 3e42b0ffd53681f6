"""GB300 (sm_103a) first-passage-time sampler for stochastic delta-N
(arXiv:2410.13683): a C-ABI CUDA library (libfpt.so, include/fpt.h) and its
thin Python binding (``paper_2410_13683_gb300.fpt``)."""
from . import fpt  # noqa: F401

__all__ = ["fpt"]
