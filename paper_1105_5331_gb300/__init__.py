"""GB300 (sm_103a) library for rank-R canonical tensor approximation by
N-GMRES-accelerated ALS (De Sterck, arXiv 1105.5331).

The compute path is the CUDA shared library ``libcp_gb300.so`` behind the C
ABI of ``include/cp.h``; this package only marshals arguments to it.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import CpError, Ctx, Tensor, library  # noqa: F401
