"""GB300 (sm_103a) segment cost-volume library for multiview depth estimation (arXiv:1909.02294).

The compute path is the C ABI of include/ftv.h, implemented by hand-written CUDA kernels in
csrc/ and built into libftv.so by build.py. `ftv` is its thin Python binding; `batch` drives
the batched and served forms. Importing this package fails if libftv.so has not been built.
"""
from .ftv import *  # noqa: F401,F403
from . import ftv  # noqa: F401
