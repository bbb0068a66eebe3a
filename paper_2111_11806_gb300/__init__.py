"""GB300-native (sm_103a) diffuse rigid-body finite-volume solver: the
explicit Eulerian cell update of Wallis, Barton & Nikiforakis
(arXiv:2111.11806) behind the C ABI of include/dfvrb.h.

The CUDA library is paper_2111_11806_gb300/libdfvrb.so, built in-tree by
`paper_2111_11806_gb300._build.build()`; `binding` is its ctypes binding.
Importing this package does not load the library; `binding.load()` does, and
raises if it is missing.
"""
from . import binding  # noqa: F401
from .binding import Grid, DFV_FP32, DFV_FP64  # noqa: F401
