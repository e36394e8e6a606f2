"""GB300 (sm_103a) block-Toeplitz Bayesian inversion: Python binding of libbti.

The compute path is the CUDA library ``libbti.so`` built from ``csrc/``
(C ABI in ``include/bti.h``).  This package only marshals arguments: every
step of every call runs in the library's kernels.  The library is loaded on
first use, so importing the package (or its ``synthetic`` input generator)
works on a machine without a GPU; any call into the library fails loudly if
the shared object is missing.  There is no CPU fallback.

Layouts (all row-major, float64 unless a call says otherwise):
  time-domain blocks [N_t][R][N_m], parameter vectors [B][N_t][N_m],
  data vectors [B][N_t][N_d], QoI vectors [B][N_t][N_q].
"""

from ._binding import (  # noqa: F401
    BtiError,
    Handle,
    OP_F,
    OP_G,
    OP_FQ,
    F64,
    F32,
    DF64,
    F16,
    lib,
    lib_path,
    header_symbols,
    KCLASSES,
)
from .autograd import EllipticOp, FOp, apply_F_autograd, map_loss  # noqa: F401
