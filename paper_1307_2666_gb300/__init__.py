"""HIF-IE on GB300: hierarchical interpolative factorization of discretized
integral operators (Ho & Ying), hot path in hand-written sm_103a CUDA.

``hif`` is the ctypes binding of the C ABI (``include/hif.h``);
``Factorization`` wraps one handle for torch tensors; ``HIFSolve`` is the
autograd function whose backward runs the adjoint (transposed) solve.
"""
from __future__ import annotations

from . import hif  # noqa: F401
from .hif import (  # noqa: F401
    hif_apply,
    hif_apply_transpose,
    hif_destroy,
    hif_factor,
    hif_id_batched,
    hif_kernel_block,
    hif_matvec,
    hif_matvec_digits,
    hif_options_default,
    hif_solve,
    hif_solve_refined,
    hif_solve_transpose,
    hif_stats,
)
from .api import Factorization, HIFSolve  # noqa: F401
