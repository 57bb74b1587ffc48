"""Dense FP64 ground truth (oracle; test infrastructure).

Assembles A (Sec. 3.1, Eq. (3.1)) and solves A u = f by LU with partial
pivoting (LAPACK getrf/getrs through scipy).  Feasible for N up to a few
thousand; it is the reference every HIF result is measured against.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import lu_factor, lu_solve

from .kernels import Operator


class DenseSolver:
    def __init__(self, op: Operator):
        self.op = op
        self.A = op.dense()
        self.lu = lu_factor(self.A)

    def solve(self, f, trans: bool = False):
        return lu_solve(self.lu, f, trans=1 if trans else 0)

    def matvec(self, x, trans: bool = False):
        return (self.A.T if trans else self.A) @ x
