"""Kernel functions and the discretized operator (oracle; test infrastructure).

Discretization (Sec. 3.1, Eq. (3.1); quadrature rule of Sec. 5): piecewise
constant collocation at cell centres x_j with cell volumes w_j,

    A_ij = a_i delta_ij + b_i K_ij c_j,
    K_ij = G(|x_i - x_j|) w_j            (i != j, one-point rule),
    K_ii = integral of G(|x_i - y|) over the cell of x_i,

where G is the Laplace fundamental solution of Eq. (1.4):
G(r) = -log(r) / (2 pi) in 2D (kernel_id 0) and 1 / (4 pi r) in 3D
(kernel_id 1).  The cell of DOF i is the square/cube of side w_i^(1/d)
centred at x_i.  The paper computes the diagonal "adaptively"; here it is the
exact integral in closed form:

  2D: int_{[-h/2,h/2]^2} log|y| dy = h^2 (ln h - ln(2)/2 - 3/2 + pi/4)
  3D: int_{[-h/2,h/2]^3} 1/|y| dy  = h^2 (3 ln(2 + sqrt 3) - pi/2)
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi
FOUR_PI = 4.0 * math.pi


def green(kernel_id: int, r: np.ndarray) -> np.ndarray:
    """G(r) of Eq. (1.4): kernel 0 = -log(r)/(2 pi), kernel 1 = 1/(4 pi r)."""
    r = np.asarray(r, dtype=np.float64)
    if kernel_id == 0:
        return -np.log(r) / TWO_PI
    if kernel_id == 1:
        return 1.0 / (FOUR_PI * r)
    raise ValueError("kernel_id must be 0 or 1")


def self_integral(kernel_id: int, w: np.ndarray) -> np.ndarray:
    """Exact K_ii: the integral of G over the DOF's own cell of volume w."""
    w = np.asarray(w, dtype=np.float64)
    if kernel_id == 0:
        h = np.sqrt(w)
        return -(h * h / TWO_PI) * (np.log(h) - 0.5 * math.log(2.0) - 1.5 + 0.25 * math.pi)
    if kernel_id == 1:
        h = np.cbrt(w)
        return (h * h / FOUR_PI) * (3.0 * math.log(2.0 + math.sqrt(3.0)) - 0.5 * math.pi)
    raise ValueError("kernel_id must be 0 or 1")


def double_layer_2d(x: np.ndarray, y: np.ndarray, ny: np.ndarray) -> np.ndarray:
    """dG/dnu_y for the 2D Laplace kernel (Sec. 1, Eqs. (1.3), (1.5)): (x-y).nu_y / (2 pi |x-y|^2).

    Only used to check the sign convention of the second-kind boundary IE.
    """
    d = x - y
    return (d * ny).sum(axis=-1) / (TWO_PI * (d * d).sum(axis=-1))


class Operator:
    """The dense operator A = diag(a) + diag(b) K diag(c), entries on demand.

    ``A`` is never stored for large N (Sec. 3.1: entries are generated as
    needed); ``entries(rows, cols)`` returns the submatrix A[rows][:, cols].
    """

    def __init__(self, points, weights, a, b, c, kernel_id):
        self.x = np.ascontiguousarray(points, dtype=np.float64)
        self.w = np.asarray(weights, dtype=np.float64)
        self.a = np.asarray(a, dtype=np.float64)
        self.b = np.asarray(b, dtype=np.float64)
        self.c = np.asarray(c, dtype=np.float64)
        self.kernel_id = int(kernel_id)
        self.N, self.dim = self.x.shape
        self.kself = self_integral(self.kernel_id, self.w)

    def kernel_entries(self, rows, cols) -> np.ndarray:
        """b_i K_ij c_j (no a_i term) for i in rows, j in cols."""
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        d = self.x[rows][:, None, :] - self.x[cols][None, :, :]
        r = np.sqrt((d * d).sum(axis=2))
        same = rows[:, None] == cols[None, :]
        r_safe = np.where(same, 1.0, r)
        K = green(self.kernel_id, r_safe) * self.w[cols][None, :]
        if same.any():
            K = np.where(same, self.kself[rows][:, None], K)
        return self.b[rows][:, None] * K * self.c[cols][None, :]

    def entries(self, rows, cols) -> np.ndarray:
        """A_ij = a_i delta_ij + b_i K_ij c_j for i in rows, j in cols."""
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        out = self.kernel_entries(rows, cols)
        same = rows[:, None] == cols[None, :]
        if same.any():
            out = out + np.where(same, self.a[rows][:, None], 0.0)
        return out

    def dense(self) -> np.ndarray:
        idx = np.arange(self.N)
        return self.entries(idx, idx)

    def proxy_out(self, xE, cols) -> np.ndarray:
        """Outgoing proxy rows Y_{cE,c} (Lemma 3.3 with quadrature weights):
        G(|x^E_e - x_j|) w_j c_j for proxy points xE (P x d)."""
        cols = np.asarray(cols, dtype=np.int64)
        d = xE[:, None, :] - self.x[cols][None, :, :]
        return green(self.kernel_id, np.sqrt((d * d).sum(axis=2))) * (self.w[cols] * self.c[cols])[None, :]

    def proxy_in(self, xE, cols) -> np.ndarray:
        """Incoming proxy rows (Y_{c,cE})^T: b_j G(|x_j - x^E_e|) w_j."""
        cols = np.asarray(cols, dtype=np.int64)
        d = xE[:, None, :] - self.x[cols][None, :, :]
        return green(self.kernel_id, np.sqrt((d * d).sum(axis=2))) * (self.b[cols] * self.w[cols])[None, :]

    def matvec(self, x: np.ndarray, trans: bool = False, block: int = 512) -> np.ndarray:
        """Direct sum y = A x (or A^T x), row block by row block, FP64."""
        x = np.asarray(x, dtype=np.float64)
        vec = x.ndim == 1
        X = x[:, None] if vec else x
        Y = np.empty_like(X)
        idx = np.arange(self.N)
        for s in range(0, self.N, block):
            rows = idx[s:s + block]
            if not trans:
                Y[rows] = self.entries(rows, idx) @ X
            else:
                Y[rows] = self.entries(idx, rows).T @ X
        return Y[:, 0] if vec else Y

    def matvec_rows(self, x: np.ndarray, rows, trans: bool = False) -> np.ndarray:
        """(A x)_i (or (A^T x)_i) for the listed rows only; any N."""
        x = np.asarray(x, dtype=np.float64)
        X = x[:, None] if x.ndim == 1 else x
        idx = np.arange(self.N)
        out = []
        for i in np.asarray(rows, dtype=np.int64):
            if not trans:
                row = self.entries(np.array([i]), idx)[0]
            else:
                row = self.entries(idx, np.array([i]))[:, 0]
            out.append(row @ X)
        out = np.asarray(out)
        return out[:, 0] if x.ndim == 1 else out
