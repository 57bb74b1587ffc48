"""Interpolative decomposition (oracle; test infrastructure).

Sec. 2.2, Lemma 2.2: a thin column-pivoted QR  Y Pi = Q [R1 R2]  gives the
skeleton columns (first k pivots) and the interpolation matrix T = R1^{-1} R2
with Y[:, redundant] = Y[:, skeleton] T.  The rank is adaptive (Sec. 2.2,
last paragraph): pivoting continues while the pivot magnitude |R_jj| exceeds
tol * |R_11|.

Readings fixed here (the paper leaves them open):
* pivot = remaining column of largest 2-norm over the not-yet-reduced rows,
  ties broken by the lowest original column index;
* column norms are recomputed exactly after every Householder step;
* k = the number of steps j with |R_jj| > tol |R_11| (k = 0 for a zero
  matrix); at most min(m, n) steps;
* skeleton order = pivot order; redundant order = ascending column index,
  and the columns of T follow that order.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular


def interp_decomp(Y: np.ndarray, tol: float):
    """Adaptive-rank ID of Y (m x n) to relative tolerance ``tol``.

    Returns (sk, rd, T): sk, rd index arrays into the columns of Y and
    T of shape (len(sk), len(rd)) with Y[:, rd] ~= Y[:, sk] @ T.
    """
    R = np.array(Y, dtype=np.float64, copy=True)
    m, n = R.shape
    perm = np.arange(n)
    kmax = min(m, n)
    k = 0
    nu0 = None
    for j in range(kmax):
        norms = np.sqrt((R[j:, j:] ** 2).sum(axis=0))
        best = norms.max() if norms.size else 0.0
        # lowest original index among the columns that attain the maximum
        cand = np.nonzero(norms == best)[0]
        p = j + cand[np.argmin(perm[j + cand])]
        if j == 0:
            nu0 = best
        if best <= tol * nu0 or best == 0.0:
            break
        if p != j:
            R[:, [j, p]] = R[:, [p, j]]
            perm[[j, p]] = perm[[p, j]]
        # Householder reflector that maps R[j:, j] onto -sign * |x| e_1
        x = R[j:, j].copy()
        alpha = np.linalg.norm(x)
        sgn = 1.0 if x[0] >= 0 else -1.0
        v = x.copy()
        v[0] += sgn * alpha
        vnorm2 = v @ v
        if vnorm2 > 0.0:
            R[j:, j:] -= np.outer(v, (2.0 / vnorm2) * (v @ R[j:, j:]))
        R[j + 1:, j] = 0.0
        k = j + 1
    R1 = R[:k, :k]
    R2 = R[:k, k:]
    T = solve_triangular(R1, R2, lower=False) if k > 0 else np.zeros((0, n))
    sk = perm[:k].copy()
    rd_unsorted = perm[k:].copy()
    order = np.argsort(rd_unsorted, kind="stable")
    rd = rd_unsorted[order]
    T = T[:, order]
    return sk, rd, T


def norm2_estimate(Y: np.ndarray, iters: int = 8) -> float:
    """Estimate of |Y|_2 by ``iters`` power iterations on Y^T Y from the
    normalized all-ones vector; returns |Y v| for the final iterate v.
    Used for rho_g = min(1, |Y^K_g| / |Y^S_g|) (Sec. 4.4)."""
    Y = np.asarray(Y, dtype=np.float64)
    n = Y.shape[1]
    if n == 0 or Y.shape[0] == 0:
        return 0.0
    v = np.ones(n) / np.sqrt(n)
    for _ in range(iters):
        w = Y.T @ (Y @ v)
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        v = w / nw
    return float(np.linalg.norm(Y @ v))
