"""Iterative solvers and error estimates (oracle; test infrastructure).

* GMRES (Saad & Schultz) with right preconditioning, restart ``restart``,
  modified Gram-Schmidt Arnoldi in FP64, stopped on the true relative residual
  |f - A u| / |f| (Sec. 5 uses F^{-1} as the preconditioner; Lemma 5.1 and
  Corollary 5.2 bound the iteration count).
* Iterative refinement u <- u + F^{-1}(f - A u).
* e_a ~ |A - F| / |A| and e_s ~ |I - A F^{-1}| by power iteration from a
  standard uniform start vector, stopped at 1e-2 relative change (Sec. 5).
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, f, precond=None, tol=1e-10, restart=20, maxit=200, x0=None):
    """Right-preconditioned restarted GMRES for A u = f (one right-hand side).

    Returns (u, iterations, relative residual history)."""
    f = np.asarray(f, dtype=np.float64)
    M = precond if precond is not None else (lambda v: v)
    u = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    fnorm = np.linalg.norm(f)
    if fnorm == 0.0:
        return u, 0, [0.0]
    hist = []
    its = 0
    r = f - matvec(u)
    beta = np.linalg.norm(r)
    hist.append(beta / fnorm)
    while its < maxit and beta / fnorm > tol:
        m = restart
        V = np.zeros((f.size, m + 1))
        Z = np.zeros((f.size, m))
        H = np.zeros((m + 1, m))
        V[:, 0] = r / beta
        g = np.zeros(m + 1)
        g[0] = beta
        cs = np.zeros(m)
        sn = np.zeros(m)
        j_done = 0
        for j in range(m):
            Z[:, j] = M(V[:, j])
            wv = matvec(Z[:, j])
            for i in range(j + 1):                 # modified Gram-Schmidt
                H[i, j] = V[:, i] @ wv
                wv = wv - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(wv)
            if H[j + 1, j] > 0.0:
                V[:, j + 1] = wv / H[j + 1, j]
            for i in range(j):                     # apply earlier Givens rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den if den > 0 else 1.0
            sn[j] = H[j + 1, j] / den if den > 0 else 0.0
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            if abs(g[j + 1]) / fnorm <= tol or its >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        u = u + Z[:, :j_done] @ y
        r = f - matvec(u)
        beta = np.linalg.norm(r)
        hist.append(beta / fnorm)
    return u, its, hist


def refine(matvec, f, solve, tol=1e-10, maxit=50):
    """Iterative refinement u_{k+1} = u_k + F^{-1}(f - A u_k)."""
    f = np.asarray(f, dtype=np.float64)
    u = solve(f)
    fn = np.linalg.norm(f)
    hist = []
    for it in range(maxit):
        r = f - matvec(u)
        rel = np.linalg.norm(r) / fn
        hist.append(rel)
        if rel <= tol:
            return u, it, hist
        u = u + solve(r)
    return u, maxit, hist


def power_norm(apply_op, apply_op_t, N, seed=0, rtol=1e-2, maxit=200, v0=None, return_iters=False):
    """|E|_2 by power iteration on E^T E from a standard uniform start (Sec. 5).

    v <- v / |v|; each step w = E^T E v, estimate sqrt(|w|), v = w / |w|; stop
    when the estimate moved by at most rtol of itself.  ``v0`` replaces the
    seeded start vector when given."""
    if v0 is None:
        rng = np.random.default_rng(seed)
        v = rng.uniform(size=N)
    else:
        v = np.array(v0, dtype=np.float64)
    v /= np.linalg.norm(v)
    est = 0.0
    it = 0
    for it in range(1, maxit + 1):
        w = apply_op_t(apply_op(v))
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return (0.0, it) if return_iters else 0.0
        new = np.sqrt(nw)
        v = w / nw
        if est > 0.0 and abs(new - est) <= rtol * new:
            return (new, it) if return_iters else new
        est = new
    return (est, it) if return_iters else est


def error_estimates(A_mv, At_mv, F_mv, Ft_mv, Fi_mv, Fit_mv, N, seed=0, v0=None, rtol=1e-2, maxit=200):
    """(e_a, e_s) of Sec. 5: |A - F| / |A| and |I - A F^{-1}|."""
    kw = dict(seed=seed, v0=v0, rtol=rtol, maxit=maxit)
    nA = power_norm(A_mv, At_mv, N, **kw)
    nE = power_norm(lambda v: A_mv(v) - F_mv(v), lambda v: At_mv(v) - Ft_mv(v), N, **kw)
    nS = power_norm(lambda v: v - A_mv(Fi_mv(v)), lambda v: v - Fit_mv(At_mv(v)), N, **kw)
    return nE / nA, nS
