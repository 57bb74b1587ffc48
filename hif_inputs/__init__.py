"""Seeded synthetic inputs for the HIF-IE volume integral equations.

This module is shared, as data only, by the CPU oracle and by the GPU library's
callers (tests, bench).  It holds none of the factorization's arithmetic: it
only lays out collocation points, draws coefficient fields and right-hand
sides, and supplies the proxy-surface directions that the method draws at
random (Sec. 3.3: a circle of 64 uniform points in 2D, 512 normalized Gaussian
vectors on the sphere in 3D).

Every generator uses numpy's PCG64 ``default_rng`` with an explicit seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "grid_points",
    "smooth_field",
    "gaussian_rhs",
    "proxy_directions",
    "Problem",
    "volume_problem",
    "batched_sizes",
    "helmholtz_problem",
]


def grid_points(n: int, dim: int) -> tuple[np.ndarray, np.ndarray]:
    """Cell centres of the uniform n^dim grid on the unit square/cube (Sec. 3.1).

    Returns ``(points, weights)``: points is N x dim row-major FP64 with
    x_j = h (j - 1/2) per coordinate, j = 1..n; weights are the cell volumes
    h^dim.  DOF order: the first coordinate varies slowest.
    """
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    h = 1.0 / n
    g = (np.arange(n, dtype=np.float64) + 0.5) * h
    mesh = np.meshgrid(*([g] * dim), indexing="ij")
    pts = np.stack([m.reshape(-1) for m in mesh], axis=1).copy()
    w = np.full(pts.shape[0], h**dim, dtype=np.float64)
    return pts, w


def smooth_field(points: np.ndarray, seed: int, terms: int = 16, kmax: int = 4) -> np.ndarray:
    """phi(x) = (1/terms) sum_j cos(2 pi k_j . x + theta_j), values in [-1, 1].

    k_j are integer wave vectors drawn uniformly from {-kmax..kmax}^dim minus
    the zero vector, theta_j ~ U[0, 2 pi).  Coefficient fields are then
    b = c = 1 + 0.5 phi, which stay inside [0.5, 1.5].
    """
    rng = np.random.default_rng(seed)
    dim = points.shape[1]
    ks = []
    while len(ks) < terms:
        k = rng.integers(-kmax, kmax + 1, size=dim)
        if np.any(k != 0):
            ks.append(k)
    ks = np.asarray(ks, dtype=np.float64)
    theta = rng.uniform(0.0, 2.0 * math.pi, size=terms)
    phase = 2.0 * math.pi * (points @ ks.T) + theta[None, :]
    return np.cos(phase).sum(axis=1) / terms


def gaussian_rhs(N: int, nrhs: int, seed: int) -> np.ndarray:
    """N x nrhs standard normal right-hand sides, column-major (Fortran order)."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((N, nrhs)))


def uniform_vector(N: int, seed: int) -> np.ndarray:
    """N standard uniform values on [0, 1): the start vector of the power
    iterations and the right-hand side of the first-kind GMRES runs."""
    return np.random.default_rng(seed).uniform(size=N)


def proxy_directions(dim: int, count: int | None = None, seed: int = 7) -> np.ndarray:
    """Unit vectors of the proxy surface (Sec. 3.3).

    2D: ``count`` (default 64) equispaced angles 2 pi k / count.
    3D: ``count`` (default 512) standard normal vectors, normalized, from ``seed``.
    Returned as count x dim row-major FP64.
    """
    if dim == 2:
        P = 64 if count is None else count
        t = 2.0 * math.pi * np.arange(P, dtype=np.float64) / P
        return np.stack([np.cos(t), np.sin(t)], axis=1).copy()
    if dim == 3:
        P = 512 if count is None else count
        rng = np.random.default_rng(seed)
        g = rng.standard_normal((P, 3))
        return g / np.linalg.norm(g, axis=1, keepdims=True)
    raise ValueError("dim must be 2 or 3")


@dataclass
class Problem:
    """One discretized volume IE a u + b K(c u) = f on a uniform grid."""

    n: int
    dim: int
    kernel_id: int  # 0: -log(r)/(2 pi) (2D), 1: 1/(4 pi r) (3D)
    points: np.ndarray
    weights: np.ndarray
    a: np.ndarray
    b: np.ndarray
    c: np.ndarray
    f: np.ndarray
    proxy: np.ndarray = field(default=None)

    @property
    def N(self) -> int:
        return self.points.shape[0]


def volume_problem(n: int, dim: int = 2, *, smooth_seed: int | None = None,
                   rhs_seed: int = 1001, nrhs: int = 1, proxy_seed: int = 7,
                   a_value: float = 1.0) -> Problem:
    """Second-kind volume IE on the unit square (dim 2) or cube (dim 3).

    a = a_value; b = c = 1 when ``smooth_seed`` is None, otherwise
    b = c = 1 + 0.5 phi with phi = smooth_field(points, smooth_seed).
    """
    pts, w = grid_points(n, dim)
    N = pts.shape[0]
    if smooth_seed is None:
        bc = np.ones(N)
    else:
        bc = 1.0 + 0.5 * smooth_field(pts, smooth_seed)
    a = np.full(N, float(a_value))
    f = gaussian_rhs(N, nrhs, rhs_seed)
    return Problem(n=n, dim=dim, kernel_id=0 if dim == 2 else 1, points=pts, weights=w,
                   a=a, b=bc.copy(), c=bc.copy(), f=f, proxy=proxy_directions(dim, seed=proxy_seed))


def helmholtz_problem(n: int, kappa: float, *, rhs_seed: int = 1101, nrhs: int = 1) -> Problem:
    """Lippmann-Schwinger scattering on the unit square (Sec. 5, Example 3).

    Wavenumber k = 2 pi kappa (kappa wavelengths across the domain), scatterer
    omega(x) = exp(-32 |x - (1/2, 1/2)|^2), a = 1 and b = c = k sqrt(omega);
    the kernel (kernel_id 2) is (i/4) H_0^(1)(k r).  Right-hand sides are
    complex with independent standard normal real and imaginary parts.
    """
    pts, w = grid_points(n, 2)
    N = pts.shape[0]
    k = 2.0 * math.pi * kappa
    d = pts - 0.5
    omega = np.exp(-32.0 * (d * d).sum(axis=1))
    bc = k * np.sqrt(omega)
    rng = np.random.default_rng(rhs_seed)
    f = np.asfortranarray(rng.standard_normal((N, nrhs)) + 1j * rng.standard_normal((N, nrhs)))
    pb = Problem(n=n, dim=2, kernel_id=2, points=pts, weights=w, a=np.ones(N), b=bc.copy(), c=bc.copy(), f=f,
                 proxy=proxy_directions(2))
    pb.k = k
    return pb


def batched_sizes(P: int, seed: int, choices=tuple(range(32, 257, 16))) -> list[int]:
    """Grid sizes n_p drawn uniformly from ``choices`` (default {32, 48, ..., 256})."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, len(choices), size=P)
    return [int(choices[i]) for i in idx]
