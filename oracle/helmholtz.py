"""The Lippmann-Schwinger operator of Sec. 5, Example 3 (oracle; test infrastructure).

The equation u + k sqrt(w) int K(|x - y|) [k sqrt(w)] u dy = sqrt(w) f on the
unit square is the integral equation of Eq. (1.1) with a = 1 and
b = c = k sqrt(omega), where K(r) = (i/4) H_0^(1)(k r) is the fundamental
solution of the Helmholtz equation with the Sommerfeld condition and omega is
the scatterer.  The discretization is that of the volume examples (Sec. 3.1,
Eq. (3.1); quadrature of Sec. 5): collocation at cell centres x_j with cell
areas w_j,

    A_ij = a_i delta_ij + b_i K_ij c_j,   K_ij = G(|x_i - x_j|) w_j (i != j),
    K_ii = integral of G over the cell of x_i,

a complex symmetric matrix when b = c and the weights are equal.

The factorization works over the reals through the 2 x 2 embedding of every
complex entry z = x + i y as [[x, -y], [y, x]]: DOF j becomes the two real DOFs
2j (real part) and 2j + 1 (imaginary part) at the same point, and a complex
vector is its interleaved real form.  The embedding maps a product of complex
matrices to the product of their embeddings and the conjugate transpose to
the real transpose, so the HIF-IE of the real operator (Sec. 4; Lemma 2.4 with
real transposes) is a factorization of the complex operator, and its
transposed solve is the complex adjoint solve.

Hankel function: scipy.special.hankel1 (a library routine).  Self term:
G's integral over the square in polar coordinates about the centre,
8 int_0^{pi/4} int_0^{h / (2 cos t)} G(r) r dr dt, by adaptive quadrature
(the integrand r G(r) ~ r log r is integrable and continuous).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.integrate as si
import scipy.special as ss

from .kernels import Operator


def green_helmholtz(k: float, r) -> np.ndarray:
    """G(r) = (i / 4) H_0^(1)(k r) (Sec. 5, Example 3)."""
    return 0.25j * ss.hankel1(0, k * np.asarray(r, dtype=np.float64))


def self_integral_helmholtz(k: float, h: float) -> complex:
    """Integral of G over the square of side h centred at the singularity."""
    def part(fn):
        def inner(t):
            R = 0.5 * h / math.cos(t)
            return si.quad(lambda r: fn(r) * r, 0.0, R, limit=200, epsabs=0.0, epsrel=1e-13)[0]
        return 8.0 * si.quad(inner, 0.0, 0.25 * math.pi, limit=200, epsabs=0.0, epsrel=1e-13)[0]
    re = part(lambda r: -0.25 * ss.y0(k * r))
    im = part(lambda r: 0.25 * ss.j0(k * r))
    return complex(re, im)


class HelmholtzOperator:
    """The complex N x N operator A = diag(a) + diag(b) K diag(c)."""

    def __init__(self, points, weights, a, b, c, k):
        self.x = np.ascontiguousarray(points, dtype=np.float64)
        self.w = np.asarray(weights, dtype=np.float64)
        self.a = np.asarray(a, dtype=np.float64)
        self.b = np.asarray(b, dtype=np.float64)
        self.c = np.asarray(c, dtype=np.float64)
        self.k = float(k)
        self.N, self.dim = self.x.shape
        if self.dim != 2:
            raise ValueError("the Helmholtz kernel is two-dimensional")
        cache = {}
        ks = np.empty(self.N, dtype=np.complex128)
        for i, wi in enumerate(self.w):
            key = float(wi)
            if key not in cache:
                cache[key] = self_integral_helmholtz(self.k, math.sqrt(key))
            ks[i] = cache[key]
        self.kself = ks

    def kernel_entries(self, rows, cols) -> np.ndarray:
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        d = self.x[rows][:, None, :] - self.x[cols][None, :, :]
        r = np.sqrt((d * d).sum(axis=2))
        same = rows[:, None] == cols[None, :]
        K = green_helmholtz(self.k, np.where(same, 1.0, r)) * self.w[cols][None, :]
        if same.any():
            K = np.where(same, self.kself[rows][:, None], K)
        return self.b[rows][:, None] * K * self.c[cols][None, :]

    def entries(self, rows, cols) -> np.ndarray:
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        out = self.kernel_entries(rows, cols)
        same = rows[:, None] == cols[None, :]
        return out + np.where(same, self.a[rows][:, None], 0.0)

    def dense(self) -> np.ndarray:
        idx = np.arange(self.N)
        return self.entries(idx, idx)

    def matvec(self, x, adjoint: bool = False, block: int = 512) -> np.ndarray:
        """y = A x (or A^H x), row block by row block."""
        x = np.asarray(x, dtype=np.complex128)
        X = x[:, None] if x.ndim == 1 else x
        Y = np.empty_like(X)
        idx = np.arange(self.N)
        for s in range(0, self.N, block):
            rows = idx[s:s + block]
            Y[rows] = (self.entries(idx, rows).conj().T if adjoint else self.entries(rows, idx)) @ X
        return Y[:, 0] if x.ndim == 1 else Y


def embed_matrix(Z: np.ndarray) -> np.ndarray:
    """Real 2 x 2 embedding of a complex matrix (rows 2i + a, columns 2j + b)."""
    m, n = Z.shape
    E = np.empty((2 * m, 2 * n))
    E[0::2, 0::2] = Z.real
    E[0::2, 1::2] = -Z.imag
    E[1::2, 0::2] = Z.imag
    E[1::2, 1::2] = Z.real
    return E


def to_real(v) -> np.ndarray:
    """Interleaved real form of a complex vector or block of vectors."""
    v = np.asarray(v, dtype=np.complex128)
    out = np.empty((2 * v.shape[0],) + v.shape[1:])
    out[0::2] = v.real
    out[1::2] = v.imag
    return out


def to_complex(v) -> np.ndarray:
    v = np.asarray(v, dtype=np.float64)
    return v[0::2] + 1j * v[1::2]


class EmbeddedOperator(Operator):
    """The real 2N x 2N embedding of a HelmholtzOperator, with the interface
    of kernels.Operator (entries on demand, dense, matvec), so that the
    sequential HIF-IE runs on it unchanged.  Points, weights and coefficients
    are repeated for the two components of every DOF."""

    def __init__(self, points, weights, a, b, c, k):
        self.cop = HelmholtzOperator(points, weights, a, b, c, k)
        rep = lambda v: np.repeat(np.asarray(v, dtype=np.float64), 2, axis=0)
        self.x = rep(self.cop.x)
        self.w = rep(self.cop.w)
        self.a = rep(self.cop.a)
        self.b = rep(self.cop.b)
        self.c = rep(self.cop.c)
        self.kernel_id = 2
        self.k = self.cop.k
        self.N, self.dim = self.x.shape
        self.kself = None

    def kernel_entries(self, rows, cols) -> np.ndarray:
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        Z = self.cop.kernel_entries(rows // 2, cols // 2)
        ra = (rows % 2)[:, None]
        cb = (cols % 2)[None, :]
        # [[Re, -Im], [Im, Re]] picked by (row component, column component)
        return np.where(ra == cb, Z.real, np.where(ra == 1, Z.imag, -Z.imag))

    def proxy_out(self, xE, cols) -> np.ndarray:
        """Rows (e, component) of the outgoing proxy block Y_{cE,c} (Lemma 3.3):
        the entries G(|x^E_e - x_j|) w_j c_j, embedded."""
        cols = np.asarray(cols, dtype=np.int64)
        d = xE[:, None, :] - self.x[cols][None, :, :]
        Z = green_helmholtz(self.k, np.sqrt((d * d).sum(axis=2))) * (self.w[cols] * self.c[cols])[None, :]
        return _embed_rows(Z, cols % 2)

    def proxy_in(self, xE, cols) -> np.ndarray:
        """Rows (e, component) of (A_{c,cE})^T for the incoming proxy block,
        A_{j,e} = b_j G(|x_j - x^E_e|) w_j, embedded and transposed."""
        cols = np.asarray(cols, dtype=np.int64)
        d = xE[:, None, :] - self.x[cols][None, :, :]
        Z = green_helmholtz(self.k, np.sqrt((d * d).sum(axis=2))) * (self.b[cols] * self.w[cols])[None, :]
        # the embedding of A_{c,cE} has block(z)[b][a] at (2j + b, 2e + a);
        # row (e, a) of its transpose: a = 0 -> (Re, Im), a = 1 -> (-Im, Re)
        # for column component b = 0, 1
        cb = (cols % 2)[None, :]
        out = np.empty((2 * Z.shape[0], Z.shape[1]))
        out[0::2] = np.where(cb == 0, Z.real, Z.imag)
        out[1::2] = np.where(cb == 0, -Z.imag, Z.real)
        return out


def _embed_rows(Z: np.ndarray, ccomp: np.ndarray) -> np.ndarray:
    """Rows (e, a) of the embedding of a complex block Z (P x n) whose columns
    are already real DOFs of component ccomp: block(z)[a][b]."""
    P, n = Z.shape
    E = np.empty((2 * P, n))
    cb = ccomp[None, :]
    E[0::2] = np.where(cb == 0, Z.real, -Z.imag)
    E[1::2] = np.where(cb == 0, Z.imag, Z.real)
    return E
