"""torch-facing wrappers of the C ABI: one factorization handle per object,
and the autograd function of the adjoint method.  Argument marshalling only;
the arithmetic runs in the library's kernels."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import hif as _h


def _colmajor(x: torch.Tensor) -> torch.Tensor:
    """View/copy of an (N,) or (N, nrhs) FP64 tensor in column-major layout."""
    if x.dtype != torch.float64:
        raise TypeError("vectors must be float64")
    if x.ndim == 1:
        return x.contiguous()
    if x.shape[1] == 1:
        return x.contiguous()
    if x.stride(0) == 1 and x.stride(1) >= x.shape[0]:
        return x
    return x.t().contiguous().t()


def _to_real(x: torch.Tensor) -> torch.Tensor:
    """A complex (N,) or (N, nrhs) tensor as its interleaved real form, the
    vectors of the real 2 x 2 embedding (2N,) or (2N, nrhs), column-major."""
    if x.ndim == 1:
        return torch.view_as_real(x.contiguous()).reshape(-1)
    return torch.view_as_real(x.t().contiguous()).reshape(x.shape[1], -1).t()


def _to_complex(y: torch.Tensor) -> torch.Tensor:
    if y.ndim == 1:
        return torch.view_as_complex(y.contiguous().reshape(-1, 2))
    return torch.view_as_complex(y.t().contiguous().reshape(y.shape[1], -1, 2)).t()


def _empty_like_cm(x: torch.Tensor) -> torch.Tensor:
    if x.ndim == 1:
        return torch.empty_like(x)
    return torch.empty((x.shape[1], x.shape[0]), dtype=x.dtype, device=x.device).t()


class Factorization:
    """HIF-IE factorization F ~ A of A = diag(a) + diag(b) K diag(c).

    points (N, dim), weights/a/b/c (N,) FP64 tensors (CUDA or CPU).
    precision: "fp64" or "fp32" (factorization precision; vectors stay FP64).
    direct: direct sum on uniform grids, "tc" (tensor cores on exact 8-bit
    digits), "df64" (paired FP32) or "fp64".
    graphs: replay the factored-form sweeps from captured CUDA graphs.
    autotune: pick each sublevel's sweep CTA size by timing after factoring.
    kernel_id 2: the Helmholtz kernel (i/4) H_0^(1)(k r) of Sec. 5, Example 3,
    with ``wavenumber`` k; a, b, c stay real, vectors are complex (complex128
    tensors), and the library works on the real 2 x 2 embedding of the
    complex operator; the transposed operations are the complex adjoints.
    symmetric: compress the one-sided Y'_c when b == c and the weights are
    equal (A symmetric; Sec. 5); False always compresses the full Y_c.
    ldl: with the symmetric shortcut, factor the diagonal blocks by LDL and
    keep X only (Sec. 5); False always uses LU with partial pivoting.
    """

    def __init__(self, points, weights, a, b, c, kernel_id: int, eps: float, *, precision: str = "fp64",
                 second_kind: bool = True, occupancy: int = 64, proxy_dirs=None, fractional: bool = True,
                 skip_levels: int = 0, proxy_radius: float = 1.5, fp32_tol_floor: float | None = None,
                 root=None, stream=None, direct: str = "tc", graphs: bool = True, autotune: bool = True,
                 symmetric: bool = True, ldl: bool = True, wavenumber: float | None = None):
        dim = (points[0][0] if isinstance(points, (list, tuple)) else points).shape[1]
        opt = _h.hif_options_default(dim)
        opt.leaf_occupancy = int(occupancy)
        opt.second_kind = 1 if second_kind else 0
        opt.precision = 0 if precision == "fp64" else 1
        opt.fractional_levels = 1 if fractional else 0
        opt.skip_levels = int(skip_levels)
        opt.proxy_radius = float(proxy_radius)
        opt.direct_precision = {"df64": 0, "fp64": 1, "tc": 2}[direct]
        opt.use_graphs = 1 if graphs else 0
        opt.autotune = 1 if autotune else 0
        opt.symmetric = 1 if symmetric else 0
        opt.ldl = 1 if ldl else 0
        if wavenumber is not None:
            opt.wavenumber = float(wavenumber)
        self.complex = kernel_id == 2
        self._keep = []
        if proxy_dirs is not None:
            pd = np.ascontiguousarray(np.asarray(proxy_dirs.cpu() if hasattr(proxy_dirs, "cpu") else proxy_dirs,
                                                 dtype=np.float64))
            self._keep.append(pd)
            opt.proxy_points = pd.shape[0]
            opt.proxy_dirs = pd.ctypes.data
        if fp32_tol_floor is not None:
            opt.fp32_tol_floor = float(fp32_tol_floor)
        if root is not None:
            lo, width = root
            for k in range(dim):
                opt.root_lo[k] = float(lo[k])
            opt.root_width = float(width)
        if stream is not None:
            opt.stream = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self.kernel_id = kernel_id
        self.eps = eps
        self.a, self.b, self.c = a, b, c
        if isinstance(points, (list, tuple)):
            # a batch of independent problems: points = [(points, weights, a, b, c), ...]
            probs = [tuple(t.contiguous() for t in pr) for pr in points]
            self._keep.append(probs)
            self.offsets = np.cumsum([0] + [pr[0].shape[0] for pr in probs])
            self.N, self.dim = int(self.offsets[-1]), probs[0][0].shape[1]
            self.device = probs[0][0].device
            self.h = _h.hif_factor_batched(probs, kernel_id, eps, opt)
            return
        self.N, self.dim = points.shape
        self.offsets = np.array([0, self.N])
        self.device = points.device if hasattr(points, "device") else torch.device("cpu")
        self.h = _h.hif_factor(points.contiguous(), weights.contiguous(), a.contiguous(), b.contiguous(),
                               c.contiguous(), kernel_id, eps, opt)

    @classmethod
    def batched(cls, problems, kernel_id: int, eps: float, **kw):
        """One handle over independent problems [(points, weights, a, b, c), ...];
        vectors are their concatenation (see ``offsets``)."""
        return cls(list(problems), None, None, None, None, kernel_id, eps, **kw)

    # -- factored operators ------------------------------------------------
    def _real_in(self, x):
        if self.complex:
            if not torch.is_complex(x):
                x = x.to(torch.complex128)
            return _to_real(x.to(torch.complex128))
        return x

    def _real_out(self, y):
        return _to_complex(y) if self.complex else y

    def _op(self, fn, x):
        xin = _colmajor(self._real_in(x))
        out = _empty_like_cm(xin)
        fn(self.h, xin, out)
        return self._real_out(out)

    def solve(self, b):
        return self._op(_h.hif_solve, b)

    def solve_transpose(self, b):
        return self._op(_h.hif_solve_transpose, b)

    def apply(self, x):
        return self._op(_h.hif_apply, x)

    def apply_transpose(self, x):
        return self._op(_h.hif_apply_transpose, x)

    def matvec(self, x, trans: bool = False, classes: int = 8):
        """A x (or A^T x) by the direct sum; classes 5 or 6 takes the short
        digit sets of the tensor-core sum (hif_matvec_digits)."""
        xin = _colmajor(self._real_in(x))
        out = _empty_like_cm(xin)
        if classes == 8:
            _h.hif_matvec(self.h, 1 if trans else 0, xin, out)
        else:
            _h.hif_matvec_digits(self.h, 1 if trans else 0, int(classes), xin, out)
        return self._real_out(out)

    def solve_refined(self, f, trans: bool = False, tol: float = 1e-10, maxit: int = 50, method: str = "ir"):
        fin = _colmajor(self._real_in(f))
        out = _empty_like_cm(fin)
        st, its, rel = _h.hif_solve_refined(self.h, 1 if trans else 0, fin, out, tol, maxit,
                                            0 if method == "ir" else 1)
        return self._real_out(out), its, rel

    def eliminated_dofs(self, sublevel: int):
        """numpy int32 array of the DOFs eliminated at a sublevel; the index
        ``stats()["sublevels"]`` is the top block."""
        return _h.hif_eliminated_dofs(self.h, sublevel)

    def adjoint_gradients(self, u, lam):
        """(dL/da, dL/db, dL/dc) of the adjoint method from the solution u
        and the adjoint solution lam = A^{-T} dL/du (same shape)."""
        uc = _colmajor(u)
        lc = _colmajor(lam)
        if uc.ndim == 2 and (uc.stride(1) != uc.shape[0] or lc.stride(1) != lc.shape[0]):
            uc = uc.t().contiguous().t()
            lc = lc.t().contiguous().t()
        N = uc.shape[0]
        ga, gb, gc = (torch.empty(N, dtype=torch.float64, device=uc.device) for _ in range(3))
        _h.hif_adjoint_gradients(self.h, uc, lc, ga, gb, gc)
        return ga, gb, gc

    def error_estimates(self, v0, rtol: float = 1e-2, maxit: int = 200) -> dict:
        """e_a ~ |A - F| / |A| and e_s ~ |I - A F^{-1}| (Sec. 5) by power
        iteration from the start vector v0 (N,)."""
        norms, its, conv = _h.hif_error_estimates(self.h, v0.contiguous() if hasattr(v0, "contiguous") else v0,
                                                  rtol, maxit)
        return {"e_a": norms[1] / norms[0], "e_s": norms[2], "norm_A": norms[0], "norm_E": norms[1],
                "iters": its, "converged": conv}

    def stats(self) -> dict:
        return _h.hif_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            _h.hif_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HIFSolve(torch.autograd.Function):
    """u = A^{-1} f through a refined solve with the factorization as
    preconditioner; backward is the adjoint method:

        lambda = A^{-T} g            (transposed refined solve)
        dL/df = lambda,  dL/da = -lambda * u,
        dL/db = -lambda * K(c u),     K(c u)     = (F u - a u) / b,
        dL/dc = -u * K^T(b lambda),   K^T(b l)   = (F^T lambda - a lambda) / c,

    with F the factorization's fast apply; the three coefficient gradients
    come from one library call (``hif_adjoint_gradients``).  ``fac`` must have been built from
    the same a, b, c."""

    @staticmethod
    def forward(ctx, f, a, b, c, fac: Factorization, tol: float = 1e-12):
        u, _, _ = fac.solve_refined(f, tol=tol)
        ctx.fac = fac
        ctx.tol = tol
        ctx.save_for_backward(u, a, b, c)
        return u

    @staticmethod
    def backward(ctx, g):
        u, a, b, c = ctx.saved_tensors
        fac = ctx.fac
        lam, _, _ = fac.solve_refined(g, trans=True, tol=ctx.tol)
        ga, gb, gc = fac.adjoint_gradients(u, lam)
        return lam, ga, gb, gc, None, None
