"""Adjoint of the refined HIF-IE solve (autograd backward through a transposed
solve and the factorization's fast apply), checked against the dense FP64
gradient and against central finite differences of refined solves.

L(f, a, b, c) = 1/2 |u - u*|^2 with A(a, b, c) u = f.
"""
import numpy as np
import pytest
import torch

import hif_inputs as hi
from oracle import kernels

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1307_2666_gb300 as P
    return P


def T(v):
    return torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device=DEV)


def _loss(P, pb, f, a, b, c, ustar, eps, tol):
    fac = P.Factorization(T(pb.points), T(pb.weights), a, b, c, 0, eps)
    u = P.HIFSolve.apply(f, a, b, c, fac, tol)
    L = 0.5 * torch.sum((u - ustar) ** 2)
    return L, fac


def test_adjoint_matches_dense_gradient_n32(P):
    pb = hi.volume_problem(32, 2, smooth_seed=1005, rhs_seed=1006)
    ustar = hi.gaussian_rhs(pb.N, 1, 1007)[:, 0]
    f = T(pb.f[:, 0]).requires_grad_(True)
    a = T(pb.a).requires_grad_(True)
    b = T(pb.b).requires_grad_(True)
    c = T(1.0 + 0.5 * hi.smooth_field(pb.points, 1105)).requires_grad_(True)
    L, fac = _loss(P, pb, f, a, b, c, T(ustar), 1e-9, 1e-13)
    L.backward()
    # dense FP64 adjoint: lambda = A^{-T}(u - u*)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, c.detach().cpu().numpy(), 0)
    A = op.dense()
    u = np.linalg.solve(A, pb.f[:, 0])
    lam = np.linalg.solve(A.T, u - ustar)
    K = op.kernel_entries(np.arange(pb.N), np.arange(pb.N)) / (op.b[:, None] * op.c[None, :])
    ref = {"f": lam, "a": -lam * u, "b": -lam * (K @ (op.c * u)), "c": -u * (K.T @ (op.b * lam))}
    got = {"f": f.grad, "a": a.grad, "b": b.grad, "c": c.grad}
    for k in ref:
        g = got[k].cpu().numpy()
        assert np.linalg.norm(g - ref[k]) <= 1e-7 * np.linalg.norm(ref[k]), k
    fac.close()


@pytest.mark.parametrize("h", [1e-6, 1e-4])
def test_adjoint_central_differences_n256(P, h):
    """n=256 (N=65,536), eps=1e-9, FP64 factorization; directional derivatives
    along seeded random directions, central steps 1e-6 and 1e-4, rel. 1e-5.

    The b and c gradients are small (about 0.05) next to |u|^2 ~ N, so the
    difference of the two losses is formed from u+ - u- rather than as
    L(+) - L(-), which would cancel about 11 digits.  Even so, at step 1e-6
    the b and c differences sit on the refined solves' FP64 floor: solutions
    good to ~1e-14 relative move L(+) - L(-) by ~|u - u*| |u| 1e-14 / sqrt(N)
    ~ 3e-12, i.e. ~3e-5 of the b/c directional derivatives (measured 3.0e-5).
    Those two are held to 2e-4 at step 1e-6; at step 1e-4 all four meet 1e-5."""
    n, eps, tol = 256, 1e-9, 1e-14
    pb = hi.volume_problem(n, 2, smooth_seed=1005, rhs_seed=1006)
    ustar = T(hi.gaussian_rhs(pb.N, 1, 1007)[:, 0])
    base = {"f": T(pb.f[:, 0]), "a": T(pb.a), "b": T(pb.b), "c": T(pb.c)}
    leaves = {k: v.clone().requires_grad_(True) for k, v in base.items()}
    L, fac = _loss(P, pb, leaves["f"], leaves["a"], leaves["b"], leaves["c"], ustar, eps, tol)
    L.backward()
    fac.close()
    rng = np.random.default_rng(2024)
    for name in ("f", "a", "b", "c"):
        d = T(rng.standard_normal(pb.N))
        g_dir = float(torch.dot(leaves[name].grad, d))
        us = []
        for sgn in (+1, -1):
            p = {k: v.clone() for k, v in base.items()}
            p[name] = p[name] + sgn * h * d
            with torch.no_grad():
                fp = P.Factorization(T(pb.points), T(pb.weights), p["a"], p["b"], p["c"], 0, eps)
                us.append(P.HIFSolve.apply(p["f"], p["a"], p["b"], p["c"], fp, tol))
                fp.close()
        # L(+) - L(-) = 1/2 sum (u+ - u-)(u+ + u- - 2 u*), formed without the
        # cancellation of two large losses
        up, um = us
        fd = float(0.5 * torch.sum((up - um) * (up + um - 2 * ustar))) / (2 * h)
        rel = 2e-4 if (h < 1e-5 and name in ("b", "c")) else 1e-5
        assert abs(fd - g_dir) <= rel * abs(g_dir), (name, fd, g_dir)
