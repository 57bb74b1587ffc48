"""Helmholtz (Lippmann-Schwinger, Sec. 5 Example 3) on the GPU, through the C ABI.

The library factors the real 2 x 2 embedding of the complex operator
(kernel_id 2); complex vectors go in and out as complex tensors.  Checked
against the oracle's complex operator: the direct sum and its adjoint element
by element, apply <= 10 eps and solve <= 100 eps against the complex dense
solve, the adjoint solve, refined solves to 1e-10 from FP64 and FP32
factorizations, and skeleton totals within 10% of the oracle's HIF-IE on the
same embedding.
"""
import numpy as np
import pytest
import torch

import hif_inputs as hi
from oracle import helmholtz as hz, hifie

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
    return torch.as_tensor(np.ascontiguousarray(v), device=DEV)


def factor(P, pb, eps, **kw):
    return P.Factorization(T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c), 2, eps, wavenumber=pb.k, **kw)


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def ls32():
    pb = hi.helmholtz_problem(32, 2.0, nrhs=2)
    cop = hz.HelmholtzOperator(pb.points, pb.weights, pb.a, pb.b, pb.c, pb.k)
    return pb, cop, cop.dense()


def test_direct_sum_and_adjoint_match_oracle(P, ls32):
    pb, cop, A = ls32
    fac = factor(P, pb, 1e-3)
    X = pb.f
    Y = fac.matvec(T(X)).cpu().numpy()
    np.testing.assert_allclose(Y, A @ X, rtol=0, atol=1e-12 * np.abs(A @ X).max())
    Yh = fac.matvec(T(X), trans=True).cpu().numpy()
    np.testing.assert_allclose(Yh, A.conj().T @ X, rtol=0, atol=1e-12 * np.abs(A @ X).max())
    fac.close()


@pytest.mark.parametrize("eps", [1e-3, 1e-6])
def test_factorization_accuracy_against_complex_dense(P, ls32, eps):
    pb, cop, A = ls32
    fac = factor(P, pb, eps)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(pb.N) + 1j * rng.standard_normal(pb.N)
    assert relerr(fac.apply(T(x)).cpu().numpy(), A @ x) <= 10 * eps
    f = pb.f[:, 0]
    assert relerr(fac.solve(T(f)).cpu().numpy(), np.linalg.solve(A, f)) <= 100 * eps
    # the transposed solve of the real embedding is the complex adjoint solve
    assert relerr(fac.solve_transpose(T(f)).cpu().numpy(), np.linalg.solve(A.conj().T, f)) <= 100 * eps
    # multi-RHS equal to column by column
    U = fac.solve(T(pb.f)).cpu().numpy()
    np.testing.assert_allclose(U[:, 1], fac.solve(T(pb.f[:, 1])).cpu().numpy(), rtol=1e-13, atol=1e-15)
    # skeleton totals against the oracle on the same embedding
    Fo = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 2, eps, pb.proxy, wavenumber=pb.k)
    st = fac.stats()
    for s, sl in zip(st["per_sublevel"], Fo.sublevels):
        ko = sum(b.sk.size for b in sl.boxes)
        assert abs(s["skeletons"] - ko) <= 0.1 * ko + 2
    assert abs(st["top_size"] - Fo.sL) <= 0.1 * Fo.sL + 2
    fac.close()


@pytest.mark.parametrize("precision,method", [("fp64", "gmres"), ("fp32", "ir"), ("fp32", "gmres")])
def test_refined_solve_to_1e10(P, ls32, precision, method):
    pb, cop, A = ls32
    fac = factor(P, pb, 1e-6, precision=precision)
    u, its, rel = fac.solve_refined(T(pb.f), tol=1e-10, method=method)
    assert rel <= 1e-10
    ud = np.linalg.solve(A, pb.f)
    assert relerr(u.cpu().numpy(), ud) <= 1e-8
    r = pb.f - A @ u.cpu().numpy()
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(pb.f) * 1.01
    fac.close()


def test_higher_frequency_preconditioner(P):
    # kappa = 4 wavelengths across the n = 64 grid (16 points per wavelength):
    # F^{-1} preconditions GMRES to a few iterations (Sec. 5, Example 3)
    pb = hi.helmholtz_problem(64, 4.0)
    fac = factor(P, pb, 1e-6)
    u, its, rel = fac.solve_refined(T(pb.f), tol=1e-10, method="gmres")
    assert rel <= 1e-10 and its <= 6
    cop = hz.HelmholtzOperator(pb.points, pb.weights, pb.a, pb.b, pb.c, pb.k)
    rows = np.random.default_rng(7).choice(pb.N, 16, replace=False)
    r = pb.f[rows, 0] - cop.entries(rows, np.arange(pb.N)) @ u.cpu().numpy()[:, 0]
    assert np.sqrt(pb.N / 16) * np.linalg.norm(r) <= 3e-10 * np.linalg.norm(pb.f)
    fac.close()
