"""First-kind problems (Example 1: a = 0, b = c = 1), the RSF ablation
(Algorithm 3.1: cells only) and the a posteriori error estimates e_a, e_s of
Sec. 5, on the GPU through the C ABI, against the oracle.

The power iterations run on the GPU with the direct sum for A and the
factored form for F; the oracle runs the same iteration on the dense A and on
the GPU's own F made dense column by column, from the same start vector, so
the two must agree to rounding, step for step.
"""
import numpy as np
import pytest
import torch

import hif_inputs as hi
from oracle import dense, kernels, krylov

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


def factor(P, pb, eps, **kw):
    return P.Factorization(T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c), pb.kernel_id, eps,
                           proxy_dirs=pb.proxy if pb.dim == 3 else None, **kw)


def dense_of(fn, N):
    return fn(T(np.eye(N, order="F"))).cpu().numpy()


@pytest.mark.parametrize("direct", ["tc", "fp64"])
def test_error_estimates_match_oracle_power_iteration(P, direct):
    pb = hi.volume_problem(32, 2, a_value=0.0)
    N = pb.N
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    A = op.dense()
    fac = factor(P, pb, 1e-4, direct=direct)
    Fd = dense_of(fac.apply, N)
    Ftd = dense_of(fac.apply_transpose, N)
    Fi = dense_of(fac.solve, N)
    Fit = dense_of(fac.solve_transpose, N)
    v0 = hi.uniform_vector(N, 3)
    est = fac.error_estimates(T(v0))
    assert est["converged"]
    kw = dict(v0=v0, return_iters=True)
    ref = [krylov.power_norm(lambda v: A @ v, lambda v: A.T @ v, N, **kw),
           krylov.power_norm(lambda v: A @ v - Fd @ v, lambda v: A.T @ v - Ftd @ v, N, **kw),
           krylov.power_norm(lambda v: v - A @ (Fi @ v), lambda v: v - Fit @ (A.T @ v), N, **kw)]
    got = [est["norm_A"], est["norm_E"], est["e_s"]]
    for (r, its), g, gi in zip(ref, got, est["iters"]):
        assert gi == its
        assert abs(g - r) <= 1e-8 * r
    # and from below, within the paper's 1e-2 stopping rule, of the exact norms
    ex_a = np.linalg.norm(A - Fd, 2) / np.linalg.norm(A, 2)
    ex_s = np.linalg.norm(np.eye(N) - A @ Fi, 2)
    assert 0.8 * ex_a <= est["e_a"] <= 1.01 * ex_a
    assert 0.8 * ex_s <= est["e_s"] <= 1.01 * ex_s
    fac.close()


@pytest.mark.parametrize("eps,ni_max", [(1e-3, 10), (1e-6, 5), (1e-9, 3)])
def test_first_kind_gmres_iterations(P, eps, ni_max):
    # Example 1 on the n = 64 grid: e_a = O(eps), e_s much larger, and GMRES
    # with F^{-1} as preconditioner reaches 1e-12 in a few steps from a
    # uniform random right-hand side
    pb = hi.volume_problem(64, 2, a_value=0.0)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    ds = dense.DenseSolver(op)
    fac = factor(P, pb, eps)
    est = fac.error_estimates(T(hi.uniform_vector(pb.N, 3)))
    assert est["e_a"] <= 10 * eps and est["e_s"] >= 10 * est["e_a"]
    f = hi.uniform_vector(pb.N, 5)
    u, its, rel = fac.solve_refined(T(f), tol=1e-12, method="gmres")
    assert rel <= 1e-12 and its <= ni_max
    ud = ds.solve(f)
    assert np.linalg.norm(u.cpu().numpy() - ud) <= 1e-8 * np.linalg.norm(ud)
    fac.close()


def test_rsf_ablation_top_block(P):
    # Algorithm 3.1 (fractional levels off) against HIF-IE on the same
    # first-kind problem: cells only, a larger top block, the same accuracy
    eps = 1e-6
    pb = hi.volume_problem(64, 2, a_value=0.0)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    ds = dense.DenseSolver(op)
    hif = factor(P, pb, eps)
    rsf = factor(P, pb, eps, fractional=False)
    sh, sr = hif.stats(), rsf.stats()
    assert all(s["kind"] == "cell" for s in sr["per_sublevel"])
    assert any(s["kind"] == "edge" for s in sh["per_sublevel"])
    assert sr["top_size"] > 1.2 * sh["top_size"]
    f = hi.uniform_vector(pb.N, 5)
    ud = ds.solve(f)
    for fac in (hif, rsf):
        u, its, rel = fac.solve_refined(T(f), tol=1e-12, method="gmres")
        assert rel <= 1e-12 and its <= 5
        assert np.linalg.norm(u.cpu().numpy() - ud) <= 1e-8 * np.linalg.norm(ud)
        est = fac.error_estimates(T(hi.uniform_vector(pb.N, 3)))
        assert est["e_a"] <= 10 * eps
    hif.close()
    rsf.close()


def test_error_estimates_argument_errors(P):
    from paper_1307_2666_gb300 import hif as H
    pb = hi.volume_problem(16, 2)
    fac = factor(P, pb, 1e-6)
    with pytest.raises(H.HIFError) as err:
        fac.error_estimates(T(np.zeros(pb.N)))
    assert err.value.status == H.HIF_EINVAL
    norms, its, conv = H.hif_error_estimates(fac.h, T(hi.uniform_vector(pb.N, 1)), 1e-12, 2)
    assert not conv and its == (2, 2, 2) and all(np.isfinite(norms))
    fac.close()
