"""Batched factorization: independent problems of uneven size in one handle,
the boxes of each sublevel of all problems skeletonized in the same launches.

Each problem must come out as if it were factored alone: the same tree and
boxes go through the same kernels, but a sublevel's launch shape (rows per
proxy chunk, shared-memory staging) follows its largest box, so the rounding
of a small problem can change when it shares launches with a big one. FP64
results therefore agree to 1e-12 and FP32 results to the FP32 factorization's
accuracy. Each problem must also be accurate against its own dense FP64 solve,
and the handle's operator must be block diagonal.
"""
import numpy as np
import pytest
import torch

import hif_inputs as hi
from oracle import dense, kernels

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


def _problems(sizes, seed0=2000):
    pbs = []
    for q, n in enumerate(sizes):
        pb = hi.volume_problem(n, 2, smooth_seed=seed0 + q, rhs_seed=3000 + q, nrhs=2)
        pbs.append(pb)
    return pbs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_equals_individual_and_dense(P, precision):
    sizes = [16, 40, 24, 64, 32, 48]
    eps = 1e-6
    pbs = _problems(sizes)
    probs = [(T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c)) for pb in pbs]
    fb = P.Factorization.batched(probs, 0, eps, precision=precision)
    off = fb.offsets
    F = np.vstack([pb.f for pb in pbs])
    ub = fb.solve(T(F)).cpu().numpy()
    yb = fb.matvec(T(F)).cpu().numpy()
    tops = 0
    for q, pb in enumerate(pbs):
        fi = P.Factorization(*probs[q], 0, eps, precision=precision)
        ui = fi.solve(T(pb.f)).cpu().numpy()
        tops += fi.stats()["top_size"]
        if precision == "fp64":
            np.testing.assert_allclose(ub[off[q]:off[q + 1]], ui, rtol=1e-12, atol=1e-13)
        else:
            assert np.linalg.norm(ub[off[q]:off[q + 1]] - ui) <= 1e-4 * np.linalg.norm(ui)
        op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
        ud = dense.DenseSolver(op).solve(pb.f)
        bound = 100 * eps if precision == "fp64" else 1e-4
        assert np.linalg.norm(ub[off[q]:off[q + 1]] - ud) <= bound * np.linalg.norm(ud)
        # block diagonal direct sum
        np.testing.assert_allclose(yb[off[q]:off[q + 1]], op.matvec(pb.f), rtol=1e-12, atol=1e-13)
        fi.close()
    if precision == "fp64":
        assert fb.stats()["top_size"] == tops
    else:
        # FP32: the batched and the single-problem factorizations run
        # different launches (one plan for all problems), whose rounding
        # differs; a rank at the tolerance can move by one
        assert abs(fb.stats()["top_size"] - tops) <= max(2, 0.005 * tops)
    fb.close()


def test_batched_refined_solve_per_problem(P):
    sizes = [32, 48, 64, 80, 96]
    pbs = _problems(sizes, seed0=2100)
    probs = [(T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c)) for pb in pbs]
    fb = P.Factorization.batched(probs, 0, 1e-6, precision="fp32")
    off = fb.offsets
    F = np.vstack([pb.f for pb in pbs])
    F[off[1]:off[2]] *= 1e-6                 # a problem with a much smaller right-hand side
    u, its, rel = fb.solve_refined(T(F), tol=1e-10)
    assert rel <= 1e-10
    u = u.cpu().numpy()
    for q, pb in enumerate(pbs):
        op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
        fq = F[off[q]:off[q + 1]]
        r = fq - op.matvec(u[off[q]:off[q + 1]])
        assert np.linalg.norm(r, axis=0).max() <= 1e-10 * np.linalg.norm(fq, axis=0).min()
    fb.close()


def test_graphs_and_autotune_leave_results_unchanged(P):
    # the sweeps replayed from captured CUDA graphs with tuned CTA sizes give
    # bitwise the same solves and applies as plain launches at 256 threads,
    # and the launch counter still counts every kernel that ran
    from paper_1307_2666_gb300 import hif as H
    sizes = [24, 64, 40]
    pbs = _problems(sizes, seed0=2300)
    probs = [(T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c)) for pb in pbs]
    F = T(np.vstack([pb.f for pb in pbs]))
    outs, counts = [], []
    for graphs, tune in ((True, True), (False, False)):
        # FP64: the FP32 fold's autotuned rows per chunk would change the factor itself
        fb = P.Factorization.batched(probs, 0, 1e-6, precision="fp64", graphs=graphs, autotune=tune)
        res = []
        for _ in range(2):                         # the second call replays the captured graph
            l0 = H.hif_kernel_launches()
            res.append((fb.solve(F), fb.apply(F), fb.solve_transpose(F)))
            torch.cuda.synchronize()
            counts.append(H.hif_kernel_launches() - l0)
        outs.append(res)
        fb.close()
    for k in range(2):
        for a, b in zip(outs[0][k], outs[1][k]):
            assert torch.equal(a, b)
    assert counts[0] == counts[1] == counts[2] == counts[3] > 0


def test_batched_256_problems_n32_to_256_refined(P):
    # the batched workload at full size: 256 problems with n drawn
    # from {32, 48, ..., 256} (seed 1004), b = c = 1 + 0.5 phi_p (seed
    # 2000 + p), 4 Gaussian right-hand sides each (seed 3000 + p), eps 1e-6,
    # FP32 batched handle refined to 1e-10; every problem's residual is
    # re-estimated from sampled rows of the oracle's FP64 operator, and the
    # problems with n <= 48 are compared with their dense solves
    sizes = hi.batched_sizes(256, 1004)
    pbs = [hi.volume_problem(n, 2, smooth_seed=2000 + q, rhs_seed=3000 + q, nrhs=4) for q, n in enumerate(sizes)]
    probs = [(T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c)) for pb in pbs]
    fb = P.Factorization.batched(probs, 0, 1e-6, precision="fp32")
    off = fb.offsets
    assert off[-1] == sum(pb.N for pb in pbs)
    F = np.vstack([pb.f for pb in pbs])
    u, its, rel = fb.solve_refined(T(F), tol=1e-10)
    assert rel <= 1e-10
    u = u.cpu().numpy()
    rng = np.random.default_rng(1004)
    worst = 0.0
    for q, pb in enumerate(pbs):
        op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
        uq = u[off[q]:off[q + 1]]
        rows = rng.choice(pb.N, 16, replace=False)
        r = pb.f[rows] - op.matvec_rows(uq, rows)
        est = np.sqrt(pb.N / 16) * np.linalg.norm(r, axis=0) / np.linalg.norm(pb.f, axis=0)
        worst = max(worst, float(est.max()))
        if pb.n <= 48:
            ud = dense.DenseSolver(op).solve(pb.f)
            assert np.linalg.norm(uq - ud) <= 1e-9 * np.linalg.norm(ud)
    # 16 sampled rows: an estimate within a factor ~2 of the true norm
    assert worst <= 3e-10, worst
    fb.close()
