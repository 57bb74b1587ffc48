"""The batched elimination of large boxes (Lemma 2.4 blocks, the LU of B_rr
by 32-wide panels, the unit triangular inverses by blocks, X, Z and the
Schur update by tiled products) against the one-CTA elimination and the
dense solve.

HIF_BIG_ELIM sets the box size k + r above which a box takes the batched
path; at 40 nearly every box of the n = 64 grid does, with k and r that are
not multiples of the 32 x 32 inverse blocks or the 64 x 64 product tiles.
Both paths factor the same skeletons (the elimination does not change the
IDs of its own sublevel, and FP64 keeps later rank decisions away from the
threshold), so their solves agree to rounding; each also meets the solve
bound against the dense FP64 solve.
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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
def test_batched_elimination_fp64_matches_one_cta_path(P, monkeypatch, eps):
    pb = hi.volume_problem(64, 2, smooth_seed=1002, rhs_seed=1001, nrhs=3)
    args = (T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c), 0, eps)
    monkeypatch.setenv("HIF_BIG_ELIM", "40")
    fb = P.Factorization(*args, symmetric=False)
    monkeypatch.setenv("HIF_BIG_ELIM", "100000")
    fo = P.Factorization(*args, symmetric=False)
    monkeypatch.delenv("HIF_BIG_ELIM")
    assert [s["skeletons"] for s in fb.stats()["per_sublevel"]] == [s["skeletons"] for s in fo.stats()["per_sublevel"]]
    F = T(pb.f)
    for op in ("apply", "solve", "solve_transpose"):
        assert rel(getattr(fb, op)(F).cpu().numpy(), getattr(fo, op)(F).cpu().numpy()) <= 1e-12, op
    u = dense.DenseSolver(kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)).solve(pb.f)
    assert rel(fb.solve(F).cpu().numpy(), u) <= 100 * eps
    fb.close()
    fo.close()


def test_batched_elimination_fp32_refined(P, monkeypatch):
    pb = hi.volume_problem(64, 2, smooth_seed=1002, rhs_seed=1001, nrhs=2)
    args = (T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c), 0, 1e-6)
    monkeypatch.setenv("HIF_BIG_ELIM", "40")
    fb = P.Factorization(*args, precision="fp32")
    monkeypatch.delenv("HIF_BIG_ELIM")
    u = dense.DenseSolver(kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)).solve(pb.f)
    assert rel(fb.solve(T(pb.f)).cpu().numpy(), u) <= 1e-4
    x, its, r = fb.solve_refined(T(pb.f), tol=1e-10)
    assert r <= 1e-10 and rel(x.cpu().numpy(), u) <= 1e-9
    fb.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_wide_box_sweeps_match_one_cta_sweeps(P, monkeypatch, precision, tol):
    # HIF_SWEEP_WIDE sets the k + r above which a box's sweep passes run as
    # stage launches over the GPU (gather, products with T, X, Y and the unit
    # factors or their inverses, permutations, scatter); at 30 nearly every
    # LU box of the n = 64 grid does.  All four operations, 1 and 20 RHS
    # (the stage launches take 16 at a time), against the one-CTA sweeps of
    # the same factorization.
    pb = hi.volume_problem(64, 2, smooth_seed=1002, rhs_seed=1001, nrhs=20)
    args = (T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c), 0, 1e-6)
    monkeypatch.setenv("HIF_BIG_ELIM", "40")
    monkeypatch.setenv("HIF_SWEEP_WIDE", "30")
    fw = P.Factorization(*args, symmetric=False, precision=precision)
    monkeypatch.setenv("HIF_SWEEP_WIDE", "100000")
    fo = P.Factorization(*args, symmetric=False, precision=precision)
    monkeypatch.delenv("HIF_SWEEP_WIDE")
    monkeypatch.delenv("HIF_BIG_ELIM")
    for F in (T(pb.f[:, :1]), T(pb.f)):
        for op in ("apply", "solve", "apply_transpose", "solve_transpose"):
            assert rel(getattr(fw, op)(F).cpu().numpy(), getattr(fo, op)(F).cpu().numpy()) <= tol, op
    fw.close()
    fo.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_blocked_pivoted_qr_matches_per_step_qr(P, monkeypatch, precision):
    # the large-box pivoted QR by panels of 32 pivots (delayed trailing
    # updates, downdated norms recomputed at every panel end) against one
    # launch pair per pivot; HIF_BIG_ID=40 sends the boxes above 40 columns
    # down the large-box path
    pb = hi.volume_problem(64, 2, smooth_seed=1002, rhs_seed=1001, nrhs=2)
    args = (T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c), 0, 1e-6)
    monkeypatch.setenv("HIF_BIG_ID", "40")
    monkeypatch.setenv("HIF_BIG_QP_NB", "32")
    fb = P.Factorization(*args, precision=precision)
    monkeypatch.setenv("HIF_BIG_QP_NB", "1")
    fs = P.Factorization(*args, precision=precision)
    monkeypatch.delenv("HIF_BIG_QP_NB")
    monkeypatch.delenv("HIF_BIG_ID")
    kb = [s["skeletons"] for s in fb.stats()["per_sublevel"]]
    ks = [s["skeletons"] for s in fs.stats()["per_sublevel"]]
    if precision == "fp64":
        assert kb == ks
        for sub in range(len(kb)):
            np.testing.assert_array_equal(fb.eliminated_dofs(sub), fs.eliminated_dofs(sub))
        assert rel(fb.solve(T(pb.f)).cpu().numpy(), fs.solve(T(pb.f)).cpu().numpy()) <= 1e-12
    else:
        for a, b in zip(kb, ks):
            assert abs(a - b) <= 2 + 0.05 * b
    u = dense.DenseSolver(kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)).solve(pb.f)
    x, its, r = fb.solve_refined(T(pb.f), tol=1e-10)
    assert r <= 1e-10 and rel(x.cpu().numpy(), u) <= 1e-9
    fb.close()
    fs.close()
