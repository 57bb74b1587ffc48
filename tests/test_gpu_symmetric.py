"""Symmetric fast path (Sec. 5): for A = A^T the one-sided proxy matrix
Y'_c = [A_{cN,c}; Y_{cE,c}] is compressed instead of Y_c.  Its ID is the
ID of Y_c (every dropped row repeats a kept one), so the GPU factorization
with and without the shortcut must pick the same skeletons and give the same
operator F to rounding, while the proxy matrices have half the rows.  Both
modes are also held to the dense FP64 solve and to the oracle's skeleton
counts in the same mode.
"""
import os

import numpy as np
import pytest
import torch

import hif_inputs as hi
from oracle import dense, hifie, kernels

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


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def compare_modes(P, pb, eps, tol_op, **kw):
    fs = factor(P, pb, eps, symmetric=True, **kw)
    ff = factor(P, pb, eps, symmetric=False, **kw)
    ss, sf = fs.stats(), ff.stats()
    assert ss["symmetric_problems"] == 1 and sf["symmetric_problems"] == 0
    # one row per near-field DOF and proxy point against two
    assert 2 * ss["proxy_rows"] == sf["proxy_rows"]
    assert [s["skeletons"] for s in ss["per_sublevel"]] == [s["skeletons"] for s in sf["per_sublevel"]]
    assert ss["top_size"] == sf["top_size"]
    X = hi.gaussian_rhs(pb.N, 3, 21)
    for op in ("apply", "solve", "solve_transpose"):
        ys = getattr(fs, op)(T(X)).cpu().numpy()
        yf = getattr(ff, op)(T(X)).cpu().numpy()
        assert relerr(ys, yf) <= tol_op, op
    return fs, ff


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_symmetric_and_full_compression_agree_2d(P, eps):
    pb = hi.volume_problem(64, 2, smooth_seed=1002, rhs_seed=1001)
    fs, ff = compare_modes(P, pb, eps, 1e-10)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    ds = dense.DenseSolver(op)
    f = pb.f[:, 0]
    u = ds.solve(f)
    for fac in (fs, ff):
        assert relerr(fac.solve(T(f)).cpu().numpy(), u) <= 100 * eps
    # skeleton counts against the oracle, which takes the same shortcut
    Fo = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, eps, pb.proxy)
    for s, sl in zip(fs.stats()["per_sublevel"], Fo.sublevels):
        ko = sum(b.sk.size for b in sl.boxes)
        assert abs(s["skeletons"] - ko) <= 0.1 * ko + 2
    fs.close()
    ff.close()


def test_symmetric_and_full_compression_agree_3d(P):
    pb = hi.volume_problem(12, 3, smooth_seed=5)
    fs, ff = compare_modes(P, pb, 1e-3, 1e-10, occupancy=27)
    fs.close()
    ff.close()


def test_symmetric_large_box_path(P):
    # boxes above 40 columns take the materialized-Y_c path (one launch per
    # pivot step) instead of the shared-memory fold
    os.environ["HIF_BIG_ID"] = "40"
    try:
        pb = hi.volume_problem(64, 2, smooth_seed=1002, rhs_seed=1001)
        fs, ff = compare_modes(P, pb, 1e-6, 1e-10)
        op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
        f = pb.f[:, 0]
        u = dense.DenseSolver(op).solve(f)
        assert relerr(fs.solve(T(f)).cpu().numpy(), u) <= 1e-4
    finally:
        os.environ.pop("HIF_BIG_ID", None)
    fs.close()
    ff.close()


def test_symmetric_fp32_factorization(P):
    pb = hi.volume_problem(64, 2, smooth_seed=1002, rhs_seed=1001)
    fs = factor(P, pb, 1e-6, precision="fp32")
    assert fs.stats()["symmetric_problems"] == 1
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    f = pb.f[:, 0]
    u = dense.DenseSolver(op).solve(f)
    assert relerr(fs.solve(T(f)).cpu().numpy(), u) <= 1e-4
    x, its, rel = fs.solve_refined(T(f), tol=1e-10)
    assert relerr(x.cpu().numpy(), u) <= 1e-9
    fs.close()


def test_batched_mixes_symmetric_and_general_problems(P):
    # b != c or unequal weights turn the shortcut off for that problem only
    sizes = [40, 33, 48]
    pbs = [hi.volume_problem(n, 2, smooth_seed=700 + q) for q, n in enumerate(sizes)]
    pbs[1].c = 1.0 + 0.5 * hi.smooth_field(pbs[1].points, 9)
    probs = [(T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c)) for pb in pbs]
    eps = 1e-6
    fb = P.Factorization.batched(probs, 0, eps)
    st = fb.stats()
    assert st["symmetric_problems"] == 2
    f = np.concatenate([pb.f[:, 0] for pb in pbs])
    u = fb.solve(T(f)).cpu().numpy()
    off = fb.offsets
    for q, pb in enumerate(pbs):
        op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
        uq = dense.DenseSolver(op).solve(pb.f[:, 0])
        assert relerr(u[off[q]:off[q + 1]], uq) <= 100 * eps
    fb.close()


# ------------------------------------------------ LDL (Sec. 5, opening) ---

@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_ldl_equals_lu_and_stores_less(P, precision, tol):
    # symmetric A: the diagonal blocks factored by LDL keep X only (Y = X^T)
    # and one r x r array for L and L^{-1}; the block inverse is the same, so
    # F and F^{-1} agree with the LU path to rounding
    pb = hi.volume_problem(64, 2, smooth_seed=1002, rhs_seed=1001)
    fl = factor(P, pb, 1e-6, precision=precision, ldl=True)
    fu = factor(P, pb, 1e-6, precision=precision, ldl=False)
    sl, su = fl.stats(), fu.stats()
    assert sl["ldl_boxes"] > 0 and sl["ldl_fallbacks"] == 0 and su["ldl_boxes"] == 0
    ks_l = [s["skeletons"] for s in sl["per_sublevel"]]
    ks_u = [s["skeletons"] for s in su["per_sublevel"]]
    if precision == "fp64":
        assert ks_l == ks_u
    else:
        # FP32 rounding of the Schur updates differs between the two forms
        # and can move a later rank decision by one
        assert ks_l[0] == ks_u[0] and all(abs(a - b) <= 2 + 0.005 * b for a, b in zip(ks_l, ks_u))
    assert sl["factor_bytes"] < 0.8 * su["factor_bytes"]
    X = T(hi.gaussian_rhs(pb.N, 3, 31))
    for op in ("apply", "solve", "solve_transpose", "apply_transpose"):
        assert relerr(getattr(fl, op)(X).cpu().numpy(), getattr(fu, op)(X).cpu().numpy()) <= tol, op
    if precision == "fp64":
        # every LDL box is symmetric, so F^{-1} and F^{-T} agree to rounding
        assert relerr(fl.solve(X).cpu().numpy(), fl.solve_transpose(X).cpu().numpy()) <= 1e-12
        assert relerr(fl.apply(X).cpu().numpy(), fl.apply_transpose(X).cpu().numpy()) <= 1e-12
        op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
        u = dense.DenseSolver(op).solve(pb.f[:, 0])
        assert relerr(fl.solve(T(pb.f[:, 0])).cpu().numpy(), u) <= 100e-6
    else:
        x, its, rel = fl.solve_refined(T(pb.f[:, 0]), tol=1e-10)
        assert rel <= 1e-10
    fl.close()
    fu.close()


def test_ldl_falls_back_to_lu_per_box(P, monkeypatch):
    # an acceptance constant no pivot can meet: every LDL box with r > 1
    # takes the LU form, and the result is the LU path's
    pb = hi.volume_problem(48, 2, smooth_seed=1002, rhs_seed=1001)
    fu = factor(P, pb, 1e-6, ldl=False)
    monkeypatch.setenv("HIF_LDL_TEST_ALPHA", "1e30")
    fl = factor(P, pb, 1e-6, ldl=True)
    monkeypatch.delenv("HIF_LDL_TEST_ALPHA")
    st = fl.stats()
    assert st["ldl_fallbacks"] > 0
    X = T(hi.gaussian_rhs(pb.N, 2, 32))
    for op in ("apply", "solve", "solve_transpose"):
        assert relerr(getattr(fl, op)(X).cpu().numpy(), getattr(fu, op)(X).cpu().numpy()) <= 1e-12, op
    fl.close()
    fu.close()


def test_ldl_not_used_for_nonsymmetric_problems(P):
    pb = hi.volume_problem(32, 2, smooth_seed=1002)
    pb.c = 1.0 + 0.5 * hi.smooth_field(pb.points, 99)
    f = factor(P, pb, 1e-6)
    assert f.stats()["ldl_boxes"] == 0 and f.stats()["symmetric_problems"] == 0
    f.close()


def test_large_boxes_folded_to_R_fp32(P, monkeypatch):
    # FP32 boxes above the one-column-per-thread width are folded to R by the
    # multi-column fold and their pivoted QR runs on R (Sec. 2.2: the ID of
    # R[:, g] is that of Y_c[:, g]); against the materialized-Y_c path and the
    # dense solve, with boxes above 40 columns sent down the large-box paths
    pb = hi.volume_problem(64, 2, smooth_seed=1002, rhs_seed=1001)
    monkeypatch.setenv("HIF_BIG_ID", "40")
    monkeypatch.setenv("HIF_FOLD_BIG", "1")
    fr = factor(P, pb, 1e-6, precision="fp32")
    monkeypatch.setenv("HIF_FOLD_BIG", "0")
    fm = factor(P, pb, 1e-6, precision="fp32")
    monkeypatch.delenv("HIF_FOLD_BIG")
    monkeypatch.delenv("HIF_BIG_ID")
    sr, sm = fr.stats(), fm.stats()
    # FP32 rank decisions at the tolerance floor follow the rounding of two
    # different reductions (R by Householder folds, or the proxy matrix itself)
    for a, b in zip(sr["per_sublevel"], sm["per_sublevel"]):
        assert abs(a["skeletons"] - b["skeletons"]) <= 2 + 0.05 * b["skeletons"]
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    f = pb.f[:, 0]
    u = dense.DenseSolver(op).solve(f)
    assert relerr(fr.solve(T(f)).cpu().numpy(), u) <= 1e-4
    assert relerr(fr.solve(T(f)).cpu().numpy(), fm.solve(T(f)).cpu().numpy()) <= 1e-4
    x, its, rel = fr.solve_refined(T(f), tol=1e-10)
    assert rel <= 1e-10 and relerr(x.cpu().numpy(), u) <= 1e-9
    fr.close()
    fm.close()
