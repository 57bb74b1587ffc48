"""Tensor-core direct sum (exact 8-bit digits, integer class sums) vs the
oracle's FP64 direct sum, element by element.

The sum is the refinement residual operator (Sec. 5) over all N^2 pairs of
the assembled K (Sec. 3.1, Eq. (3.1)).  The only rounding is the digits it
drops (below 2^-55 of max|K| max|x| per term) and the FP64 combination of
the class sums, so every entry must agree with FP64 to 1e-13 of the largest
entry of its column.
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


def handle(P, pb, direct="tc", eps=1e-3, precision="fp32"):
    return P.Factorization(T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c), pb.kernel_id, eps,
                           proxy_dirs=pb.proxy if pb.dim == 3 else None, precision=precision, direct=direct)


def close_cols(y, ref, tol=1e-13):
    y = np.atleast_2d(y.T).T
    ref = np.atleast_2d(ref.T).T
    scale = np.abs(ref).max(axis=0)
    err = np.abs(y - ref).max(axis=0)
    assert np.all(err <= tol * scale), (err / np.maximum(scale, 1e-300))


# 2D: one tile and chunk, ragged tiles/chunks, exactly two, several; nrhs
# below, at and above the 8 columns of one launch
@pytest.mark.parametrize("n,nrhs", [(64, 1), (100, 3), (128, 8), (130, 11), (47, 16)])
def test_tc_sum_2d_matches_oracle(P, n, nrhs):
    pb = hi.volume_problem(n, 2, smooth_seed=1002 + n)
    x = hi.gaussian_rhs(pb.N, nrhs, 40 + n)
    fac = handle(P, pb)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    for trans in (False, True):
        y = fac.matvec(T(x), trans=trans).cpu().numpy()
        close_cols(y, op.matvec(x, trans=trans))
    fac.close()


@pytest.mark.parametrize("n,nrhs", [(12, 2), (20, 9)])
def test_tc_sum_3d_matches_oracle(P, n, nrhs):
    pb = hi.volume_problem(n, 3, smooth_seed=77 + n)
    x = hi.gaussian_rhs(pb.N, nrhs, 50 + n)
    fac = handle(P, pb)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 1)
    for trans in (False, True):
        y = fac.matvec(T(x), trans=trans).cpu().numpy()
        close_cols(y, op.matvec(x, trans=trans))
    fac.close()


def test_tc_sum_matches_fp64_grid_sum(P):
    # two ragged tiles per line, 8 + 2 right-hand sides, with column scales
    # spread over 40 orders of magnitude and an all-zero column
    pb = hi.volume_problem(200, 2, smooth_seed=31)
    x = hi.gaussian_rhs(pb.N, 10, 7)
    x *= np.logspace(-20, 20, 10)[None, :]
    x[:, 3] = 0.0
    f_tc = handle(P, pb)
    f_64 = handle(P, pb, direct="fp64")
    for trans in (False, True):
        y = f_tc.matvec(T(x), trans=trans).cpu().numpy()
        ref = f_64.matvec(T(x), trans=trans).cpu().numpy()
        assert np.all(y[:, 3] == 0.0)
        cols = [c for c in range(10) if c != 3]
        close_cols(y[:, cols], ref[:, cols])
    f_tc.close()
    f_64.close()


def test_tc_sum_batched_segments(P):
    sizes = [40, 17, 64, 33]
    pbs = [hi.volume_problem(n, 2, smooth_seed=900 + q) for q, n in enumerate(sizes)]
    probs = [(T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c)) for pb in pbs]
    fb = P.Factorization.batched(probs, 0, 1e-3, precision="fp32", direct="tc")
    x = hi.gaussian_rhs(sum(pb.N for pb in pbs), 3, 5)
    y = fb.matvec(T(x)).cpu().numpy()
    off = fb.offsets
    for q, pb in enumerate(pbs):
        op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
        close_cols(y[off[q]:off[q + 1]], op.matvec(x[off[q]:off[q + 1]]))
    fb.close()


def test_tc_sum_full_size_sampled_rows(P):
    # the refinement workload: n = 1024 (N = 1,048,576), 8 right-hand sides,
    # one launch over all 8192 tiles; rows sampled at tile and chunk edges
    n = 1024
    pb = hi.volume_problem(n, 2, smooth_seed=1002, rhs_seed=1003, nrhs=8)
    fac = handle(P, pb, eps=1e-6)
    y = fac.matvec(T(pb.f)).cpu().numpy()
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    rng = np.random.default_rng(11)
    rows = np.unique(np.concatenate([[0, 127, 128, n - 1, n, n * n - 1, 511 * n + 383],
                                     rng.integers(0, pb.N, 9)]))
    ref = op.matvec_rows(pb.f, rows)
    scale = np.abs(ref).max(axis=0)
    err = np.abs(y[rows] - ref).max(axis=0)
    assert np.all(err <= 1e-13 * scale), err / scale
    fac.close()


def test_tc_sum_bounded_wait_reports_timeout_and_context_survives(P):
    # the MMA thread is told to issue nothing: the builders' waits for their
    # shared-memory stages run out (~2 s), the kernel drains its copies,
    # frees TMEM and returns; the call reports HIF_ETIMEOUT and the same
    # handle then computes a correct sum
    import os
    from paper_1307_2666_gb300 import hif as H
    pb = hi.volume_problem(64, 2, smooth_seed=4)
    x = hi.gaussian_rhs(pb.N, 2, 6)
    fac = handle(P, pb)
    os.environ["HIF_TC_TEST_STALL"] = "1"
    try:
        with pytest.raises(H.HIFError) as err:
            fac.matvec(T(x))
        assert err.value.status == H.HIF_ETIMEOUT
    finally:
        os.environ.pop("HIF_TC_TEST_STALL", None)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    close_cols(fac.matvec(T(x)).cpu().numpy(), op.matvec(x))
    fac.close()


# ---- short digit sets (the refinement's intermediate residuals) -------------

def _short_bounds(pb, x, classes, trans):
    """Per-term bound of the pairs a short sum drops, from the oracle's K
    (b = c = 1): (classes + 1) 2^(-2 - 8 classes) x 2^(eT + eX), with
    2^(eT + eX) <= 16 max|K| max|s x| per column (s = c, or b for A^T), and
    2% for the classes further down."""
    one = np.ones(pb.N)
    K0 = kernels.Operator(pb.points, pb.weights, pb.a, one, one, 0).kernel_entries(np.array([0]), np.arange(pb.N))
    kmax = np.abs(K0).max()                  # on the grid every |offset| occurs in row 0
    vmax = np.abs((pb.b if trans else pb.c)[:, None] * x).max(axis=0)
    return 1.02 * (classes + 1) * 2.0 ** (-2 - 8 * classes) * 16.0 * kmax * vmax


@pytest.mark.parametrize("classes", [4, 5, 6])
@pytest.mark.parametrize("n,nrhs", [(100, 3), (130, 11)])
def test_short_sums_within_their_bounds(P, n, nrhs, classes):
    # the kernel part of the error, (A_short x - A x) / b (or / c for A^T),
    # against the dropped pairs: every entry below N per-term bounds (worst
    # case) and, as a sum of N terms of mean zero, every entry below
    # 8 sqrt(N) and the column norm below N per-term bounds
    pb = hi.volume_problem(n, 2, smooth_seed=1002 + n)
    x = hi.gaussian_rhs(pb.N, nrhs, 40 + n)
    fac = handle(P, pb)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    N = pb.N
    for trans in (False, True):
        beta = _short_bounds(pb, x, classes, trans)
        y = fac.matvec(T(x), trans=trans, classes=classes).cpu().numpy()
        ref = op.matvec(x, trans=trans)
        ek = np.abs(y - ref) / np.abs((pb.c if trans else pb.b)[:, None])
        assert np.all(ek.max(axis=0) <= N * beta)
        assert np.all(ek.max(axis=0) <= 8.0 * np.sqrt(N) * beta), ek.max(axis=0) / (np.sqrt(N) * beta)
        assert np.all(np.linalg.norm(ek, axis=0) <= N * beta)
        # the short kernel ran: its result is not the full sum's
        full = fac.matvec(T(x), trans=trans).cpu().numpy()
        assert np.any(full != y)
    fac.close()


def test_refinement_short_residuals_reach_the_full_residual(P, capfd, monkeypatch):
    # FP32 factor, 4 RHS: the refinement with short intermediate residuals
    # and with every residual in full reach the same iteration count, and the
    # returned residual (always a full sum) is the oracle's at the returned u
    n = 128
    pb = hi.volume_problem(n, 2, smooth_seed=1002, rhs_seed=1003, nrhs=4)
    fac = handle(P, pb, eps=1e-6)
    monkeypatch.setenv("HIF_TRACE", "1")
    u_s, its_s, rel_s = fac.solve_refined(T(pb.f), tol=1e-10)
    trace = capfd.readouterr().err
    monkeypatch.setenv("HIF_SHORT_RESIDUAL", "0")
    u_f, its_f, rel_f = fac.solve_refined(T(pb.f), tol=1e-10)
    trace_f = capfd.readouterr().err
    assert "(5 digit classes" in trace and "(8 digit classes" in trace
    assert all(f"({kd} digit classes" not in trace_f for kd in (4, 5, 6))
    assert its_s == its_f and rel_s <= 1e-10 and rel_f <= 1e-10
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    u = u_s.cpu().numpy()
    r = pb.f - op.matvec(u)
    rel = np.max(np.linalg.norm(r, axis=0) / np.linalg.norm(pb.f, axis=0))
    assert abs(rel - rel_s) <= 1e-3 * rel_s + 1e-16
    uf = u_f.cpu().numpy()
    assert np.linalg.norm(u - uf) <= 1e-9 * np.linalg.norm(uf)
    fac.close()
