"""hif_gemm_batched_f32: the FP32 products of the large-box elimination
(Lemma 2.4 blocks, Schur update) on the tcgen05 tensor cores.

Every result is compared element by element with the FP64 product of the same
FP32 inputs.  The three-piece BF16 split drops only piece products of weight
below 2^-16 * 2^-8, so the error is that of FP32 accumulation:
|C - C_ref| <= 2^-18 (1 + k / 256) (|op(A)| |op(B)|)_ij, checked on shapes that
cover whole tiles (128 x 256 x 32), ragged tails in every dimension, both
transposes, padded leading dimensions, beta = 0 and 1, k = 0 and a batch of
problems of different sizes in one launch.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def H():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1307_2666_gb300 import hif
    return hif


def _problem(rng, m, n, k, ta, tb, alpha, beta, pad=0):
    ra, ca = (k, m) if ta else (m, k)
    rb, cb = (n, k) if tb else (k, n)
    A = rng.standard_normal((ra + pad, ca)).astype(np.float32)
    B = rng.standard_normal((rb + pad, cb)).astype(np.float32)
    C0 = rng.standard_normal((m + pad, n)).astype(np.float32)
    dA = torch.as_tensor(np.asfortranarray(A).reshape(-1, order="F"), device=DEV)
    dB = torch.as_tensor(np.asfortranarray(B).reshape(-1, order="F"), device=DEV)
    dC = torch.as_tensor(np.asfortranarray(C0).reshape(-1, order="F"), device=DEV)
    q = dict(A=dA, B=dB, C=dC, lda=ra + pad, ldb=rb + pad, ldc=m + pad, m=m, n=n, k=k, trans_a=ta, trans_b=tb,
             alpha=alpha, beta=beta)
    opA = (A[:k, :m].T if ta else A[:m, :k]).astype(np.float64)
    opB = (B[:n, :k].T if tb else B[:k, :n]).astype(np.float64)
    ref = alpha * (opA @ opB) + (C0[:m, :n].astype(np.float64) if beta else 0.0)
    mag = np.abs(alpha) * (np.abs(opA) @ np.abs(opB))
    return q, ref, mag


def _result(q):
    m, n, ldc = q["m"], q["n"], q["ldc"]
    return q["C"].cpu().numpy().reshape(ldc, n, order="F")[:m, :n].astype(np.float64)


def _check(q, ref, mag):
    got = _result(q)
    tol = 2.0 ** -18 * (1 + q["k"] / 256) * mag + 1e-30
    err = np.abs(got - ref)
    assert np.all(err <= tol), f"max err/tol {np.max(err / tol):.3g} for m={q['m']} n={q['n']} k={q['k']}"
    return float(np.max(err / np.maximum(mag, 1e-30)))


@pytest.mark.parametrize("m,n,k", [(128, 256, 32), (1, 1, 1), (129, 257, 33), (300, 70, 1000), (37, 513, 5),
                                   (256, 512, 64), (64, 64, 2048)])
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_products_match_fp64(H, m, n, k, ta, tb):
    rng = np.random.default_rng(m * 7 + n * 13 + k + 100 * ta + 10 * tb)
    q, ref, mag = _problem(rng, m, n, k, ta, tb, alpha=-1.0, beta=1)
    assert H.hif_gemm_batched_f32([q]) == H.HIF_OK
    _check(q, ref, mag)


def test_beta_zero_alpha_scaled_and_padded(H):
    rng = np.random.default_rng(5)
    q, ref, mag = _problem(rng, 150, 300, 77, 1, 0, alpha=0.375, beta=0, pad=3)
    assert H.hif_gemm_batched_f32([q]) == H.HIF_OK
    _check(q, ref, mag)
    # the padding rows of C are untouched
    C = q["C"].cpu().numpy().reshape(q["ldc"], q["n"], order="F")
    rng2 = np.random.default_rng(5)
    _ = rng2.standard_normal((77 + 3, 150)), rng2.standard_normal((77 + 3, 300))
    C0 = rng2.standard_normal((150 + 3, 300)).astype(np.float32)
    np.testing.assert_array_equal(C[150:], C0[150:])


def test_k_zero(H):
    rng = np.random.default_rng(6)
    q0, _, _ = _problem(rng, 40, 50, 0, 0, 0, alpha=1.0, beta=0)
    q1, _, _ = _problem(rng, 40, 50, 0, 0, 0, alpha=1.0, beta=1)
    before = _result(q1)
    assert H.hif_gemm_batched_f32([q0, q1]) == H.HIF_OK
    assert np.all(_result(q0) == 0.0)
    np.testing.assert_array_equal(_result(q1), before)


def test_batch_of_uneven_problems(H):
    rng = np.random.default_rng(7)
    qs, refs = [], []
    for i in range(40):
        m, n, k = (int(x) for x in rng.integers(1, 400, size=3))
        q, ref, mag = _problem(rng, m, n, k, int(rng.integers(2)), int(rng.integers(2)), alpha=-1.0,
                               beta=int(rng.integers(2)))
        qs.append(q)
        refs.append((ref, mag))
    assert H.hif_gemm_batched_f32(qs) == H.HIF_OK
    for q, (ref, mag) in zip(qs, refs):
        _check(q, ref, mag)


def test_invalid_arguments(H):
    lib = H.load()
    rng = np.random.default_rng(8)
    q, _, _ = _problem(rng, 10, 10, 10, 0, 0, alpha=1.0, beta=1)
    bad = dict(q, lda=5)
    assert H.hif_gemm_batched_f32([bad]) == H.HIF_EINVAL
    assert b"invalid" in lib.hif_last_error()
    bad = dict(q, beta=2)
    assert H.hif_gemm_batched_f32([bad]) == H.HIF_EINVAL
    assert lib.hif_gemm_batched_f32(-1, None, None) == H.HIF_EINVAL
    assert b"negative count" in lib.hif_last_error()
    assert H.hif_gemm_batched_f32([]) == H.HIF_OK


def test_elimination_products_on_tensor_cores(H, monkeypatch):
    # the FP32 factorization with the Lemma 2.4 products and the Schur update
    # of the batched large-box elimination on the tensor cores (HIF_TC_GEMM=1,
    # boxes above 64 DOFs sent to that elimination) against the SIMT products
    # and the dense solve
    import hif_inputs as hi
    import paper_1307_2666_gb300 as P
    from oracle import dense, kernels
    pb = hi.volume_problem(64, 2, smooth_seed=1002, rhs_seed=1001)
    T = lambda v: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device=DEV)
    args = (T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c), 0, 1e-6)
    monkeypatch.setenv("HIF_BIG_ELIM", "64")
    monkeypatch.setenv("HIF_TC_GEMM", "1")
    ft = P.Factorization(*args, precision="fp32")
    monkeypatch.setenv("HIF_TC_GEMM", "0")
    fs = P.Factorization(*args, precision="fp32")
    st, ss = ft.stats(), fs.stats()
    for a, b in zip(st["per_sublevel"], ss["per_sublevel"]):
        assert abs(a["skeletons"] - b["skeletons"]) <= 2 + 0.05 * b["skeletons"]
    f = pb.f[:, 0]
    u = dense.DenseSolver(kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)).solve(f)
    rel = lambda x, y: float(np.linalg.norm(x - y) / np.linalg.norm(y))
    assert rel(ft.solve(T(f)).cpu().numpy(), u) <= 1e-4
    x, its, r = ft.solve_refined(T(f), tol=1e-10)
    assert r <= 1e-10 and rel(x.cpu().numpy(), u) <= 1e-9
    ft.close()
    fs.close()
