"""hif_id_batched_noalloc: the batched interpolative decomposition for callers
that cannot allocate device memory (a device-memory budget fixed at start-up,
or code that may not call cudaMalloc/cudaFree because they can synchronize the
whole device).

Its results must equal those of hif_id_batched on the same inputs, call after
call: the fixed device work space is shared by all calls and keeps the last
call's contents, so two different calls in a row check that nothing stale
leaks into the second one.  The ranks, pivots and T are also compared with the
oracle's interpolative decomposition (Sec. 2.2, Lemma 2.2).  Inputs beyond any
of the three limits of the fixed work space (matrix count, columns per matrix,
total work space) are refused with HIF_EINVAL and leave the outputs untouched;
a valid call right after a refused one is still correct.
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


def _batch(seed):
    """A batch of matrices: exact low rank with separated pivots, and a matrix
    whose rank is set by the tolerance."""
    rng = np.random.default_rng(seed)
    mats, tols = [], []
    for (m, n, k) in [(60, 25, 25), (100, 40, 12), (37, 53, 9), (129, 64, 64), (3, 5, 3), (64, 1, 1)]:
        A = rng.standard_normal((m, k)) @ rng.standard_normal((k, n))
        A *= (1.3 ** np.arange(n))[None, :]
        mats.append(A)
        tols.append(1e-11)
    U, _ = np.linalg.qr(rng.standard_normal((90, 30)))
    V, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    mats.append((U * 10.0 ** (-np.arange(30) / 4)) @ V.T)
    tols.append(1e-5)
    return mats, tols


def _layout(mats, tols):
    off, m, n, poff, toff = [], [], [], [], []
    o = po = to = 0
    for M in mats:
        off.append(o); m.append(M.shape[0]); n.append(M.shape[1]); poff.append(po); toff.append(to)
        o += M.size; po += M.shape[1]; to += M.shape[1] ** 2 // 4 + M.shape[1]
    buf = np.concatenate([np.asfortranarray(M).reshape(-1, order="F") for M in mats])
    d = lambda a, t: torch.as_tensor(np.asarray(a, dtype=t), device=DEV)
    args = dict(mats=d(buf, np.float64), off=d(off, np.int64), m=d(m, np.int32), n=d(n, np.int32),
                tol=d(tols, np.float64), poff=d(poff, np.int64), toff=d(toff, np.int64))
    return args, po, to


def _run(fn, args, po, to, count):
    # device arrays throughout (what the no-allocation entry point requires)
    k = torch.full((count,), -7, dtype=torch.int32, device=DEV)
    perm = torch.full((po,), -7, dtype=torch.int32, device=DEV)
    T = torch.full((to,), np.nan, dtype=torch.float64, device=DEV)
    st = fn(args["mats"], args["off"], args["m"], args["n"], args["tol"], k, perm, args["poff"], T, args["toff"])
    torch.cuda.synchronize()
    return st, k.cpu().numpy(), perm.cpu().numpy(), T.cpu().numpy()


def _run_allocating(H, args, po, to, count):
    # hif_id_batched reads its index and tolerance arrays on the host
    h = {key: v.cpu().numpy() for key, v in args.items()}
    k = np.full(count, -7, dtype=np.int32)
    perm = np.full(po, -7, dtype=np.int32)
    T = np.full(to, np.nan)
    H.hif_id_batched(h["mats"], h["off"], h["m"], h["n"], h["tol"], k, perm, h["poff"], T, h["toff"])
    return H.HIF_OK, k, perm, T


def test_noalloc_matches_allocating_entry_point_twice(H):
    for seed in (11, 12):                       # two different calls in a row
        mats, tols = _batch(seed)
        args, po, to = _layout(mats, tols)
        st0, k0, p0, T0 = _run_allocating(H, args, po, to, len(mats))
        st1, k1, p1, T1 = _run(H.hif_id_batched_noalloc, args, po, to, len(mats))
        assert st1 == H.HIF_OK
        np.testing.assert_array_equal(k1, k0)
        np.testing.assert_array_equal(p1, p0)
        toff = args["toff"].cpu().numpy()
        for i, M in enumerate(mats):
            ki, ni = int(k0[i]), M.shape[1]
            a = T0[toff[i]:toff[i] + ki * (ni - ki)]
            b = T1[toff[i]:toff[i] + ki * (ni - ki)]
            if a.size:
                np.testing.assert_allclose(b, a, rtol=1e-8, atol=1e-9 * max(1.0, np.abs(a).max()))


def test_noalloc_matches_oracle_interp_decomp(H):
    from oracle import idqr
    mats, tols = _batch(12)
    args, po, to = _layout(mats, tols)
    st, k, perm, T = _run(H.hif_id_batched_noalloc, args, po, to, len(mats))
    assert st == H.HIF_OK
    poff = args["poff"].cpu().numpy()
    toff = args["toff"].cpu().numpy()
    for i, (M, tol) in enumerate(zip(mats, tols)):
        sk, rd, To = idqr.interp_decomp(M, tol)
        ki, ni = int(k[i]), M.shape[1]
        assert ki == sk.size
        np.testing.assert_array_equal(perm[poff[i]:poff[i] + ki], sk)
        np.testing.assert_array_equal(perm[poff[i] + ki:poff[i] + ni], rd)
        if To.size:
            got = T[toff[i]:toff[i] + ki * (ni - ki)].reshape(ki, ni - ki, order="F")
            np.testing.assert_allclose(got, To, rtol=1e-8, atol=1e-8 * max(1.0, np.abs(To).max()))


def _valid_call_still_matches(H, seed):
    mats, tols = _batch(seed)
    args, po, to = _layout(mats, tols)
    st0, k0, p0, T0 = _run_allocating(H, args, po, to, len(mats))
    st1, k1, p1, T1 = _run(H.hif_id_batched_noalloc, args, po, to, len(mats))
    assert st1 == H.HIF_OK
    np.testing.assert_array_equal(k1, k0)
    np.testing.assert_array_equal(p1, p0)
    toff = args["toff"].cpu().numpy()
    for i, M in enumerate(mats):                 # the k x (n - k) block of each matrix
        ki, ni = int(k0[i]), M.shape[1]
        a = T0[toff[i]:toff[i] + ki * (ni - ki)]
        b = T1[toff[i]:toff[i] + ki * (ni - ki)]
        if a.size:
            np.testing.assert_allclose(b, a, rtol=1e-8, atol=1e-9 * max(1.0, np.abs(a).max()))


def _refused(H, mats, tols):
    args, po, to = _layout(mats, tols)
    st, k, perm, T = _run(H.hif_id_batched_noalloc, args, po, to, len(mats))
    assert st == H.HIF_EINVAL
    assert b"work space" in H.load().hif_last_error()
    assert np.all(k == -7) and np.all(perm == -7) and np.all(np.isnan(T))   # outputs untouched


def test_noalloc_refuses_too_many_columns(H):
    A = np.random.default_rng(3).standard_normal((8, 1100))      # more columns than the fixed limit
    _refused(H, [A], [1e-6])
    _valid_call_still_matches(H, 21)


def test_noalloc_refuses_total_work_space(H):
    # every matrix within 1024 columns, but 2 * 1023 * 600 doubles > 2^20
    rng = np.random.default_rng(4)
    _refused(H, [rng.standard_normal((1023, 600)) for _ in range(2)], [1e-6, 1e-6])
    _valid_call_still_matches(H, 22)


def test_noalloc_refuses_too_many_matrices(H):
    rng = np.random.default_rng(5)
    _refused(H, [rng.standard_normal((2, 2)) for _ in range(4097)], [1e-6] * 4097)
    _valid_call_still_matches(H, 23)


def test_noalloc_null_and_negative_arguments_set_last_error(H):
    lib = H.load()
    assert lib.hif_id_batched_noalloc(-1, None, None, None, None, None, None, None, None, None, None,
                                      None) == H.HIF_EINVAL
    assert b"negative count" in lib.hif_last_error()
    assert lib.hif_id_batched_noalloc(1, None, None, None, None, None, None, None, None, None, None,
                                      None) == H.HIF_EINVAL
    assert b"NULL" in lib.hif_last_error()
