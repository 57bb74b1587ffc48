"""hif_id_batched_noalloc: the batched interpolative decomposition for callers
that cannot allocate device memory (graph capture, fixed memory budgets).

Its results must equal those of hif_id_batched on the same inputs, call after
call: the fixed device work space is shared by all calls and keeps the last
call's contents, so two different calls in a row check that nothing stale
leaks into the second one.  Inputs beyond the fixed work space are refused
with HIF_EINVAL, before any matrix is touched.
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


def test_noalloc_refuses_inputs_beyond_its_work_space(H):
    A = np.random.default_rng(3).standard_normal((8, 1100))      # more columns than the fixed limit
    args, po, to = _layout([A], [1e-6])
    st, k, perm, T = _run(H.hif_id_batched_noalloc, args, po, to, 1)
    assert st == H.HIF_EINVAL
    assert b"work space" in H.load().hif_last_error()
    assert k[0] == -7                                                 # outputs untouched
