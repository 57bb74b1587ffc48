"""GPU path vs the CPU oracle, through the C ABI.

Component parity is element by element (kernel entries, batched ID, direct
sum); the factorization is judged the way the method is defined: apply error
<= 10 eps and solve error <= 100 eps against the dense FP64 solve, skeleton
totals within 10% of the sequential CPU HIF-IE, and the algebraic identities
of the factored form to rounding.
"""
import numpy as np
import pytest
import torch

import hif_inputs as hi
from oracle import dense, hifie, idqr, kernels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1307_2666_gb300 as P
    return P


DEV = "cuda:0"


def T(v):
    return torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device=DEV)


def factor(P, pb, eps, **kw):
    return P.Factorization(T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c), pb.kernel_id, eps,
                           proxy_dirs=pb.proxy if pb.dim == 3 else None, **kw)


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


_oracle_cache = {}


def oracle_setup(n, dim=2, smooth=1002, eps=1e-6, occupancy=64, second_kind=True):
    key = (n, dim, smooth, eps, occupancy, second_kind)
    if key not in _oracle_cache:
        pb = hi.volume_problem(n, dim, smooth_seed=smooth)
        op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, pb.kernel_id)
        F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, pb.kernel_id, eps, pb.proxy,
                         occupancy=occupancy, second_kind=second_kind)
        _oracle_cache[key] = (pb, op, dense.DenseSolver(op), F)
    return _oracle_cache[key]


# ---------------------------------------------------------------- entries --

def test_kernel_block_matches_oracle_entries(lib):
    P = lib
    for dim, n in [(2, 64), (3, 12)]:
        pb = hi.volume_problem(n, dim, smooth_seed=3)
        pb.c = 1.0 + 0.25 * hi.smooth_field(pb.points, 4)
        rng = np.random.default_rng(0)
        rows = np.concatenate([rng.integers(0, pb.N, 37), [5, 6]]).astype(np.int32)
        cols = np.concatenate([rng.integers(0, pb.N, 23), [5, 7]]).astype(np.int32)
        out = torch.empty((len(cols), len(rows)), dtype=torch.float64, device=DEV).t()
        P.hif_kernel_block(T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c), pb.kernel_id,
                           torch.as_tensor(rows, device=DEV), torch.as_tensor(cols, device=DEV), out)
        op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, pb.kernel_id)
        ref = op.entries(rows, cols)
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=1e-16)


def test_kernel_block_host_pointers(lib):
    P = lib
    pb = hi.volume_problem(16, 2, smooth_seed=3)
    rows = np.arange(0, 256, 7, dtype=np.int32)
    cols = np.arange(3, 256, 11, dtype=np.int32)
    out = np.zeros((len(rows), len(cols)), order="F")
    P.hif_kernel_block(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, rows, cols, out)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    np.testing.assert_allclose(out, op.entries(rows, cols), rtol=1e-13, atol=1e-16)


# --------------------------------------------------------------------- ID --

def _run_id_batched(P, mats, tols):
    off, m, n, poff, toff = [], [], [], [], []
    buf = []
    o = po = to = 0
    for M in mats:
        off.append(o); m.append(M.shape[0]); n.append(M.shape[1]); poff.append(po); toff.append(to)
        buf.append(np.asfortranarray(M).reshape(-1, order="F"))
        o += M.size; po += M.shape[1]; to += M.shape[1] ** 2 // 4 + M.shape[1]
    allm = np.concatenate(buf)
    k = np.zeros(len(mats), dtype=np.int32)
    perm = np.zeros(po, dtype=np.int32)
    Tb = np.zeros(to)
    P.hif_id_batched(allm, np.array(off, dtype=np.int64), np.array(m, dtype=np.int32), np.array(n, dtype=np.int32),
                     np.array(tols, dtype=np.float64), k, perm, np.array(poff, dtype=np.int64), Tb,
                     np.array(toff, dtype=np.int64))
    out = []
    for i, M in enumerate(mats):
        ki, ni = int(k[i]), M.shape[1]
        pm = perm[poff[i]:poff[i] + ni]
        Tm = Tb[toff[i]:toff[i] + ki * (ni - ki)].reshape((ki, ni - ki), order="F")
        out.append((ki, pm, Tm))
    return out


def test_id_batched_matches_oracle(lib):
    P = lib
    rng = np.random.default_rng(1)
    mats, tols = [], []
    for (m, n, k) in [(60, 25, 25), (100, 40, 12), (37, 53, 9), (129, 64, 64), (3, 5, 3), (64, 1, 1)]:
        A = rng.standard_normal((m, min(k, n))) @ rng.standard_normal((min(k, n), n))
        A *= (1.3 ** np.arange(n))[None, :]           # well separated pivots
        mats.append(A)
        tols.append(1e-11)
    # geometric singular values: rank set by the tolerance
    U, _ = np.linalg.qr(rng.standard_normal((90, 30)))
    V, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    mats.append((U * 10.0 ** (-np.arange(30) / 4)) @ V.T)
    tols.append(1e-5)
    mats.append(np.zeros((8, 6)))
    tols.append(1e-6)
    res = _run_id_batched(P, mats, tols)
    for A, tol, (k, pm, Tm) in zip(mats, tols, res):
        sk, rd, Tref = idqr.interp_decomp(A, tol)
        assert k == sk.size
        assert list(pm[:k]) == list(sk)
        assert list(pm[k:]) == list(rd)
        if k and rd.size:
            np.testing.assert_allclose(Tm, Tref, rtol=1e-8, atol=1e-9 * max(1.0, np.abs(Tref).max()))


# ------------------------------------------------------------ direct sum --

@pytest.mark.parametrize("trans", [0, 1])
def test_direct_sum_grid_matches_oracle(lib, trans):
    P = lib
    pb = hi.volume_problem(64, 2, smooth_seed=1002)
    pb.c = 1.0 + 0.3 * hi.smooth_field(pb.points, 17)
    pb.a = 1.0 + 0.1 * hi.smooth_field(pb.points, 18)
    fac = factor(P, pb, 1e-3)
    x = hi.gaussian_rhs(pb.N, 3, 5)
    y = fac.matvec(T(x), trans=bool(trans)).cpu().numpy()
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    np.testing.assert_allclose(y, op.matvec(x, trans=bool(trans)), rtol=1e-12, atol=1e-13)
    fac.close()


def test_direct_sum_paired_fp32_matches_fp64(lib):
    # the paired-FP32 convolution agrees with the FP64 one to ~1e-14
    P = lib
    pb = hi.volume_problem(96, 2, smooth_seed=1002)
    x = T(hi.gaussian_rhs(pb.N, 5, 8))
    f1 = factor(P, pb, 1e-3, direct="df64")
    f2 = factor(P, pb, 1e-3, direct="fp64")
    for trans in (False, True):
        y1 = f1.matvec(x, trans=trans).cpu().numpy()
        y2 = f2.matvec(x, trans=trans).cpu().numpy()
        assert np.abs(y1 - y2).max() <= 1e-13 * np.abs(y2).max()
    f1.close()
    f2.close()


def test_direct_sum_general_points_matches_oracle(lib):
    P = lib
    pb = hi.volume_problem(24, 2, smooth_seed=5)
    rng = np.random.default_rng(2)
    pts = pb.points + rng.uniform(-0.2, 0.2, pb.points.shape) / 24      # breaks the grid structure
    pb.points = pts
    fac = factor(P, pb, 1e-6)
    x = hi.gaussian_rhs(pb.N, 2, 9)
    op = kernels.Operator(pts, pb.weights, pb.a, pb.b, pb.c, 0)
    for trans in (False, True):
        y = fac.matvec(T(x), trans=trans).cpu().numpy()
        np.testing.assert_allclose(y, op.matvec(x, trans=trans), rtol=1e-12, atol=1e-13)
    # the factorization of the jittered points is accurate too
    u = fac.solve(T(pb.f[:, 0])).cpu().numpy()
    assert relerr(u, dense.DenseSolver(op).solve(pb.f[:, 0])) <= 100e-6
    fac.close()


def test_direct_sum_3d_grid(lib):
    P = lib
    pb = hi.volume_problem(12, 3, smooth_seed=8)
    fac = factor(P, pb, 1e-3, occupancy=27)
    x = hi.gaussian_rhs(pb.N, 2, 3)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 1)
    np.testing.assert_allclose(fac.matvec(T(x)).cpu().numpy(), op.matvec(x), rtol=1e-12, atol=1e-13)
    fac.close()


# ---------------------------------------------------------- factorization --

def test_n64_eps1e6_accuracy_and_rank_parity(lib):
    """n=64 (N=4096), log kernel, a=1, b=c=1, eps=1e-6, FP64, 1 RHS."""
    P = lib
    eps = 1e-6
    pb = hi.volume_problem(64, 2, rhs_seed=1001)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    ds = dense.DenseSolver(op)
    Fo = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, eps, pb.proxy)
    fac = factor(P, pb, eps)
    st = fac.stats()
    # same partition: boxes per sublevel
    assert [s["boxes"] for s in st["per_sublevel"]] == [len(sl.boxes) for sl in Fo.sublevels]
    # skeleton totals within 10% of the CPU HIF, sublevel by sublevel, and |s_L|
    for s, sl in zip(st["per_sublevel"], Fo.sublevels):
        ko = sum(b.sk.size for b in sl.boxes)
        assert abs(s["skeletons"] - ko) <= 0.1 * ko + 2
    assert abs(st["top_size"] - Fo.sL) <= 0.1 * Fo.sL
    f = pb.f[:, 0]
    u = fac.solve(T(f)).cpu().numpy()
    assert relerr(u, ds.solve(f)) <= 100 * eps
    x = hi.gaussian_rhs(pb.N, 1, 77)[:, 0]
    assert relerr(fac.apply(T(x)).cpu().numpy(), ds.matvec(x)) <= 10 * eps
    # GPU and CPU factorizations agree with each other to the same order
    assert relerr(u, Fo.solve(f)) <= 100 * eps
    fac.close()


@pytest.mark.parametrize("eps", [1e-3, 1e-9])
def test_accuracy_bounds_smooth_coefficients(lib, eps):
    P = lib
    pb, op, ds, _ = oracle_setup(32, smooth=1002, eps=1e-6)
    fac = factor(P, pb, eps)
    f = pb.f[:, 0]
    assert relerr(fac.solve(T(f)).cpu().numpy(), ds.solve(f)) <= 100 * eps
    x = hi.gaussian_rhs(pb.N, 1, 3)[:, 0]
    assert relerr(fac.apply(T(x)).cpu().numpy(), ds.matvec(x)) <= 10 * eps
    fac.close()


def test_transposes_and_identities(lib):
    P = lib
    eps = 1e-6
    pb, op, ds, Fo = oracle_setup(32, smooth=1002, eps=eps)
    pb = hi.volume_problem(32, 2, smooth_seed=1002)
    pb.c = 1.0 + 0.5 * hi.smooth_field(pb.points, 99)   # b != c: A not symmetric
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    ds = dense.DenseSolver(op)
    fac = factor(P, pb, eps)
    X = hi.gaussian_rhs(pb.N, 4, 11)
    Xt = T(X)
    np.testing.assert_allclose(fac.apply(fac.solve(Xt)).cpu().numpy(), X, rtol=0, atol=1e-12 * np.abs(X).max())
    np.testing.assert_allclose(fac.apply_transpose(fac.solve_transpose(Xt)).cpu().numpy(), X, rtol=0,
                               atol=1e-12 * np.abs(X).max())
    assert relerr(fac.solve_transpose(Xt).cpu().numpy(), ds.solve(X, trans=True)) <= 100 * eps
    assert relerr(fac.apply_transpose(Xt).cpu().numpy(), ds.matvec(X, trans=True)) <= 10 * eps
    Y = hi.gaussian_rhs(pb.N, 4, 12)
    lhs = np.sum(fac.solve(Xt).cpu().numpy() * Y)
    rhs = np.sum(X * fac.solve_transpose(T(Y)).cpu().numpy())
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
    # multi-RHS equals column-by-column
    one = fac.solve(T(X[:, 2])).cpu().numpy()
    np.testing.assert_allclose(fac.solve(Xt).cpu().numpy()[:, 2], one, rtol=1e-14, atol=1e-15)
    fac.close()


def test_eps_zero_is_dense_lu(lib):
    P = lib
    pb = hi.volume_problem(16, 2, smooth_seed=2)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    fac = factor(P, pb, 0.0, occupancy=16)
    I = T(np.eye(pb.N))
    Fd = fac.apply(I).cpu().numpy()
    A = op.dense()
    assert np.abs(Fd - A).max() <= 1e-12 * np.abs(A).max()
    fac.close()


@pytest.mark.parametrize("n,occ", [(4, 64), (4, 1), (7, 4), (48, 64), (20, 16)])
def test_edge_sizes_against_dense(lib, n, occ):
    # N below the leaf size (top block only), single-DOF leaves, ragged grids
    P = lib
    eps = 1e-8
    pb = hi.volume_problem(n, 2, smooth_seed=6)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    ds = dense.DenseSolver(op)
    fac = factor(P, pb, eps, occupancy=occ)
    f = pb.f[:, 0]
    assert relerr(fac.solve(T(f)).cpu().numpy(), ds.solve(f)) <= 100 * eps
    fac.close()


def test_second_kind_modification_on_gpu(lib):
    P = lib
    pb, op, ds, _ = oracle_setup(32, smooth=1002)
    x = hi.gaussian_rhs(pb.N, 1, 0)[:, 0]
    Ax = ds.matvec(x)
    errs = {}
    for mode in (False, True):
        fac = factor(P, pb, 1e-6, second_kind=mode)
        errs[mode] = relerr(fac.apply(T(x)).cpu().numpy(), Ax)
        fac.close()
    assert errs[False] > 5 * errs[True]


def test_3d_cells_faces_edges(lib):
    P = lib
    eps = 1e-3
    pb = hi.volume_problem(12, 3)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 1)
    ds = dense.DenseSolver(op)
    fac = factor(P, pb, eps, occupancy=27)
    st = fac.stats()
    assert [s["kind"] for s in st["per_sublevel"][:3]] == ["cell", "face", "edge"]
    f = pb.f[:, 0]
    assert relerr(fac.solve(T(f)).cpu().numpy(), ds.solve(f)) <= 100 * eps
    x = hi.gaussian_rhs(pb.N, 1, 5)[:, 0]
    assert relerr(fac.apply(T(x)).cpu().numpy(), ds.matvec(x)) <= 10 * eps
    Fo = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 1, eps, pb.proxy, occupancy=27)
    assert abs(st["top_size"] - Fo.sL) <= 0.1 * Fo.sL
    fac.close()


# -------------------------------------------------------------- refinement --

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("method", ["ir", "gmres"])
def test_refined_solve_to_1e10(lib, precision, method):
    P = lib
    pb, op, ds, _ = oracle_setup(64, smooth=1002, eps=1e-6)
    fac = factor(P, pb, 1e-6, precision=precision)
    F = hi.gaussian_rhs(pb.N, 3, 21)
    u, its, rel = fac.solve_refined(T(F), tol=1e-10, method=method)
    assert rel <= 1e-10
    ud = ds.solve(F)
    assert relerr(u.cpu().numpy(), ud) <= 1e-9
    r = F - op.matvec(u.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(F) <= 1e-10
    fac.close()


def test_fp32_factorization_accuracy(lib):
    P = lib
    pb, op, ds, _ = oracle_setup(64, smooth=1002, eps=1e-6)
    fac = factor(P, pb, 1e-6, precision="fp32")
    f = pb.f[:, 0]
    e = relerr(fac.solve(T(f)).cpu().numpy(), ds.solve(f))
    assert e <= 1e-4
    fac.close()


def test_host_and_device_pointers_agree(lib):
    P = lib
    pb = hi.volume_problem(32, 2, smooth_seed=4)
    h1 = P.hif_factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, 1e-6)          # host arrays
    fac = factor(P, pb, 1e-6)                                                      # device arrays
    f = np.asfortranarray(pb.f)
    x_host = np.zeros_like(f)
    P.hif_solve(h1, f, x_host)
    x_dev = fac.solve(T(f)).cpu().numpy()
    np.testing.assert_allclose(x_host, x_dev, rtol=1e-13, atol=1e-15)
    P.hif_destroy(h1)
    fac.close()


def test_full_size_refined_solve_residual_by_oracle_rows(lib):
    # the bench workload end to end: n = 1024 (N = 1,048,576), FP32
    # factorization, 8 right-hand sides refined to 1e-10; the residual
    # f - A u is then recomputed at sampled rows by the oracle's own FP64
    # operator, independent of the GPU direct sum
    P = lib
    pb = hi.volume_problem(1024, 2, smooth_seed=1002, rhs_seed=1003, nrhs=8)
    fac = factor(P, pb, 1e-6, precision="fp32")
    u, its, rel = fac.solve_refined(T(pb.f), tol=1e-10)
    assert rel <= 1e-10
    u = u.cpu().numpy()
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    _check_residual_norm_by_rows(op, pb.f, u, seed=5)
    fac.close()


def _check_residual_norm_by_rows(op, F, u, seed, rows_n=64):
    """Estimate |f - A u| per column from uniformly sampled rows of the
    oracle's FP64 operator: sqrt(N / |rows|) |r_rows| is an unbiased
    estimate of |r|^2 under the square root.  With 64 rows its relative
    spread is about 10% for residuals without a few dominant entries, so a
    bound of 3e-10 |f| separates a 1e-10 residual from anything near 1e-9."""
    N = F.shape[0]
    rows = np.random.default_rng(seed).choice(N, rows_n, replace=False)
    r = F[rows] - op.matvec_rows(u, rows)
    est = np.sqrt(N / rows_n) * np.linalg.norm(r, axis=0)
    fn = np.linalg.norm(F, axis=0)
    assert np.all(est <= 3e-10 * fn), (est / fn)
    return est / fn


@pytest.mark.slow
def test_full_size_3d_refined_solve_residual_by_oracle_rows(lib):
    # the 3D workload: n = 64 cube (N = 262,144), eps = 1e-3, FP32
    # factorization, 16 right-hand sides refined to 1e-10
    P = lib
    pb = hi.volume_problem(64, 3, smooth_seed=2002, rhs_seed=2003, nrhs=16)
    fac = factor(P, pb, 1e-3, precision="fp32")
    u, its, rel = fac.solve_refined(T(pb.f), tol=1e-10, maxit=60)
    assert rel <= 1e-10
    u = u.cpu().numpy()
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 1)
    _check_residual_norm_by_rows(op, pb.f, u, seed=6)
    fac.close()


@pytest.mark.parametrize("n,occ", [(12, 27), (16, 64)])
def test_3d_eps_1e6_against_dense(lib, n, occ):
    # the 3D grid at the tighter tolerance: cells -> faces -> edges at
    # eps = 1e-6 with b = c = 1 + 0.5 phi, FP64, against the dense solve
    P = lib
    eps = 1e-6
    pb = hi.volume_problem(n, 3, smooth_seed=1008, rhs_seed=1009, nrhs=2)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 1)
    ds = dense.DenseSolver(op)
    fac = factor(P, pb, eps, occupancy=occ)
    st = fac.stats()
    assert [s["kind"] for s in st["per_sublevel"][:3]] == ["cell", "face", "edge"]
    assert relerr(fac.solve(T(pb.f)).cpu().numpy(), ds.solve(pb.f)) <= 100 * eps
    x = hi.gaussian_rhs(pb.N, 2, 9)
    assert relerr(fac.apply(T(x)).cpu().numpy(), ds.matvec(x)) <= 10 * eps
    # refined to 1e-10 against the dense solution
    u, its, rel = fac.solve_refined(T(pb.f), tol=1e-10)
    assert rel <= 1e-10 and relerr(u.cpu().numpy(), ds.solve(pb.f)) <= 1e-9
    fac.close()
