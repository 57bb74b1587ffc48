"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms verified by independent quadrature, potential-theory identities, exact
low-rank reconstruction, LAPACK's pivoted QR, the paper's product formula
(Eq. (4.1)) multiplied out densely, the dense LU solve, and the paper's
accuracy and second-kind claims (Sec. 4.4, Sec. 5 Example 2).
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.linalg as sla

import hif_inputs as hi
from oracle import dense, hifie, idqr, kernels, krylov


def _golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")
    out = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, val, _cite = line.split()
        out[name] = float(val)
    return out


GOLD = _golden()


# ----------------------------------------------------------------- kernels ---

def test_green_functions_eq_1_4():
    # G(1) = 0 for the log kernel, G(r) = -log(r)/(2 pi); 1/(4 pi r) in 3D
    assert kernels.green(0, np.array([1.0]))[0] == 0.0
    assert kernels.green(0, np.array([math.e]))[0] == pytest.approx(-1 / (2 * math.pi))
    assert kernels.green(1, np.array([2.0]))[0] == pytest.approx(1 / (8 * math.pi))


@pytest.mark.parametrize("h", [1.0, 1.0 / 64, 1.0 / 1024])
def test_self_cell_2d_matches_quadrature(h):
    # independent quadrature: polar coordinates over 1/8 of the square,
    # integrand log(r) r is smooth; 8 symmetric triangles
    a = h / 2
    val, _ = si.dblquad(lambda r, t: math.log(r) * r, 0.0, math.pi / 4,
                        lambda t: 0.0, lambda t: a / math.cos(t), epsabs=1e-15, epsrel=1e-12)
    ref = -(8 * val) / (2 * math.pi)
    got = kernels.self_integral(0, np.array([h * h]))[0]
    assert got == pytest.approx(ref, rel=1e-10)


def test_unit_square_log_integral_textbook():
    # int_0^1 int_0^1 ln(s^2 + t^2) = ln 2 - 3 + pi/2 (closed form the 2D self term rests on)
    val, _ = si.dblquad(lambda r, t: math.log(r * r) * r, 0.0, math.pi / 4,
                        lambda t: 0.0, lambda t: 1.0 / math.cos(t), epsabs=1e-14)
    assert 2 * val == pytest.approx(math.log(2) - 3 + math.pi / 2, rel=1e-10)


@pytest.mark.parametrize("h", [1.0, 1.0 / 64])
def test_self_cell_3d_matches_quadrature(h):
    # six pyramids with apex at the centre: y = x (1, u, v), dy = x^2 dx du dv,
    # int_{[-a,a]^3} 1/|y| = 6 (a^2/2) int_{[-1,1]^2} (1 + u^2 + v^2)^(-1/2) du dv
    a = h / 2
    val, _ = si.dblquad(lambda u, v: 1.0 / math.sqrt(1 + u * u + v * v), -1, 1, -1, 1,
                        epsabs=1e-14, epsrel=1e-12)
    ref = 6 * (a * a / 2) * val / (4 * math.pi)
    got = kernels.self_integral(1, np.array([h ** 3]))[0]
    assert got == pytest.approx(ref, rel=1e-10)


def test_double_layer_gauss_identity_sign():
    # Eq. (1.5): on a circle the double-layer kernel is the constant -1/(4 pi R);
    # the principal value of sigma = 1 is -1/2, the jump adds -1/2, and the total
    # equals the interior value int dG/dnu = -1 (trapezoid rule is exact here).
    R, M = 0.7, 400
    t = 2 * math.pi * np.arange(M) / M
    y = R * np.stack([np.cos(t), np.sin(t)], axis=1)
    nu = y / R
    ds = 2 * math.pi * R / M
    x0 = y[0]
    pv = kernels.double_layer_2d(x0[None, :], y[1:], nu[1:]).sum() * ds
    # the constant kernel value, integrated over the whole circle
    assert pv + (-1 / (4 * math.pi * R)) * ds == pytest.approx(-0.5, abs=1e-12)
    inner = kernels.double_layer_2d(np.array([[0.1, -0.2]]), y, nu).sum() * ds
    assert inner == pytest.approx(-1.0, abs=1e-12)
    assert GOLD["double_layer_jump"] + pv + (-1 / (4 * math.pi * R)) * ds == pytest.approx(inner, abs=1e-12)


def test_operator_structure():
    pb = hi.volume_problem(12, 2)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    A = op.dense()
    # b = c = 1: K symmetric
    assert np.allclose(A, A.T, atol=0, rtol=1e-15)
    # translation invariance of the one-point rule on the uniform grid
    n = 12
    i, j = 3 * n + 4, 7 * n + 2
    assert A[i, j] == pytest.approx(A[i + n + 1, j + n + 1], rel=1e-14)
    # diagonal: a + b K_ii c with the closed-form K_ii
    assert A[5, 5] == pytest.approx(1.0 + kernels.self_integral(0, pb.weights[:1])[0], rel=1e-15)
    # one-point off-diagonal: -log(r)/(2 pi) h^2
    h = 1.0 / n
    assert A[0, 1] == pytest.approx(-math.log(h) / (2 * math.pi) * h * h, rel=1e-14)


def test_operator_b_scales_rows_c_scales_columns():
    # Eq. (1.1): b multiplies the integral (the row of DOF i), c sits inside it
    # (the column of DOF j), a only the diagonal; scaling one coefficient
    # entry must move exactly that row, column or diagonal entry
    pb = hi.volume_problem(10, 2, smooth_seed=5)
    N = pb.N
    A = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0).dense()
    Kpart = A - np.diag(pb.a)
    i, j = 17, 42
    b2, c2, a2 = pb.b.copy(), pb.c.copy(), pb.a.copy()
    b2[i] *= 3.0
    c2[j] *= 3.0
    a2[i] += 0.5
    Db = kernels.Operator(pb.points, pb.weights, pb.a, b2, pb.c, 0).dense() - A
    Dc = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, c2, 0).dense() - A
    Da = kernels.Operator(pb.points, pb.weights, a2, pb.b, pb.c, 0).dense() - A
    others = np.arange(N) != i
    assert np.all(Db[others] == 0.0)
    np.testing.assert_allclose(Db[i], 2.0 * Kpart[i], rtol=1e-13, atol=0)
    others = np.arange(N) != j
    assert np.all(Dc[:, others] == 0.0)
    np.testing.assert_allclose(Dc[:, j], 2.0 * Kpart[:, j], rtol=1e-13, atol=0)
    E = np.zeros((N, N))
    E[i, i] = 0.5
    np.testing.assert_allclose(Da, E, rtol=0, atol=1e-15)


def test_direct_sum_rows_match_full():
    pb = hi.volume_problem(10, 2, smooth_seed=5)
    c = pb.c * (1.0 + 0.5 * hi.smooth_field(pb.points, 6))          # b != c: A^T != A
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, c, 0)
    x = np.random.default_rng(3).standard_normal(op.N)
    y = op.matvec(x, block=37)
    yt = op.matvec(x, trans=True, block=29)
    rows = [0, 17, 55, 99]
    assert np.allclose(op.matvec_rows(x, rows), y[rows], rtol=1e-14, atol=1e-15)
    assert np.allclose(op.matvec_rows(x, rows, trans=True), yt[rows], rtol=1e-14, atol=1e-15)
    # A^T x differs from A x when b != c only through the scaling: check with the dense matrix
    A = op.dense()
    assert np.allclose(A.T @ x, yt, rtol=1e-13, atol=1e-15)
    assert not np.allclose(y, yt, rtol=1e-6)


# ---------------------------------------------------------------------- ID ---

def test_id_exact_low_rank():
    rng = np.random.default_rng(0)
    for m, n, k in [(50, 20, 7), (30, 30, 12), (10, 40, 10)]:
        Y = rng.standard_normal((m, k)) @ rng.standard_normal((k, n))
        sk, rd, T = idqr.interp_decomp(Y, 1e-12)
        assert sk.size == k
        assert sorted(np.concatenate([sk, rd]).tolist()) == list(range(n))
        err = np.linalg.norm(Y[:, rd] - Y[:, sk] @ T, 2)
        assert err <= 1e-11 * np.linalg.norm(Y, 2)


def test_id_bounds_eq_2_3():
    rng = np.random.default_rng(1)
    m, n = 80, 40
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sv = 10.0 ** (-np.arange(n) / 3.0)
    Y = (U * sv) @ V.T
    f = GOLD["id_f"]
    for tol in [1e-2, 1e-5, 1e-9]:
        sk, rd, T = idqr.interp_decomp(Y, tol)
        k = sk.size
        assert np.linalg.norm(T, 2) <= math.sqrt(f * f * k * (n - k)) + 1e-12
        E = np.linalg.norm(Y[:, rd] - Y[:, sk] @ T, 2)
        assert E <= math.sqrt(1 + f * f * k * (n - k)) * sv[k]
        # the adaptive rank keeps E near tol |Y|
        assert E <= 10 * tol * sv[0] * math.sqrt(1 + f * f * k * (n - k))


def test_id_pivots_match_lapack_geqp3():
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((60, 25)) * (1.5 ** np.arange(25))[None, :]
    _, R, piv = sla.qr(Y, pivoting=True, mode="economic")
    sk, rd, T = idqr.interp_decomp(Y, 1e-13)
    assert sk.size == 25
    assert list(sk[:10]) == list(piv[:10])


def test_id_tie_break_lowest_index():
    Y = np.zeros((5, 4))
    Y[:, 1] = [1, 2, 3, 4, 5]
    Y[:, 3] = [1, 2, 3, 4, 5]
    Y[:, 0] = [0.1, 0, 0, 0, 0]
    sk, rd, T = idqr.interp_decomp(Y, 1e-6)
    assert sk[0] == 1
    assert 3 in rd


def test_norm2_estimate():
    rng = np.random.default_rng(4)
    U, _ = np.linalg.qr(rng.standard_normal((40, 10)))
    V, _ = np.linalg.qr(rng.standard_normal((10, 10)))
    s = np.array([3.0, 1.0, 0.9, 0.5, 0.3, 0.2, 0.1, 0.05, 0.01, 0.0])
    Y = (U * s) @ V.T
    assert idqr.norm2_estimate(Y) == pytest.approx(3.0, rel=1e-6)
    assert idqr.norm2_estimate(np.zeros((4, 3))) == 0.0


# --------------------------------------------------------- factorization ---

def _setup(n, dim=2, smooth=None, **kw):
    pb = hi.volume_problem(n, dim, smooth_seed=smooth)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, pb.kernel_id)
    return pb, op


@pytest.mark.parametrize("b_ne_c", [False, True])
def test_sweeps_match_product_formula_eq_4_1(b_ne_c):
    # the four factored-form sweeps against the dense product of Eq. (4.1);
    # with b != c (LU boxes, a non-symmetric top block) every transpose shows
    pb, op = _setup(12 if b_ne_c else 8, smooth=11)
    c = pb.c * (1.0 + 0.5 * hi.smooth_field(pb.points, 12)) if b_ne_c else pb.c
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, c, 0)
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, c, 0, 1e-4, pb.proxy, occupancy=4)
    assert any(bf.rd.size for sl in F.sublevels for bf in sl.boxes)
    if b_ne_c:
        assert not np.allclose(F.top_A, F.top_A.T)
    Fd = F.dense_F()
    I = np.eye(op.N)
    assert np.allclose(F.apply(I), Fd, rtol=0, atol=1e-13)
    assert np.allclose(F.apply_transpose(I), Fd.T, rtol=0, atol=1e-13)
    Fi = np.linalg.inv(Fd)
    assert np.allclose(F.solve(I), Fi, rtol=0, atol=1e-11)
    assert np.allclose(F.solve_transpose(I), Fi.T, rtol=0, atol=1e-11)


def test_skeletonization_decouples_redundant_dofs_lemma_2_3():
    # U_0^T A V_0 over the first sublevel: each box's redundant block is D_c and
    # its rows/columns are decoupled from everything else up to the ID error.
    pb, op = _setup(16, smooth=3)
    eps = 1e-5
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, eps, pb.proxy, occupancy=64)
    Us, Vs, _ = F.dense_factors()
    A = op.dense()
    Z = Us[0].T @ A @ Vs[0]
    first = F.sublevels[0]
    rd_all = np.concatenate([bf.rd for bf in first.boxes])
    assert rd_all.size > 0
    scale = np.abs(A - np.diag(np.diag(A))).max()
    for bf in first.boxes:
        if not bf.rd.size:
            continue
        assert np.allclose(Z[np.ix_(bf.rd, bf.rd)], np.diag(bf.D), atol=50 * eps * scale)
        others = np.setdiff1d(np.arange(op.N), bf.rd)
        assert np.abs(Z[np.ix_(bf.rd, others)]).max() <= 50 * eps * scale
        assert np.abs(Z[np.ix_(others, bf.rd)]).max() <= 50 * eps * scale


def test_proxy_id_interpolates_full_far_field_lemma_3_1():
    # b != c so that the incoming and outgoing proxy rows span different spaces
    pb, _ = _setup(32, smooth=7)
    pb.c = 1.0 + 0.5 * hi.smooth_field(pb.points, 8)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    eps = 1e-6
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, eps, pb.proxy)
    A = op.dense()
    checked = 0
    for bf in F.sublevels[0].boxes[:6]:
        c = np.concatenate([bf.sk, bf.rd])
        rest = np.setdiff1d(np.arange(op.N), c)
        W = np.vstack([A[np.ix_(rest, c)], A[np.ix_(c, rest)].T])
        ci = {g: i for i, g in enumerate(c)}
        sk = [ci[g] for g in bf.sk]
        rd = [ci[g] for g in bf.rd]
        err = np.linalg.norm(W[:, rd] - W[:, sk] @ bf.T, 2)
        assert err <= 100 * eps * np.linalg.norm(W, 2)
        checked += 1
    assert checked == 6


def test_sci_coupled_dofs_join_near_field_sec_4_3():
    # With a proxy circle of radius 1.0 w the SCI-coupled DOFs of an edge reach
    # outside it; the near field must include them (Sec. 4.3) for the error to
    # stay at the level reached with the standard radius 1.5 w.
    pb, op = _setup(32, smooth=1002)
    x = np.random.default_rng(0).standard_normal(op.N)
    Ax = op.matvec(x)
    errs = []
    for R in (1.5, 1.0):
        F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, 1e-6, pb.proxy, proxy_radius=R)
        errs.append(np.linalg.norm(F.apply(x) - Ax) / np.linalg.norm(Ax))
    assert errs[1] <= 2 * errs[0]


def test_proxy_rows_span_far_field_lemma_3_3():
    # Four tight clusters in the corner cells: each near field is empty, so the
    # ID rests on the proxy rows alone.  With b != c the outgoing rows (scaled
    # by c_j) and the incoming rows (scaled by b_j) are both needed to
    # interpolate the full far field W_c = [A_{F,c}; A_{c,F}^T].
    g = 0.0025 + 0.005 * np.arange(4)
    blob = np.stack(np.meshgrid(g, g, indexing="ij"), axis=-1).reshape(-1, 2)
    pts = np.vstack([blob, blob * [1, -1] + [0, 1], blob * [-1, 1] + [1, 0], 1 - blob])
    N = pts.shape[0]
    w = np.full(N, 0.005 ** 2)
    rng = np.random.default_rng(9)
    a = np.ones(N)
    b = 1.0 + 0.5 * rng.uniform(-1, 1, N)
    c = 1.0 + 0.5 * rng.uniform(-1, 1, N)
    eps = 1e-8
    F = hifie.factor(pts, w, a, b, c, 0, eps, hi.proxy_directions(2), occupancy=16)
    op = kernels.Operator(pts, w, a, b, c, 0)
    A = op.dense()
    boxes = [bf for bf in F.sublevels[0].boxes]
    assert len(boxes) == 4 and all(bf.m == 128 for bf in boxes)
    assert sum(bf.rd.size for bf in boxes) > 0
    for bf in boxes:
        cidx = np.concatenate([bf.sk, bf.rd])
        rest = np.setdiff1d(np.arange(N), cidx)
        W = np.vstack([A[np.ix_(rest, cidx)], A[np.ix_(cidx, rest)].T])
        pos = {gg: i for i, gg in enumerate(cidx)}
        sk = [pos[gg] for gg in bf.sk]
        rd = [pos[gg] for gg in bf.rd]
        err = np.linalg.norm(W[:, rd] - W[:, sk] @ bf.T, 2)
        assert err <= 100 * eps * np.linalg.norm(W, 2)


def test_sci_groups_lemma_4_2_and_half_edges():
    # Lemma 4.2: columns i, j share a sparsity pattern iff
    # (S^T S)_ij = max(nnz_i, nnz_j)
    rng = np.random.default_rng(3)
    base = rng.uniform(size=(30, 5)) < 0.4
    pat = base[:, rng.integers(0, 5, size=40)]
    groups = hifie.sci_groups(pat)
    Bm = pat.T.astype(int) @ pat.astype(int)
    nnz = pat.sum(axis=0)
    gid = np.empty(40, dtype=int)
    for q, gg in enumerate(groups):
        gid[gg] = q
    for i in range(40):
        for j in range(40):
            assert (gid[i] == gid[j]) == (Bm[i, j] == max(nnz[i], nnz[j]))
    # Fig. 4.4: after cell skeletonization an edge splits into the half-edges of
    # its two cells, so the first edge sublevel compresses at least two groups
    pb, _ = _setup(32, smooth=1)
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, 1e-6, pb.proxy)
    edges = F.sublevels[1]
    assert edges.kind == "edge"
    assert np.median([bf.ngroups for bf in edges.boxes]) >= 2
    F1 = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, 1e-6, pb.proxy, second_kind=False)
    assert all(bf.ngroups == 1 for sl in F1.sublevels for bf in sl.boxes)


def test_eps_zero_reproduces_dense():
    pb, op = _setup(16, smooth=2)
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, 0.0, pb.proxy, occupancy=16)
    A = op.dense()
    I = np.eye(op.N)
    assert np.abs(F.apply(I) - A).max() <= 1e-12 * np.abs(A).max()
    ds = dense.DenseSolver(op)
    f = pb.f[:, 0]
    assert np.linalg.norm(F.solve(f) - ds.solve(f)) <= 1e-12 * np.linalg.norm(ds.solve(f))


@pytest.mark.parametrize("n,occ", [(4, 1), (4, 4), (8, 1), (8, 4)])
def test_brute_force_tiny(n, occ):
    pb, op = _setup(n, smooth=1)
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, 1e-12, pb.proxy, occupancy=occ)
    A = op.dense()
    Fd = F.apply(np.eye(op.N))
    assert np.linalg.norm(Fd - A, 2) <= 1e-10 * np.linalg.norm(A, 2)


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_accuracy_bounds_2d(eps):
    pb, op = _setup(32, smooth=1002)
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, eps, pb.proxy)
    ds = dense.DenseSolver(op)
    x = np.random.default_rng(0).standard_normal(op.N)
    Ax = ds.matvec(x)
    assert np.linalg.norm(F.apply(x) - Ax) <= 10 * eps * np.linalg.norm(Ax)
    f = pb.f[:, 0]
    u = ds.solve(f)
    assert np.linalg.norm(F.solve(f) - u) <= 100 * eps * np.linalg.norm(u)
    # factored inverse is an exact inverse of the factored operator
    assert np.linalg.norm(F.apply(F.solve(x)) - x) <= 1e-13 * np.linalg.norm(x)
    y = np.random.default_rng(1).standard_normal(op.N)
    assert abs(F.solve(x) @ y - x @ F.solve_transpose(y)) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)


def test_symmetry_test_matches_dense_transpose():
    # b = c with equal weights gives A = A^T; b != c or unequal weights do not
    pb, op = _setup(8, smooth=5)
    A = op.dense()
    assert hifie.is_symmetric(op)
    assert np.allclose(A, A.T, rtol=1e-15, atol=0)
    c2 = pb.c * (1.0 + 0.1 * hi.smooth_field(pb.points, 6))
    op2 = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, c2, 0)
    A2 = op2.dense()
    assert not hifie.is_symmetric(op2)
    assert np.abs(A2 - A2.T).max() > 1e-6 * np.abs(A2).max()
    w3 = pb.weights.copy()
    w3[0] *= 1.5
    op3 = kernels.Operator(pb.points, w3, pb.a, pb.b, pb.c, 0)
    assert not hifie.is_symmetric(op3)
    assert not np.allclose(op3.dense(), op3.dense().T, rtol=1e-12, atol=0)
    with pytest.raises(ValueError):
        hifie.factor(pb.points, pb.weights, pb.a, pb.b, c2, 0, 1e-6, pb.proxy, symmetric=True)


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_symmetric_compression_equals_full_sec_5(eps):
    # Sec. 5: for symmetric A the one-sided Y'_c holds every row of Y_c once,
    # so Y_c^T Y_c = 2 Y'_c^T Y'_c: the same skeletons in the same pivot
    # order with half the rows, and the same factorization F.  T itself is
    # only as stable as the ID's R_11 (rounding in the SCI blocks moves it by
    # up to ~1e-16 / eps^2 on the later sublevels), so it is compared on the
    # first sublevel, and F as an operator
    pb, op = _setup(32, smooth=1002)
    Fs = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, eps, pb.proxy, symmetric=True)
    Ff = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, eps, pb.proxy, symmetric=False)
    assert len(Fs.sublevels) == len(Ff.sublevels)
    nbox = 0
    for t, (ss, sf) in enumerate(zip(Fs.sublevels, Ff.sublevels)):
        assert len(ss.boxes) == len(sf.boxes)
        for bs, bf in zip(ss.boxes, sf.boxes):
            assert 2 * bs.m == bf.m
            assert np.array_equal(bs.sk, bf.sk) and np.array_equal(bs.rd, bf.rd)
            if t == 0 and bs.T.size:
                assert np.abs(bs.T - bf.T).max() <= 1e-6 * max(1.0, np.abs(bf.T).max())
            nbox += 1
    assert nbox >= 40
    assert np.array_equal(Fs.top, Ff.top)
    x = np.random.default_rng(2).standard_normal(op.N)
    for fs, ff in ((Fs.apply, Ff.apply), (Fs.solve, Ff.solve), (Fs.solve_transpose, Ff.solve_transpose)):
        ys, yf = fs(x), ff(x)
        assert np.linalg.norm(ys - yf) <= 1e-12 * np.linalg.norm(yf)


def test_nonsymmetric_accuracy_full_compression():
    # b != c: the full Y_c is compressed and the factorization keeps the
    # accuracy of the symmetric case (Theorem 3.1 / Sec. 4 error model)
    pb, _ = _setup(32, smooth=1002)
    c = 1.0 + 0.5 * hi.smooth_field(pb.points, 1003)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, c, 0)
    assert not hifie.is_symmetric(op)
    eps = 1e-6
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, c, 0, eps, pb.proxy)
    P = pb.proxy.shape[0]
    Fs = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.b, 0, eps, pb.proxy)
    # two rows per near-field DOF and per proxy point, against one when b = c
    assert all(bf.m % 2 == 0 and bf.m >= 2 * P for sl in F.sublevels for bf in sl.boxes)
    assert all(bf.m >= P for sl in Fs.sublevels for bf in sl.boxes)
    assert sum(bf.m for sl in Fs.sublevels for bf in sl.boxes) < sum(bf.m for sl in F.sublevels for bf in sl.boxes)
    ds = dense.DenseSolver(op)
    x = np.random.default_rng(0).standard_normal(op.N)
    Ax = ds.matvec(x)
    assert np.linalg.norm(F.apply(x) - Ax) <= 10 * eps * np.linalg.norm(Ax)
    f = pb.f[:, 0]
    u = ds.solve(f)
    assert np.linalg.norm(F.solve(f) - u) <= 100 * eps * np.linalg.norm(u)


def test_second_kind_fix_matters_sec_4_4():
    # Sec. 4.4 / Example 2: without the rho_c tolerance and split compression the
    # error of hifie2 grows well above that of hifie2x (4.1e-4 vs 5.9e-7 at 512^2).
    assert GOLD["ex2_hifie2_ea_1e-6_512"] > 100 * GOLD["ex2_hifie2x_ea_1e-6_512"]
    pb, op = _setup(32, smooth=1002)
    x = np.random.default_rng(0).standard_normal(op.N)
    Ax = op.matvec(x)
    errs = {}
    for mode in (False, True):
        F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, 1e-6, pb.proxy, second_kind=mode)
        errs[mode] = np.linalg.norm(F.apply(x) - Ax) / np.linalg.norm(Ax)
    assert errs[False] > 5 * errs[True]


def test_3d_accuracy_and_identities():
    pb, op = _setup(12, dim=3)
    eps = 1e-3
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 1, eps, pb.proxy, occupancy=27)
    assert sum(bf.rd.size for sl in F.sublevels for bf in sl.boxes) > 0
    assert [sl.kind for sl in F.sublevels][:3] == ["cell", "face", "edge"]
    ds = dense.DenseSolver(op)
    x = np.random.default_rng(0).standard_normal(op.N)
    Ax = ds.matvec(x)
    assert np.linalg.norm(F.apply(x) - Ax) <= 10 * eps * np.linalg.norm(Ax)
    f = pb.f[:, 0]
    u = ds.solve(f)
    assert np.linalg.norm(F.solve(f) - u) <= 100 * eps * np.linalg.norm(u)
    assert np.linalg.norm(F.apply_transpose(F.solve_transpose(x)) - x) <= 1e-13 * np.linalg.norm(x)


def test_voronoi_partition_covers_and_ties():
    # every active DOF lands in exactly one edge; grid points equidistant from
    # two edge centres go to the lower id
    lo, W = np.zeros(2), 1.0
    s = 4
    ctr = hifie.centers("edge", 2, s, lo, W / s)
    assert ctr.shape[0] == 2 * s * (s - 1)
    p = np.array([[0.25, 0.25]])          # a cell corner: 4 edges at distance 1/8
    d2 = ((p[:, None, :] - ctr[None]) ** 2).sum(axis=2)
    owner = np.argmin(d2, axis=1)[0]
    ties = np.nonzero(d2[0] == d2[0].min())[0]
    assert ties.size == 4 and owner == ties.min()
    c3 = hifie.centers("face", 3, 3, np.zeros(3), 1 / 3)
    assert c3.shape[0] == 3 * 2 * 9
    e3 = hifie.centers("edge", 3, 3, np.zeros(3), 1 / 3)
    assert e3.shape[0] == 3 * 4 * 3


# ----------------------------------------------------------------- krylov ---

def test_gmres_lemma_5_1_iteration_bound():
    rng = np.random.default_rng(5)
    N = 120
    E = rng.standard_normal((N, N))
    E *= 0.1 / np.linalg.norm(E, 2)
    A = np.eye(N) + E
    f = rng.standard_normal(N)
    u, its, hist = krylov.gmres(lambda v: A @ v, f, tol=1e-10)
    assert np.linalg.norm(A @ u - f) <= 1e-10 * np.linalg.norm(f)
    assert its <= math.ceil(math.log(1e-10) / math.log(0.1))
    assert np.allclose(u, np.linalg.solve(A, f), rtol=1e-8)


def test_gmres_exact_preconditioner_one_step():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((50, 50)) + 10 * np.eye(50)
    Ai = np.linalg.inv(A)
    f = rng.standard_normal(50)
    u, its, _ = krylov.gmres(lambda v: A @ v, f, precond=lambda v: Ai @ v, tol=1e-12)
    assert its == 1


def test_error_estimates_match_dense_two_norms():
    # Sec. 5 estimators against the exact 2-norms of the assembled matrices
    pb, op = _setup(16, smooth=4)
    pb.a = np.zeros(op.N)                                     # first kind, Example 1
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    A = op.dense()
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, 1e-4, pb.proxy, occupancy=16)
    I = np.eye(op.N)
    Fd = F.apply(I)
    Fi = F.solve(I)
    ex_a = np.linalg.norm(A - Fd, 2) / np.linalg.norm(A, 2)
    ex_s = np.linalg.norm(I - A @ Fi, 2)
    mv = [lambda v: A @ v, lambda v: A.T @ v, F.apply, F.apply_transpose, F.solve, F.solve_transpose]
    v0 = hi.uniform_vector(op.N, 3)
    ea, es = krylov.error_estimates(*mv, op.N, v0=v0, rtol=1e-12, maxit=5000)
    assert ea == pytest.approx(ex_a, rel=1e-6) and es == pytest.approx(ex_s, rel=1e-6)
    # the paper's stopping rule: from below, within a few percent
    ea2, es2 = krylov.error_estimates(*mv, op.N, v0=v0)
    assert 0.8 * ex_a <= ea2 <= ex_a * (1 + 1e-12)
    assert 0.8 * ex_s <= es2 <= ex_s * (1 + 1e-12)
    # a planted rank-one error of known size
    u = np.random.default_rng(1).standard_normal(op.N)
    u /= np.linalg.norm(u)
    d = 1e-3 * np.linalg.norm(A, 2)
    nE = krylov.power_norm(lambda v: d * u * (u @ v), lambda v: d * u * (u @ v), op.N, v0=v0)
    assert nE == pytest.approx(d, rel=1e-12)


@pytest.mark.parametrize("eps,ni_max", [(1e-3, 8), (1e-6, 4), (1e-9, 3)])
def test_first_kind_example_1_preconditioner(eps, ni_max):
    # Example 1 (a = 0, b = c = 1): F approximates A to O(eps) while
    # |I - A F^{-1}| is far larger (an ill-conditioned first-kind system),
    # and GMRES with F^{-1} as preconditioner still needs only a few steps
    pb = hi.volume_problem(32, 2, a_value=0.0)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    A = op.dense()
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, eps, pb.proxy)
    I = np.eye(op.N)
    Fd = F.apply(I)
    ea = np.linalg.norm(A - Fd, 2) / np.linalg.norm(A, 2)
    es = np.linalg.norm(I - A @ np.linalg.inv(Fd), 2)
    assert ea <= 10 * eps and es >= 20 * ea
    f = hi.uniform_vector(op.N, 5)
    u, its, hist = krylov.gmres(lambda v: A @ v, f, precond=F.solve, tol=1e-12)
    assert hist[-1] <= 1e-12 and its <= ni_max
    assert np.linalg.norm(u - np.linalg.solve(A, f)) <= 1e-8 * np.linalg.norm(u)


def test_rsf_top_block_exceeds_hif():
    # Algorithm 3.1 (cells only) against Algorithm 4.1: without the edge
    # sublevels the top skeleton set |s_L| is larger, and it grows faster
    # with N (Tables of Examples 1-2)
    tops = {}
    for n in (16, 32):
        pb = hi.volume_problem(n, 2, a_value=0.0)
        for frac in (True, False):
            F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, 1e-6, pb.proxy, fractional=frac,
                             occupancy=16)
            assert all(sl.kind == "cell" for sl in F.sublevels) == (not frac)
            tops[n, frac] = F.sL
    assert tops[32, False] > tops[32, True] and tops[16, False] >= tops[16, True]
    assert tops[32, False] - tops[16, False] > tops[32, True] - tops[16, True]


def test_power_iteration_error_estimate():
    d = np.linspace(0.1, 2.0, 64)
    est = krylov.power_norm(lambda v: d * v, lambda v: d * v, 64, rtol=1e-6, maxit=2000)
    assert est == pytest.approx(2.0, rel=1e-3)


# -------------------------------------------------------------------- LDL ---

def test_ldl_diag_pivot_reconstructs_and_pivots_on_largest_diagonal():
    rng = np.random.default_rng(31)
    r = 40
    G = rng.standard_normal((r, r))
    B = 0.1 * (G + G.T) + np.diag(rng.uniform(0.5, 2.0, r) * np.where(rng.random(r) < 0.5, -1.0, 1.0))
    perm, L, D = hifie.ldl_diag_pivot(B)
    Pb = B[np.ix_(perm, perm)]
    np.testing.assert_allclose(L @ np.diag(D) @ L.T, Pb, rtol=0, atol=1e-13 * np.abs(B).max())
    assert np.allclose(np.triu(L, 1), 0.0) and np.allclose(np.diag(L), 1.0)
    # the first pivot is the diagonal entry of largest magnitude
    assert perm[0] == int(np.argmax(np.abs(np.diag(B))))
    # every pivot passes the 1 x 1 Bunch-Kaufman test in its own Schur complement
    Bw = Pb.copy()
    for j in range(r):
        col = np.abs(Bw[j:, j])
        assert abs(Bw[j, j]) >= hifie.LDL_ALPHA * np.delete(col, 0).max(initial=0.0) - 1e-15
        assert abs(Bw[j, j]) >= np.abs(np.diag(Bw)[j:]).max() - 1e-15
        Bw[j + 1:, j + 1:] -= np.outer(Bw[j + 1:, j], Bw[j, j + 1:]) / Bw[j, j]
    # block inverse from the factors equals the dense inverse
    Binv = np.linalg.inv(B)
    Lp = np.zeros_like(L)
    Lp[perm, :] = L
    np.testing.assert_allclose(np.linalg.inv(Lp).T @ np.diag(1 / D) @ np.linalg.inv(Lp), Binv, rtol=1e-10,
                               atol=1e-12 * np.abs(Binv).max())


def test_ldl_diag_pivot_refuses_weak_pivots():
    # [[0, 1], [1, 0]] needs a 2 x 2 pivot; a diagonal below alpha times the
    # column maximum is refused too
    assert hifie.ldl_diag_pivot(np.array([[0.0, 1.0], [1.0, 0.0]])) is None
    assert hifie.ldl_diag_pivot(np.array([[0.5, 1.0], [1.0, 0.4]])) is None
    assert hifie.ldl_diag_pivot(np.array([[0.7, 1.0], [1.0, 2.0]])) is not None


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
def test_ldl_factor_equals_lu_factor(eps):
    # Sec. 5: LDL changes how the block inverse is formed, not its value;
    # same skeletons, same F and F^{-1} to rounding, Y = X^T, a symmetric
    # factorization (F = F^T) and a smaller store
    pb = hi.volume_problem(32, 2, smooth_seed=1002)
    args = (pb.points, pb.weights, pb.a, pb.b, pb.c, 0, eps, pb.proxy)
    Fl = hifie.factor(*args, ldl=True)
    Fu = hifie.factor(*args, ldl=False)
    nl = sum(bf.ldl for sl in Fl.sublevels for bf in sl.boxes)
    assert nl == sum(bf.rd.size > 0 for sl in Fl.sublevels for bf in sl.boxes) > 0
    assert not any(bf.ldl for sl in Fu.sublevels for bf in sl.boxes)
    for sa, sb in zip(Fl.sublevels, Fu.sublevels):
        for ba, bb in zip(sa.boxes, sb.boxes):
            np.testing.assert_array_equal(ba.sk, bb.sk)
            np.testing.assert_array_equal(ba.rd, bb.rd)
            if ba.ldl:
                np.testing.assert_array_equal(ba.Y, ba.X.T)
    X = hi.gaussian_rhs(pb.N, 3, 4)
    for fa, fb in [(Fl.solve, Fu.solve), (Fl.apply, Fu.apply), (Fl.solve_transpose, Fu.solve_transpose),
                   (Fl.apply_transpose, Fu.apply_transpose)]:
        ya, yb = fa(X), fb(X)
        assert np.linalg.norm(ya - yb) <= 1e-11 * np.linalg.norm(yb)
    assert np.linalg.norm(Fl.solve(X) - Fl.solve_transpose(X)) <= 1e-12 * np.linalg.norm(X)
    assert np.linalg.norm(Fl.apply(X) - Fl.apply_transpose(X)) <= 1e-12 * np.linalg.norm(X)
    assert Fl.storage_doubles() < 0.8 * Fu.storage_doubles()


def test_ldl_dense_factors_match_sweeps():
    # the factored form of Eq. (4.1) multiplied out densely, with LDL boxes
    pb = hi.volume_problem(8, 2, smooth_seed=5)
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, 1e-3, pb.proxy, occupancy=4, ldl=True)
    assert any(bf.ldl for sl in F.sublevels for bf in sl.boxes)
    Fd = F.dense_F()
    I = np.eye(pb.N)
    np.testing.assert_allclose(F.apply(I), Fd, rtol=0, atol=1e-12 * np.abs(Fd).max())
    np.testing.assert_allclose(F.solve(Fd), I, rtol=0, atol=1e-11)
