"""Pins of the Helmholtz (Lippmann-Schwinger, Sec. 5 Example 3) oracle.

* G(r) = (i/4) H_0^(1)(k r) against its small- and large-argument forms
  (series of J_0 and Y_0; the Hankel asymptotic expansion).
* The self-cell integral against the k -> 0 limit, where (i/4) H_0^(1)(k r)
  = -(1/2 pi)(log(k r / 2) + gamma) + i/4 + O((k r)^2 log(k r)), i.e. the
  Laplace closed form minus (h^2 / 2 pi)(log(k/2) + gamma) plus i h^2 / 4.
* The real 2 x 2 embedding: entries, products, the adjoint as the transpose,
  and the embedded dense solve equal to the complex dense solve.
* The sequential HIF-IE on the embedding against the complex dense solve:
  apply error <= 10 eps, solve error <= 100 eps, and the proxy rows of
  Lemma 3.3 interpolating the whole far field for the Helmholtz kernel.
"""
import math

import numpy as np
import pytest
import scipy.special as ss

import hif_inputs as hi
from oracle import helmholtz as hz, hifie, kernels, krylov


def test_green_small_and_large_argument():
    gamma = 0.5772156649015329
    for r in (1e-6, 1e-4):
        k = 3.0
        g = hz.green_helmholtz(k, r)
        approx = -(math.log(k * r / 2) + gamma) / (2 * math.pi) + 0.25j
        assert abs(g - approx) <= 1e-6 * abs(approx)
    for x in (200.0, 1000.0):
        g = hz.green_helmholtz(1.0, x)
        asym = 0.25j * math.sqrt(2 / (math.pi * x)) * np.exp(1j * (x - math.pi / 4)) * (1 - 1j / (8 * x))
        assert abs(g - asym) <= 2e-6 * abs(asym)


@pytest.mark.parametrize("h", [1.0, 1.0 / 64])
def test_self_integral_small_k_limit(h):
    gamma = 0.5772156649015329
    k = 1e-4
    got = hz.self_integral_helmholtz(k, h)
    lap = kernels.self_integral(0, np.array([h * h]))[0]
    limit = lap - h * h / (2 * math.pi) * (math.log(k / 2) + gamma) + 0.25j * h * h
    assert abs(got - limit) <= 1e-7 * abs(limit)


def test_self_integral_matches_brute_force_quadrature():
    # singularity-subtracted tensor Gauss quadrature on the cell, independent
    # of the polar rule: G minus its logarithmic part is bounded
    k, h = 25.0, 1.0 / 16
    gamma = 0.5772156649015329
    x, wq = np.polynomial.legendre.leggauss(60)
    sub = 4
    tot = 0.0 + 0.0j
    for i in range(sub):
        for j in range(sub):
            xa = (-0.5 + (i + 0.5 * (x + 1)) / sub) * h
            ya = (-0.5 + (j + 0.5 * (x + 1)) / sub) * h
            X, Y = np.meshgrid(xa, ya, indexing="ij")
            R = np.sqrt(X * X + Y * Y)
            f = hz.green_helmholtz(k, R) + np.log(R) / (2 * math.pi)
            tot += (f * np.outer(wq, wq)).sum() * (h / sub / 2) ** 2
    lap = kernels.self_integral(0, np.array([h * h]))[0]
    got = hz.self_integral_helmholtz(k, h)
    assert abs(got - (tot + lap)) <= 1e-8 * abs(got)


def test_embedding_is_an_algebra_map():
    rng = np.random.default_rng(2)
    Z = rng.standard_normal((5, 7)) + 1j * rng.standard_normal((5, 7))
    W = rng.standard_normal((7, 3)) + 1j * rng.standard_normal((7, 3))
    v = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    np.testing.assert_allclose(hz.embed_matrix(Z) @ hz.embed_matrix(W), hz.embed_matrix(Z @ W), atol=1e-13)
    np.testing.assert_allclose(hz.embed_matrix(Z).T, hz.embed_matrix(Z.conj().T), atol=0)
    np.testing.assert_allclose(hz.to_complex(hz.embed_matrix(Z) @ hz.to_real(v)), Z @ v, atol=1e-13)


def _ls_problem(n, kappa=1.0):
    pb = hi.helmholtz_problem(n, kappa)
    return pb


def test_embedded_operator_entries_and_dense_solve():
    pb = _ls_problem(12, 2.0)
    cop = hz.HelmholtzOperator(pb.points, pb.weights, pb.a, pb.b, pb.c, pb.k)
    eop = hz.EmbeddedOperator(pb.points, pb.weights, pb.a, pb.b, pb.c, pb.k)
    Ac = cop.dense()
    # complex symmetric with b = c
    np.testing.assert_allclose(Ac, Ac.T, atol=1e-15)
    E = eop.dense()
    np.testing.assert_allclose(E, hz.embed_matrix(Ac), atol=0, rtol=0)
    f = pb.f[:, 0]
    u = np.linalg.solve(Ac, f)
    ue = hz.to_complex(np.linalg.solve(E, hz.to_real(f)))
    np.testing.assert_allclose(ue, u, rtol=1e-12, atol=1e-13)
    # the embedded transpose is the complex adjoint
    x = pb.f[:, 0] * (1 + 0.3j)
    np.testing.assert_allclose(hz.to_complex(E.T @ hz.to_real(x)), Ac.conj().T @ x, atol=1e-12)
    np.testing.assert_allclose(cop.matvec(x, adjoint=True), Ac.conj().T @ x, atol=1e-12)


@pytest.mark.parametrize("eps", [1e-3, 1e-6])
def test_hifie_on_embedding_matches_complex_dense(eps):
    pb = _ls_problem(24, 2.0)
    cop = hz.HelmholtzOperator(pb.points, pb.weights, pb.a, pb.b, pb.c, pb.k)
    Ac = cop.dense()
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 2, eps, pb.proxy, wavenumber=pb.k, occupancy=32)
    assert F.N == 2 * pb.N and len(F.sublevels) >= 2
    rng = np.random.default_rng(4)
    x = rng.standard_normal(pb.N) + 1j * rng.standard_normal(pb.N)
    Ax = Ac @ x
    Fx = hz.to_complex(F.apply(hz.to_real(x)))
    assert np.linalg.norm(Fx - Ax) <= 10 * eps * np.linalg.norm(Ax)
    f = pb.f[:, 0]
    u = np.linalg.solve(Ac, f)
    uf = hz.to_complex(F.solve(hz.to_real(f)))
    assert np.linalg.norm(uf - u) <= 100 * eps * np.linalg.norm(u)
    # F^{-1} preconditions GMRES to a few iterations (Sec. 5, Lemma 5.1)
    E = hz.embed_matrix(Ac)
    ug, its, hist = krylov.gmres(lambda v: E @ v, hz.to_real(f), precond=F.solve, tol=1e-12)
    assert hist[-1] <= 1e-12 and its <= 6
    np.testing.assert_allclose(hz.to_complex(ug), u, rtol=1e-10, atol=1e-12)


def test_embedded_proxy_blocks_are_operator_blocks():
    # Lemma 3.3's proxy blocks are interactions with the proxy points taken as
    # extra DOFs (unit b and c, the box's quadrature weight): Y_{cE,c} =
    # A_{E,c} and the incoming rows (A_{c,E})^T, i.e. the transpose of the
    # embedded block (the embedding of the conjugate-transposed complex block)
    pb = _ls_problem(8, 1.0)
    pb.c = pb.b * (1.0 + 0.5 * hi.smooth_field(pb.points, 77)) + 0.3       # b != c
    box = np.array([9, 10, 17, 18])                                         # complex DOFs
    ctr = pb.points[box].mean(axis=0)
    xE = ctr[None, :] + 0.3 * pb.proxy[:16]
    eop = hz.EmbeddedOperator(pb.points, pb.weights, pb.a, pb.b, pb.c, pb.k)
    cols = np.sort(np.concatenate([2 * box, 2 * box + 1]))                  # real DOFs of the box
    pts = np.vstack([pb.points[box], xE])
    nb, ne = box.size, xE.shape[0]
    one = np.ones(ne)
    ext = hz.EmbeddedOperator(pts, np.full(nb + ne, pb.weights[0]), np.ones(nb + ne),
                              np.concatenate([pb.b[box], one]), np.concatenate([pb.c[box], one]), pb.k)
    bcols = np.arange(2 * nb)                                               # box DOFs in ext, same order
    erows = np.arange(2 * nb, 2 * (nb + ne))                                # proxy points as DOFs
    np.testing.assert_allclose(eop.proxy_out(xE, cols), ext.kernel_entries(erows, bcols), rtol=1e-13, atol=0)
    np.testing.assert_allclose(eop.proxy_in(xE, cols), ext.kernel_entries(bcols, erows).T, rtol=1e-13, atol=0)


@pytest.mark.parametrize("b_ne_c", [False, True])
def test_helmholtz_proxy_rows_span_far_field_lemma_3_3(b_ne_c):
    # the proxy argument of Lemma 3.3 holds for the Helmholtz kernel: the ID
    # of each leaf's Y_c (near rows plus proxy rows) interpolates the leaf's
    # whole far field W_c = [A_{F,c}; A_{c,F}^T] of the embedded operator;
    # with b != c the incoming rows (b_j G w_j, transposed 2 x 2 blocks) carry
    # information the outgoing ones do not
    pb = _ls_problem(32, 1.5)
    if b_ne_c:
        pb.c = pb.b * (1.0 + 0.5 * hi.smooth_field(pb.points, 77)) + 0.3
    eps = 1e-8
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 2, eps, pb.proxy, wavenumber=pb.k, occupancy=128)
    eop = hz.EmbeddedOperator(pb.points, pb.weights, pb.a, pb.b, pb.c, pb.k)
    A = eop.dense()
    N = A.shape[0]
    checked = 0
    for bf in F.sublevels[0].boxes:
        if bf.rd.size == 0:
            continue
        cidx = np.concatenate([bf.sk, bf.rd])
        ctr = eop.x[cidx].mean(axis=0)
        w = 0.25                                   # leaf width: 8 x 8 points (128 real DOFs) of the 32^2 grid
        far = np.nonzero(np.abs(eop.x - ctr).max(axis=1) > 1.5 * w)[0]
        if far.size == 0:
            continue
        W = np.vstack([A[np.ix_(far, cidx)], A[np.ix_(cidx, far)].T])
        pos = {gg: i for i, gg in enumerate(cidx)}
        sk = [pos[gg] for gg in bf.sk]
        rd = [pos[gg] for gg in bf.rd]
        err = np.linalg.norm(W[:, rd] - W[:, sk] @ bf.T, 2)
        assert err <= 100 * eps * np.linalg.norm(W, 2)
        checked += 1
    assert checked > 0
