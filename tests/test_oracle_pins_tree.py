"""Pins of the oracle's tree and of its iterative refinement.

The tree depth and the box counts per sublevel are fixed by the grid
arithmetic of Sec. 4.1/4.2: a level with s cells per side holds s^d cells;
the interior edges of a 2D level are the 2 s (s - 1) sides shared by two
cells; in 3D the interior faces are the 3 (s - 1) s^2 faces shared by two
cells and the interior edges the 3 (s - 1)^2 s edges shared by four.  The
tests count these by brute-force adjacency of cells, independently of the
oracle's index ranges.  Iterative refinement u <- u + F^{-1}(f - A u) is
pinned on A = I + E with a symmetric E whose eigenvalues are +-0.1, where the
residual after k corrections is exactly 0.1^(k+1) |f| with F = I.
"""
import itertools
import math

import numpy as np
import pytest

import hif_inputs as hi
from oracle import hifie, krylov


# ------------------------------------------------------- tree depth -------

@pytest.mark.parametrize("n,dim,occ,L", [(64, 2, 64, 3), (1024, 2, 64, 7), (256, 2, 64, 5),
                                         (64, 3, 64, 4), (32, 2, 64, 2), (64, 2, 16, 4)])
def test_depth_is_smallest_with_occupancy_met(n, dim, occ, L):
    # uniform n^d grid: a leaf of side 2^-L holds (n / 2^L)^d points, so L is
    # the smallest depth with (n / 2^L)^d <= occ
    if dim == 3 and n > 64:
        pytest.skip("large 3D grid")
    pts, w = hi.grid_points(n, dim)
    lo, W = hifie.root_box(pts, w)
    assert W == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(lo, 0.0, atol=1e-15)
    got = hifie.num_levels(pts, lo, W, occ)
    assert got == L
    expect = next(l for l in range(30) if (n // 2**l) ** dim <= occ)
    assert got == expect
    # every leaf cell holds exactly (n / 2^L)^d DOFs
    s = 2**L
    t = hifie.cell_index(pts, lo, W, s)
    flat = np.ravel_multi_index(tuple(t.T), (s,) * dim)
    counts = np.bincount(flat, minlength=s**dim)
    assert counts.min() == counts.max() == (n // s) ** dim


# ------------------------------------------------------- box centres ------

def _cell_centres(s, dim):
    g = (np.arange(s) + 0.5) / s
    mesh = np.meshgrid(*([g] * dim), indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], axis=1), np.stack(
        np.meshgrid(*([np.arange(s)] * dim), indexing="ij"), axis=-1).reshape(-1, dim)


def _shared_entities(s, dim, ncoords):
    """Centres of the entities shared by cells whose integer indices differ
    by one in exactly ``ncoords`` coordinates (1: faces/2D edges, 2: 3D
    edges): the mean of the 2^ncoords cells around each."""
    ctr, idx = _cell_centres(s, dim)
    out = set()
    for axes in itertools.combinations(range(dim), ncoords):
        for base in itertools.product(range(s), repeat=dim):
            if any(base[a] + 1 >= s for a in axes):
                continue
            members = []
            for bits in itertools.product((0, 1), repeat=ncoords):
                j = list(base)
                for a, bb in zip(axes, bits):
                    j[a] += bb
                members.append(np.ravel_multi_index(tuple(j), (s,) * dim))
            c = ctr[members].mean(axis=0)
            out.add(tuple(np.round(c * s * 2).astype(np.int64)))
    return out


@pytest.mark.parametrize("s", [2, 4, 8, 32, 128])
def test_2d_edge_centres_are_interior_cell_sides(s):
    lo = np.zeros(2)
    c = hifie.centers("edge", 2, s, lo, 1.0 / s)
    assert c.shape == (2 * s * (s - 1), 2)
    got = {tuple(v) for v in np.round(c * s * 2).astype(np.int64)}
    assert len(got) == c.shape[0]
    if s <= 32:
        assert got == _shared_entities(s, 2, 1)
    cells = hifie.centers("cell", 2, s, lo, 1.0 / s)
    assert cells.shape == (s * s, 2)


@pytest.mark.parametrize("s", [2, 4, 8, 16])
def test_3d_face_and_edge_centres_are_interior(s):
    lo = np.zeros(3)
    faces = hifie.centers("face", 3, s, lo, 1.0 / s)
    edges = hifie.centers("edge", 3, s, lo, 1.0 / s)
    assert faces.shape == (3 * (s - 1) * s * s, 3)
    assert edges.shape == (3 * (s - 1) ** 2 * s, 3)
    gf = {tuple(v) for v in np.round(faces * s * 2).astype(np.int64)}
    ge = {tuple(v) for v in np.round(edges * s * 2).astype(np.int64)}
    assert len(gf) == faces.shape[0] and len(ge) == edges.shape[0]
    if s <= 8:
        assert gf == _shared_entities(s, 3, 1)
        assert ge == _shared_entities(s, 3, 2)


def test_box_counts_per_level_2d_n64_n1024_3d_n64():
    # n = 64 (2D, occupancy 64): L = 3, cells 64/16/4, edges 112/24/4;
    # n = 1024: edges 2 s (s - 1) = 32512, 8064, 1984, 480, 112, 24, 4;
    # 3D n = 64 (occupancy 64): L = 4, faces 11520/1344/144/12, edges
    # 10800/1176/108/6
    lo2, lo3 = np.zeros(2), np.zeros(3)
    cells = [hifie.centers("cell", 2, 2 ** (3 - l), lo2, 1.0).shape[0] for l in range(3)]
    edges = [hifie.centers("edge", 2, 2 ** (3 - l), lo2, 1.0).shape[0] for l in range(3)]
    assert cells == [64, 16, 4] and edges == [112, 24, 4]
    e1024 = [hifie.centers("edge", 2, 2 ** (7 - l), lo2, 1.0).shape[0] for l in range(7)]
    assert e1024 == [32512, 8064, 1984, 480, 112, 24, 4]
    f3 = [hifie.centers("face", 3, 2 ** (4 - l), lo3, 1.0).shape[0] for l in range(4)]
    e3 = [hifie.centers("edge", 3, 2 ** (4 - l), lo3, 1.0).shape[0] for l in range(4)]
    c3 = [hifie.centers("cell", 3, 2 ** (4 - l), lo3, 1.0).shape[0] for l in range(4)]
    assert c3 == [4096, 512, 64, 8]
    assert f3 == [11520, 1344, 144, 12]
    assert e3 == [10800, 1176, 108, 6]
    assert hifie.sublevel_plan(2, 3) == [("cell", 0), ("edge", 0), ("cell", 1), ("edge", 1),
                                         ("cell", 2), ("edge", 2)]
    assert [k for k, _ in hifie.sublevel_plan(3, 2)] == ["cell", "face", "edge", "cell", "face", "edge"]


def test_n64_factor_visits_every_box():
    # the oracle's sublevel loop on the 2D n = 64 grid at eps = 1e-6: every cell
    # and every interior edge holds active DOFs, so the non-empty boxes per
    # sublevel are exactly the counts above
    pb = hi.volume_problem(64, 2, rhs_seed=1001)
    trace = []
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, 1e-6, pb.proxy, trace=trace)
    per = {}
    for kind, ell, *_ in trace:
        per[(kind, ell)] = per.get((kind, ell), 0) + 1
    assert [per[(k, l)] for k, l in hifie.sublevel_plan(2, 3)] == [64, 112, 16, 24, 4, 4]
    assert [(sl.kind, sl.level, len(sl.boxes)) for sl in F.sublevels] == [
        ("cell", 0, 64), ("edge", 0, 112), ("cell", 1, 16), ("edge", 1, 24), ("cell", 2, 4), ("edge", 2, 4)]
    # every leaf cell of the n = 64 grid compresses all 64 of its DOFs
    assert all(b.n == 64 for b in F.sublevels[0].boxes)


# --------------------------------------------------- iterative refinement --

def _two_level_E(N, seed, mag=0.1):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    lam = mag * np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    return (Q * lam) @ Q.T


@pytest.mark.parametrize("tol", [3e-10, 2e-7, 5e-3])
def test_refine_contracts_by_norm_of_E(tol):
    # F = I: u_0 = f, r_k = (-E)^(k+1) f, so |r_k| / |f| = 0.1^(k+1) exactly
    # (E = 0.1 Q diag(+-1) Q^T), and refinement stops after the first k with
    # 0.1^(k+1) <= tol
    N = 64
    E = _two_level_E(N, 11)
    A = np.eye(N) + E
    f = np.random.default_rng(12).standard_normal(N)
    u, its, hist = krylov.refine(lambda v: A @ v, f, lambda v: v.copy(), tol=tol)
    expect = math.ceil(math.log(tol) / math.log(0.1)) - 1
    assert its == expect
    assert len(hist) == its + 1
    assert np.allclose(hist, [0.1 ** (k + 1) for k in range(its + 1)], rtol=1e-9)
    assert hist[-1] <= tol < hist[-2] if its else hist[-1] <= tol
    # the returned u is the last iterate, whose residual is the last entry
    assert np.linalg.norm(f - A @ u) / np.linalg.norm(f) == pytest.approx(hist[-1], rel=1e-9)
    ue = np.linalg.solve(A, f)
    assert np.linalg.norm(u - ue) <= 1.2 * tol * np.linalg.norm(f) / 0.9


def test_refine_exact_solver_needs_no_correction():
    rng = np.random.default_rng(13)
    A = rng.standard_normal((40, 40)) + 8 * np.eye(40)
    Ai = np.linalg.inv(A)
    f = rng.standard_normal(40)
    u, its, hist = krylov.refine(lambda v: A @ v, f, lambda v: Ai @ v, tol=1e-12)
    assert its == 0 and len(hist) == 1 and hist[0] <= 1e-12
    assert np.allclose(u, np.linalg.solve(A, f), rtol=1e-12, atol=1e-13)


def test_refine_with_approximate_inverse_reaches_dense_solution():
    # F^{-1} = (I + E')^{-1} for a perturbation E' of E: contraction
    # |I - A F^{-1}| = |(E - E') (I + E')^{-1}| <= 0.02 / 0.9
    N = 80
    E = _two_level_E(N, 14)
    A = np.eye(N) + E
    rng = np.random.default_rng(15)
    P = rng.standard_normal((N, N))
    Ep = E + 0.02 * P / np.linalg.norm(P, 2)
    Fi = np.linalg.inv(np.eye(N) + Ep)
    f = rng.standard_normal(N)
    u, its, hist = krylov.refine(lambda v: A @ v, f, lambda v: Fi @ v, tol=1e-12)
    rate = 0.02 / 0.9
    assert its <= math.ceil(math.log(1e-12) / math.log(rate))
    assert all(h1 <= rate * h0 * 1.0001 for h0, h1 in zip(hist, hist[1:]))
    assert np.linalg.norm(u - np.linalg.solve(A, f)) <= 1e-11 * np.linalg.norm(f)
