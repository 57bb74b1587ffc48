"""The seeded synthetic inputs (hif_inputs): the recipe the oracle and the GPU
path both read, checked against its own description -- grid points at cell
centres with weights h^d, coefficient fields inside [0.5, 1.5], unit proxy
directions, Gaussian right-hand sides, batched sizes from their set -- and
reproducible from their seeds."""
import math

import numpy as np

import hif_inputs as hi


def test_grid_points_are_cell_centres():
    for n, d in [(4, 2), (3, 3)]:
        pts, w = hi.grid_points(n, d)
        h = 1.0 / n
        assert pts.shape == (n ** d, d) and np.all(w == h ** d)
        assert set(np.round(pts[:, 0] / h - 0.5, 12)) == set(range(n))
        # the first coordinate varies slowest
        assert np.all(np.diff(pts[:, 0]) >= 0) and pts[1, d - 1] > pts[0, d - 1]


def test_coefficients_and_rhs():
    pb = hi.volume_problem(16, 2, smooth_seed=1002, rhs_seed=1003, nrhs=3)
    assert np.array_equal(pb.b, pb.c) and np.all(pb.a == 1.0)
    assert 0.5 <= pb.b.min() and pb.b.max() <= 1.5 and pb.b.std() > 0.01
    assert pb.f.shape == (256, 3) and pb.f.flags["F_CONTIGUOUS"]
    assert abs(pb.f.mean()) < 0.2 and abs(pb.f.std() - 1.0) < 0.1
    # reproducible from the seeds, different for other seeds
    pb2 = hi.volume_problem(16, 2, smooth_seed=1002, rhs_seed=1003, nrhs=3)
    assert np.array_equal(pb.b, pb2.b) and np.array_equal(pb.f, pb2.f)
    assert not np.array_equal(pb.b, hi.volume_problem(16, 2, smooth_seed=1004).b)
    assert np.all(hi.volume_problem(8, 2).b == 1.0)


def test_proxy_directions_are_unit_vectors():
    d2 = hi.proxy_directions(2)
    assert d2.shape == (64, 2) and np.allclose(np.linalg.norm(d2, axis=1), 1.0, atol=1e-15)
    ang = np.mod(np.arctan2(d2[:, 1], d2[:, 0]), 2 * math.pi)
    assert np.allclose(np.sort(ang), 2 * math.pi * np.arange(64) / 64, atol=1e-12)
    d3 = hi.proxy_directions(3)
    assert d3.shape == (512, 3) and np.allclose(np.linalg.norm(d3, axis=1), 1.0, atol=1e-15)
    assert np.array_equal(d3, hi.proxy_directions(3))
    assert np.abs(d3.mean(axis=0)).max() < 0.1                       # spread over the sphere


def test_batched_sizes_and_helmholtz():
    sizes = hi.batched_sizes(256, 1004)
    assert len(sizes) == 256 and set(sizes) <= set(range(32, 257, 16)) and len(set(sizes)) > 10
    assert sizes == hi.batched_sizes(256, 1004)
    pb = hi.helmholtz_problem(16, 0.5)
    assert pb.kernel_id == 2 and abs(pb.k - math.pi) < 1e-15
    assert np.array_equal(pb.b, pb.c) and pb.b.max() <= pb.k and np.iscomplexobj(pb.f)
