"""Large-box path with the proxy matrix first reduced to its R factor by the
blocked unpivoted QR (opt-in, HIF_BIG_RFIRST=1; then pivoted QR on R, Lemma
2.2): forced onto small problems by lowering the large-box threshold, and
judged like every factorization: solve error against the dense FP64 solve,
skeleton totals against the same path without the reduction, refined
residuals."""
import os

import numpy as np
import pytest
import torch

import hif_inputs as hi
from oracle import dense, kernels

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


def factor(P, pb, eps, precision, big, rfirst):
    old = {k: os.environ.get(k) for k in ("HIF_BIG_ID", "HIF_BIG_RFIRST")}
    os.environ["HIF_BIG_ID"] = str(big)
    os.environ["HIF_BIG_RFIRST"] = "1" if rfirst else "0"
    try:
        return P.Factorization(T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c), pb.kernel_id, eps,
                               proxy_dirs=pb.proxy if pb.dim == 3 else None, precision=precision)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def skeletons(fac):
    return [s["skeletons"] for s in fac.stats()["per_sublevel"]]


@pytest.mark.parametrize("dim,n,big", [(2, 64, 24), (2, 96, 40), (3, 12, 24)])
def test_r_first_large_boxes_accuracy_fp64(P, dim, n, big):
    eps = 1e-6
    pb = hi.volume_problem(n, dim, smooth_seed=700 + n)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, pb.kernel_id)
    ud = dense.DenseSolver(op).solve(pb.f[:, 0])
    f_r = factor(P, pb, eps, "fp64", big, True)
    f_0 = factor(P, pb, eps, "fp64", big, False)
    for f in (f_r, f_0):
        u = f.solve(T(pb.f[:, 0])).cpu().numpy()
        assert np.linalg.norm(u - ud) <= 100 * eps * np.linalg.norm(ud)
    # the same ID up to rounding: skeleton totals per sublevel within 10%
    for a, b in zip(skeletons(f_r), skeletons(f_0)):
        assert abs(a - b) <= 0.1 * max(b, 10)
    f_r.close()
    f_0.close()


@pytest.mark.parametrize("dim,n,big", [(2, 96, 40), (3, 12, 24)])
def test_r_first_large_boxes_fp32_refined(P, dim, n, big):
    pb = hi.volume_problem(n, dim, smooth_seed=800 + n, nrhs=3)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, pb.kernel_id)
    fac = factor(P, pb, 1e-6, "fp32", big, True)
    u, its, rel = fac.solve_refined(T(pb.f), tol=1e-10)
    assert rel <= 1e-10 and its <= 6
    r = pb.f - op.matvec(u.cpu().numpy())
    assert np.linalg.norm(r, axis=0).max() <= 1e-10 * np.linalg.norm(pb.f, axis=0).min() * 1.01
    fac.close()
