"""The benchmark's own workload at full size (128^3 inclusion field, contrast 1e6,
8^3 elements, 4 levels, 6 eigenvectors per local problem), in the launch
configuration bench.py times, checked through properties the oracle computes
at any size: the residual b - A x recomputed with the oracle's operator is below
rtol in both forms, x has zero mean, and the two forms agree to the accuracy
their residuals allow."""
import numpy as np
import pytest
import torch

import bench
import fields
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_19342_gb300 as p
    return p


def abs_apply(T, x):
    """|A| |x|: per face T (|x_i| + |x_j|) added to both cells (rounding bound of a
    residual evaluation)."""
    ax = np.abs(x)
    q = np.zeros_like(ax)
    for d, (lo, hi) in enumerate(((np.s_[:, :, :-1], np.s_[:, :, 1:]), (np.s_[:, :-1, :], np.s_[:, 1:, :]),
                                  (np.s_[:-1, :, :], np.s_[1:, :, :]))):
        f = T[d][lo] * (ax[lo] + ax[hi])
        q[lo] += f
        q[hi] += f
    return q


def test_bench_workload_full_size(pkg):
    kappa = bench.field()
    shape = kappa.shape
    f = bench.rhs(shape)
    b = f - f.mean()
    T = oracle.face_transmissibilities(kappa, (1.0 / shape[2], 1.0 / shape[1], 1.0 / shape[0]))
    xs = {}
    for form, prec in (("fp64", pkg.FP64), ("mixed", pkg.MIXED)):
        opts = pkg.Options(n_levels=bench.N_LEVELS, block=bench.BLOCK, ratio=bench.RATIO, n_eig=bench.N_EIG,
                           precision=prec, eig_tol=1e-8)
        S = pkg.Solver(torch.tensor(kappa, device="cuda"), opts)
        x, info, st = S.solve(torch.tensor(f, device="cuda"), rtol=bench.RTOL, max_iter=1000)
        assert st == 0 and info["converged"], info
        x = x.cpu().numpy()
        res = np.linalg.norm(b - oracle.apply_A(T, x)) / np.linalg.norm(b)
        slack = 32 * np.finfo(np.float64).eps * np.linalg.norm(abs_apply(T, x)) / np.linalg.norm(b)
        assert res <= bench.RTOL + slack, (form, res, slack, info)
        assert abs(x.mean()) <= 1e-13 * np.abs(x).max()
        xs[form] = x
        S.close()
    # both solutions meet the residual tolerance; their difference is bounded by the
    # tolerance times the conditioning (not small at contrast 1e6): a sanity bound
    diff = np.linalg.norm(xs["fp64"] - xs["mixed"]) / np.linalg.norm(xs["fp64"])
    print(f"fp64 vs mixed solution: relative difference {diff:.2e}")
    assert diff < 1e-2, diff
