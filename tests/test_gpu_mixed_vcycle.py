"""The mixed form's V-cycle (level 1 in FP32, coarse levels and the coarsest
solve in FP64) through the C-ABI, element by element, on seeded 32^3 fields
with the oracle's bases imported, against two oracles: the FP64 V-cycle
(Algorithm 1) and the same V-cycle with level 1's data and arithmetic rounded
to FP32 where the mixed form rounds them (``oracle.vcycle_mixed``).

Tolerance: an FP32 evaluation of the V-cycle carries an error e32 relative to
the FP64 result, set by the unit roundoff (6e-8) and its growth through the
smoother sweeps, restriction and prolongation (large at high contrast).  The
GPU kernels perform the same FP32 operations in another summation order, so
their error must be of the same size: ||z_gpu - z64|| <= 4 e32 ||z64||, and two
FP32 evaluations can differ by at most the sum of their errors, so
||z_gpu - z32|| <= 5 e32 ||z64||.  A dropped term, a wrong sign or index, or an
operand read in the wrong precision would give an error far above e32."""
import numpy as np
import pytest
import torch

import fields
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_19342_gb300 as p
    return p


def _case(pkg, kappa, block, n_eig):
    N = kappa.shape[-1]
    nl = len(n_eig) + 1
    oo = oracle.Options(n_levels=nl, block=block, ratio=[(2, 2, 2)] * (nl - 2), n_eig=n_eig, nu=[1] * (nl - 1))
    H = oracle.setup(kappa, (1.0 / N,) * 3, oo)
    out = {}
    for prec in (pkg.FP64, pkg.MIXED):
        go = pkg.Options(n_levels=nl, block=block, ratio=[(2, 2, 2)] * (nl - 2), n_eig=n_eig, precision=prec,
                         eig_tol=1e-10)
        S = pkg.Solver(torch.tensor(kappa, device="cuda"), go)
        assert S.import_bases(H.basis[:nl - 1]) == 0
        out[prec] = S
    return H, out


CASES = {
    "grf32_b4": dict(kappa=lambda: fields.grf_lognormal((32, 32, 32), seed=0, contrast=1e3), block=(4, 4, 4),
                     n_eig=[4, 4]),
    "incl32_b8": dict(kappa=lambda: fields.inclusions(32, seed=1, n_spheres=25, n_channels=5, k_hi=1e6),
                      block=(8, 8, 8), n_eig=[6, 6]),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, pkg):
    c = CASES[request.param]
    H, S = _case(pkg, c["kappa"](), c["block"], c["n_eig"])
    return request.param, H, S


def test_mixed_vcycle_elementwise(pkg, case):
    name, H, S = case
    rng = np.random.default_rng(11)
    n = H.dims[0]
    worst = []
    for trial in range(2):
        r = rng.standard_normal(n) if trial == 0 else fields.rhs_corners(H.shape).ravel()
        r = r - r.mean()
        z64 = oracle.vcycle(H, r)
        z32 = oracle.vcycle_mixed(H, r)
        zg = S[pkg.MIXED].apply_precond(torch.tensor(r.reshape(H.shape), device="cuda")).cpu().numpy().ravel()
        nz = np.linalg.norm(z64)
        e32 = np.linalg.norm(z32 - z64) / nz
        eg = np.linalg.norm(zg - z64) / nz
        d = np.linalg.norm(zg - z32) / nz
        print(f"{name} trial {trial}: e32 = {e32:.3e}  e_gpu = {eg:.3e}  |gpu - fp32 oracle| = {d:.3e}")
        assert e32 > 0
        assert eg <= 4 * e32, (eg, e32)
        assert d <= 5 * e32, (d, e32)
        # the FP64 form of the same context matches the FP64 oracle to FP64 rounding
        zf = S[pkg.FP64].apply_precond(torch.tensor(r.reshape(H.shape), device="cuda")).cpu().numpy().ravel()
        assert np.linalg.norm(zf - z64) <= 1e-9 * nz
        worst.append(eg / e32)


def test_mixed_iterations_with_the_oracles_bases(pkg, case):
    # the same preconditioner in both forms: any gap in iteration counts between the
    # FP64 and mixed forms is reproduced by the FP32 oracle (a rounding cost)
    name, H, S = case
    b = fields.rhs_corners(H.shape)
    o64 = oracle.solve(H, b.ravel(), rtol=1e-8)
    o32 = oracle.solve(H, b.ravel(), rtol=1e-8, mixed=True)
    _, i64, _ = S[pkg.FP64].solve(torch.tensor(b, device="cuda"), rtol=1e-8)
    _, i32, _ = S[pkg.MIXED].solve(torch.tensor(b, device="cuda"), rtol=1e-8)
    print(f"{name}: iterations FP64 oracle {o64.iterations} gpu {i64['iterations']}; "
          f"mixed oracle {o32.iterations} gpu {i32['iterations']}")
    assert abs(i64["iterations"] - o64.iterations) <= 1
    assert abs(i32["iterations"] - o32.iterations) <= max(3, o32.iterations // 10)
    assert i32["true_rel_residual"] <= 1e-8
