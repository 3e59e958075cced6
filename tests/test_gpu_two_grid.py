"""The exact two-grid preconditioner P_TG (Eq. (B_TG); options.two_grid)
through the C-ABI against the oracle's vcycle_two_grid, which applies the dense
pseudo-inverse of A_2, with the oracle's bases imported.

Tolerance: the GPU solves A_2 e_c = r_c by an inner PCG to ||r|| <= rho ||r_c||,
so ||e_c - A_2^+ r_c|| <= cond+(A_2) rho ||A_2^+ r_c|| (cond+ over the range of
A_2); the fine steps around it are linear with norm of order one, so the
preconditioner's output carries a relative error of at most a small multiple
of cond+(A_2) rho.  The test takes rho = 1e-13 and allows 10 cond+(A_2) rho; in
the mixed form the FP32 restriction's rounding (a few unit roundoffs of 2^-24)
is amplified the same way, and the bound is 100 cond+(A_2) 2^-24."""
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


@pytest.mark.parametrize("n_levels,n_eig,contrast", [(3, [4, 4], 1e3), (4, [4, 4, 4], 1e5)])
@pytest.mark.parametrize("precision", [0, 1])
def test_two_grid_against_oracle(pkg, n_levels, n_eig, contrast, precision):
    N = 32
    kap = fields.grf_lognormal((N, N, N), seed=1, contrast=contrast)
    ratio = [(2, 2, 2)] * (n_levels - 2)
    H = oracle.setup(kap, (1 / N,) * 3, oracle.Options(n_levels=n_levels, block=(4, 4, 4), ratio=ratio,
                                                       n_eig=n_eig, nu=[1] * (n_levels - 1)))
    rho = 1e-13
    S = pkg.Solver(torch.tensor(kap, device="cuda"),
                   pkg.Options(n_levels=n_levels, block=(4, 4, 4), ratio=ratio, n_eig=n_eig, two_grid=True,
                               inner_rtol=rho, inner_max_iter=400, precision=precision))
    assert S.import_bases(H.basis[:n_levels - 1]) == 0
    Ac = H.A[1].toarray()
    w = np.linalg.eigvalsh(0.5 * (Ac + Ac.T))
    wpos = w[w > 1e-12 * w[-1]]
    cond = wpos[-1] / wpos[0]
    rng = np.random.default_rng(2)
    r = rng.standard_normal(H.dims[0])
    r -= r.mean()
    ref = oracle.vcycle_two_grid(H, r)
    z = S.apply_precond(torch.tensor(r.reshape(H.shape), device="cuda")).cpu().numpy().ravel()
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    # mixed form: level 1 in FP32, so r_c carries relative errors of a few unit roundoffs
    # u32 = 2^-24 (grown through the sweeps), which the exact coarse solve amplifies by up
    # to cond+(A_2)
    tol = 10 * cond * rho if precision == 0 else 100 * cond * 2.0 ** -24
    print(f"P_TG levels {n_levels} contrast {contrast:g} precision {precision}: cond+(A_2) = {cond:.2e}, "
          f"rel. error {err:.2e} (bound {tol:.2e})")
    assert err <= tol
    # solves: iteration counts of P_TG against the oracle, and against the V-cycle (P_ITG)
    b = fields.rhs_corners(H.shape)
    o_tg = oracle.solve(H, b.ravel(), rtol=1e-8, two_grid=True)
    o_itg = oracle.solve(H, b.ravel(), rtol=1e-8)
    x, info, st = S.solve(torch.tensor(b, device="cuda"), rtol=1e-8)
    print(f"  iterations: P_TG gpu {info['iterations']} (inner {info['inner_iterations']}) oracle "
          f"{o_tg.iterations}; P_ITG oracle {o_itg.iterations}")
    assert info["converged"] and info["true_rel_residual"] <= 1e-8
    assert abs(info["iterations"] - o_tg.iterations) <= 1
    assert info["inner_iterations"] >= info["iterations"]
    if precision == 0:
        xe = x.cpu().numpy().ravel()
        k = o_tg.iterations
        assert np.linalg.norm(xe - o_tg.x) <= 1e-7 * np.linalg.norm(o_tg.x)
