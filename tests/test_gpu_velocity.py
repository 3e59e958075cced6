"""Velocity recovery and the mass-balance check (Eq. (velocity); msmg_velocity)
through the C-ABI against the oracle: face velocities element by element on
the oracle's own solution (two FP64 products per face: 1e-13 of the largest
velocity), and after a GPU solve the cell balance div v - b relative to b
equal to the solve's true relative residual (at most rtol)."""
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


@pytest.mark.parametrize("shape,block,comps", [((32, 32, 32), (4, 4, 4), 1), ((16, 24, 40), (4, 4, 8), 3)])
def test_velocity_and_mass_balance(pkg, shape, block, comps):
    nz, ny, nx = shape
    rng = np.random.default_rng(9)
    kap = np.exp(rng.normal(0, 2, size=(comps,) + shape)) if comps == 3 else \
        fields.grf_lognormal(shape, seed=4, contrast=1e4)
    h = (1 / nx, 1 / ny, 1 / nz)
    oo = oracle.Options(n_levels=3, block=block, ratio=[(2, 2, 2)], n_eig=[4, 4], nu=[1, 1])
    H = oracle.setup(kap, h, oo)
    f = fields.rhs_line_sources(shape)
    ref = oracle.solve(H, f.ravel(), rtol=1e-10)
    S = pkg.Solver(torch.tensor(kap, device="cuda"), pkg.Options(n_levels=3, block=block, ratio=[(2, 2, 2)],
                                                                  n_eig=[4, 4]), h=h)
    # face velocities of a given pressure: the oracle's solution
    v, bal = S.velocity(torch.tensor(ref.x.reshape(shape), device="cuda"), torch.tensor(f, device="cuda"))
    vo = oracle.velocity(H.T, ref.x, h)
    scale = np.abs(vo).max()
    assert np.abs(v.cpu().numpy() - vo).max() <= 1e-13 * scale
    bm = f.ravel() - f.mean()
    div_ref = oracle.divergence(vo, h).ravel()
    np.testing.assert_allclose(bal[1], np.linalg.norm(bm), rtol=1e-12)
    # a residual of about 1e-10 ||b||: compared to its own rounding noise (face terms of
    # size |T| |p| summed in another order)
    res_ref = np.linalg.norm(div_ref - bm)
    assert abs(bal[0] - res_ref) <= 1e-3 * res_ref + 1e-12 * bal[1]
    # after the GPU's own solve the balance is the solve's residual
    x, info, _ = S.solve(torch.tensor(f, device="cuda"), rtol=1e-8)
    v2, bal2 = S.velocity(x, torch.tensor(f, device="cuda"))
    assert bal2[0] / bal2[1] <= 1e-8 * (1 + 1e-6)
    np.testing.assert_allclose(bal2[0] / bal2[1], info["true_rel_residual"], rtol=1e-4)
