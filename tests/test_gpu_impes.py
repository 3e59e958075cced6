"""Two-phase flow (Section 6) through the C-ABI against the oracle: the well
term of A (options.cell_diag) in the V-cycle and the nonsingular solve, the
pressure terms of Eq. (IMP), the upstream saturation sub-steps of Eq. (ES), and
three coupled IMPES time steps (pressure solve warm-started from the previous
step, velocity, sub-steps) on an SPE10-shaped synthetic field.

Tolerances: the pressure terms and the sub-steps are a few FP64 operations per
value (1e-13 relative); the V-cycle with the oracle's bases as the Strategy-1
parity test (1e-11, times eps cond of the coarsest level); solves to rtol 1e-10
agree to 1e-10 cond-ish (1e-7 relative on p); the saturations inherit that
through v (absolute 1e-8), the sub-steps' time through max |dS/dt| (1e-6)."""
import numpy as np
import pytest
import torch

import fields
import oracle
from oracle import impes

pytestmark = pytest.mark.gpu

SHAPE = (8, 16, 16)              # nz, ny, nx
H_CELL = (20.0, 10.0, 2.0)       # hx, hy, hz (ft), the SPE10 cell
P_BH = 4000.0


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_19342_gb300 as p
    return p


def reservoir(seed=0):
    kx = fields.grf_lognormal(SHAPE, seed=seed, contrast=1e4)
    kappa3 = np.stack([kx, kx, 0.1 * kx])
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.05, 0.3, size=SHAPE)
    wi = np.zeros(SHAPE)
    nz, ny, nx = SHAPE
    for (j, i) in ((0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1)):   # producers in the corners
        wi[:, j, i] = impes.well_index(H_CELL[0], H_CELL[1], 1.0)
    q = np.zeros(SHAPE)
    q[:, ny // 2, nx // 2] = 50.0                                        # injector in the centre
    return kappa3, phi, wi, q


def opts(pkg, W, precision=0):
    return (pkg.Options(n_levels=3, block=(4, 4, 4), ratio=[(2, 2, 2)], n_eig=[4, 4], precision=precision,
                        cell_diag=W, eig_tol=1e-12),
            oracle.Options(n_levels=3, block=(4, 4, 4), ratio=[(2, 2, 2)], n_eig=[4, 4], nu=[1, 1],
                           cell_diag=None if W is None else W.cpu().numpy()))


def test_cell_term_vcycle_and_solve(pkg):
    kappa3, phi, wi, q = reservoir(1)
    fl = impes.Fluid()
    S0 = np.full(SHAPE, 0.2)
    ke, W, b = impes.pressure_terms(S0, kappa3, wi, q, P_BH, fl)
    Wt = torch.tensor(W, device="cuda")
    go, oo = opts(pkg, Wt)
    H = oracle.setup(ke, H_CELL, oo)
    Si = pkg.Solver(torch.tensor(ke, device="cuda"), go, h=H_CELL)
    assert Si.import_bases(H.basis[:2]) == 0
    rng = np.random.default_rng(0)
    r = rng.standard_normal(H.dims[0])
    z = Si.apply_precond(torch.tensor(r.reshape(SHAPE), device="cuda")).cpu().numpy().ravel()
    zr = oracle.vcycle(H, r)
    assert np.linalg.norm(z - zr) <= 1e-11 * np.linalg.norm(zr)
    ref = oracle.solve(H, b.ravel(), rtol=1e-10)
    for prec in (0, 1):
        S = pkg.Solver(torch.tensor(ke, device="cuda"), opts(pkg, Wt, prec)[0], h=H_CELL)
        x, info, _ = S.solve(torch.tensor(b, device="cuda"), rtol=1e-10)
        xe = x.cpu().numpy().ravel()
        err = np.linalg.norm(xe - ref.x) / np.linalg.norm(ref.x)
        print(f"precision {prec}: iterations {info['iterations']} (oracle {ref.iterations}), rel. error {err:.2e}, "
              f"mean {xe.mean():.2f}")
        assert info["converged"] and info["true_rel_residual"] <= 1e-10 * (1 + 1e-6)
        assert err <= 1e-8
        if prec == 0:
            assert abs(info["iterations"] - ref.iterations) <= 1
        # the cell balance div v = q_inj + W (p_BH - p) up to the solve's residual ||b - (A + W) p||
        _, bal = S.velocity(x, torch.tensor(b, device="cuda"))
        assert bal[0] <= 1e-10 * (1 + 1e-6) * np.linalg.norm(b)
        S.close()


def test_pressure_terms_and_substeps(pkg):
    kappa3, phi, wi, q = reservoir(2)
    fl = impes.Fluid()
    rng = np.random.default_rng(5)
    S = rng.uniform(0.2, 0.8, size=SHAPE)
    fg = pkg.make_fluid()
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    ke, w, b = pkg.msmg_impes_pressure_terms(fg, t(S), t(kappa3), t(wi), t(q), P_BH)
    ke_r, W_r, b_r = impes.pressure_terms(S, kappa3, wi, q, P_BH, fl)
    np.testing.assert_allclose(ke.cpu().numpy(), ke_r, rtol=1e-13)
    np.testing.assert_allclose(w.cpu().numpy(), W_r, rtol=1e-13, atol=0)
    np.testing.assert_allclose(b.cpu().numpy(), b_r, rtol=1e-13)
    # sub-steps on a given pressure and velocity field
    Sol = pkg.Solver(t(ke_r), opts(pkg, t(W_r))[0], h=H_CELL)
    p = P_BH + rng.normal(0, 50.0, size=SHAPE)
    v = impes.face_velocity(Sol.export_faces().cpu().numpy(), p, H_CELL)
    Sg = t(S)
    dt = pkg.msmg_impes_transport(Sol.ctx, fg, t(v), t(p), t(W_r), P_BH, t(q), t(phi), Sg, 20, 0.001)
    Sr, dtr = impes.transport(S, v, p, W_r, P_BH, q, phi, H_CELL, 20, 0.001, fl)
    np.testing.assert_allclose(Sg.cpu().numpy(), Sr, rtol=0, atol=1e-13)
    np.testing.assert_allclose(dt, dtr, rtol=1e-13)


@pytest.mark.parametrize("precision", [0, 1])
def test_impes_steps_against_oracle(pkg, precision):
    kappa3, phi, wi, q = reservoir(3)
    fl = impes.Fluid()
    fg = pkg.make_fluid()
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    S_g, S_o = t(np.full(SHAPE, 0.2)), np.full(SHAPE, 0.2)
    p_g, p_o = None, None
    kg, wig, qg, phig = t(kappa3), t(wi), t(q), t(phi)
    for step in range(3):
        ke, w, b = pkg.msmg_impes_pressure_terms(fg, S_g, kg, wig, qg, P_BH)
        Sol = pkg.Solver(ke, opts(pkg, w, precision)[0], h=H_CELL)
        p_g, info, _ = Sol.solve(b, rtol=1e-10, x0=p_g)
        v, bal = Sol.velocity(p_g, b)
        dt_g = pkg.msmg_impes_transport(Sol.ctx, fg, v, p_g, w, P_BH, qg, phig, S_g, 10, 0.001)
        Sol.close()
        ke_r, W_r, b_r = impes.pressure_terms(S_o, kappa3, wi, q, P_BH, fl)
        H = oracle.setup(ke_r, H_CELL, opts(pkg, None)[1].__class__(**{**opts(pkg, None)[1].__dict__,
                                                                         "cell_diag": W_r}))
        x0 = None if p_o is None else p_o.ravel()
        res = oracle.pcg(H.A[0], b_r.ravel(), lambda r: oracle.vcycle(H, r), rtol=1e-10, x0=x0, singular=False)
        p_o = res.x.reshape(SHAPE)
        v_o = impes.face_velocity(H.T, p_o, H_CELL)
        S_o, dt_o = impes.transport(S_o, v_o, p_o, W_r, P_BH, q, phi, H_CELL, 10, 0.001, fl)
        ep = np.linalg.norm(p_g.cpu().numpy() - p_o) / np.linalg.norm(p_o)
        eS = np.abs(S_g.cpu().numpy() - S_o).max()
        print(f"step {step}: PCG {info['iterations']} (oracle {res.iterations}), |p| rel. error {ep:.2e}, "
              f"|S| max error {eS:.2e}, dt {dt_g:.4e} (oracle {dt_o:.4e}), balance {bal[0] / bal[1]:.1e}")
        assert ep <= 1e-7 and eS <= 1e-8
        assert abs(dt_g - dt_o) <= 1e-6 * dt_o
        assert S_g.min().item() >= 0.2 - 1e-12 and S_g.max().item() <= 0.8 + 1e-12


@pytest.mark.gpu
def test_refresh_equals_a_fresh_setup(pkg):
    # a time loop sets up again in the workspace it holds: the same bits as a new solver
    kappa3, phi, wi, q = reservoir(5)
    fg = pkg.make_fluid()
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    kg, wig, qg = t(kappa3), t(wi), t(q)
    ke1, w1, b1 = pkg.msmg_impes_pressure_terms(fg, t(np.full(SHAPE, 0.2)), kg, wig, qg, P_BH)
    ke2, w2, b2 = pkg.msmg_impes_pressure_terms(fg, t(np.linspace(0.2, 0.8, int(np.prod(SHAPE))).reshape(SHAPE)),
                                                 kg, wig, qg, P_BH)
    for precision in (0, 1):
        Sol = pkg.Solver(ke1, opts(pkg, w1, precision)[0], h=H_CELL)
        x1, _, _ = Sol.solve(b1, rtol=1e-10)
        Sol.refresh(ke2, cell_diag=w2)
        x_ref, info_r, _ = Sol.solve(b2, rtol=1e-10)
        Sol.close()
        Fresh = pkg.Solver(ke2, opts(pkg, w2, precision)[0], h=H_CELL)
        x_new, info_n, _ = Fresh.solve(b2, rtol=1e-10)
        Fresh.close()
        assert info_r["iterations"] == info_n["iterations"]
        assert torch.equal(x_ref, x_new)
        with pytest.raises(ValueError):                 # the cell term must stay present
            Fresh2 = pkg.Solver(ke2, opts(pkg, w2, precision)[0], h=H_CELL)
            try:
                Fresh2.refresh(ke1, cell_diag=None)
            finally:
                Fresh2.close()
