"""8^3 elements: the subspace-iteration eigensolver (Eq. (spepb)) against
LAPACK in the oracle, and the solve built on it, on a high-contrast
inclusion field (spheres and channels at 1e6) and on the homogeneous case."""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def incl(pkg):
    N = 32
    kappa = fields.inclusions(N, seed=1, n_spheres=12, n_channels=3, k_hi=1e6)
    # L = 7 closes the multiplicity groups 1 + 3 + 3 of homogeneous 8^3 elements, so every
    # local coarse space is uniquely defined and the two preconditioners coincide
    go = pkg.Options(n_levels=3, block=(8, 8, 8), ratio=[(2, 2, 2)], n_eig=[7, 7], eig_tol=1e-12)
    oo = oracle.Options(n_levels=3, block=(8, 8, 8), ratio=[(2, 2, 2)], n_eig=[7, 7], nu=[1, 1])
    H = oracle.setup(kappa, (1 / N,) * 3, oo)
    S = pkg.Solver(torch.tensor(kappa, device="cuda"), go)
    return kappa, H, S


def test_subspace_eigenpairs_high_contrast(incl):
    kappa, H, S = incl
    Phi, lam = S.export_basis(1)
    Phi, lam = Phi.cpu().numpy(), lam.cpu().numpy()
    info = S.info
    assert S.setup_status == 0
    assert info["eig_residual_max"] <= 1e-12
    np.testing.assert_allclose(lam, H.lam[0], atol=1e-10)
    Po = H.basis[0]
    L = Po.shape[1]
    lam_next, _, _ = oracle.level1_eigenpairs(H.T, H.S, (8, 8, 8), L + 1)
    checked = 0
    for e in range(Phi.shape[0]):
        gap = lam_next[e, L] - lam_next[e, L - 1]
        if gap < 1e-6:
            continue          # a cluster straddles the cutoff: the span is not unique
        P1, P2 = Phi[e].T @ Phi[e], Po[e].T @ Po[e]
        # subspace perturbation ~ residual / gap
        assert np.abs(P1 - P2).max() <= max(1e-8, 1e-10 / gap) * np.abs(P2).max(), (e, gap)
        checked += 1
    assert checked >= Phi.shape[0] // 2


def test_solve_parity_large_elements(pkg, incl):
    kappa, H, S = incl
    f = fields.rhs_corners(kappa.shape).ravel()
    ref = oracle.solve(H, f, rtol=1e-8)
    # own bases: iteration count within one; iterates differ by the eigensolver's
    # span error, about eig_tol / gap (gap ~1e-3 here), so 1e-8
    x, info, st = S.solve(torch.tensor(f, device="cuda"), rtol=1e-8)
    assert info["converged"] and abs(info["iterations"] - ref.iterations) <= 1
    xk, _, _ = S.solve(torch.tensor(f, device="cuda"), rtol=0.0, max_iter=ref.iterations)
    assert rel(xk.cpu().numpy().ravel(), ref.x) < 1e-8
    # the oracle's bases: identical preconditioner, iterates equal to FP64 rounding
    go = pkg.Options(n_levels=3, block=(8, 8, 8), ratio=[(2, 2, 2)], n_eig=[7, 7], eig_tol=1e-12)
    S2 = pkg.Solver(torch.tensor(kappa, device="cuda"), go)
    assert S2.import_bases([H.basis[0], H.basis[1]]) == 0
    xk2, info2, _ = S2.solve(torch.tensor(f, device="cuda"), rtol=0.0, max_iter=ref.iterations)
    assert info2["iterations"] == ref.iterations
    # both sides round differently inside the coarsest pseudo-inverse, whose relative
    # error is about eps * cond(A_L) (cond ~1e7 at contrast 1e6): tolerance derived from it
    w = np.linalg.eigvalsh(H.A[-1].toarray())
    tol = max(1e-10, np.finfo(float).eps * w[-1] / w[1])
    assert rel(xk2.cpu().numpy().ravel(), ref.x) < tol
    S2.close()


def test_homogeneous_closed_form_eigenvalues(pkg):
    N = 16
    go = pkg.Options(n_levels=3, block=(8, 8, 8), ratio=[(1, 1, 2)], n_eig=[7, 4], eig_tol=1e-12)
    S = pkg.Solver(torch.ones((N, N, N), dtype=torch.float64, device="cuda"), go)
    _, lam = S.export_basis(1)
    k = np.arange(8)
    vals = np.sort((2 * (1 - np.cos(np.pi * k[:, None, None] / 8)) + 2 * (1 - np.cos(np.pi * k[None, :, None] / 8))
                    + 2 * (1 - np.cos(np.pi * k[None, None, :] / 8))).ravel() / 3)[:7]
    np.testing.assert_allclose(lam.cpu().numpy(), np.tile(vals, (8, 1)), atol=1e-12)


def test_mixed_form_two_phase_eigenpairs(pkg, incl):
    """The mixed form's eigensolve (an FP32 phase, then FP64 polishing of the
    whole block) reaches the same tolerance and the same eigenpairs as LAPACK."""
    kappa, H, _ = incl
    go = pkg.Options(n_levels=3, block=(8, 8, 8), ratio=[(2, 2, 2)], n_eig=[7, 7], eig_tol=1e-12,
                     precision=pkg.MIXED)
    S = pkg.Solver(torch.tensor(kappa, device="cuda"), go)
    assert S.setup_status == 0
    assert S.info["eig_residual_max"] <= 1e-12
    Phi, lam = S.export_basis(1)
    Phi, lam = Phi.cpu().numpy(), lam.cpu().numpy()
    np.testing.assert_allclose(lam, H.lam[0], atol=1e-10)
    Po = H.basis[0]
    L = Po.shape[1]
    lam_next, _, _ = oracle.level1_eigenpairs(H.T, H.S, (8, 8, 8), L + 1)
    for e in range(Phi.shape[0]):
        gap = lam_next[e, L] - lam_next[e, L - 1]
        if gap < 1e-6:
            continue
        P1, P2 = Phi[e].T @ Phi[e], Po[e].T @ Po[e]
        assert np.abs(P1 - P2).max() <= max(1e-8, 1e-10 / gap) * np.abs(P2).max(), (e, gap)
    S.close()
