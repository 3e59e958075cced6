"""Pins for the oracle's V-cycle and PCG: the closed-form operators of
Eq. (B_ITG) and Eq. (B_c), the eigenvalue bound of Section 4, the full-space
special case, an exact cosine solution and a dense least-squares solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle


def make(shape=(8, 8, 8), box=(2, 2, 2), L=(3, 4), n_levels=3, seed=4, sigma=2.0):
    rng = np.random.default_rng(seed)
    kap = np.exp(rng.normal(0, sigma, size=shape))
    h = (1.0 / shape[2], 1.0 / shape[1], 1.0 / shape[0])
    opts = oracle.Options(n_levels=n_levels, block=box, ratio=[(2, 2, 2)] * (n_levels - 2),
                          n_eig=list(L), nu=[1] * (n_levels - 1))
    return oracle.setup(kap, h, opts)


def dense_op(apply, n):
    return np.column_stack([apply(np.eye(n)[:, j]) for j in range(n)])


def test_vcycle_matches_closed_form_three_grid_operator():
    # Eq. (B_c): B_c^{-1} = Mc^-T + Mc^-1 - Mc^-T Ac Mc^-1 + (I - Mc^-T Ac) Rcc^T Acc^+ Rcc (I - Ac Mc^-1)
    # Eq. (B_ITG): P^{-1} = M^-T + M^-1 - M^-T A M^-1 + (I - M^-T A) Rc^T B_c^{-1} Rc (I - A M^-1)
    H = make()
    n, nc = H.dims[0], H.dims[1]
    A, Ac = H.A[0].toarray(), H.A[1].toarray()
    Rc, Rcc = H.R[0].toarray(), H.R[1].toarray()
    Mi = dense_op(H.M[0].solve, n)
    Mci = dense_op(H.M[1].solve, nc)
    Ic, I = np.eye(nc), np.eye(n)
    Bc = Mci.T + Mci - Mci.T @ Ac @ Mci + (Ic - Mci.T @ Ac) @ Rcc.T @ H.coarsest_pinv @ Rcc @ (Ic - Ac @ Mci)
    P = Mi.T + Mi - Mi.T @ A @ Mi + (I - Mi.T @ A) @ Rc.T @ Bc @ Rc @ (I - A @ Mi)
    V = dense_op(lambda r: oracle.vcycle(H, r), n)
    np.testing.assert_allclose(V, P, atol=1e-9 * np.abs(P).max())


@pytest.mark.parametrize("n_levels,L", [(2, (3,)), (3, (3, 4)), (4, (2, 3, 3))])
def test_preconditioned_spectrum_in_unit_interval(n_levels, L):
    # Section 4: lambda_max(P^{-1} A) <= 1 (exact two-grid: = 1; the inexact cycle stays
    # below by induction) and lambda_min > 0 on range(A)
    H = make(n_levels=n_levels, L=L, shape=(8, 8, 16) if n_levels == 4 else (8, 8, 8))
    n = H.dims[0]
    A = H.A[0].toarray()
    V = dense_op(lambda r: oracle.vcycle(H, r), n)
    np.testing.assert_allclose(V, V.T, atol=1e-9 * np.abs(V).max())
    Q = np.linalg.qr(np.c_[np.ones(n), np.eye(n)[:, :n - 1]])[0][:, 1:]   # basis of range(A)
    # eigenvalues of V A restricted to range(A): similar to V^{1/2} A V^{1/2}
    Vr = Q.T @ V @ Q
    Ar = Q.T @ A @ Q
    C = np.linalg.cholesky(0.5 * (Vr + Vr.T))
    w = np.linalg.eigvalsh(C.T @ Ar @ C)
    assert w[-1] <= 1.0 + 1e-9
    assert w[0] > 1e-6
    if n_levels == 2:
        assert w[-1] == pytest.approx(1.0, abs=1e-8)   # lambda_max(P_TG^{-1} A) = 1


def test_full_space_two_grid_is_exact():
    # L_1 = number of cells per element: W_2 = W_h, the two-grid cycle is A^dagger
    H = make(shape=(4, 4, 4), box=(2, 2, 2), L=(8,), n_levels=2)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(64)
    res = oracle.solve(H, b, rtol=1e-10)
    assert res.iterations == 1
    x_ref = np.linalg.lstsq(H.A[0].toarray(), b - b.mean(), rcond=None)[0]
    np.testing.assert_allclose(res.x, x_ref - x_ref.mean(), atol=1e-9 * np.abs(x_ref).max())


def test_cosine_rhs_exact_solution():
    # kappa = 1: a DCT-II mode f is an eigenvector of A, so x = f / lambda exactly
    N = 8
    shape = (N, N, N)
    opts = oracle.Options(n_levels=3, block=(2, 2, 2), ratio=[(2, 2, 2)], n_eig=[4, 4], nu=[1, 1])
    H = oracle.setup(np.ones(shape), (1 / N,) * 3, opts)
    k = np.arange(N)
    f = (np.cos(np.pi * 3 * (k[None, None, :] + 0.5) / N) * np.cos(np.pi * 1 * (k[:, None, None] + 0.5) / N)
         * np.ones((1, N, 1))).ravel()
    lam = N * N * 2 * (1 - np.cos(3 * np.pi / N)) + N * N * 2 * (1 - np.cos(np.pi / N))
    res = oracle.solve(H, f, rtol=1e-12)
    np.testing.assert_allclose(res.x, f / lam, atol=1e-11 * np.abs(f / lam).max())


def test_unpreconditioned_pcg_matches_library_cg_and_lstsq():
    H = make()
    A = H.A[0]
    rng = np.random.default_rng(2)
    b = rng.standard_normal(A.shape[0])
    res = oracle.pcg(A, b, None, rtol=1e-10, max_iter=2000)
    bb = b - b.mean()
    x_ref = np.linalg.lstsq(A.toarray(), bb, rcond=None)[0]
    x_ref -= x_ref.mean()
    np.testing.assert_allclose(res.x, x_ref, atol=1e-7 * np.abs(x_ref).max())
    assert res.rhs_mean == pytest.approx(b.mean())
    # the same iterates as a library CG on the same system: compare the solution at
    # a fixed iteration count
    k = 15
    r1 = oracle.pcg(A, bb, None, rtol=0.0, max_iter=k)
    x_lib, _ = spla.cg(A, bb, rtol=0.0, atol=0.0, maxiter=k)
    np.testing.assert_allclose(r1.x, x_lib - x_lib.mean(), atol=1e-9 * np.abs(x_lib).max())


def test_mean_removed_and_solution_zero_mean():
    H = make()
    b = np.ones(H.dims[0])
    b[0] += 5.0
    res = oracle.solve(H, b, rtol=1e-10)
    assert abs(res.x.mean()) < 1e-14 * np.abs(res.x).max()
    assert res.rhs_mean == pytest.approx(b.mean())
    assert np.linalg.norm((b - b.mean()) - H.A[0] @ res.x) <= 1e-10 * np.linalg.norm(b - b.mean()) * 1.01


def test_more_coarse_vectors_fewer_iterations():
    # Section 5.2 trend: enlarging the coarse-coarse space lowers the iteration count
    rng = np.random.default_rng(9)
    kap = np.where(rng.random((16, 16, 16)) < 0.2, 1e5, 1.0)
    its = []
    for Lcc in (1, 4, 8):
        opts = oracle.Options(n_levels=3, block=(4, 4, 4), ratio=[(2, 2, 2)], n_eig=[8, Lcc], nu=[1, 1])
        H = oracle.setup(kap, (1 / 16,) * 3, opts)
        b = np.zeros(4096)
        b[0], b[-1] = 1.0, -1.0
        its.append(oracle.solve(H, b, 1e-8).iterations)
    assert its[0] >= its[1] >= its[2]


# ------------------------------------------------------------------ the mixed form's V-cycle and flexible PCG
def _small_hierarchy(contrast=1e2, seed=3):
    import fields
    N = 16
    kap = fields.grf_lognormal((N, N, N), seed=seed, contrast=contrast)
    opts = oracle.Options(n_levels=3, block=(4, 4, 4), ratio=[(2, 2, 2)], n_eig=[4, 4], nu=[1, 1])
    return oracle.setup(kap, (1 / N,) * 3, opts)


def test_mixed_vcycle_is_the_vcycle_in_single_precision():
    H = _small_hierarchy()
    rng = np.random.default_rng(0)
    r = rng.standard_normal(H.dims[0])
    r -= r.mean()
    z64 = oracle.vcycle(H, r)
    z32 = oracle.vcycle_mixed(H, r)
    d = np.linalg.norm(z32 - z64) / np.linalg.norm(z64)
    # level 1 really runs in FP32 (differs from FP64 by rounding), and only by rounding:
    # unit roundoff 6e-8 times the growth through the smoother at contrast 1e2
    assert 1e-9 < d < 1e-4, d
    assert z32.dtype == np.float64


def test_flexible_pcg_equals_standard_with_a_fixed_preconditioner():
    # with an exactly repeatable (linear, symmetric) preconditioner the Polak-Ribiere beta
    # equals the Fletcher-Reeves one in exact arithmetic: same iterations, same iterates
    H = _small_hierarchy()
    b = np.zeros(H.dims[0])
    b[0], b[-1] = 1.0, -1.0
    std = oracle.pcg(H.A[0], b, lambda r: oracle.vcycle(H, r), rtol=1e-10)
    flx = oracle.pcg(H.A[0], b, lambda r: oracle.vcycle(H, r), rtol=1e-10, flexible=True)
    assert abs(std.iterations - flx.iterations) <= 1
    k = min(std.iterations, flx.iterations)
    np.testing.assert_allclose(flx.residuals[:k], std.residuals[:k], rtol=1e-6)
    assert np.linalg.norm(flx.x - std.x) <= 1e-8 * np.linalg.norm(std.x)


def test_mixed_solve_reaches_the_tolerance():
    H = _small_hierarchy(contrast=1e3)
    b = np.zeros(H.dims[0])
    b[0], b[-1] = 1.0, -1.0
    res = oracle.solve(H, b, rtol=1e-8, mixed=True)
    assert res.converged
    bm = b - b.mean()
    assert np.linalg.norm(bm - H.A[0] @ res.x) <= 2e-8 * np.linalg.norm(bm)


# ------------------------------------------------------------------ exact two-grid P_TG (Eq. (B_TG))
def test_two_grid_matches_closed_form():
    # Eq. (B_TG): P_TG^{-1} = M^-T + M^-1 - M^-T A M^-1 + (I - M^-T A) Rc^T Ac^+ Rc (I - A M^-1),
    # with Ac^+ the pseudo-inverse of the singular coarse operator, here from an SVD
    H = make()
    n = H.dims[0]
    A, Ac, Rc = H.A[0].toarray(), H.A[1].toarray(), H.R[0].toarray()
    U, sv, Vt = np.linalg.svd(Ac)
    keep = sv > 1e-12 * sv[0]
    Acp = (Vt[keep].T / sv[keep]) @ U[:, keep].T
    Mi = dense_op(H.M[0].solve, n)
    I = np.eye(n)
    P = Mi.T + Mi - Mi.T @ A @ Mi + (I - Mi.T @ A) @ Rc.T @ Acp @ Rc @ (I - A @ Mi)
    V = dense_op(lambda r: oracle.vcycle_two_grid(H, r), n)
    np.testing.assert_allclose(V, P, atol=1e-9 * np.abs(P).max())


def test_two_grid_spectrum_top_is_one():
    # Section 4 (after Eq. (B_TG)): lambda_max(P_TG^{-1} A) = 1, and lambda_min > 0 on range(A)
    H = make()
    n = H.dims[0]
    A = H.A[0].toarray()
    V = dense_op(lambda r: oracle.vcycle_two_grid(H, r), n)
    Q = np.linalg.qr(np.c_[np.ones(n), np.eye(n)[:, :n - 1]])[0][:, 1:]
    Vr, Ar = Q.T @ V @ Q, Q.T @ A @ Q
    C = np.linalg.cholesky(0.5 * (Vr + Vr.T))
    w = np.linalg.eigvalsh(C.T @ Ar @ C)
    assert abs(w[-1] - 1.0) < 1e-9
    assert w[0] > 1e-6


def test_two_grid_equals_vcycle_with_two_levels():
    # with two levels the V-cycle's coarse step already is the exact pseudo-inverse
    H = make(n_levels=2, L=(3,))
    r = np.random.default_rng(2).standard_normal(H.dims[0])
    r -= r.mean()
    np.testing.assert_allclose(oracle.vcycle_two_grid(H, r), oracle.vcycle(H, r), rtol=1e-10, atol=1e-12)


# ------------------------------------------------------------------ cell term (wells, Section 6)
def test_cell_term_shifts_local_spectrum_by_its_weight():
    # with W = c S cell by cell, A_K phi + W phi = lambda S phi has the W-free eigenvectors
    # and eigenvalues shifted by exactly c (the right-hand form is S)
    rng = np.random.default_rng(8)
    shape = (8, 8, 8)
    h = (1 / 8,) * 3
    kap = np.exp(rng.normal(0, 1.5, size=shape))
    T = oracle.face_transmissibilities(kap, h)
    S = oracle.trace_weight(kap, h)
    lam0, Phi0, _ = oracle.level1_eigenpairs(T, S, (4, 4, 4), 5)
    lam1, Phi1, _ = oracle.level1_eigenpairs(T, S, (4, 4, 4), 5, W=0.37 * S)
    np.testing.assert_allclose(lam1, lam0 + 0.37, rtol=0, atol=1e-10)
    for e in range(8):       # same spans (projectors, S-orthonormal bases)
        np.testing.assert_allclose(Phi1[e].T @ Phi1[e], Phi0[e].T @ Phi0[e], atol=1e-8)


def test_cell_term_nonsingular_solve():
    rng = np.random.default_rng(9)
    shape = (8, 8, 16)
    h = (1 / 16, 1 / 8, 1 / 8)
    kap = np.exp(rng.normal(0, 2, size=shape))
    W = np.zeros(shape)
    W[:, 0, 0] = 50.0                      # a producer column
    W[:, -1, -1] = 80.0
    opts = oracle.Options(n_levels=3, block=(2, 2, 2), ratio=[(2, 2, 2)], n_eig=[3, 4], nu=[1, 1], cell_diag=W)
    H = oracle.setup(kap, h, opts)
    A = H.A[0].toarray()
    np.testing.assert_allclose(A - oracle.assemble(H.T).toarray(), np.diag(W.ravel()), atol=1e-12)
    assert np.linalg.eigvalsh(A).min() > 0
    b = rng.standard_normal(A.shape[0]) + 3.0          # a mean that must not be removed
    res = oracle.solve(H, b, rtol=1e-10)
    np.testing.assert_allclose(res.x, np.linalg.solve(A, b), rtol=1e-8, atol=1e-12)
    # the preconditioned spectrum stays in (0, 1] (Section 4 with a positive definite A)
    n = A.shape[0]
    V = np.column_stack([oracle.vcycle(H, np.eye(n)[:, j]) for j in range(n)])
    C = np.linalg.cholesky(0.5 * (V + V.T))
    w = np.linalg.eigvalsh(C.T @ A @ C)
    assert w[-1] <= 1.0 + 1e-9 and w[0] > 1e-6
