"""Pins for the oracle's local spectral problems (Eq. (spepb), Eq. (spectral cc))
against closed forms, the ladder the paper prints and brute force."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def homogeneous_local_eigs(box, h):
    """Closed form for kappa = 1: A_K = sum_d h_d^-2 L_d(b_d), S = sum_d h_d^-2, so
    lambda = sum_d h_d^-2 2(1 - cos(pi k_d / b_d)) / sum_d h_d^-2."""
    bx, by, bz = box
    w = [1.0 / h[0] ** 2, 1.0 / h[1] ** 2, 1.0 / h[2] ** 2]
    vals = []
    for kz in range(bz):
        for ky in range(by):
            for kx in range(bx):
                vals.append(sum(w[d] * 2 * (1 - np.cos(np.pi * k / b))
                                for d, (k, b) in enumerate(((kx, bx), (ky, by), (kz, bz)))) / sum(w))
    return np.sort(vals)


@pytest.mark.parametrize("shape,box,h", [((8, 8, 8), (4, 4, 4), (1 / 8, 1 / 8, 1 / 8)),
                                         ((8, 6, 4), (2, 3, 4), (1 / 4, 1 / 6, 1 / 8))])
def test_homogeneous_closed_form(shape, box, h):
    kap = np.ones(shape)
    T = oracle.face_transmissibilities(kap, h)
    S = oracle.trace_weight(kap, h)
    nb = box[0] * box[1] * box[2]
    lam, Phi, cells = oracle.level1_eigenpairs(T, S, box, nb)
    ref = homogeneous_local_eigs(box, h)
    for e in range(lam.shape[0]):
        np.testing.assert_allclose(lam[e], ref, atol=1e-12)


def test_ladder_multiplicities_match_paper():
    ladder = np.loadtxt(os.path.join(GOLDEN, "laplace_ladder.txt"))
    runs = np.diff(np.flatnonzero(np.diff(np.r_[-1, ladder, 1e9]) != 0))
    kap = np.ones((8, 8, 8))
    h = (1 / 8,) * 3
    lam, _, _ = oracle.level1_eigenpairs(oracle.face_transmissibilities(kap, h),
                                         oracle.trace_weight(kap, h), (8, 8, 8), 18)
    w = lam[0]
    groups = np.diff(np.flatnonzero(np.diff(np.r_[-1.0, w[:17], 1e9]) > 1e-9))
    assert list(groups) == list(runs)
    assert list(np.cumsum(groups)) == [1, 4, 7, 8, 11, 17]
    assert w[17] > w[16] + 1e-6          # 17 closes a multiplicity group


def random_field(shape, seed, sigma=2.0, comps=3):
    rng = np.random.default_rng(seed)
    return np.exp(rng.normal(0, sigma, size=(comps,) + shape))


def test_eigen_relations_heterogeneous():
    shape, box, h = (6, 4, 8), (2, 2, 3), (1 / 8, 1 / 4, 1 / 6)
    kap = random_field(shape, 11)
    T = oracle.face_transmissibilities(kap, h)
    S = oracle.trace_weight(kap, h)
    L = 5
    lam, Phi, cells = oracle.level1_eigenpairs(T, S, box, L)
    An = oracle.assemble(T * oracle.interior_face_mask(shape, box)).toarray()
    s = S.ravel()
    for e in range(cells.shape[0]):
        idx = cells[e]
        Ae = An[np.ix_(idx, idx)]
        V = Phi[e]
        np.testing.assert_allclose(V @ np.diag(s[idx]) @ V.T, np.eye(L), atol=1e-12)
        np.testing.assert_allclose(V @ Ae @ V.T, np.diag(lam[e]), atol=1e-10 * np.abs(Ae).max())
        # smallest eigenvalue zero with a constant eigenvector (Section 3 remark)
        assert abs(lam[e, 0]) < 1e-12 * lam[e, -1] + 1e-14
        v0 = V[0] / V[0][0]
        np.testing.assert_allclose(v0, 1.0, atol=1e-9)
        # residual of the generalised problem
        R = Ae @ V.T - (s[idx][:, None] * V.T) * lam[e][None, :]
        assert np.abs(R).max() < 1e-10 * np.abs(Ae).max()


def test_two_cell_element_closed_form():
    # element of two cells: A_K = [[t, -t], [-t, t]], S = diag(s1, s2):
    # eigenvalues 0 and t (1/s1 + 1/s2)
    kap = np.array([[[2.0, 9.0]]])
    h = (0.5, 1.0, 1.0)
    T = oracle.face_transmissibilities(kap, h)
    S = oracle.trace_weight(kap, h)
    lam, Phi, _ = oracle.level1_eigenpairs(T, S, (2, 1, 1), 2)
    t = T[0, 0, 0, 0]
    s1, s2 = S.ravel()
    np.testing.assert_allclose(lam[0], [0.0, t * (1 / s1 + 1 / s2)], atol=1e-12 * t)
    v = Phi[0, 1]
    assert v[0] / v[1] == pytest.approx(-s2 / s1, rel=1e-12)


def test_courant_fischer_random_subspaces():
    # the k-th eigenvalue is the min over k-dim subspaces of the max Rayleigh quotient;
    # a random (k+1)-dim subspace never beats the computed lambda_k
    shape, box, h = (4, 4, 4), (4, 4, 4), (0.25,) * 3
    kap = random_field(shape, 2, comps=1)
    T = oracle.face_transmissibilities(kap, h)
    S = oracle.trace_weight(kap, h)
    lam, Phi, cells = oracle.level1_eigenpairs(T, S, box, 6)
    An = oracle.assemble(T).toarray()
    s = S.ravel()[cells[0]]
    rng = np.random.default_rng(0)
    for k in range(6):
        for _ in range(20):
            Q = rng.standard_normal((64, k + 1))
            # generalized Ritz values of the subspace
            G = Q.T @ (s[:, None] * Q)
            H = Q.T @ An @ Q
            ritz = np.linalg.eigvalsh(np.linalg.solve(np.linalg.cholesky(G), np.linalg.solve(np.linalg.cholesky(G), H).T))
            assert ritz[-1] >= lam[0, k] - 1e-9 * lam[0, -1]
