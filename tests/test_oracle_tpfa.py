"""Pins for the oracle's fine operator (Section 2.2) against hand-computed
values, the closed-form homogeneous spectrum and a brute-force face loop."""
import itertools

import numpy as np
import pytest

import oracle


def test_two_cell_harmonic_average_x():
    # Fig. (kappa edge): kappa~_{i+1/2} = 2 / (1/kappa~_i + 1/kappa~_{i+1}), kappa~ = kappa/h^2
    h = (0.5, 0.25, 0.125)
    kap = np.zeros((3, 1, 1, 2))
    kap[0] = [[[3.0, 7.0]]]          # kappa^x used by the x face
    kap[1] = [[[1e9, 1e-9]]]         # other components must not enter
    kap[2] = [[[5e5, 2e-3]]]
    T = oracle.face_transmissibilities(kap, h)
    expect = 2.0 / (h[0] ** 2 / 3.0 + h[0] ** 2 / 7.0)
    assert T[0, 0, 0, 0] == pytest.approx(expect, rel=1e-15)
    assert T[0, 0, 0, 1] == 0.0 and np.all(T[1] == 0) and np.all(T[2] == 0)
    A = oracle.assemble(T).toarray()
    np.testing.assert_allclose(A, [[expect, -expect], [-expect, expect]], rtol=1e-15)


def test_orthotropic_component_per_direction():
    h = (1.0, 1.0, 0.5)
    kap = np.zeros((3, 2, 1, 1))     # two cells stacked in z
    kap[0] = 1e6
    kap[1] = 1e6
    kap[2][:, 0, 0] = [2.0, 3.0]
    T = oracle.face_transmissibilities(kap, h)
    assert T[2, 0, 0, 0] == pytest.approx(2.0 / (0.25 / 2.0 + 0.25 / 3.0), rel=1e-15)
    assert np.all(T[0] == 0) and np.all(T[1] == 0) and T[2, 1, 0, 0] == 0.0


@pytest.mark.parametrize("shape", [(4, 5, 6), (3, 3, 3), (2, 7, 1)])
def test_homogeneous_cosine_modes_are_eigenvectors(shape):
    # kappa = 1, h_d = 1/N_d: A = sum_d N_d^2 L_d (Neumann second differences); the
    # DCT-II products cos(pi k_d (i_d + 1/2) / N_d) are eigenvectors with eigenvalue
    # sum_d N_d^2 * 2 (1 - cos(pi k_d / N_d)).
    nz, ny, nx = shape
    h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    A = oracle.assemble(oracle.face_transmissibilities(np.ones(shape), h))
    k_idx = np.arange(nz)[:, None, None], np.arange(ny)[None, :, None], np.arange(nx)[None, None, :]
    for kx, ky, kz in itertools.product(range(nx), range(ny), range(nz)):
        v = (np.cos(np.pi * kx * (k_idx[2] + 0.5) / nx) * np.cos(np.pi * ky * (k_idx[1] + 0.5) / ny)
             * np.cos(np.pi * kz * (k_idx[0] + 0.5) / nz)).ravel()
        lam = (nx ** 2 * 2 * (1 - np.cos(np.pi * kx / nx)) + ny ** 2 * 2 * (1 - np.cos(np.pi * ky / ny))
               + nz ** 2 * 2 * (1 - np.cos(np.pi * kz / nz)))
        np.testing.assert_allclose(A @ v, lam * v, atol=1e-10 * max(lam, 1.0))


def test_variational_form_brute_force():
    # Eq. (discrete varia): q^T A p = sum over internal faces of T (p_j - p_i)(q_j - q_i)
    rng = np.random.default_rng(3)
    shape = (2, 3, 4)
    h = (0.3, 0.2, 0.7)
    kap = np.exp(rng.normal(0, 2, size=(3,) + shape))
    A = oracle.assemble(oracle.face_transmissibilities(kap, h))
    p = rng.standard_normal(np.prod(shape))
    q = rng.standard_normal(np.prod(shape))
    nz, ny, nx = shape
    total = 0.0
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = i + nx * (j + ny * k)
                for d, (di, dj, dk) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                    i2, j2, k2 = i + di, j + dj, k + dk
                    if i2 >= nx or j2 >= ny or k2 >= nz:
                        continue
                    c2 = i2 + nx * (j2 + ny * k2)
                    a = kap[d, k, j, i] / h[d] ** 2
                    b = kap[d, k2, j2, i2] / h[d] ** 2
                    t = 2.0 / (1.0 / a + 1.0 / b)
                    total += t * (p[c2] - p[c]) * (q[c2] - q[c])
    assert q @ (A @ p) == pytest.approx(total, rel=1e-12)


def test_symmetric_psd_constant_null_space():
    rng = np.random.default_rng(5)
    shape = (3, 4, 5)
    kap = np.exp(rng.normal(0, 3, size=(3,) + shape))
    A = oracle.assemble(oracle.face_transmissibilities(kap, (0.2, 0.25, 1 / 3))).toarray()
    np.testing.assert_allclose(A, A.T, rtol=0, atol=0)
    np.testing.assert_allclose(A @ np.ones(A.shape[0]), 0.0, atol=1e-12 * np.abs(A).max())
    w = np.linalg.eigvalsh(A)
    assert w[0] > -1e-12 * w[-1]
    assert w[1] > 1e-9 * w[-1]          # exactly one null direction (connected grid)


def test_face_coefficient_bounds():
    # Section 4: the harmonic average lies between min and 2*min of the two cells
    rng = np.random.default_rng(7)
    shape = (4, 4, 4)
    kap = np.exp(rng.normal(0, 4, size=shape))
    h = (0.25, 0.25, 0.25)
    T = oracle.face_transmissibilities(kap, h)
    kt = kap / 0.0625
    lo = np.minimum(kt[:, :, :-1], kt[:, :, 1:])
    assert np.all(T[0][:, :, :-1] <= 2 * lo * (1 + 1e-15))
    assert np.all(T[0][:, :, :-1] >= lo * (1 - 1e-15))


@pytest.mark.parametrize("shape", [(4, 5, 6), (2, 7, 1)])
def test_matrix_free_apply_closed_form_and_assembled(shape):
    # the matrix-free form reproduces the closed-form DCT eigenpairs of the homogeneous
    # operator and the assembled matrix on a heterogeneous orthotropic field
    nz, ny, nx = shape
    h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    T1 = oracle.face_transmissibilities(np.ones(shape), h)
    iz, iy, ix = np.arange(nz)[:, None, None], np.arange(ny)[None, :, None], np.arange(nx)[None, None, :]
    for kx, ky, kz in [(1, 0, 0), (0, min(2, ny - 1), 0), (nx - 1, ny - 1, nz - 1)]:
        v = (np.cos(np.pi * kx * (ix + 0.5) / nx) * np.cos(np.pi * ky * (iy + 0.5) / ny)
             * np.cos(np.pi * kz * (iz + 0.5) / nz))
        lam = (nx ** 2 * 2 * (1 - np.cos(np.pi * kx / nx)) + ny ** 2 * 2 * (1 - np.cos(np.pi * ky / ny))
               + nz ** 2 * 2 * (1 - np.cos(np.pi * kz / nz)))
        np.testing.assert_allclose(oracle.apply_A(T1, v), lam * v, atol=1e-10 * max(lam, 1.0))
    rng = np.random.default_rng(11)
    kap = np.exp(rng.normal(0, 3, size=(3,) + shape))
    T = oracle.face_transmissibilities(kap, (0.3, 0.2, 0.7))
    p = rng.standard_normal(shape)
    q = oracle.apply_A(T, p)
    ref = oracle.assemble(T) @ p.ravel()
    np.testing.assert_allclose(q.ravel(), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    assert abs(q.sum()) < 1e-12 * np.abs(q).max()          # A 1 = 0 implies 1^T A p = 0


# ------------------------------------------------------------------ velocity recovery (Eq. (velocity))
def test_velocity_two_cells_by_hand():
    # kappa^x = (1, 3) on a 2 x 1 x 1 grid, h = (1/2, 1, 1): normalised 4 and 12, harmonic
    # face coefficient 2 / (1/4 + 1/12) = 6, kappa_e = 6 h^2 = 1.5; p = (1, 3):
    # v = -1.5 (3 - 1) / (1/2) = -6 on the interior face, 0 on the boundary
    kap = np.array([[[1.0, 3.0]]])
    h = (0.5, 1.0, 1.0)
    T = oracle.face_transmissibilities(kap, h)
    v = oracle.velocity(T, np.array([1.0, 3.0]), h)
    np.testing.assert_allclose(v[0].ravel(), [-6.0, 0.0], rtol=1e-15)
    assert not v[1].any() and not v[2].any()
    # divergence: cell 0 loses -6 through +x (-6 / 0.5 = -12), cell 1 gains it
    np.testing.assert_allclose(oracle.divergence(v, h).ravel(), [-12.0, 12.0], rtol=1e-15)


def test_velocity_of_linear_pressure_is_darcy_flux():
    # homogeneous kappa = 5, p = x at the cell centres: v_x = -kappa dp/dx = -5 on interior
    # x faces, 0 on the x boundary faces, v_y = v_z = 0
    shape = (3, 4, 6)
    h = (1 / 6, 1 / 4, 1 / 3)
    T = oracle.face_transmissibilities(np.full(shape, 5.0), h)
    x = (np.arange(6) + 0.5) * h[0]
    p = np.broadcast_to(x[None, None, :], shape)
    v = oracle.velocity(T, p, h)
    np.testing.assert_allclose(v[0][:, :, :-1], -5.0, rtol=1e-13)
    assert not v[0][:, :, -1].any() and not v[1].any() and not v[2].any()


def test_divergence_of_velocity_is_A_p_and_conserves_mass():
    # div v = A p (the assembled matrix of Eq. (discrete varia), an independent route), and
    # with no-flow boundaries the cell balances sum to zero
    rng = np.random.default_rng(7)
    shape = (5, 4, 6)
    h = (1 / 6, 1 / 4, 1 / 5)
    kap = np.exp(rng.normal(0, 2, size=(3,) + shape))
    T = oracle.face_transmissibilities(kap, h)
    p = rng.standard_normal(shape)
    div = oracle.divergence(oracle.velocity(T, p, h), h)
    Ap = oracle.assemble(T) @ p.ravel()
    np.testing.assert_allclose(div.ravel(), Ap, rtol=0, atol=1e-11 * np.abs(Ap).max())
    assert abs(div.sum()) < 1e-10 * np.abs(div).sum()
