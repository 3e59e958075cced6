"""Pins for the oracle's hierarchy: Galerkin operators against face-by-face
constructions, the null vector and S-orthonormality of Section 3, the
level-2 local operator by an independent (recursive face-term) route,
piecewise-constant aggregation for L = 1, the IC(0) one-pivot identity and
the pseudo-inverse."""
import numpy as np
import pytest

import oracle


def make(shape=(8, 8, 8), box=(2, 2, 2), L=(3, 4), n_levels=3, seed=1, sigma=2.0, comps=3):
    rng = np.random.default_rng(seed)
    kap = np.exp(rng.normal(0, sigma, size=(comps,) + shape))
    h = (1.0 / shape[2], 1.0 / shape[1], 1.0 / shape[0])
    opts = oracle.Options(n_levels=n_levels, block=box, ratio=[(2, 2, 2)] * (n_levels - 2),
                          n_eig=list(L), nu=[1] * (n_levels - 1))
    return oracle.setup(kap, h, opts), kap, h


def boundary_diag(T, shape, box):
    """For every cell: sum of the coefficients of its faces that cross the
    boundary of its element (computed face by face)."""
    nz, ny, nx = shape
    D = np.zeros(shape)
    bx, by, bz = box
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for d, (di, dj, dk, c, b) in enumerate(((1, 0, 0, i, bx), (0, 1, 0, j, by), (0, 0, 1, k, bz))):
                    # + face
                    if (c + 1) % b == 0:
                        D[k, j, i] += T[d, k, j, i]
                    # - face
                    if c % b == 0 and c > 0:
                        D[k, j, i] += T[d, k - dk, j - dj, i - di]
    return D.ravel()


def test_dimensions():
    H, _, _ = make()
    assert H.dims == [512, 64 * 3, 8 * 4]


def test_galerkin_diagonal_block_identity():
    # diagonal block of A_2 = Lambda_a + Phi_a^T D_a Phi_a, D_a = faces crossing the element boundary
    H, kap, h = make()
    D = boundary_diag(H.T, H.shape, H.opts.block)
    Phi, cells = H.basis[0], oracle.element_cells(H.shape, H.opts.block)
    A2 = H.A[1].toarray()
    L = Phi.shape[1]
    for e in range(cells.shape[0]):
        V = Phi[e]
        ref = np.diag(H.lam[0][e]) + V @ (D[cells[e]][:, None] * V.T)
        np.testing.assert_allclose(A2[e * L:(e + 1) * L, e * L:(e + 1) * L], ref,
                                   atol=1e-10 * np.abs(ref).max())


def test_galerkin_off_diagonal_face_sum():
    # A_2[a, b] = - sum over faces (c in a, c' in b) of T_f Phi_a(c) Phi_b(c')^T
    H, kap, h = make()
    nz, ny, nx = H.shape
    bx, by, bz = H.opts.block
    ex, ey, ez = nx // bx, ny // by, nz // bz
    Phi = H.basis[0]
    L = Phi.shape[1]
    A2 = H.A[1].toarray()
    cells = oracle.element_cells(H.shape, H.opts.block)
    pos = {int(c): (e, p) for e in range(cells.shape[0]) for p, c in enumerate(cells[e])}
    for a in [0, 5, 17, 40]:
        ax, ay, az = a % ex, (a // ex) % ey, a // (ex * ey)
        for d, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            if ax + dx >= ex or ay + dy >= ey or az + dz >= ez:
                continue
            b = (ax + dx) + ex * ((ay + dy) + ey * (az + dz))
            ref = np.zeros((L, L))
            stride = (1, nx, nx * ny)[d]
            for c in cells[a]:
                c2 = c + stride
                e2, p2 = pos.get(int(c2), (None, None))
                if e2 != b:
                    continue
                k, j, i = np.unravel_index(c, H.shape)
                t = H.T[d, k, j, i]
                _, p = pos[int(c)]
                ref -= t * np.outer(Phi[a][:, p], Phi[b][:, p2])
            np.testing.assert_allclose(A2[a * L:(a + 1) * L, b * L:(b + 1) * L], ref,
                                       atol=1e-10 * np.abs(A2).max())
    # non-adjacent elements do not couple
    assert np.abs(A2[0:L, 2 * L:3 * L]).max() == 0.0


def test_constant_lies_in_every_coarse_space():
    # Section 3: the smallest eigenvalue is zero with a constant eigenvector, so the
    # kernel of A is contained in every W_l; z_l = R_{l-1}..R_1 S 1 spans null(A_l)
    H, _, _ = make(n_levels=4, shape=(8, 8, 16), box=(2, 2, 2), L=(3, 4, 3))
    B = np.eye(H.dims[0])
    for l in range(1, H.opts.n_levels):
        B = B @ H.R[l - 1].T.toarray()
        z = H.null_vectors[l]
        np.testing.assert_allclose(B @ z, 1.0, atol=1e-10)
        Az = H.A[l] @ z
        assert np.abs(Az).max() < 1e-10 * abs(H.A[l]).max()


def test_composed_basis_is_s_orthonormal():
    # Section 3: with S-normalised level-1 vectors the right-hand matrix of every
    # higher-level problem is the identity
    H, _, _ = make(n_levels=4, shape=(8, 8, 16), L=(3, 4, 3))
    s = H.S.ravel()
    B = np.eye(H.dims[0])
    for l in range(1, H.opts.n_levels):
        B = B @ H.R[l - 1].T.toarray()
        np.testing.assert_allclose(B.T @ (s[:, None] * B), np.eye(B.shape[1]), atol=1e-11)


def test_level2_operator_by_recursive_face_terms():
    # Independent route to the left matrix of Eq. (spectral cc) on each parent P:
    # children blocks Lambda_a + sum over a's faces inside P of Phi_a^T diag(T_face) Phi_a,
    # sibling blocks = A_2[a, b].  Its smallest eigenvalues must equal the oracle's.
    H, kap, h = make()
    nz, ny, nx = H.shape
    bx, by, bz = H.opts.block
    ex, ey, ez = nx // bx, ny // by, nz // bz
    Phi = H.basis[0]
    L = Phi.shape[1]
    cells = oracle.element_cells(H.shape, H.opts.block)
    A2 = H.A[1].toarray()
    pdofs = H.parent_dofs[1]
    for P in range(pdofs.shape[0]):
        children = pdofs[P][::L] // L
        N = A2[np.ix_(pdofs[P], pdofs[P])].copy()
        for ci, a in enumerate(children):
            ax, ay, az = a % ex, (a // ex) % ey, a // (ex * ey)
            blk = np.diag(H.lam[0][a]).copy()
            for c_idx, c in enumerate(cells[a]):
                k, j, i = np.unravel_index(c, H.shape)
                li, lj, lk = i - ax * bx, j - ay * by, k - az * bz
                for d, (cc, b, ec) in enumerate(((li, bx, ax), (lj, by, ay), (lk, bz, az))):
                    # + face of a at this cell: inside P iff the neighbour element is a sibling
                    if cc == b - 1 and ec % 2 == 0:
                        blk += H.T[d, k, j, i] * np.outer(Phi[a][:, c_idx], Phi[a][:, c_idx])
                    if cc == 0 and ec % 2 == 1:
                        kk, jj, ii = (k, j, i - 1) if d == 0 else ((k, j - 1, i) if d == 1 else (k - 1, j, i))
                        blk += H.T[d, kk, jj, ii] * np.outer(Phi[a][:, c_idx], Phi[a][:, c_idx])
            N[ci * L:(ci + 1) * L, ci * L:(ci + 1) * L] = blk
        w = np.linalg.eigvalsh(0.5 * (N + N.T))
        np.testing.assert_allclose(w[:H.lam[1].shape[1]], H.lam[1][P], atol=1e-9 * max(1.0, abs(w).max()))


def test_single_eigenvector_is_aggregation():
    # L_1 = 1: W_2 is piecewise constant; Phi_e = c_e 1 with c_e = (sum_K S)^(-1/2) and
    # A_2[a, b] = -c_a c_b * (sum of face coefficients between a and b)
    H, kap, h = make(L=(1, 1), n_levels=3)
    cells = oracle.element_cells(H.shape, H.opts.block)
    s = H.S.ravel()
    c = 1.0 / np.sqrt(s[cells].sum(axis=1))
    np.testing.assert_allclose(np.abs(H.basis[0][:, 0, :]), c[:, None] * np.ones(cells.shape[1]), rtol=1e-10)
    sign = np.sign(H.basis[0][:, 0, 0])
    A2 = H.A[1].toarray() * np.outer(sign, sign)
    nz, ny, nx = H.shape
    elem_of = np.empty(nx * ny * nz, dtype=int)
    for e in range(cells.shape[0]):
        elem_of[cells[e]] = e
    ref = np.zeros_like(A2)
    for d, stride in enumerate((1, nx, nx * ny)):
        t = H.T[d].ravel()
        for cidx in np.nonzero(t)[0]:
            a, b = elem_of[cidx], elem_of[cidx + stride]
            if a != b:
                ref[a, b] -= t[cidx] * c[a] * c[b]
                ref[b, a] -= t[cidx] * c[a] * c[b]
                ref[a, a] += t[cidx] * c[a] * c[a]     # Phi_a^T A Phi_a: faces leaving a
                ref[b, b] += t[cidx] * c[b] * c[b]
    np.testing.assert_allclose(A2, ref, atol=1e-10 * np.abs(ref).max())


def test_ic0_one_pivot_form():
    # IC(0) of a 7-point block in natural order has no fill: L_ij = a_ij / sqrt(d_j),
    # L_ii = sqrt(d_i), d_i = a_ii - sum_{j<i, j~i} a_ij^2 / d_j; and L L^T = A on the pattern
    H, _, _ = make(shape=(8, 8, 16), box=(4, 4, 4), L=(4, 4))
    M = H.M[0]
    cells = M.cells
    A = H.A[0].toarray()
    for e in [0, 3, 7]:
        Ab = A[np.ix_(cells[e], cells[e])]
        nb = Ab.shape[0]
        d = np.zeros(nb)
        for i in range(nb):
            d[i] = Ab[i, i] - sum(Ab[i, j] ** 2 / d[j] for j in range(i) if Ab[i, j] != 0)
        Lm = M.factor_dense(e)
        np.testing.assert_allclose(np.diag(Lm) ** 2, d, rtol=1e-12)
        off = np.tril(Ab, -1)
        mask = off != 0
        np.testing.assert_allclose(Lm[mask], (off / np.sqrt(d)[None, :])[mask], rtol=1e-12)
        LLt = Lm @ Lm.T
        pat = Ab != 0
        np.testing.assert_allclose(LLt[pat], Ab[pat], rtol=1e-11, atol=1e-12 * np.abs(Ab).max())


def test_coarse_block_cholesky_inverts_blocks():
    H, _, _ = make()
    M = H.M[1]
    A2 = H.A[1].toarray()
    for P in range(3):
        idx = H.parent_dofs[1][P]
        e = np.zeros(A2.shape[0])
        for col in range(4):
            e[:] = 0
            e[idx[col]] = 1.0
            z = M.solve(e)
            np.testing.assert_allclose(A2[np.ix_(idx, idx)] @ z[idx], e[idx], atol=1e-10)


def test_pseudo_inverse():
    H, _, _ = make()
    Ac = H.A[-1].toarray()
    z = H.null_vectors[-1]
    zh = z / np.linalg.norm(z)
    rng = np.random.default_rng(0)
    r = rng.standard_normal(Ac.shape[0])
    r -= zh * (zh @ r)
    x = H.coarsest_pinv @ r
    np.testing.assert_allclose(Ac @ x, r, atol=1e-9 * np.linalg.norm(r))
    assert abs(zh @ x) < 1e-10 * np.linalg.norm(x)
    # Moore-Penrose: pinv annihilates the null vector
    assert np.linalg.norm(H.coarsest_pinv @ zh) < 1e-8 * np.linalg.norm(H.coarsest_pinv)


def test_coarse_ic0_option_runs():
    rng = np.random.default_rng(1)
    kap = np.exp(rng.normal(0, 1, size=(8, 8, 8)))
    opts = oracle.Options(n_levels=3, block=(2, 2, 2), ratio=[(2, 2, 2)], n_eig=[2, 3], nu=[1, 1],
                          coarse_smoother="ic0")
    H = oracle.setup(kap, (1 / 8,) * 3, opts)
    res = oracle.solve(H, np.r_[1.0, np.zeros(510), -1.0], 1e-8)
    assert res.converged


def test_single_element_level_is_rejected():
    with pytest.raises(ValueError):
        make(shape=(8, 8, 8), box=(4, 4, 4), L=(4, 4))


# ------------------------------------------------------------------ coarse IC(0) (Section 5: incomplete Cholesky for M_c)
def test_ic0_dense_hand_worked_3x3():
    # one structural zero at (2, 1): the fill -l21 l31 / l22 = -1/2 that exact
    # Cholesky would put there is dropped, so l33 = sqrt(6 - 1) instead of sqrt(4.75)
    A = np.array([[4.0, 2.0, 2.0], [2.0, 5.0, 0.0], [2.0, 0.0, 6.0]])
    L = oracle.ic0_dense(A, A != 0)
    ref = np.array([[2.0, 0.0, 0.0], [1.0, 2.0, 0.0], [1.0, 0.0, np.sqrt(5.0)]])
    np.testing.assert_allclose(L, ref, rtol=0, atol=1e-15)


def test_ic0_dense_full_pattern_is_cholesky():
    import scipy.linalg as sla
    rng = np.random.default_rng(4)
    X = rng.standard_normal((12, 12))
    A = X @ X.T + 12 * np.eye(12)
    L = oracle.ic0_dense(A, np.ones_like(A, dtype=bool))
    np.testing.assert_allclose(L, sla.cholesky(A, lower=True), rtol=1e-13, atol=1e-13)


def test_ic0_dense_matches_A_on_its_pattern():
    # 2-D five-point matrix on a 4 x 4 grid: exact Cholesky fills the band, IC(0) keeps the
    # pattern; L L^T equals A on the pattern (the defining property) and differs off it
    rng = np.random.default_rng(5)
    m = 4
    n = m * m
    A = np.zeros((n, n))
    for i in range(n):
        x, y = i % m, i // m
        for j, ok in ((i + 1, x + 1 < m), (i + m, y + 1 < m)):
            if ok:
                t = rng.uniform(0.5, 2.0)
                A[i, j] = A[j, i] = -t
                A[i, i] += t
                A[j, j] += t
    A += np.diag(rng.uniform(0.1, 0.3, n))
    pat = A != 0
    L = oracle.ic0_dense(A, pat)
    assert np.all(L[~np.tril(pat)] == 0.0)
    LLt = L @ L.T
    np.testing.assert_allclose(LLt[pat], A[pat], rtol=0, atol=1e-13 * np.abs(A).max())
    assert np.abs(LLt[~pat]).max() > 1e-3              # the dropped fill
    assert not np.allclose(L, np.linalg.cholesky(A))


def test_block_ic0_falls_back_to_cholesky_on_breakdown():
    import scipy.sparse as sps
    # Kershaw's 4 x 4 SPD matrix: IC(0) on its nonzero pattern meets a negative pivot
    K = np.array([[3.0, -2.0, 0.0, 2.0], [-2.0, 3.0, -2.0, 0.0], [0.0, -2.0, 3.0, -2.0], [2.0, 0.0, -2.0, 3.0]])
    assert np.linalg.eigvalsh(K).min() > 0
    with pytest.raises(FloatingPointError):
        oracle.ic0_dense(K, K != 0)
    good = np.diag([2.0, 3.0, 4.0, 5.0]) + np.diag([-0.5] * 3, 1) + np.diag([-0.5] * 3, -1)
    A = sps.block_diag([good, K]).tocsr()
    M = oracle.BlockIC0Dense(A, np.array([[0, 1, 2, 3], [4, 5, 6, 7]]))
    assert M.fallback == [1]
    np.testing.assert_allclose(M.factors[1], np.linalg.cholesky(K), rtol=1e-14)
    r = np.arange(1.0, 9.0)
    z = M.solve(r)
    np.testing.assert_allclose(K @ z[4:], r[4:], rtol=1e-12)        # exact on the fallback block
    np.testing.assert_allclose(good @ z[:4], r[:4], rtol=1e-12)     # tridiagonal: IC(0) is exact


def test_sibling_pattern():
    P = oracle.sibling_pattern((2, 2, 2), 1)
    # child 0 of a 2 x 2 x 2 parent shares faces with children 1 (x), 2 (y), 4 (z)
    assert list(np.flatnonzero(P[0])) == [0, 1, 2, 4]
    assert list(np.flatnonzero(P[7])) == [3, 5, 6, 7]
    assert (P == P.T).all() and P.sum() == 8 * 4
    P3 = oracle.sibling_pattern((2, 1, 1), 3)
    assert P3.shape == (6, 6) and P3.all()


# ------------------------------------------------------------------ Strategy 2 (Section 5: thresholds B_c, B_cc)
def _inertia_below(Am: np.ndarray, Sm: np.ndarray, B: float) -> int:
    """Eigenvalues of A x = lambda S x below B, by Sylvester's law of inertia: the
    negative eigenvalues of D in the LDL^T factorisation of A - B S."""
    import scipy.linalg as sla
    _, D, _ = sla.ldl(Am - B * Sm, lower=True)
    return int(np.count_nonzero(np.linalg.eigvalsh(D) < 0))


def _strategy2(B1, B2, n_levels=3, shape=(8, 8, 16), L=(6, 8), seed=3, sigma=2.0):
    rng = np.random.default_rng(seed)
    kap = np.exp(rng.normal(0, sigma, size=shape))
    h = (1.0 / shape[2], 1.0 / shape[1], 1.0 / shape[0])
    opts = oracle.Options(n_levels=n_levels, block=(2, 2, 2), ratio=[(2, 2, 2)] * (n_levels - 2), n_eig=list(L),
                          nu=[1] * (n_levels - 1), eig_threshold=[B1, B2][:n_levels - 1])
    return oracle.setup(kap, h, opts)


def test_strategy2_level1_counts_by_inertia():
    B = 0.35
    H = _strategy2(B, 0.0)
    An = oracle.assemble(H.T * oracle.interior_face_mask(H.shape, (2, 2, 2))).tocsr()
    cells = oracle.element_cells(H.shape, (2, 2, 2))
    s = H.S.ravel()
    for e in range(cells.shape[0]):
        idx = cells[e]
        c = _inertia_below(An[idx][:, idx].toarray(), np.diag(s[idx]), B)
        assert H.counts[0][e] == min(max(c, 1), 6)
        assert np.all(H.basis[0][e, H.counts[0][e]:] == 0.0)
    assert H.dims[1] == H.counts[0].sum()
    assert 1 < H.counts[0].min() < H.counts[0].max() <= 6         # ragged in this field


def test_strategy2_homogeneous_ladder():
    # kappa = 1 on 4^3 elements of a 8^3 grid: the local spectrum is the ladder of Section 5.2,
    # lambda = (1/3) sum_d 2 (1 - cos(pi k_d / 4)) / ... ; the first distinct values have
    # multiplicities 1, 3, 3, 1: a threshold between the 2nd and 3rd distinct value keeps 4
    shape = (8, 8, 8)
    h = (1 / 8,) * 3
    lam_all, _, _ = oracle.level1_eigenpairs(oracle.face_transmissibilities(np.ones(shape), h),
                                             oracle.trace_weight(np.ones(shape), h), (4, 4, 4), 12)
    d = np.unique(np.round(lam_all[0], 10))
    for B, expect in (((d[1] + d[2]) / 2, 4), ((d[2] + d[3]) / 2, 7), ((d[3] + d[4]) / 2, 8)):
        opts = oracle.Options(n_levels=2, block=(4, 4, 4), ratio=[], n_eig=[12], nu=[1], eig_threshold=[B])
        H = oracle.setup(np.ones(shape), h, opts)
        assert list(H.counts[0]) == [expect] * 8


def test_strategy2_huge_threshold_is_strategy1():
    # Table (second approach), last row: B = 1e12 keeps every candidate
    H2 = _strategy2(1e12, 1e12)
    H1 = _strategy2(0.0, 0.0)
    assert H2.dims == H1.dims
    for l in range(3):
        assert abs(H2.A[l] - H1.A[l]).max() == 0.0


@pytest.mark.parametrize("n_levels", [3, 4])
def test_strategy2_ragged_hierarchy_invariants(n_levels):
    H = _strategy2(0.35, 0.05, n_levels=n_levels, shape=(8, 16, 16) if n_levels == 4 else (8, 8, 16),
                   L=(6, 8, 4) if n_levels == 4 else (6, 8))
    n = H.dims[0]
    # W_{l+1} coordinates: one per kept vector; Psi rows orthonormal (Eq. (spectral cc), right matrix I)
    for l in range(2, n_levels):
        assert H.dims[l] == H.counts[l - 1].sum()
        Rl = H.R[l - 1].toarray()
        np.testing.assert_allclose(Rl @ Rl.T, np.eye(Rl.shape[0]), atol=1e-12)
    assert len(set(H.counts[1].tolist())) > 1                    # the level-2 spaces are ragged
    # the composed basis is S-orthonormal and the constant stays in every space
    Bc = np.eye(n)
    for Rm in H.R:
        Bc = Bc @ Rm.T.toarray()
    np.testing.assert_allclose(Bc.T @ (H.S.ravel()[:, None] * Bc), np.eye(Bc.shape[1]), atol=1e-10)
    for l in range(1, n_levels):
        np.testing.assert_allclose(H.A[l] @ H.null_vectors[l], 0.0, atol=1e-9 * abs(H.A[l]).max())
    # the preconditioner keeps its spectrum in (0, 1] on range(A) (Section 4)
    A = H.A[0].toarray()
    V = np.column_stack([oracle.vcycle(H, np.eye(n)[:, j]) for j in range(n)])
    Q = np.linalg.qr(np.c_[np.ones(n), np.eye(n)[:, :n - 1]])[0][:, 1:]
    Vr, Ar = Q.T @ V @ Q, Q.T @ A @ Q
    C = np.linalg.cholesky(0.5 * (Vr + Vr.T))
    w = np.linalg.eigvalsh(C.T @ Ar @ C)
    assert w[-1] <= 1.0 + 1e-9 and w[0] > 1e-6


def test_ragged_pattern_uniform_equals_sibling_pattern():
    P = oracle.ragged_pattern((2, 2, 2), np.full(8, 3))
    assert (P == oracle.sibling_pattern((2, 2, 2), 3)).all()
    Q = oracle.ragged_pattern((2, 1, 1), np.array([1, 2]))
    assert Q.shape == (3, 3) and Q.all()
