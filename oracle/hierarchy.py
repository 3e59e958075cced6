"""Set-up phase of the spectral multigrid preconditioner, FP64.

Test infrastructure only (see the package docstring).

Levels are numbered l = 1 .. n_levels with W_1 = W_h the fine space and
W_{n_levels} the coarsest (Section 3: W_L c ... c W_1 = W_h).  Elements:
E_1 partitions the fine grid into boxes of ``block`` cells (the coarse
elements of Section 3); E_l (l >= 2) groups ``ratio[l-2]`` elements of
E_{l-1} per direction (coarse-coarse elements and beyond).  W_{l+1} is
spanned by the ``n_eig[l-1]`` smallest local eigenvectors on every element
of E_l, and its coordinates are ordered (element of E_l lexicographic, then
eigenvector index).

Per level the oracle builds:
* R_l, the restriction with one row per local eigenvector (Section 3),
* A_{l+1} = R_l A_l R_l^T (Section 3, the Galerkin relations stated before
  Eq. (B_c)),
* the smoother M_l: block Jacobi over the elements of E_l; incomplete Cholesky
  (no fill) of each block on the fine level and exact Cholesky of each block
  on coarse levels (Section 5 names incomplete Cholesky for both; the exact
  coarse factor is this build's reading, recorded with the design notes),
* the Moore-Penrose pseudo-inverse of the coarsest operator (Algorithm 1's
  A_cc^dagger), dense.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .tpfa import (assemble, face_transmissibilities, interior_face_mask, trace_weight)
from .spectral import coarse_eigenpairs, coarse_eigenpairs_kept, element_cells, level1_eigenpairs


@dataclass
class Options:
    """Hierarchy parameters (Section 5: sd, nu, nu_c, L_c, L_cc generalised to
    any number of levels)."""
    n_levels: int = 3
    block: tuple = (4, 4, 4)                 # E_1 element size in cells (bx, by, bz)
    ratio: list = field(default_factory=lambda: [(2, 2, 2)])  # E_l, l >= 2, per direction
    n_eig: list = field(default_factory=lambda: [4, 4])       # L_1 .. L_{n_levels-1}
    nu: list = field(default_factory=lambda: [1, 1])          # sweeps on levels 1 .. n_levels-1
    coarse_smoother: str = "chol"            # "chol" (exact block Cholesky) or "ic0"
    # Strategy 2 of Section 5: eig_threshold[l-1] > 0 keeps, on every element of E_l, the
    # candidate eigenvectors (n_eig[l-1] of them) whose eigenvalues lie below the threshold
    # (B_c, B_cc), at least one; 0 (or a short list) keeps all n_eig[l-1] (Strategy 1)
    eig_threshold: list = field(default_factory=list)
    # a nonnegative term added to the diagonal of A cell by cell (the well terms of
    # Section 6: W_i = WI kappa lambda / mu at the cells a producer crosses), and to
    # the left-hand forms of the local problems, as Section 6 modifies them; None: none
    cell_diag: object = None

    def singular(self) -> bool:
        """A has the constant null space (no cell term)."""
        return self.cell_diag is None or not np.any(np.asarray(self.cell_diag) > 0)

    def threshold(self, l: int) -> float:
        """B for the local problems on the elements of E_l (0: Strategy 1)."""
        return float(self.eig_threshold[l - 1]) if l - 1 < len(self.eig_threshold) else 0.0

    def check(self):
        if self.n_levels < 2:
            raise ValueError("need at least two levels")
        if len(self.ratio) < self.n_levels - 2 or len(self.n_eig) < self.n_levels - 1 \
                or len(self.nu) < self.n_levels - 1:
            raise ValueError("per-level option lists too short")


class BlockIC0:
    """Block-Jacobi smoother whose blocks are factorised by incomplete Cholesky
    with no fill (Section 5).  Each block is the diagonal sub-matrix A[c, c] of
    the global matrix over one element's cells, taken in the element's
    lexicographic order.  The algorithm is the generic pattern-restricted
    IC(0): a right-looking Cholesky that drops every update falling outside the
    block's nonzero pattern.  All blocks share one pattern (same element
    shape), so the loops run over pattern entries and vectorise over blocks."""

    def __init__(self, A: sp.spmatrix, cells: np.ndarray, box):
        A = sp.csr_matrix(A)
        self.cells = cells
        m, nb = cells.shape
        bx, by, bz = box
        # structural pattern of one block: i == j or face neighbours in the box
        lz, ly, lx = np.unravel_index(np.arange(nb), (bz, by, bx))
        self.nb = nb
        lower = [[] for _ in range(nb)]       # lower[i] = columns j < i in row i
        for i in range(nb):
            for d, (c, n_c, step) in enumerate(((lx, bx, 1), (ly, by, bx), (lz, bz, bx * by))):
                if c[i] > 0:
                    lower[i].append(i - step)
            lower[i].sort()
        self.lower = lower
        upper = [[] for _ in range(nb)]       # upper[j] = rows i > j with (i, j) in pattern
        for i in range(nb):
            for j in lower[i]:
                upper[j].append(i)
        self.upper = upper
        pattern = set()
        for i in range(nb):
            pattern.add((i, i))
            for j in lower[i]:
                pattern.add((i, j))
        # block values on the pattern, vectorised over blocks
        W = {}
        for (i, j) in pattern:
            W[(i, j)] = np.asarray(A[cells[:, i], cells[:, j]]).ravel().astype(np.float64)
        # right-looking IC(0) restricted to the pattern
        for k in range(nb):
            if np.any(W[(k, k)] <= 0):
                raise FloatingPointError("IC(0) pivot is not positive")
            W[(k, k)] = np.sqrt(W[(k, k)])
            col = upper[k]
            for i in col:
                W[(i, k)] = W[(i, k)] / W[(k, k)]
            for j in col:
                for i in col:
                    if i >= j and (i, j) in pattern:
                        W[(i, j)] = W[(i, j)] - W[(i, k)] * W[(j, k)]
        self.L = W                            # lower factor on the pattern

    def factor_dense(self, e: int) -> np.ndarray:
        """Dense lower-triangular factor of block ``e`` (for tests)."""
        Lm = np.zeros((self.nb, self.nb))
        for (i, j), v in self.L.items():
            Lm[i, j] = v[e]
        return Lm

    def solve(self, r: np.ndarray) -> np.ndarray:
        """z = M^{-1} r = L^{-T} L^{-1} r on every block (M = L L^T is
        symmetric, so this is also M^{-T} r)."""
        rb = r[self.cells]                    # (m, nb)
        y = np.empty_like(rb)
        for i in range(self.nb):
            acc = rb[:, i].copy()
            for j in self.lower[i]:
                acc -= self.L[(i, j)] * y[:, j]
            y[:, i] = acc / self.L[(i, i)]
        z = np.empty_like(rb)
        for i in range(self.nb - 1, -1, -1):
            acc = y[:, i].copy()
            for j in self.upper[i]:
                acc -= self.L[(j, i)] * z[:, j]
            z[:, i] = acc / self.L[(i, i)]
        out = np.empty_like(r)
        out[self.cells] = z
        return out


class BlockCholesky:
    """Block-Jacobi smoother with an exact dense Cholesky factor of each block
    A[idx, idx] (coarse levels)."""

    def __init__(self, A: sp.spmatrix, dofs: np.ndarray):
        A = sp.csr_matrix(A)
        self.dofs = dofs
        self.factors = []
        for idx in dofs:
            blk = A[idx][:, idx].toarray()
            self.factors.append(sla.cho_factor(0.5 * (blk + blk.T), lower=True))

    def solve(self, r: np.ndarray) -> np.ndarray:
        out = np.empty_like(r)
        for idx, f in zip(self.dofs, self.factors):
            out[idx] = sla.cho_solve(f, r[idx])
        return out


def kept_count(lam_candidates: np.ndarray, B: float) -> int:
    """Number of local eigenvectors kept (Section 5): all candidates under
    Strategy 1 (B = 0); under Strategy 2 those with eigenvalue below B, at
    least one (the constant, eigenvalue 0, is always among them)."""
    if B <= 0:
        return int(len(lam_candidates))
    return max(1, int(np.count_nonzero(np.asarray(lam_candidates) < B)))


def ragged_pattern(ratio, counts_children) -> np.ndarray:
    """sibling_pattern for children carrying different numbers of coordinates
    (Strategy 2): the dofs of child a and child b couple when a == b or the
    two share a face."""
    rx, ry, rz = ratio
    nch = rx * ry * rz
    cz, cy, cx = np.unravel_index(np.arange(nch), (rz, ry, rx))
    owner = np.repeat(np.arange(nch), counts_children)
    dist = np.abs(cx[owner][:, None] - cx[owner][None, :]) + np.abs(cy[owner][:, None] - cy[owner][None, :]) \
        + np.abs(cz[owner][:, None] - cz[owner][None, :])
    return dist <= 1


def ic0_dense(blk: np.ndarray, pat: np.ndarray) -> np.ndarray:
    """Incomplete Cholesky with no fill of one dense symmetric block: the
    right-looking Cholesky factorisation in which every update that would land
    outside the pattern ``pat`` (boolean, symmetric, true on the diagonal) is
    dropped.  Returns the lower factor L (zero off the pattern); raises
    FloatingPointError on a pivot that is not positive."""
    n = blk.shape[0]
    W = np.tril(np.array(blk, dtype=np.float64)) * np.tril(pat)
    for k in range(n):
        if not W[k, k] > 0:
            raise FloatingPointError("IC(0) pivot is not positive")
        W[k, k] = np.sqrt(W[k, k])
        for i in range(k + 1, n):
            if pat[i, k]:
                W[i, k] /= W[k, k]
        for j in range(k + 1, n):
            if not pat[j, k]:
                continue
            for i in range(j, n):
                if pat[i, k] and pat[i, j]:
                    W[i, j] -= W[i, k] * W[j, k]
    return W


def sibling_pattern(ratio, L: int) -> np.ndarray:
    """Structural pattern of one parent's diagonal block of a coarse operator
    A_l (l >= 2): the parent's children, lexicographic inside the parent (x
    fastest) with L coordinates each, couple only to themselves and to their
    face neighbours (A_l is a block 7-point stencil, Section 3), so the block
    (child a, child b) is in the pattern when a == b or a, b share a face."""
    rx, ry, rz = ratio
    nch = rx * ry * rz
    cz, cy, cx = np.unravel_index(np.arange(nch), (rz, ry, rx))
    dist = np.abs(cx[:, None] - cx[None, :]) + np.abs(cy[:, None] - cy[None, :]) + np.abs(cz[:, None] - cz[None, :])
    return np.kron(dist <= 1, np.ones((L, L), dtype=bool))


class BlockIC0Dense:
    """Coarse-level IC(0) smoother (Section 5 names incomplete Cholesky for
    M_c): block Jacobi over the parents, each parent's diagonal block
    A[idx, idx] factorised by ``ic0_dense`` on ``pattern`` (one boolean matrix
    shared by all parents; by default each block's nonzero entries).  A parent
    whose incomplete factorisation meets a pivot that is not positive is
    factorised exactly instead (dense Cholesky; A_l is not an M-matrix, so IC(0)
    can break down) and its index is listed in ``fallback``."""

    def __init__(self, A: sp.spmatrix, dofs: np.ndarray, pattern: np.ndarray | None = None):
        A = sp.csr_matrix(A)
        self.dofs = dofs
        self.factors = []
        self.fallback = []
        for P, idx in enumerate(dofs):
            blk = A[idx][:, idx].toarray()
            blk = 0.5 * (blk + blk.T)
            if pattern is None:
                pat = blk != 0.0
            else:
                pat = pattern[P] if isinstance(pattern, list) else pattern
            try:
                W = ic0_dense(blk, pat)
            except FloatingPointError:
                W = np.linalg.cholesky(blk)
                self.fallback.append(P)
            self.factors.append(W)

    def solve(self, r: np.ndarray) -> np.ndarray:
        out = np.empty_like(r)
        for idx, Lm in zip(self.dofs, self.factors):
            y = sla.solve_triangular(Lm, r[idx], lower=True)
            out[idx] = sla.solve_triangular(Lm.T, y, lower=False)
        return out


@dataclass
class Hierarchy:
    opts: Options
    shape: tuple
    h: tuple
    T: np.ndarray                        # (3, nz, ny, nx) face coefficients
    S: np.ndarray                        # (nz, ny, nx) Tr K~
    A: list                              # A[l-1] = A_l (sparse), l = 1 .. n_levels
    R: list                              # R[l-1] = R_l (n_{l+1} x n_l)
    M: list                              # M[l-1] = smoother of level l, l < n_levels
    lam: list                            # eigenvalues per level: lam[l-1] (m_l, L_l)
    basis: list                          # Phi (m_1, L_1, nb) then Psi (m_l, L_l, nP)
    grids: list                          # element grid (gz, gy, gx) of E_l
    parent_dofs: list                    # parent_dofs[l-1] (m_l, nP) for l >= 2; None for l = 1
    coarsest_pinv: np.ndarray            # dense A_L^dagger
    null_vectors: list                   # null vector of A_l in level-l coordinates
    counts: list = field(default_factory=list)  # counts[l-1][e]: vectors kept on element e of E_l

    @property
    def dims(self):
        return [a.shape[0] for a in self.A]


def setup(kappa, h, opts: Options) -> Hierarchy:
    """Build every level of the hierarchy from the permeability (Section 3)."""
    opts.check()
    kappa = np.asarray(kappa, dtype=np.float64)
    shape = kappa.shape[-3:]
    T = face_transmissibilities(kappa, h)
    S = trace_weight(kappa, h)
    W = None if opts.cell_diag is None else np.asarray(opts.cell_diag, dtype=np.float64).reshape(shape)
    A1 = assemble(T)
    if W is not None:
        A1 = (A1 + sp.diags(W.ravel())).tocsr()
    nL = opts.n_levels

    # level 1 -> 2: Eq. (spepb) on the elements of E_1; the candidates' unused slots
    # (Strategy 2) are zero rows of the padded basis array and no rows of R_1
    lam1, Phi, cells = level1_eigenpairs(T, S, opts.block, opts.n_eig[0], W)
    m1, L1, nb = Phi.shape
    cnt = np.array([kept_count(lam1[e], opts.threshold(1)) for e in range(m1)])
    keep = np.arange(L1)[None, :] < cnt[:, None]
    Phi = np.where(keep[:, :, None], Phi, 0.0)
    off = np.concatenate([[0], np.cumsum(cnt)])
    row_of = off[:-1, None] + np.arange(L1)[None, :]
    rows = np.repeat(row_of[keep][:, None], nb, axis=1).ravel()
    cols = cells[np.nonzero(keep)[0]].ravel()
    R1 = sp.csr_matrix((Phi[keep].ravel(), (rows, cols)), shape=(int(off[-1]), A1.shape[0]))
    A = [A1, (R1 @ A1 @ R1.T).tocsr()]
    R = [R1]
    lam = [lam1]
    basis = [Phi]
    counts = [cnt]
    grids = [(shape[0] // opts.block[2], shape[1] // opts.block[1], shape[2] // opts.block[0])]
    parent_dofs = [None]
    B = R1.T.tocsr()                          # composed basis of W_2 in fine coordinates
    fine_box = list(opts.block)
    s = S.ravel()
    z = [np.ones(A1.shape[0]), R1 @ s]        # null vector of A_l: R ... R_1 S 1 (Section 3 remark)

    # levels l >= 2: Eq. (spectral cc) on the elements of E_l, posed in W_l
    for l in range(2, nL):
        r = opts.ratio[l - 2]
        g = grids[-1]                          # grid of E_{l-1}
        if g[2] % r[0] or g[1] % r[1] or g[0] % r[2]:
            raise ValueError("ratio does not divide the element grid")
        children = element_cells(g, r)         # (mP, r^3) indices into E_{l-1}
        Lprev = basis[-1].shape[1]
        cprev = counts[-1]                     # coordinates carried by each element of E_{l-1}
        oprev = np.concatenate([[0], np.cumsum(cprev)])
        pd = [np.concatenate([oprev[c] + np.arange(cprev[c]) for c in ch]) for ch in children]
        if np.all(cprev == Lprev):
            pd = np.array(pd)
        fine_box = [fine_box[d] * r[d] for d in range(3)]
        An = assemble(T * interior_face_mask(shape, fine_box))
        if W is not None:
            An = (An + sp.diags(W.ravel())).tocsr()
        An_coarse = (B.T @ An @ B).tocsr()
        Ll = opts.n_eig[l - 1]
        lam_c, vecs = coarse_eigenpairs_kept(An_coarse, list(pd), Ll, opts.threshold(l))
        mP, nch = children.shape
        cnt = np.array([v.shape[0] for v in vecs])
        off = np.concatenate([[0], np.cumsum(cnt)])
        rows = np.concatenate([np.repeat(off[P] + np.arange(cnt[P]), len(pd[P])) for P in range(mP)])
        cols = np.concatenate([np.tile(pd[P], cnt[P]) for P in range(mP)])
        vals = np.concatenate([vecs[P].ravel() for P in range(mP)])
        Rl = sp.csr_matrix((vals, (rows, cols)), shape=(int(off[-1]), A[-1].shape[0]))
        # padded arrays (the layout of the library's exports): slot ci * Lprev + k of a
        # parent holds coordinate k of its child ci; unused slots and rows are zero
        Psi = np.zeros((mP, Ll, nch * Lprev))
        lamP = np.full((mP, Ll), np.inf)
        for P in range(mP):
            slots = np.concatenate([ci * Lprev + np.arange(cprev[c]) for ci, c in enumerate(children[P])])
            Psi[P, :cnt[P]][:, slots] = vecs[P]
            lamP[P, :len(lam_c[P])] = lam_c[P]
        A.append((Rl @ A[-1] @ Rl.T).tocsr())
        R.append(Rl)
        lam.append(lamP)
        basis.append(Psi)
        counts.append(cnt)
        grids.append((g[0] // r[2], g[1] // r[1], g[2] // r[0]))
        parent_dofs.append(pd)
        B = (B @ Rl.T).tocsr()
        z.append(Rl @ z[-1])

    # Block Jacobi over E_l needs at least two elements on every smoothed level:
    # a single block would be the whole singular operator.
    for l, g in enumerate(grids, start=1):
        if g[0] * g[1] * g[2] < 2:
            raise ValueError(f"level {l} has a single element; its smoother block would be singular")

    # smoothers: block Jacobi over E_l on level l (Section 5)
    M = [BlockIC0(A1, cells, opts.block)]
    for l in range(2, nL):
        pd = parent_dofs[l - 1]
        if opts.coarse_smoother == "chol":
            M.append(BlockCholesky(A[l - 1], pd))
        elif isinstance(pd, np.ndarray):
            M.append(BlockIC0Dense(A[l - 1], pd, sibling_pattern(opts.ratio[l - 2], basis[l - 2].shape[1])))
        else:
            ch = element_cells(grids[l - 2], opts.ratio[l - 2])
            pats = [ragged_pattern(opts.ratio[l - 2], counts[l - 2][c]) for c in ch]
            M.append(BlockIC0Dense(A[l - 1], pd, pats))

    # coarsest: Moore-Penrose pseudo-inverse (Algorithm 1, A_cc^dagger)
    Ac = A[-1].toarray()
    Ac = 0.5 * (Ac + Ac.T)
    pinv = np.linalg.pinv(Ac, rcond=1e-13, hermitian=True)
    return Hierarchy(opts, tuple(shape), tuple(h), T, S, A, R, M, lam, basis, grids,
                     parent_dofs, pinv, z, counts)
