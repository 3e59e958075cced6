"""Local spectral problems of Section 3, FP64 (LAPACK ``eigh``).

Test infrastructure only (see the package docstring).

Level 1 (Eq. (spepb)): on each coarse element K (a box of fine cells) solve
    A_K Phi = lambda S_K Phi,
where A_K is the two-point-flux matrix built from the faces inside K only
(Neumann on the element boundary) and S_K = diag(Tr K~) on K's cells.  The
L smallest eigenpairs are kept, normalised so that Phi^T S_K Phi = I.

Level l >= 2 (Eq. (spectral cc)): on each element P of level l (a box of
level-(l-1) elements) the same bilinear forms are restricted to W_l(P), the
span of the level-l basis functions supported in P.  With the basis of
W_l(P) written in fine-grid coordinates as the columns of B_P, the left
matrix is B_P^T A_P B_P (A_P: fine faces inside P only) and the right matrix
B_P^T S B_P, which is the identity because the basis is S-orthonormal
(Section 3, the remark after Eq. (spectral cc)).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .tpfa import assemble, interior_face_mask


def element_cells(shape, box) -> np.ndarray:
    """Global flat indices of the cells of each element of a partition of the
    (nz, ny, nx) grid into boxes of (bx, by, bz) cells.  Returns (m, bx*by*bz):
    elements in lexicographic order (x fastest), cells in the element in
    lexicographic order (x fastest)."""
    nz, ny, nx = shape
    bx, by, bz = box
    if nx % bx or ny % by or nz % bz:
        raise ValueError("element size does not divide the grid")
    ex, ey, ez = nx // bx, ny // by, nz // bz
    lz, ly, lx = np.meshgrid(np.arange(bz), np.arange(by), np.arange(bx), indexing="ij")
    local = (lx + nx * (ly + ny * lz)).ravel()
    EZ, EY, EX = np.meshgrid(np.arange(ez), np.arange(ey), np.arange(ex), indexing="ij")
    origin = (EX * bx + nx * (EY * by + ny * (EZ * bz))).ravel()
    return origin[:, None] + local[None, :]


def level1_eigenpairs(T: np.ndarray, S: np.ndarray, box, L: int, W: np.ndarray | None = None):
    """Smallest ``L`` eigenpairs of Eq. (spepb) on every level-1 element, with the
    cell term W (wells, Section 6) added to the left-hand form when given.

    Returns (lam (m, L), Phi (m, L, nb), cells (m, nb)); Phi[e, k] is the k-th
    eigenvector on element e's cells (in element order), S-orthonormal."""
    shape = T.shape[1:]
    An = assemble(T * interior_face_mask(shape, box))
    if W is not None:
        An = (An + sp.diags(np.asarray(W, dtype=np.float64).ravel())).tocsr()
    cells = element_cells(shape, box)
    s = S.ravel()
    m, nb = cells.shape
    if not 1 <= L <= nb:
        raise ValueError("number of eigenvectors out of range")
    lam = np.empty((m, L))
    Phi = np.empty((m, L, nb))
    An = An.tocsr()
    for e in range(m):
        idx = cells[e]
        Ae = An[idx][:, idx].toarray()
        w, V = sla.eigh(Ae, np.diag(s[idx]))      # V^T S V = I
        lam[e] = w[:L]
        Phi[e] = V[:, :L].T
    return lam, Phi, cells


def coarse_eigenpairs(An_coarse: sp.spmatrix, parent_dofs: np.ndarray, L: int):
    """Smallest ``L`` eigenpairs of Eq. (spectral cc) on every level-l element.

    ``An_coarse`` is B^T A_N B in the current coarse coordinates, where A_N is
    the fine two-point-flux matrix keeping only faces inside level-l elements;
    its diagonal block on ``parent_dofs[P]`` is the left matrix of the local
    problem on P.  The right matrix is the identity (S-orthonormal basis).
    Returns (lam (mP, L), Psi (mP, L, nP))."""
    mP, nP = parent_dofs.shape
    if not 1 <= L <= nP:
        raise ValueError("number of eigenvectors out of range")
    An_coarse = sp.csr_matrix(An_coarse)
    lam = np.empty((mP, L))
    Psi = np.empty((mP, L, nP))
    for P in range(mP):
        idx = parent_dofs[P]
        N = An_coarse[idx][:, idx].toarray()
        N = 0.5 * (N + N.T)
        w, V = np.linalg.eigh(N)
        lam[P] = w[:L]
        Psi[P] = V[:, :L].T
    return lam, Psi


def coarse_eigenpairs_kept(An_coarse: sp.spmatrix, parent_dofs: list, L: int, B: float):
    """Eq. (spectral cc) on every level-l element whose coordinates
    ``parent_dofs[P]`` may differ in number (Strategy 2 below), with the
    selection of Section 5: the ``L`` smallest eigenpairs are the candidates
    (fewer if the local space is smaller), of which Strategy 1 (B = 0) keeps
    all and Strategy 2 keeps those with eigenvalue below B, at least one.
    Returns (lam [mP] arrays of the candidates' eigenvalues, vecs [mP] arrays
    (kept, len(parent_dofs[P])) of the kept eigenvectors as rows)."""
    from .hierarchy import kept_count
    An_coarse = sp.csr_matrix(An_coarse)
    lam, vecs = [], []
    for idx in parent_dofs:
        N = An_coarse[idx][:, idx].toarray()
        N = 0.5 * (N + N.T)
        w, V = np.linalg.eigh(N)
        nc = min(L, len(idx))
        c = kept_count(w[:nc], B)
        lam.append(w[:nc])
        vecs.append(V[:, :c].T)
    return lam, vecs
