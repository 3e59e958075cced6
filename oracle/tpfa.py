"""Fine-scale operator of the paper (Section 2.2), FP64.

Test infrastructure only (see the package docstring).

Arrays use numpy shape (nz, ny, nx): flat cell index i + nx*(j + ny*k).
Direction d = 0, 1, 2 means x, y, z.  Face coefficient T[d][c] belongs to the
face between cell c and its +d neighbour; it is zero on domain-boundary faces
(no-flow condition, Eq. (ell2): only internal faces carry a term).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def as_components(kappa) -> np.ndarray:
    """Orthotropic permeability as (3, nz, ny, nx) float64.  Accepts an isotropic
    (nz, ny, nx) field, a (1, nz, ny, nx) field or a (3, nz, ny, nx) field
    (Section 2.1: K = diag(kappa^x, kappa^y, kappa^z))."""
    k = np.asarray(kappa, dtype=np.float64)
    if k.ndim == 3:
        k = k[None]
    if k.shape[0] == 1:
        k = np.repeat(k, 3, axis=0)
    if k.shape[0] != 3:
        raise ValueError("kappa must have 1 or 3 components")
    return k


def normalized_permeability(kappa, h) -> np.ndarray:
    """K~ = diag(kappa^d / (h^d)^2) per cell (Section 2.2, the normalisation
    that makes the face coefficients dimensionless)."""
    k = as_components(kappa)
    return np.stack([k[d] / (h[d] * h[d]) for d in range(3)])


def trace_weight(kappa, h) -> np.ndarray:
    """Tr K~ per cell: the weight of the right-hand side of the local spectral
    problems, Eq. (spepb) and Eq. (spectral cc)."""
    return normalized_permeability(kappa, h).sum(axis=0)


def face_transmissibilities(kappa, h) -> np.ndarray:
    """Face coefficients kappa~_e: harmonic average of the two cells' normalised
    permeability in the face's direction (Section 2.2 and Fig. (kappa edge)):
    kappa~_{i+1/2} = 2 / (1/kappa~_i + 1/kappa~_{i+1}).  Zero on boundary faces."""
    kt = normalized_permeability(kappa, h)
    T = np.zeros_like(kt)
    T[0][:, :, :-1] = 2.0 / (1.0 / kt[0][:, :, :-1] + 1.0 / kt[0][:, :, 1:])
    T[1][:, :-1, :] = 2.0 / (1.0 / kt[1][:, :-1, :] + 1.0 / kt[1][:, 1:, :])
    T[2][:-1, :, :] = 2.0 / (1.0 / kt[2][:-1, :, :] + 1.0 / kt[2][1:, :, :])
    return T


def interior_face_mask(shape, box) -> np.ndarray:
    """Boolean (3, nz, ny, nx): True where the face between c and c+e_d lies
    inside one element of a partition of the grid into boxes of ``box`` =
    (bx, by, bz) cells, i.e. the face set E_h^0(K) of Eq. (spepb)."""
    nz, ny, nx = shape
    bx, by, bz = box
    m = np.zeros((3, nz, ny, nx), dtype=bool)
    m[0] = ((np.arange(nx) + 1) % bx != 0)[None, None, :]
    m[1] = ((np.arange(ny) + 1) % by != 0)[None, :, None]
    m[2] = ((np.arange(nz) + 1) % bz != 0)[:, None, None]
    return m


def apply_A(T: np.ndarray, p: np.ndarray) -> np.ndarray:
    """q = A p without forming A (Eq. (discrete varia) read face by face): the
    flux T_e (p_i - p_j) across every internal face e between cells i and j
    (j the +d neighbour of i) is added to q_i and subtracted from q_j.
    T as returned by face_transmissibilities, p of shape (nz, ny, nx) or flat."""
    _, nz, ny, nx = T.shape
    pp = np.asarray(p, dtype=np.float64).reshape(nz, ny, nx)
    q = np.zeros_like(pp)
    fx = T[0][:, :, :-1] * (pp[:, :, :-1] - pp[:, :, 1:])
    q[:, :, :-1] += fx
    q[:, :, 1:] -= fx
    fy = T[1][:, :-1, :] * (pp[:, :-1, :] - pp[:, 1:, :])
    q[:, :-1, :] += fy
    q[:, 1:, :] -= fy
    fz = T[2][:-1, :, :] * (pp[:-1, :, :] - pp[1:, :, :])
    q[:-1, :, :] += fz
    q[1:, :, :] -= fz
    return q.reshape(np.shape(p))


def assemble(T: np.ndarray) -> sp.csr_matrix:
    """The symmetric positive semidefinite matrix of Eq. (discrete varia):
    q^T A p = sum over faces e of T_e (p_j - p_i)(q_j - q_i).  Each face with
    coefficient T between cells i and j adds T to A_ii and A_jj and -T to
    A_ij and A_ji."""
    _, nz, ny, nx = T.shape
    n = nx * ny * nz
    idx = np.arange(n).reshape(nz, ny, nx)
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    for d, stride in enumerate((1, nx, nx * ny)):
        t = T[d].ravel()
        nz_faces = np.nonzero(t)[0]
        i = idx.ravel()[nz_faces]
        j = i + stride
        tv = t[nz_faces]
        rows += [i, j]
        cols += [j, i]
        vals += [-tv, -tv]
        np.add.at(diag, i, tv)
        np.add.at(diag, j, tv)
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    return A.tocsr()


def velocity(T: np.ndarray, p, h) -> np.ndarray:
    """Velocity recovered from the pressure (Section 2.2: v = M_t^{-1} B^T p,
    written out in Eq. (velocity)): on the face between cell i and its +d
    neighbour j, v = -kappa_e (p_j - p_i) / h_d, where kappa_e / h_d^2 is the
    face coefficient T_e.  Returns (3, nz, ny, nx): component d at cell c is the
    velocity on c's +d face; zero on boundary faces (no flow)."""
    _, nz, ny, nx = T.shape
    pp = np.asarray(p, dtype=np.float64).reshape(nz, ny, nx)
    v = np.zeros_like(T)
    kx = T[0][:, :, :-1] * h[0] * h[0]
    v[0][:, :, :-1] = -kx * (pp[:, :, 1:] - pp[:, :, :-1]) / h[0]
    ky = T[1][:, :-1, :] * h[1] * h[1]
    v[1][:, :-1, :] = -ky * (pp[:, 1:, :] - pp[:, :-1, :]) / h[1]
    kz = T[2][:-1, :, :] * h[2] * h[2]
    v[2][:-1, :, :] = -kz * (pp[1:, :, :] - pp[:-1, :, :]) / h[2]
    return v


def divergence(v: np.ndarray, h) -> np.ndarray:
    """Discrete divergence of a face velocity field (the cell balance stated
    after Eq. (discrete varia), divided by the cell volume): for each cell,
    sum over d of (v on its +d face - v on its -d face) / h_d; the -d face of
    a cell is the +d face of its -d neighbour, and boundary faces carry zero."""
    _, nz, ny, nx = v.shape
    out = np.zeros((nz, ny, nx))
    for d in range(3):
        vp = v[d]
        vm = np.zeros_like(vp)
        if d == 0:
            vm[:, :, 1:] = vp[:, :, :-1]
        elif d == 1:
            vm[:, 1:, :] = vp[:, :-1, :]
        else:
            vm[1:, :, :] = vp[:-1, :, :]
        out += (vp - vm) / h[d]
    return out
