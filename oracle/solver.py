"""V-cycle preconditioner and preconditioned conjugate gradients, FP64.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .hierarchy import Hierarchy


class _Level1FP32:
    """Level 1 of the hierarchy with its data rounded to FP32: the fine
    operator, the basis Phi (as R_1 and R_1^T) and the IC(0) factor.  Products
    with FP32 operands stay in FP32 (NumPy and SciPy keep the operand type)."""

    def __init__(self, H: Hierarchy):
        from .hierarchy import BlockIC0
        self.A = H.A[0].astype(np.float32)
        self.R = H.R[0].astype(np.float32).tocsr()
        self.RT = self.R.T.tocsr()
        M = H.M[0]
        M32 = BlockIC0.__new__(BlockIC0)
        M32.__dict__.update(M.__dict__)
        M32.L = {k: v.astype(np.float32) for k, v in M.L.items()}
        self.M = M32


def _level1_fp32(H: Hierarchy) -> _Level1FP32:
    cache = getattr(H, "_fp32_level1", None)
    if cache is None:
        cache = _Level1FP32(H)
        H._fp32_level1 = cache
    return cache


def vcycle_mixed(H: Hierarchy, f: np.ndarray) -> np.ndarray:
    """The V-cycle of ``vcycle`` with level 1 in single precision, the split of
    the mixed form: the right-hand side rounded to FP32; pre-smoothing,
    residual, restriction, prolongation and post-smoothing on level 1 with FP32
    data and FP32 arithmetic; the restricted residual widened to FP64; every
    coarse level and the coarsest pseudo-inverse in FP64; the coarse correction
    rounded to FP32 for the prolongation; the result widened to FP64.  The
    order of the steps is that of ``vcycle`` (Algorithm 1)."""
    L1 = _level1_fp32(H)
    f32 = np.asarray(f, dtype=np.float64).astype(np.float32)
    nu = H.opts.nu[0]
    u = np.zeros_like(f32)
    for _ in range(nu):
        u = u + L1.M.solve(f32 - L1.A @ u)
    rc = (L1.R @ (f32 - L1.A @ u)).astype(np.float64)
    e = vcycle(H, rc, 2) if H.opts.n_levels > 2 else H.coarsest_pinv @ rc
    u = u + L1.RT @ e.astype(np.float32)
    for _ in range(nu):
        u = u + L1.M.solve(f32 - L1.A @ u)
    return u.astype(np.float64)


def vcycle(H: Hierarchy, f: np.ndarray, level: int = 1) -> np.ndarray:
    """One application of the multigrid preconditioner on level ``level``
    (Algorithm 1, applied recursively: the map r_c -> e_c of Algorithm 1 is
    this same cycle one level down, Eq. (B_c)).  Starting from u = 0:

      pre-smoothing  (nu sweeps)  u <- u + M^{-1} (f - A u)
      restriction                 r' = R (f - A u)
      coarse correction           e  = cycle(level + 1, r')  (A^dagger r' at the coarsest level)
      prolongation                u <- u + R^T e
      post-smoothing (nu sweeps)  u <- u + M^{-T} (f - A u)
    """
    nL = H.opts.n_levels
    if level == nL:
        return H.coarsest_pinv @ f
    A = H.A[level - 1]
    M = H.M[level - 1]
    R = H.R[level - 1]
    nu = H.opts.nu[level - 1]
    u = np.zeros_like(f)
    for _ in range(nu):
        u = u + M.solve(f - A @ u)
    rc = R @ (f - A @ u)
    e = vcycle(H, rc, level + 1)
    u = u + R.T @ e
    for _ in range(nu):
        u = u + M.solve(f - A @ u)      # M^{-T} = M^{-1}: both factors are symmetric
    return u


def coarse_pinv(H: Hierarchy) -> np.ndarray:
    """Dense Moore-Penrose pseudo-inverse of A_2 = R_1 A R_1^T (singular, with
    the null vector of Section 3's remark), cached on the hierarchy."""
    P = getattr(H, "_coarse_pinv", None)
    if P is None:
        Ac = H.A[1].toarray()
        P = np.linalg.pinv(0.5 * (Ac + Ac.T), rcond=1e-13, hermitian=True)
        H._coarse_pinv = P
    return P


def vcycle_two_grid(H: Hierarchy, f: np.ndarray) -> np.ndarray:
    """The exact two-grid preconditioner P_TG of Eq. (B_TG): Algorithm 1's fine
    steps with the coarse correction e_c = A_c^dagger r_c solved exactly (A_c =
    A_2), in place of the recursive cycle B_c^{-1} of Eq. (B_c).  Starting from
    u = 0: pre-smoothing, restriction, exact coarse solve, prolongation,
    post-smoothing."""
    A, M, R = H.A[0], H.M[0], H.R[0]
    nu = H.opts.nu[0]
    u = np.zeros_like(f)
    for _ in range(nu):
        u = u + M.solve(f - A @ u)
    rc = R @ (f - A @ u)
    e = coarse_pinv(H) @ rc
    u = u + R.T @ e
    for _ in range(nu):
        u = u + M.solve(f - A @ u)
    return u


@dataclass
class PCGResult:
    x: np.ndarray
    iterations: int
    converged: bool
    residuals: list = field(default_factory=list)   # ||r_k||_2 for k = 0 .. iterations
    rhs_mean: float = 0.0


def pcg(A, b: np.ndarray, precond=None, rtol: float = 1e-8, max_iter: int = 1000,
        x0: np.ndarray | None = None, flexible: bool = False, singular: bool = True) -> PCGResult:
    """Preconditioned conjugate gradients (Hestenes-Stiefel recurrences) for the
    singular consistent system A x = b of Eq. (p).

    The mean of b is removed first (compatibility condition, Section 2.1) and
    the returned x has zero mean (uniqueness condition, Section 2.1).  Stops
    when ||b - A x_k||_2 <= rtol ||b||_2 on the recurrence residual.  With
    ``flexible`` the direction update takes the Polak-Ribiere coefficient
    beta = z_{k+1}^T (r_{k+1} - r_k) / z_k^T r_k, which tolerates a
    preconditioner that is not exactly the same linear map every time (the
    mixed form's rounded V-cycle).  With ``singular`` False (A has a cell term,
    the wells of Section 6) b is taken as it is and x keeps its mean."""
    b = np.asarray(b, dtype=np.float64)
    mean = float(b.mean()) if singular else 0.0
    b = b - mean
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    bnorm = float(np.linalg.norm(b))
    res = [float(np.linalg.norm(r))]
    if bnorm == 0.0 or res[0] <= rtol * bnorm:
        return PCGResult(x - x.mean() if singular else x, 0, True, res, mean)
    apply_p = precond if precond is not None else (lambda v: v.copy())
    z = apply_p(r)
    p = z.copy()
    rz = float(r @ z)
    converged = False
    k = 0
    for k in range(1, max_iter + 1):
        q = A @ p
        pq = float(p @ q)
        if not pq > 0.0:
            raise FloatingPointError(f"PCG breakdown: p^T A p = {pq} at iteration {k}")
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        res.append(float(np.linalg.norm(r)))
        if res[-1] <= rtol * bnorm:
            converged = True
            break
        z = apply_p(r)
        rz_new = float(r @ z)
        if flexible:
            beta = float(z @ (-alpha * q)) / rz      # z_{k+1}^T (r_{k+1} - r_k) / z_k^T r_k
        else:
            beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    return PCGResult(x - x.mean() if singular else x, k, converged, res, mean)


def solve(H: Hierarchy, b: np.ndarray, rtol: float = 1e-8, max_iter: int = 1000, mixed: bool = False,
          two_grid: bool = False) -> PCGResult:
    """PCG on the fine system preconditioned by one V-cycle per iteration; with
    ``mixed`` the V-cycle's level 1 runs in FP32 (``vcycle_mixed``) and the PCG
    takes the flexible beta; with ``two_grid`` the preconditioner is the exact
    two-grid P_TG (``vcycle_two_grid``)."""
    if two_grid:
        pre = lambda r: vcycle_two_grid(H, r)
    else:
        pre = (lambda r: vcycle_mixed(H, r)) if mixed else (lambda r: vcycle(H, r))
    return pcg(H.A[0], np.asarray(b, dtype=np.float64).ravel(), pre, rtol, max_iter, flexible=mixed,
               singular=H.opts.singular())
