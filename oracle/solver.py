"""V-cycle preconditioner and preconditioned conjugate gradients, FP64.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .hierarchy import Hierarchy


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


@dataclass
class PCGResult:
    x: np.ndarray
    iterations: int
    converged: bool
    residuals: list = field(default_factory=list)   # ||r_k||_2 for k = 0 .. iterations
    rhs_mean: float = 0.0


def pcg(A, b: np.ndarray, precond=None, rtol: float = 1e-8, max_iter: int = 1000,
        x0: np.ndarray | None = None) -> PCGResult:
    """Preconditioned conjugate gradients (Hestenes-Stiefel recurrences) for the
    singular consistent system A x = b of Eq. (p).

    The mean of b is removed first (compatibility condition, Section 2.1) and
    the returned x has zero mean (uniqueness condition, Section 2.1).  Stops
    when ||b - A x_k||_2 <= rtol ||b||_2 on the recurrence residual."""
    b = np.asarray(b, dtype=np.float64)
    mean = float(b.mean())
    b = b - mean
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    bnorm = float(np.linalg.norm(b))
    res = [float(np.linalg.norm(r))]
    if bnorm == 0.0 or res[0] <= rtol * bnorm:
        return PCGResult(x - x.mean(), 0, True, res, mean)
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
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    return PCGResult(x - x.mean(), k, converged, res, mean)


def solve(H: Hierarchy, b: np.ndarray, rtol: float = 1e-8, max_iter: int = 1000) -> PCGResult:
    """PCG on the fine system preconditioned by one V-cycle per iteration."""
    return pcg(H.A[0], np.asarray(b, dtype=np.float64).ravel(), lambda r: vcycle(H, r), rtol, max_iter)
