"""Plain, slow FP64 CPU oracle for the spectral multigrid PCG of
"An efficient multiscale multigrid preconditioner for Darcy flow in
high-contrast media" (arXiv 2403.19342).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The product path (the CUDA library and its Python
binding) never calls it, and the oracle shares no code with that path.

Every step restates the paper directly, with no blocking, fusion or
reordering beyond what the definition states:

* ``tpfa``       -- normalised permeability, harmonic-average face
                    coefficients and the cell-centred pressure matrix
                    A = B M_t^{-1} B^T in its two-point-flux form (Section 2.2,
                    Eq. (discrete varia), Fig. (kappa edge)); the velocity
                    recovered from the pressure (Eq. (velocity)) and its
                    discrete divergence.
* ``spectral``   -- the level-1 local generalised eigenproblem (Eq. (spepb))
                    and the level-l>=2 local problem posed in the coarse space
                    (Eq. (spectral cc)); restriction matrices R_l.
* ``hierarchy``  -- Galerkin operators A_{l+1} = R_l A_l R_l^T (Section 3),
                    block-Jacobi smoothers (Section 5: incomplete Cholesky on
                    the fine level, exact block Cholesky on coarse levels) and
                    the coarsest Moore-Penrose pseudo-inverse.
* ``solver``     -- the V-cycle (Algorithm 1, generalised recursively to any
                    number of levels) and preconditioned conjugate gradients.
* ``impes``      -- two-phase flow by the improved IMPES scheme (Section 6):
                    fluid model, well index, the pressure terms of Eq. (IMP)
                    and the upstream-weighted saturation sub-steps of
                    Eq. (ES).
* ``learned``    -- the learned warm start of the level-1 eigensolves (not a
                    step of the paper): network forward, sign-invariant loss,
                    back-propagation and the Adam step.

Pins (tests marked ``not gpu``) tie each function to closed forms, to values
the paper prints, to library routines on special cases and to brute force.
"""
from .tpfa import (as_components, normalized_permeability, trace_weight,
                   face_transmissibilities, assemble, apply_A, interior_face_mask, velocity, divergence)
from .spectral import element_cells, level1_eigenpairs, coarse_eigenpairs, coarse_eigenpairs_kept
from .hierarchy import (Options, Hierarchy, setup, BlockIC0, BlockIC0Dense, ic0_dense, sibling_pattern,
                        kept_count, ragged_pattern)
from .solver import vcycle, vcycle_mixed, vcycle_two_grid, coarse_pinv, pcg, solve, PCGResult

__all__ = [
    "as_components", "normalized_permeability", "trace_weight",
    "face_transmissibilities", "assemble", "apply_A", "interior_face_mask", "velocity", "divergence",
    "element_cells", "level1_eigenpairs", "coarse_eigenpairs", "coarse_eigenpairs_kept",
    "Options", "Hierarchy", "setup", "BlockIC0", "BlockIC0Dense", "ic0_dense", "sibling_pattern",
    "kept_count", "ragged_pattern",
    "vcycle", "vcycle_mixed", "vcycle_two_grid", "coarse_pinv", "pcg", "solve", "PCGResult",
]
