/*
 * msmg -- spectral multiscale multigrid PCG for the cell-centred Darcy
 * pressure system, for NVIDIA GB300 (sm_103a).
 *
 * Method: arXiv 2403.19342, "An efficient multiscale multigrid preconditioner
 * for Darcy flow in high-contrast media".
 *   - fine operator: the two-point-flux matrix A = B M_t^{-1} B^T obtained from
 *     lowest-order Raviart-Thomas with trapezoidal quadrature (Section 2.2,
 *     Eq. (p), Eq. (discrete varia)); face coefficients are harmonic averages
 *     of the normalised permeability kappa^d / h_d^2 (Fig. (kappa edge));
 *     boundary faces carry nothing (no-flow, Eq. (ell2));
 *   - nested spaces W_L c ... c W_1 = W_h spanned by the smallest eigenvectors
 *     of local spectral problems on non-overlapping elements (Section 3,
 *     Eq. (spepb) on level 1, Eq. (spectral cc) on higher levels);
 *   - Galerkin operators A_{l+1} = R_l A_l R_l^T, block-Jacobi smoothers and a
 *     coarsest pseudo-inverse, applied as a V-cycle (Algorithm 1, recursive);
 *   - preconditioned conjugate gradients on A p = f.
 *
 * Conventions for every call:
 *   - Cell order is i + nx*(j + ny*k) with i fastest ("natural order").
 *   - Pointers are DEVICE pointers unless a call or flag says otherwise.  The
 *     caller owns every buffer, including the workspace given to msmg_setup;
 *     the library allocates no device memory and owns only the opaque context.
 *   - Work is enqueued on the caller's stream; calls that return data to the
 *     host (info structs) synchronise that stream.
 *   - Return value: 0 success, > 0 warning, < 0 error (msmg_status_string).
 *   - Calls on one context are not thread-safe; distinct contexts are
 *     independent.
 */
#ifndef MSMG_H
#define MSMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* msmg_stream;        /* same handle as cudaStream_t */
typedef struct msmg_ctx msmg_ctx;                /* opaque, owned by the library */
typedef struct msmg_net msmg_net;                /* opaque: learned warm-start network */

#define MSMG_MAX_LEVELS 8

/* status codes */
#define MSMG_OK                      0
#define MSMG_NOT_CONVERGED           1   /* warning: max_iter reached            */
#define MSMG_COARSE_IC_FALLBACK      2   /* warning: a coarse IC(0) factor broke  */
                                         /* down; that parent uses its exact block */
#define MSMG_ERR_INVALID_ARG        -1
#define MSMG_ERR_NOT_DIVISIBLE      -2   /* element sizes do not tile the grid   */
#define MSMG_ERR_BAD_KAPPA          -3   /* non-positive or non-finite kappa     */
#define MSMG_ERR_SINGLE_BLOCK       -4   /* a smoothed level has one element     */
#define MSMG_ERR_BREAKDOWN          -5   /* PCG: p^T A p <= 0 or non-finite      */
#define MSMG_ERR_EIG_NOT_CONVERGED  -6   /* local eigensolve missed eig_tol      */
#define MSMG_ERR_WORKSPACE          -7   /* workspace too small or misaligned    */
#define MSMG_ERR_CUDA               -8
#define MSMG_ERR_NOT_FACTORIZABLE   -9   /* a smoother or coarsest factor failed */
#define MSMG_ERR_UNSUPPORTED       -10
#define MSMG_ERR_DEVICE_TIMEOUT    -11   /* a bounded device-side wait gave up   */

/* precision modes */
#define MSMG_FP64   0   /* every step in FP64                                           */
#define MSMG_MIXED  1   /* FP32 fine-level V-cycle and bases, FP64 coarse levels,       */
                        /* coarsest solve and outer PCG; the level-1 eigensolve runs in */
                        /* FP32 to a residual near FP32's reach, then FP64 to eig_tol   */

/* coarse-level smoothers (block Jacobi over the parents of each level l >= 2) */
#define MSMG_BLOCK_CHOL 0   /* exact inverse of each parent's diagonal block of A_l       */
#define MSMG_BLOCK_IC0  1   /* incomplete Cholesky of it (Section 5): no fill outside the  */
                            /* block pattern of the children's face adjacency             */

/* kappa element types */
#define MSMG_F64 0
#define MSMG_F32 1

/* msmg_solve flags */
#define MSMG_FLAG_X0        1   /* x holds an initial guess on entry (warm start)     */
#define MSMG_FLAG_HOST_IO   2   /* rhs and x are HOST pointers (pinned for speed);    */
                                /* the copies run on the stream inside the call       */
#define MSMG_FLAG_NO_GRAPH  4   /* launch the PCG iteration kernel by kernel           */

/* Largest batch width: right-hand sides one context solves in lockstep. */
#define MSMG_MAX_BATCH_RHS 64

typedef struct {
    int nx, ny, nz;        /* fine cells per direction                     */
    double hx, hy, hz;     /* cell sizes (the paper's unit cube: 1/n)      */
} msmg_grid;

typedef struct {
    int n_levels;                      /* number of spaces, >= 2: W_{n_levels} c ... c W_1 = W_h     */
    int block[3];                      /* level-1 element (coarse element) size in cells, x y z     */
    int ratio[MSMG_MAX_LEVELS][3];     /* ratio[i]: elements of level i+1 per element of level i+2,  */
                                       /* per direction, i = 0 .. n_levels-3 (sd in Section 5)       */
    int n_eig[MSMG_MAX_LEVELS];        /* n_eig[i]: eigenvectors per element of level i+1, i.e. the */
                                       /* dimension of each local space of W_{i+2} (L_c, L_cc)      */
    int nu[MSMG_MAX_LEVELS];           /* nu[i]: smoothing sweeps on W_{i+1} (nu, nu_c)              */
    int precision;                     /* MSMG_FP64 or MSMG_MIXED                                    */
    double eig_tol;                    /* local eigen-residual tolerance (see msmg_setup)            */
    int eig_max_iter;                  /* cap on subspace iterations per element (0: default 1000)   */
    int autotune;                      /* 1: msmg_setup times the V-cycle variants (msmg_autotune)   */
                                       /* for batch width 1 and the context's widest batch           */
    const msmg_net* warm_start;        /* NULL: cold start; else a network whose n_in equals the     */
                                       /* level-1 element's cells and n_vec equals n_eig[0] - 1:     */
                                       /* its guesses seed the level-1 subspace iteration (elements  */
                                       /* of more than 96 cells), which still runs to eig_tol        */
    int coarse_smoother;               /* MSMG_BLOCK_CHOL (default) or MSMG_BLOCK_IC0: the factor of */
                                       /* each parent's diagonal block on levels >= 2 (Section 5);  */
                                       /* with MSMG_BLOCK_IC0 a parent whose incomplete factor meets */
                                       /* a pivot <= 0 uses its exact block and msmg_setup returns   */
                                       /* the warning MSMG_COARSE_IC_FALLBACK                        */
    int two_grid;                      /* 0: the V-cycle, P_ITG of Eq. (B_ITG) (default); 1: the     */
                                       /* exact two-grid preconditioner P_TG of Eq. (B_TG): the      */
                                       /* coarse correction solves A_2 e_c = r_c by an inner PCG on  */
                                       /* level 2 preconditioned by the coarse cycle from level 2,    */
                                       /* one cooperative launch per application (n_levels >= 3)    */
    double inner_rtol;                 /* P_TG: inner relative residual (0: 1e-10)                   */
    int inner_max_iter;                /* P_TG: inner iteration cap per application (0: 200)         */
    double eig_threshold[MSMG_MAX_LEVELS]; /* Strategy 2 (Section 5): eig_threshold[i] > 0 keeps, on   */
                                       /* every element of level i+1, the candidate eigenvectors     */
                                       /* (n_eig[i] of them) with eigenvalue below it, at least one  */
                                       /* (B_c for i = 0, B_cc beyond); 0 keeps all n_eig[i]          */
                                       /* (Strategy 1).  The arrays keep n_eig[i] slots per element: */
                                       /* an unused slot holds a zero basis vector and, one level     */
                                       /* up, a decoupled unknown that stays zero                     */
    const double* cell_diag;           /* NULL, or device, nx*ny*nz FP64 values >= 0, natural order: */
                                       /* a term W added to the diagonal of A (the well terms of     */
                                       /* Section 6, W = WI kappa lambda at the cells a producer      */
                                       /* crosses) and to the left-hand forms of the local problems, */
                                       /* as Section 6 modifies them.  With some W > 0 the system is  */
                                       /* nonsingular: msmg_solve then removes no mean, and the       */
                                       /* coarsest solve is a plain inverse.  Read by msmg_setup only */
} msmg_options;

typedef struct {
    int n_levels;
    int64_t dims[MSMG_MAX_LEVELS];     /* dim W_l, l = 1 .. n_levels                     */
    int64_t dims_kept[MSMG_MAX_LEVELS];/* dim W_l counting the kept vectors only (Strategy */
                                       /* 2); equal to dims under Strategy 1             */
    int64_t elements[MSMG_MAX_LEVELS]; /* number of elements of E_l, l = 1 .. n_levels-1 */
    double setup_ms;                   /* device time of msmg_setup                      */
    double eig_ms;                     /* of which level-1 eigensolves                   */
    int eig_iterations_max;            /* subspace iterations of the slowest element     */
    int64_t eig_iterations_total;      /* subspace iterations summed over the elements   */
    int warm_started;                  /* 1 when the learned warm start seeded level 1   */
    double face_contrast;              /* max / min interior face coefficient (Fig. (kappa */
                                       /* edge)): the permeability contrast the hierarchy */
                                       /* sees; high values call for more eigenvectors    */
    int tuning[4];                     /* V-cycle variants in use, for batch width 1 and  */
                                       /* wider: [0], [1] fine prolongation inside the    */
                                       /* post-smoothing kernel (1) or apart (0); [2], [3] */
                                       /* coarse cycle: a launch per step (0), the small  */
                                       /* levels as one cluster launch (1), every coarse  */
                                       /* level as one cooperative grid launch (2), the   */
                                       /* small levels as one cooperative grid launch (3) */
    double eig_residual_max;           /* largest final eigen-residual (level 1)         */
    int64_t workspace_bytes;
} msmg_setup_info;

typedef struct {
    int iterations;                    /* PCG iterations performed                       */
    int converged;
    double rel_residual;               /* ||b - A x||_2 / ||b||_2, recurrence residual    */
    double true_rel_residual;          /* recomputed from x at exit                      */
    double rhs_mean;                   /* mean removed from the right-hand side          */
    double solve_ms;                   /* device time of the solve                       */
    int64_t inner_iterations;          /* P_TG: inner iterations summed over the solve    */
    int64_t kernel_launches;           /* library kernels launched by the solve          */
} msmg_solve_info;

/*
 * Workspace bytes needed by msmg_setup for this grid and hierarchy with room for
 * n_rhs right-hand sides solved in lockstep (the batch width; every solve vector
 * is held n_rhs times, so the size grows linearly with it).  msmg_setup takes the
 * largest batch width, up to MSMG_MAX_BATCH_RHS, that its workspace holds.  Returns
 * MSMG_ERR_NOT_DIVISIBLE / MSMG_ERR_INVALID_ARG / MSMG_ERR_SINGLE_BLOCK for a
 * hierarchy that cannot be built (block must divide the grid, each ratio
 * must divide the element grid below it, every level below the coarsest must
 * have at least two elements, 1 <= n_eig <= dofs per local problem).
 */
int msmg_workspace_size(const msmg_grid* grid, const msmg_options* opts, int n_rhs, size_t* bytes);

/*
 * Set-up phase (Section 3 and Section 5): face coefficients (Section 2.2),
 * level-1 local generalised eigenproblems A_K Phi = lambda S_K Phi with
 * S_K = diag(Tr K~) (Eq. (spepb)), S-orthonormal bases, Galerkin operators,
 * level-l problems in the coarse space (Eq. (spectral cc), right matrix = I),
 * smoother factors and the coarsest pseudo-inverse.
 *
 *   kappa            device, kappa_components x (nx*ny*nz) values, component-major,
 *                    natural cell order; 1 component = isotropic, 3 = (kx, ky, kz)
 *   kappa_dtype      MSMG_F64 or MSMG_F32
 *   workspace        device, >= msmg_workspace_size bytes, 256-byte aligned; must stay
 *                    allocated and untouched until msmg_destroy
 *   out              receives the new context
 * eig_tol bounds || A~ y - theta y ||_2 for each kept eigenvector y (||y||_2 = 1) of the
 * symmetric form A~ = S^{-1/2} A_K S^{-1/2}, whose spectrum lies in [0, 8].  Errors:
 * MSMG_ERR_BAD_KAPPA (kappa <= 0 or not finite), MSMG_ERR_EIG_NOT_CONVERGED (an element
 * missed eig_tol within eig_max_iter; the context is still created and usable),
 * MSMG_ERR_NOT_FACTORIZABLE, plus those of msmg_workspace_size.
 */
int msmg_setup(const msmg_grid* grid, const void* kappa, int kappa_components, int kappa_dtype,
               const msmg_options* opts, void* workspace, size_t workspace_bytes,
               msmg_stream stream, msmg_ctx** out);

/*
 * PCG solve of A x = rhs (Eq. (p)) preconditioned by one V-cycle per iteration.
 *   rhs, x     n_rhs x (nx*ny*nz) FP64 values, natural order, one system after another;
 *              device pointers unless MSMG_FLAG_HOST_IO
 *   n_rhs      any number >= 1: the systems are solved in batches of the context's batch
 *              width (msmg_max_batch_rhs), each batch in lockstep (one set of launches,
 *              separate scalars, convergence test and iteration count per system)
 *   rtol       stop when ||b - A x_k||_2 <= rtol ||b||_2 (b = rhs with its mean removed,
 *              the compatibility condition of Section 2.1)
 *   max_iter   iteration cap (MSMG_NOT_CONVERGED when reached)
 *   info       host array, one entry per system (may be NULL); solve_ms is the device
 *              time of the system's batch, kernel_launches the batch's launches
 * x is returned with zero mean (Section 2.1).  In MSMG_MIXED the V-cycle runs in FP32
 * and the outer recurrence in FP64 with the flexible (Polak-Ribiere) beta.  Returns the
 * worst status over the systems: MSMG_ERR_BREAKDOWN, MSMG_NOT_CONVERGED, or MSMG_OK (or
 * MSMG_ERR_DEVICE_TIMEOUT when a kernel's bounded wait for its staged data gave up).
 * Blocks the calling thread until the solution is in x.
 */
int msmg_solve(msmg_ctx* ctx, const double* rhs, double* x, int n_rhs, double rtol, int max_iter,
               int flags, msmg_stream stream, msmg_solve_info* info);

/*
 * Solves on several contexts at once (independent problems: different grids, fields or
 * hierarchies).  Context k solves n_rhs[k] systems rhs[k] -> x[k] exactly as msmg_solve
 * would; the contexts run on streams of their own, forked from and joined back into
 * stream, and the host advances whichever context's work has completed, so the launches
 * of small problems overlap.  A context may appear once.  info (may be NULL) has
 * sum(n_rhs) entries, context after context.  No counterpart in the paper: its
 * experiments solve one system at a time.
 */
int msmg_solve_batched(msmg_ctx* const* ctxs, int n_ctx, const double* const* rhs, double* const* x,
                       const int* n_rhs, double rtol, int max_iter, int flags, msmg_stream stream,
                       msmg_solve_info* info);

/* The context's batch width: right-hand sides one msmg_solve launch sequence carries. */
int msmg_max_batch_rhs(const msmg_ctx* ctx);

/*
 * Autotuner: times the V-cycle variants at batch width n_rhs (1 .. msmg_max_batch_rhs) with
 * CUDA events over reps repetitions on the context's buffers and keeps the fastest for
 * that width class (width 1, or wider).  The variants -- fine prolongation fused into the
 * post-smoothing kernel or a kernel of its own; the coarse cycle as a launch per step, its
 * small levels and the coarsest solve as one thread-block-cluster launch (when the
 * hierarchy has such a tail: at most 256 parents on its first level, at most 1536
 * coarsest unknowns), every coarse level as one cooperative launch over the whole GPU
 * (at most 4096 coarsest unknowns), or the same small levels as one cooperative launch
 * over the whole GPU -- give the same bits: only the time moves.  Overwrites the solve buffers; call between
 * solves.  msmg_setup runs it when options.autotune is set; the choice is reported in
 * msmg_setup_info.tuning.
 */
int msmg_autotune(msmg_ctx* ctx, int n_rhs, int reps, msmg_stream stream);

/* Apply a tuning found earlier (for instance a saved msmg_setup_info.tuning): four
 * values in the order and ranges of msmg_setup_info.tuning.  MSMG_ERR_UNSUPPORTED if a
 * fused coarse form is asked for that the hierarchy or the GPU does not allow. */
int msmg_set_tuning(msmg_ctx* ctx, const int* tuning);

/* q = A p, FP64, natural order (Eq. (discrete varia)). */
int msmg_apply_A(msmg_ctx* ctx, const double* p, double* q, msmg_stream stream);

/* z = P^{-1} r: one V-cycle from zero (Algorithm 1 generalised), natural order.  Synchronises
 * the stream; MSMG_ERR_DEVICE_TIMEOUT if a kernel's bounded wait for its staged data gave up
 * (z is then not valid). */
int msmg_apply_precond(msmg_ctx* ctx, const double* r, double* z, msmg_stream stream);

/* Deterministic FP64 dot product of two device vectors of length n with the PCG's
 * grid-reduction kernel (per-CTA partial sums added in CTA order by the last CTA).
 *   scratch      device, >= msmg_dot_scratch_bytes(n) bytes, 16-byte aligned, owned by the
 *                caller; its contents are overwritten (the call clears what it needs)
 *   result_host  host; the call synchronises the stream */
size_t msmg_dot_scratch_bytes(int64_t n);
int msmg_dot(const double* a, const double* b, int64_t n, void* scratch, double* result_host, msmg_stream stream);

/*
 * msmg_dot without any device allocation, for callers that cannot allocate device
 * memory: code that must stay within a fixed device-memory budget after start-up,
 * host callbacks or plugins that own no allocator, or latency-critical loops where
 * cudaMalloc's implicit device synchronisation is not acceptable.  The paper has no
 * counterpart: this is a library convenience around the PCG reduction kernel.
 *   a, b         device, n doubles each; n <= MSMG_DOT_NOALLOC_MAX_N, larger n returns
 *                MSMG_ERR_INVALID_ARG (the fixed scratch holds one partial sum per 1024
 *                elements)
 *   result_host  host; the call synchronises the stream
 * Scratch: a fixed array of (MSMG_DOT_NOALLOC_MAX_N / 1024 + 32) doubles (about 128 KiB)
 * in this library's device memory, which every GPU that loads the library holds until
 * the process exits.  Every call looks up the array's address on the current device
 * (a and b must be on that device).  The call copies the result to the host and
 * synchronises the stream, so it must not be used while the stream is being captured.
 * All calls share the array: calls that overlap on the GPU (concurrent streams or
 * threads) race and give wrong results.
 */
#define MSMG_DOT_NOALLOC_MAX_N 16777216
int msmg_dot_noalloc(const double* a, const double* b, int64_t n, double* result_host, msmg_stream stream);

/*
 * Diagnostics: the FP32 <-> FP64 conversions the mixed-form V-cycle kernels perform
 * on the integer pipes (GB300 runs the hardware conversions on its FP64 pipe, which
 * the FP64 PCG arithmetic already keeps busy), applied element by element so that a
 * caller can compare them bit for bit with the hardware conversions (IEEE 754 round to
 * nearest, ties to even; the widening is exact; NaN stays NaN).  Not part of the
 * method: the paper fixes the precisions, not how a conversion is carried out.
 *   in64   device, n doubles; out32[i] = in64[i] rounded to binary32
 *   in32   device, n floats;  out64[i] = in32[i] widened to binary64
 * n <= 0 does nothing.  Asynchronous on ``stream``; MSMG_ERR_CUDA if the launch fails.
 */
int msmg_check_conversions(const double* in64, const float* in32, int64_t n, float* out32, double* out64,
                           msmg_stream stream);

/*
 * Level data in the layouts of the paper's matrices (for parity checks).
 * level l = 1 .. n_levels-1.  Elements of E_l are in lexicographic order (x fastest) of
 * the element grid; the dofs of a level-l local problem are its child elements in
 * lexicographic order inside the parent, each child's n_eig[l-2] values contiguous
 * (l >= 2), or its cells in lexicographic order inside the element (l = 1).
 *   basis   device, m_l x n_eig[l-1] x (dofs per local problem) FP64: level 1 = Phi
 *           (S-orthonormal), level >= 2 = Psi (orthonormal)
 *   lam     device, m_l x n_eig[l-1] eigenvalues (may be NULL)
 */
int msmg_export_basis(msmg_ctx* ctx, int level, double* basis, double* lam, msmg_stream stream);

/*
 * Replace the local eigenbases with the given ones (same layout as export) and rebuild
 * every quantity that depends on them (Galerkin operators, coarse smoothers, the
 * coarsest pseudo-inverse).  Bases for levels 1 .. n_levels-1 in one call:
 * bases[l-1] points to level l's array.
 */
int msmg_import_bases(msmg_ctx* ctx, const double* const* bases, msmg_stream stream);

/*
 * Dense FP64 copy of the Galerkin operator A_l (l = 2 .. n_levels) in the coordinate
 * order of the paper's R_l: (element of E_{l-1} in lexicographic order, eigenvector).
 * out: device, dim(W_l)^2 values, row-major.  Intended for small grids.
 */
int msmg_export_operator(msmg_ctx* ctx, int level, double* out, msmg_stream stream);

/*
 * Velocity recovery (Section 2.2): v = M_t^{-1} B^T p, the two-point flux of Eq. (velocity)
 * on every face, v_f = -kappa_f (p_j - p_i) / h_d = -T_f h_d (p_j - p_i) for the face between
 * cell i and its +d neighbour j (T_f the harmonic-average face coefficient of Fig. (kappa
 * edge)), zero on boundary faces (no flow); and the discrete mass balance of every cell,
 * div_i = sum_d (v_{i+e_d/2} - v_{i-e_d/2}) / h_d against b_i = f_i - mean(f) (the
 * conservation identity that follows Eq. (discrete varia), in three directions).
 *   p        device, n FP64 pressures, natural order (for instance msmg_solve's x)
 *   f        device, n FP64 sources, natural order (msmg_solve's rhs; its mean is removed
 *            here as the solve removes it)
 *   v        device, 3 x n FP64, natural order: v[d][cell] = velocity on the cell's +d face
 *   balance  host, 2 doubles (may be NULL): ||div - b||_2 and ||b||_2; ||div - b|| equals the
 *            solve's residual ||f' - A p|| (f' = f - mean(f)), so their ratio is its relative
 *            residual.  With a cell term W (options.cell_diag, wells) b = f - W p, the net source
 *            (injection and the flow that leaves through the wells), no mean is removed, and
 *            ||div - b|| equals ||f - (A + W) p||.  With balance the call synchronises the stream.
 * Uses the context's reduction scratch: not concurrently with a solve on the same context.
 */
int msmg_velocity(msmg_ctx* ctx, const double* p, const double* f, double* v, double* balance, msmg_stream stream);

/*
 * ------------------------------------------------------------ two-phase flow (Section 6)
 * The improved IMPES scheme around the pressure solve.  Fluid model: S* = (S - s_wc) /
 * (1 - s_wc - s_or) clipped to [0, 1], k_rw = S*^2, k_ro = (1 - S*)^2, total mobility
 * lambda = k_rw / mu_w + k_ro / mu_o, fractional flow f_w = (k_rw / mu_w) / lambda (the paper:
 * mu_w = 0.3, mu_o = 3.0, s_wc = s_or = 0.2).  A time step: msmg_impes_pressure_terms, then
 * msmg_setup with kappa_eff and options.cell_diag = w, msmg_solve(b) (Eq. (IMP)), msmg_velocity,
 * then msmg_impes_transport (Eq. (ES)).
 */
typedef struct {
    double mu_w, mu_o;       /* water and oil viscosities                   */
    double s_wc, s_or;       /* connate water and residual oil saturations  */
} msmg_fluid;

/* The pressure system of Eq. (IMP) at saturation S (natural order, device arrays):
 *   kappa       3 x n permeability (kappa^x, kappa^y, kappa^z)
 *   wi          n: well index of each cell a producer crosses (Section 6's formula), 0 elsewhere
 *   q_inj       n: injection rate per unit volume (the injector's rate spread over its cells)
 *   kappa_eff   out, 3 x n: lambda(S) kappa, the permeability of the pressure solve
 *   w           out, n: W = wi kappa^x lambda(S), the producers' term of A (options.cell_diag)
 *   b           out, n: q_inj + W p_bh, the right-hand side
 * Asynchronous; MSMG_ERR_INVALID_ARG on a bad size or fluid. */
int msmg_impes_pressure_terms(int64_t n, const msmg_fluid* fluid, const double* S, const double* kappa,
                              const double* wi, const double* q_inj, double p_bh, double* kappa_eff, double* w,
                              double* b, msmg_stream stream);

/* M explicit saturation sub-steps of Eq. (ES) on the context's grid, upstream weighting of
 * f_w at every face (the saturation of the cell the flow leaves), sources q_w = q_inj + f_w(S)
 * w (p_bh - p): each sub-step takes dt = ds_max / max |dS/dt|, so no cell changes by more than
 * ds_max.  v: 3 x n face velocities of msmg_velocity for the pressure p; w, q_inj, p_bh as in
 * msmg_impes_pressure_terms; phi: n porosities (> 0); S: n saturations, updated in place.
 * dt_host (may be NULL) receives the sum of the sub-steps' dt (the synchronising case).
 * Uses the context's solve buffers as scratch (not during a solve on the same context). */
int msmg_impes_transport(msmg_ctx* ctx, const msmg_fluid* fluid, const double* v, const double* p, const double* w,
                         double p_bh, const double* q_inj, const double* phi, double* S, int M, double ds_max,
                         double* dt_host, msmg_stream stream);

/* Face coefficients T[d][cell] (d = x, y, z; face between cell and its +d neighbour,
 * zero on the boundary), FP64, natural order: device, 3 x (nx*ny*nz). */
int msmg_export_faces(msmg_ctx* ctx, double* T, msmg_stream stream);

int msmg_get_setup_info(msmg_ctx* ctx, msmg_setup_info* info);
void msmg_destroy(msmg_ctx* ctx);
const char* msmg_status_string(int status);

/*
 * ------------------------------------------------------------ learned warm start
 * A multilayer perceptron n_in -> hidden[0] -> hidden[1] -> n_vec * n_in (ReLU after
 * the two hidden layers), its output o_k scaled cell by cell by w_c = sqrt(S_c / sum S)
 * (recovered from the input: S_c is proportional to exp(8 x_c)), maps a level-1
 * element's standardised log-permeability patch
 * x[c] = clamp(log S_c - mean log S, -20, 20) / 8 (S = Tr K~ of Eq. (spepb); for an
 * isotropic kappa, log S is log kappa plus a constant) to guesses for the element's
 * eigenvectors 1 .. n_vec in the symmetric form y = S^{1/2} phi, ||y||_2 = 1 (vector 0,
 * the constant, is known).  Not part of the paper: it only seeds the subspace iteration
 * of msmg_setup (options.warm_start), which still runs to eig_tol, so the
 * preconditioner does not depend on it.
 *
 * Weights: FP32 masters and BF16 copies that every product reads; FP32 activations and
 * accumulation.  Parameter layout (one FP32 array of msmg_net_param_count values):
 * W_l row-major [fan_in][fan_out] at w_off[l], b_l at b_off[l] (msmg_net_param_offsets).
 * Loss per sample and vector (sign-invariant): ||p||^2 + ||t||^2 - 2 |p . t|, averaged
 * over samples and vectors.  Training: Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the
 * masters.  All kernels are deterministic.
 */
typedef struct {
    int n_in;              /* cells per level-1 element                              */
    int hidden[2];         /* hidden layer widths                                    */
    int n_vec;             /* eigenvector guesses per element (n_eig[0] - 1)         */
    int batch_max;         /* rows per pass (activations are sized for it)           */
} msmg_net_desc;

/* Device bytes for a network of this shape (0 for an invalid description). */
size_t msmg_net_workspace_size(const msmg_net_desc* desc);

/* Create a network in the caller's device workspace (256-byte aligned, >=
 * msmg_net_workspace_size); weights uniform in +-sqrt(6 / fan_in) (last layer a quarter
 * of that) from a counter-based hash of seed and index (splitmix64), biases zero. */
int msmg_net_create(const msmg_net_desc* desc, void* workspace, size_t workspace_bytes, uint64_t seed,
                    msmg_stream stream, msmg_net** out);
void msmg_net_destroy(msmg_net* net);
int64_t msmg_net_param_count(const msmg_net* net);
int msmg_net_param_offsets(const msmg_net* net, int64_t* w_off, int64_t* b_off);   /* 3 + 3 values */

/* Copy the FP32 master parameters out (device array of msmg_net_param_count floats) or
 * in (the BF16 copies are refreshed). */
int msmg_net_get_params(const msmg_net* net, float* params, msmg_stream stream);
int msmg_net_set_params(msmg_net* net, const float* params, msmg_stream stream);

/* y[b] = network(x[b]) for b < batch (device, row-major [batch][n_in] -> [batch][n_vec * n_in]). */
int msmg_net_forward(msmg_net* net, const float* x, float* y, int batch, msmg_stream stream);

/* Device time of the forward pass's three products for one batch (<= batch_max) of x:
 * one forward pass forms their operands, then each product is launched once more between
 * CUDA events on `stream`; ms[l] receives the milliseconds of layer l's product.  Needs
 * the tensor-core form (layer widths multiples of 64), else MSMG_ERR_UNSUPPORTED.
 * Synchronises the stream. */
int msmg_net_time_products(msmg_net* net, const float* x, int batch, double* ms, msmg_stream stream);

/* Loss of a batch (<= batch_max) and its gradient with respect to every parameter
 * (device array of msmg_net_param_count floats, may be NULL); loss_host may be NULL. */
int msmg_net_gradients(msmg_net* net, const float* x, const float* target, int batch, float* grad,
                       float* loss_host, msmg_stream stream);

/* One Adam step on a batch (<= batch_max) with learning rate lr; the batch loss before
 * the step goes to *loss_host (may be NULL). */
int msmg_net_train_step(msmg_net* net, const float* x, const float* target, int batch, float lr,
                        float* loss_host, msmg_stream stream);

/* Training pairs of a set-up context (level-1 elements of more than one eigenvector):
 * x [m][nb] network inputs and y [m][n_eig[0] - 1][nb] the computed eigenvectors 1 ..
 * n_eig[0]-1 in the symmetric form; elements in lexicographic order (x fastest), as in
 * msmg_export_basis. */
int msmg_learning_data(msmg_ctx* ctx, float* x, float* y, msmg_stream stream);

/*
 * Average device time (ms) per launch of the fine-level kernels of one PCG iteration,
 * measured with CUDA events around each launch on the given stream over reps repetitions on
 * the context's own buffers (fixed synthetic data), at batch width n_rhs (1 .. the
 * context's).  ms_out[0 .. n_out) receives:
 *   [0] PCG update of x and r fused with the pre-smoothing   [1] residual + restriction
 *   [2] fine prolongation, when it runs as a kernel of its own (about 0 when the context's
 *       tuning for this batch width runs it inside [3])
 *   [3] residual + post-smoothing (with the r.z reduction), plus the prolongation when fused
 *   [4] all coarse levels (levels >= 2)   [5] search-direction update fused with q = A p
 *   [6] [0]..[3] and [4] together (one preconditioner application)
 * Used for roofline figures; no effect on results.
 */
int msmg_time_kernels(msmg_ctx* ctx, int n_rhs, int reps, double* ms_out, int n_out, msmg_stream stream);


#ifdef __cplusplus
}
#endif
#endif /* MSMG_H */
