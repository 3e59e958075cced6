"""Python binding of libmsmg (include/msmg.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch
tensors to device pointers and streams, and raises on error statuses.  There
is no CPU fallback: importing works without a GPU, but every call that
reaches the library needs libmsmg.so (built by ``build.build()``) and a CUDA
device, and fails loudly otherwise.

The functions carry the C entry points' names (``msmg_setup``,
``msmg_solve``, ...).  ``Solver`` bundles them with workspace management.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import json
import os
from dataclasses import dataclass, field

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmsmg.so")

MAX_LEVELS = 8
FP64, MIXED = 0, 1
F64, F32 = 0, 1
FLAG_X0, FLAG_HOST_IO, FLAG_NO_GRAPH = 1, 2, 4

BLOCK_CHOL, BLOCK_IC0 = 0, 1

STATUS = {
    0: "MSMG_OK", 1: "MSMG_NOT_CONVERGED", 2: "MSMG_COARSE_IC_FALLBACK", -1: "MSMG_ERR_INVALID_ARG", -2: "MSMG_ERR_NOT_DIVISIBLE",
    -3: "MSMG_ERR_BAD_KAPPA", -4: "MSMG_ERR_SINGLE_BLOCK", -5: "MSMG_ERR_BREAKDOWN",
    -6: "MSMG_ERR_EIG_NOT_CONVERGED", -7: "MSMG_ERR_WORKSPACE", -8: "MSMG_ERR_CUDA",
    -9: "MSMG_ERR_NOT_FACTORIZABLE", -10: "MSMG_ERR_UNSUPPORTED",
    -11: "MSMG_ERR_DEVICE_TIMEOUT",
}


class MsmgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class msmg_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double)]


class msmg_options(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("block", C.c_int * 3), ("ratio", (C.c_int * 3) * MAX_LEVELS),
                ("n_eig", C.c_int * MAX_LEVELS), ("nu", C.c_int * MAX_LEVELS), ("precision", C.c_int),
                ("eig_tol", C.c_double), ("eig_max_iter", C.c_int), ("autotune", C.c_int),
                ("warm_start", C.c_void_p), ("coarse_smoother", C.c_int), ("two_grid", C.c_int),
                ("inner_rtol", C.c_double), ("inner_max_iter", C.c_int),
                ("eig_threshold", C.c_double * MAX_LEVELS), ("cell_diag", C.c_void_p)]


class msmg_setup_info(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("dims", C.c_int64 * MAX_LEVELS),
                ("dims_kept", C.c_int64 * MAX_LEVELS), ("elements", C.c_int64 * MAX_LEVELS),
                ("setup_ms", C.c_double), ("eig_ms", C.c_double), ("eig_iterations_max", C.c_int),
                ("eig_iterations_total", C.c_int64), ("warm_started", C.c_int), ("face_contrast", C.c_double),
                ("tuning", C.c_int * 4),
                ("eig_residual_max", C.c_double), ("workspace_bytes", C.c_int64)]


class msmg_net_desc(C.Structure):
    _fields_ = [("n_in", C.c_int), ("hidden", C.c_int * 2), ("n_vec", C.c_int), ("batch_max", C.c_int)]


class msmg_fluid(C.Structure):
    _fields_ = [("mu_w", C.c_double), ("mu_o", C.c_double), ("s_wc", C.c_double), ("s_or", C.c_double)]


class msmg_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("rel_residual", C.c_double),
                ("true_rel_residual", C.c_double), ("rhs_mean", C.c_double), ("solve_ms", C.c_double),
                ("inner_iterations", C.c_int64), ("kernel_launches", C.c_int64)]


_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libmsmg.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmsmg.so not found at {path}; run __graft_entry__.build() "
                          "(the CUDA path has no fallback)")
    lib = C.CDLL(path)
    P, I, D, S, I64 = C.c_void_p, C.c_int, C.c_double, C.c_size_t, C.c_int64
    sig = {
        "msmg_workspace_size": (I, [C.POINTER(msmg_grid), C.POINTER(msmg_options), I, C.POINTER(S)]),
        "msmg_setup": (I, [C.POINTER(msmg_grid), P, I, I, C.POINTER(msmg_options), P, S, P, C.POINTER(P)]),
        "msmg_solve": (I, [P, P, P, I, D, I, I, P, C.POINTER(msmg_solve_info)]),
        "msmg_apply_A": (I, [P, P, P, P]),
        "msmg_apply_precond": (I, [P, P, P, P]),
        "msmg_dot_scratch_bytes": (S, [I64]),
        "msmg_dot": (I, [P, P, I64, P, C.POINTER(D), P]),
        "msmg_export_basis": (I, [P, I, P, P, P]),
        "msmg_import_bases": (I, [P, C.POINTER(P), P]),
        "msmg_export_operator": (I, [P, I, P, P]),
        "msmg_export_faces": (I, [P, P, P]),
        "msmg_get_setup_info": (I, [P, C.POINTER(msmg_setup_info)]),
        "msmg_destroy": (None, [P]),
        "msmg_status_string": (C.c_char_p, [I]),
        "msmg_time_kernels": (I, [P, I, I, C.POINTER(D), I, P]),
        "msmg_solve_batched": (I, [C.POINTER(P), I, C.POINTER(P), C.POINTER(P), C.POINTER(I), D, I, I, P,
                                   C.POINTER(msmg_solve_info)]),
        "msmg_max_batch_rhs": (I, [P]),
        "msmg_autotune": (I, [P, I, I, P]),
        "msmg_set_tuning": (I, [P, C.POINTER(I)]),
        "msmg_net_workspace_size": (S, [C.POINTER(msmg_net_desc)]),
        "msmg_net_create": (I, [C.POINTER(msmg_net_desc), P, S, C.c_uint64, P, C.POINTER(P)]),
        "msmg_net_destroy": (None, [P]),
        "msmg_net_param_count": (I64, [P]),
        "msmg_net_param_offsets": (I, [P, C.POINTER(I64), C.POINTER(I64)]),
        "msmg_net_get_params": (I, [P, P, P]),
        "msmg_net_set_params": (I, [P, P, P]),
        "msmg_net_forward": (I, [P, P, P, I, P]),
        "msmg_net_time_products": (I, [P, P, I, C.POINTER(D), P]),
        "msmg_net_gradients": (I, [P, P, P, I, P, C.POINTER(C.c_float), P]),
        "msmg_net_train_step": (I, [P, P, P, I, C.c_float, C.POINTER(C.c_float), P]),
        "msmg_learning_data": (I, [P, P, P, P]),
        "msmg_dot_noalloc": (I, [P, P, I64, C.POINTER(D), P]),
        "msmg_check_conversions": (I, [P, P, I64, P, P, P]),
        "msmg_velocity": (I, [P, P, P, P, C.POINTER(D), P]),
        "msmg_impes_pressure_terms": (I, [I64, C.POINTER(msmg_fluid), P, P, P, P, D, P, P, P, P]),
        "msmg_impes_transport": (I, [P, C.POINTER(msmg_fluid), P, P, P, D, P, P, P, I, D, C.POINTER(D), P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names of the entry points the binding declares (all must be exported)."""
    return ["msmg_workspace_size", "msmg_setup", "msmg_solve", "msmg_apply_A", "msmg_apply_precond",
            "msmg_dot_scratch_bytes", "msmg_dot", "msmg_export_basis", "msmg_import_bases",
            "msmg_export_operator", "msmg_export_faces", "msmg_get_setup_info", "msmg_destroy",
            "msmg_status_string", "msmg_time_kernels", "msmg_dot_noalloc",
            "msmg_solve_batched", "msmg_max_batch_rhs", "msmg_autotune", "msmg_set_tuning",
            "msmg_net_workspace_size", "msmg_net_create",
            "msmg_net_destroy", "msmg_net_param_count", "msmg_net_param_offsets", "msmg_net_get_params",
            "msmg_net_set_params", "msmg_net_forward", "msmg_net_time_products", "msmg_net_gradients",
            "msmg_net_train_step",
            "msmg_learning_data", "msmg_check_conversions", "msmg_velocity", "msmg_impes_pressure_terms",
            "msmg_impes_transport"]


def _check(status: int) -> int:
    if status < 0:
        msg = load_library().msmg_status_string(status).decode()
        raise MsmgError(status, msg)
    return status


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _ptr(t: torch.Tensor, dtype=None, cuda: bool = True) -> int:
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if cuda and not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


@dataclass
class Options:
    n_levels: int = 3
    block: tuple = (4, 4, 4)
    ratio: list = field(default_factory=lambda: [(2, 2, 2)])
    n_eig: list = field(default_factory=lambda: [4, 4])
    nu: list | None = None
    precision: int = FP64
    eig_tol: float = 1e-12
    eig_max_iter: int = 0
    autotune: bool = False             # time the V-cycle variants at set-up (msmg_autotune)
    warm_start: object = None          # a WarmStartNet (or its handle) seeds the level-1 eigensolves
    coarse_smoother: int = BLOCK_CHOL  # BLOCK_CHOL (exact parent blocks) or BLOCK_IC0 (Section 5)
    two_grid: bool = False             # exact two-grid P_TG (Eq. (B_TG)) instead of the V-cycle
    inner_rtol: float = 0.0            # P_TG inner tolerance (0: library default 1e-10)
    inner_max_iter: int = 0            # P_TG inner iteration cap (0: library default 200)
    eig_threshold: list = field(default_factory=list)   # Strategy 2: B per level (0: keep n_eig)
    cell_diag: object = None           # CUDA FP64 tensor (nz, ny, nx) >= 0: well term W added to A

    def to_c(self) -> msmg_options:
        o = msmg_options()
        o.n_levels = self.n_levels
        for d in range(3):
            o.block[d] = self.block[d]
        for i, r in enumerate(self.ratio[:MAX_LEVELS]):
            for d in range(3):
                o.ratio[i][d] = r[d]
        for i, v in enumerate(self.n_eig[:MAX_LEVELS]):
            o.n_eig[i] = v
        nu = self.nu if self.nu is not None else [1] * (self.n_levels - 1)
        for i, v in enumerate(nu[:MAX_LEVELS]):
            o.nu[i] = v
        o.precision = self.precision
        o.eig_tol = self.eig_tol
        o.eig_max_iter = self.eig_max_iter
        o.autotune = 1 if self.autotune else 0
        ws = self.warm_start
        o.warm_start = (ws.handle if hasattr(ws, "handle") else ws) or None
        o.coarse_smoother = self.coarse_smoother
        o.two_grid = 1 if self.two_grid else 0
        o.inner_rtol = self.inner_rtol
        o.inner_max_iter = self.inner_max_iter
        for i, v in enumerate(self.eig_threshold[:MAX_LEVELS]):
            o.eig_threshold[i] = v
        if self.cell_diag is not None:
            w = self.cell_diag
            if not (isinstance(w, torch.Tensor) and w.is_cuda and w.dtype == torch.float64 and w.is_contiguous()):
                raise TypeError("cell_diag: a contiguous CUDA float64 tensor of nz*ny*nx values")
            o.cell_diag = w.data_ptr()
        return o


def make_grid(shape, h=None) -> msmg_grid:
    nz, ny, nx = shape
    g = msmg_grid()
    g.nx, g.ny, g.nz = nx, ny, nz
    hx, hy, hz = h if h is not None else (1.0 / nx, 1.0 / ny, 1.0 / nz)
    g.hx, g.hy, g.hz = hx, hy, hz
    return g


# ----------------------------------------------------------------- C names
def msmg_workspace_size(grid: msmg_grid, opts: msmg_options, n_rhs: int = 1) -> int:
    out = C.c_size_t(0)
    _check(load_library().msmg_workspace_size(C.byref(grid), C.byref(opts), n_rhs, C.byref(out)))
    return out.value


def msmg_setup(grid: msmg_grid, kappa: torch.Tensor, opts: msmg_options, workspace: torch.Tensor,
               stream=None) -> tuple[int, int]:
    """Returns (ctx handle, status).  kappa: CUDA (C, nz, ny, nx) or (nz, ny, nx), f64/f32."""
    comps = 1 if kappa.dim() == 3 else kappa.shape[0]
    dt = {torch.float64: F64, torch.float32: F32}[kappa.dtype]
    ctx = C.c_void_p(0)
    st = load_library().msmg_setup(C.byref(grid), _ptr(kappa), comps, dt, C.byref(opts), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), _stream(stream), C.byref(ctx))
    if st < 0 and st != -6:
        if ctx.value:
            load_library().msmg_destroy(ctx)
        _check(st)
    if st == -6 and not ctx.value:
        _check(st)
    return ctx.value, st


def msmg_solve(ctx: int, rhs: torch.Tensor, x: torch.Tensor, rtol: float, max_iter: int, flags: int = 0,
               stream=None) -> tuple[int, list]:
    host = bool(flags & FLAG_HOST_IO)
    n_rhs = rhs.shape[0] if rhs.dim() == 4 else 1
    infos = (msmg_solve_info * n_rhs)()
    st = load_library().msmg_solve(ctx, _ptr(rhs, torch.float64, cuda=not host), _ptr(x, torch.float64, cuda=not host),
                                   n_rhs, rtol, max_iter, flags, _stream(stream), infos)
    _check(st)
    return st, [_info_dict(i) for i in infos]


def _info_dict(i) -> dict:
    return dict(iterations=i.iterations, converged=bool(i.converged), rel_residual=i.rel_residual,
                true_rel_residual=i.true_rel_residual, rhs_mean=i.rhs_mean, solve_ms=i.solve_ms,
                inner_iterations=i.inner_iterations, kernel_launches=i.kernel_launches)


def msmg_solve_batched(ctxs: list, rhs: list, x: list, rtol: float, max_iter: int, flags: int = 0,
                       stream=None) -> tuple[int, list]:
    """Solve on several contexts at once; rhs[k] / x[k] hold context k's systems
    ([n_rhs, nz, ny, nx] or [nz, ny, nx]).  Returns the worst status and one list of
    info dicts per context."""
    host = bool(flags & FLAG_HOST_IO)
    k = len(ctxs)
    counts = [(r.shape[0] if r.dim() == 4 else 1) for r in rhs]
    infos = (msmg_solve_info * max(1, sum(counts)))()
    ca = (C.c_void_p * k)(*ctxs)
    ra = (C.c_void_p * k)(*[_ptr(r, torch.float64, cuda=not host) for r in rhs])
    xa = (C.c_void_p * k)(*[_ptr(v, torch.float64, cuda=not host) for v in x])
    na = (C.c_int * k)(*counts)
    st = load_library().msmg_solve_batched(ca, k, ra, xa, na, rtol, max_iter, flags, _stream(stream), infos)
    _check(st)
    out, o = [], 0
    for cnt in counts:
        out.append([_info_dict(infos[o + j]) for j in range(cnt)])
        o += cnt
    return st, out


def msmg_max_batch_rhs(ctx: int) -> int:
    return load_library().msmg_max_batch_rhs(ctx)


def msmg_autotune(ctx: int, n_rhs: int = 1, reps: int = 3, stream=None) -> None:
    _check(load_library().msmg_autotune(ctx, n_rhs, reps, _stream(stream)))


def msmg_set_tuning(ctx: int, tuning) -> None:
    arr = (C.c_int * 4)(*tuning)
    _check(load_library().msmg_set_tuning(ctx, arr))


def msmg_apply_A(ctx: int, p: torch.Tensor, q: torch.Tensor, stream=None) -> None:
    _check(load_library().msmg_apply_A(ctx, _ptr(p, torch.float64), _ptr(q, torch.float64), _stream(stream)))


def msmg_apply_precond(ctx: int, r: torch.Tensor, z: torch.Tensor, stream=None) -> None:
    _check(load_library().msmg_apply_precond(ctx, _ptr(r, torch.float64), _ptr(z, torch.float64), _stream(stream)))


def _same_vectors(a: torch.Tensor, b: torch.Tensor) -> None:
    """Both operands of a dot product: same length, same CUDA device (checked
    before anything reaches the library, which reads n values of each)."""
    if a.numel() != b.numel():
        raise ValueError(f"dot operands differ in length: {a.numel()} vs {b.numel()}")
    if a.device != b.device:
        raise ValueError(f"dot operands on different devices: {a.device} vs {b.device}")


def msmg_dot(a: torch.Tensor, b: torch.Tensor, scratch: torch.Tensor | None = None, stream=None) -> float:
    _same_vectors(a, b)
    lib = load_library()
    n = a.numel()
    with torch.cuda.device(a.device):
        if scratch is None:
            scratch = torch.empty(lib.msmg_dot_scratch_bytes(n), dtype=torch.uint8, device=a.device)
        elif scratch.device != a.device:
            raise ValueError("scratch must be on the operands' device")
        out = C.c_double(0.0)
        _check(lib.msmg_dot(_ptr(a, torch.float64), _ptr(b, torch.float64), n, _ptr(scratch), C.byref(out),
                            _stream(stream)))
    return out.value


DOT_NOALLOC_MAX_N = 16777216


def msmg_dot_noalloc(a: torch.Tensor, b: torch.Tensor, stream=None) -> float:
    """msmg_dot without a scratch buffer: the library's fixed device array holds the
    partial sums (for callers that cannot allocate device memory; see include/msmg.h)."""
    _same_vectors(a, b)
    out = C.c_double(0.0)
    with torch.cuda.device(a.device):
        _check(load_library().msmg_dot_noalloc(_ptr(a, torch.float64), _ptr(b, torch.float64), a.numel(),
                                               C.byref(out), _stream(stream)))
    return out.value


def msmg_check_conversions(in64: torch.Tensor, in32: torch.Tensor, stream=None):
    """The V-cycle kernels' integer-pipe conversions applied element by element:
    (in64 rounded to FP32, in32 widened to FP64), for comparison with the hardware's."""
    n = in64.numel()
    if in32.numel() != n:
        raise ValueError("in64 and in32 must have the same length")
    out32 = torch.empty(n, dtype=torch.float32, device=in64.device)
    out64 = torch.empty(n, dtype=torch.float64, device=in64.device)
    _check(load_library().msmg_check_conversions(_ptr(in64, torch.float64), _ptr(in32, torch.float32), n,
                                                 _ptr(out32), _ptr(out64), _stream(stream)))
    return out32, out64


def msmg_export_basis(ctx: int, level: int, basis: torch.Tensor, lam: torch.Tensor | None = None,
                      stream=None) -> None:
    _check(load_library().msmg_export_basis(ctx, level, _ptr(basis, torch.float64),
                                            _ptr(lam, torch.float64) if lam is not None else None,
                                            _stream(stream)))


def msmg_import_bases(ctx: int, bases: list, stream=None) -> int:
    arr = (C.c_void_p * len(bases))(*[_ptr(b, torch.float64) for b in bases])
    return _check(load_library().msmg_import_bases(ctx, arr, _stream(stream)))


def msmg_export_operator(ctx: int, level: int, out: torch.Tensor, stream=None) -> None:
    _check(load_library().msmg_export_operator(ctx, level, _ptr(out, torch.float64), _stream(stream)))


def msmg_velocity(ctx: int, p: torch.Tensor, f: torch.Tensor, v: torch.Tensor, stream=None) -> tuple[float, float]:
    """Face velocities v[3][nz][ny][nx] from the pressure p (Eq. (velocity)) and the mass
    balance (||div v - b||_2, ||b||_2), b = f - mean(f)."""
    if p.numel() * 3 != v.numel() or f.numel() != p.numel():
        raise ValueError("p, f: n values each; v: 3 n values")
    bal = (C.c_double * 2)()
    _check(load_library().msmg_velocity(ctx, _ptr(p, torch.float64), _ptr(f, torch.float64), _ptr(v, torch.float64),
                                        bal, _stream(stream)))
    return bal[0], bal[1]


def make_fluid(mu_w: float = 0.3, mu_o: float = 3.0, s_wc: float = 0.2, s_or: float = 0.2) -> msmg_fluid:
    """Section 6's fluid model (defaults: the paper's values)."""
    f = msmg_fluid()
    f.mu_w, f.mu_o, f.s_wc, f.s_or = mu_w, mu_o, s_wc, s_or
    return f


def msmg_impes_pressure_terms(fluid: msmg_fluid, S: torch.Tensor, kappa: torch.Tensor, wi: torch.Tensor,
                              q_inj: torch.Tensor, p_bh: float, stream=None):
    """(kappa_eff [3, ...], w, b) of the pressure system of Eq. (IMP) at saturation S."""
    n = S.numel()
    if kappa.numel() != 3 * n or wi.numel() != n or q_inj.numel() != n:
        raise ValueError("S, wi, q_inj: n values; kappa: 3 n values")
    ke = torch.empty_like(kappa)
    w = torch.empty_like(S)
    b = torch.empty_like(S)
    _check(load_library().msmg_impes_pressure_terms(n, C.byref(fluid), _ptr(S, torch.float64), _ptr(kappa, torch.float64),
                                                    _ptr(wi, torch.float64), _ptr(q_inj, torch.float64), p_bh,
                                                    _ptr(ke), _ptr(w), _ptr(b), _stream(stream)))
    return ke, w, b


def msmg_impes_transport(ctx: int, fluid: msmg_fluid, v: torch.Tensor, p: torch.Tensor, w: torch.Tensor, p_bh: float,
                         q_inj: torch.Tensor, phi: torch.Tensor, S: torch.Tensor, M: int, ds_max: float,
                         stream=None) -> float:
    """M saturation sub-steps of Eq. (ES) in place on S; returns the time they cover."""
    n = S.numel()
    if v.numel() != 3 * n or any(t.numel() != n for t in (p, w, q_inj, phi)):
        raise ValueError("v: 3 n values; p, w, q_inj, phi, S: n values")
    dt = C.c_double(0.0)
    _check(load_library().msmg_impes_transport(ctx, C.byref(fluid), _ptr(v, torch.float64), _ptr(p, torch.float64),
                                               _ptr(w, torch.float64), p_bh, _ptr(q_inj, torch.float64),
                                               _ptr(phi, torch.float64), _ptr(S, torch.float64), M, ds_max,
                                               C.byref(dt), _stream(stream)))
    return dt.value


def msmg_export_faces(ctx: int, out: torch.Tensor, stream=None) -> None:
    _check(load_library().msmg_export_faces(ctx, _ptr(out, torch.float64), _stream(stream)))


def msmg_get_setup_info(ctx: int) -> dict:
    i = msmg_setup_info()
    _check(load_library().msmg_get_setup_info(ctx, C.byref(i)))
    nL = i.n_levels
    return dict(n_levels=nL, dims=list(i.dims[:nL]), dims_kept=list(i.dims_kept[:nL]),
                elements=list(i.elements[:nL - 1]), setup_ms=i.setup_ms,
                eig_ms=i.eig_ms, eig_iterations_max=i.eig_iterations_max,
                eig_iterations_total=i.eig_iterations_total, warm_started=bool(i.warm_started),
                tuning=list(i.tuning), face_contrast=i.face_contrast,
                eig_residual_max=i.eig_residual_max, workspace_bytes=i.workspace_bytes)


def msmg_destroy(ctx: int) -> None:
    load_library().msmg_destroy(ctx)


def msmg_time_kernels(ctx: int, reps: int = 20, stream=None, n_rhs: int = 1) -> list:
    out = (C.c_double * 7)()
    _check(load_library().msmg_time_kernels(ctx, n_rhs, reps, out, 7, _stream(stream)))
    return list(out)


# ----------------------------------------------------------------- learned warm start
def msmg_net_workspace_size(desc: msmg_net_desc) -> int:
    return load_library().msmg_net_workspace_size(C.byref(desc))


def msmg_net_create(desc: msmg_net_desc, workspace: torch.Tensor, seed: int = 0, stream=None) -> int:
    h = C.c_void_p(0)
    _check(load_library().msmg_net_create(C.byref(desc), _ptr(workspace), workspace.numel(), seed, _stream(stream),
                                          C.byref(h)))
    return h.value


def msmg_net_forward(net: int, x: torch.Tensor, y: torch.Tensor, stream=None) -> None:
    _check(load_library().msmg_net_forward(net, _ptr(x, torch.float32), _ptr(y, torch.float32), x.shape[0],
                                           _stream(stream)))


def msmg_net_time_products(net: int, x: torch.Tensor, stream=None) -> list:
    """Device milliseconds of the forward pass's three products (tensor-core form)."""
    ms = (C.c_double * 3)()
    _check(load_library().msmg_net_time_products(net, _ptr(x, torch.float32), x.shape[0], ms, _stream(stream)))
    return [float(v) for v in ms]


def msmg_net_gradients(net: int, x: torch.Tensor, target: torch.Tensor, grad: torch.Tensor | None = None,
                       stream=None) -> float:
    loss = C.c_float(0)
    _check(load_library().msmg_net_gradients(net, _ptr(x, torch.float32), _ptr(target, torch.float32), x.shape[0],
                                             _ptr(grad, torch.float32) if grad is not None else None,
                                             C.byref(loss), _stream(stream)))
    return loss.value


def msmg_net_train_step(net: int, x: torch.Tensor, target: torch.Tensor, lr: float, stream=None) -> float:
    loss = C.c_float(0)
    _check(load_library().msmg_net_train_step(net, _ptr(x, torch.float32), _ptr(target, torch.float32), x.shape[0],
                                              lr, C.byref(loss), _stream(stream)))
    return loss.value


def msmg_learning_data(ctx: int, x: torch.Tensor, y: torch.Tensor, stream=None) -> None:
    _check(load_library().msmg_learning_data(ctx, _ptr(x, torch.float32), _ptr(y, torch.float32), _stream(stream)))


class WarmStartNet:
    """The learned warm start (include/msmg.h): a network in a torch-allocated device
    workspace.  ``train`` runs Adam steps through the library's kernels."""

    def __init__(self, n_in: int = 512, hidden=(512, 512), n_vec: int = 5, batch_max: int = 1024, seed: int = 0,
                 stream=None):
        self.desc = msmg_net_desc()
        self.desc.n_in, self.desc.n_vec, self.desc.batch_max = n_in, n_vec, batch_max
        self.desc.hidden[0], self.desc.hidden[1] = hidden
        nbytes = msmg_net_workspace_size(self.desc)
        if nbytes == 0:
            raise MsmgError(-1, "invalid network description")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream
        self.handle = msmg_net_create(self.desc, self.workspace, seed, stream)

    @property
    def n_param(self) -> int:
        return load_library().msmg_net_param_count(self.handle)

    def offsets(self):
        w = (C.c_int64 * 3)()
        b = (C.c_int64 * 3)()
        _check(load_library().msmg_net_param_offsets(self.handle, w, b))
        return list(w), list(b)

    def get_params(self) -> torch.Tensor:
        p = torch.empty(self.n_param, dtype=torch.float32, device="cuda")
        _check(load_library().msmg_net_get_params(self.handle, _ptr(p), _stream(self.stream)))
        return p

    def set_params(self, p: torch.Tensor) -> None:
        p = p.to(device="cuda", dtype=torch.float32).contiguous()
        _check(load_library().msmg_net_set_params(self.handle, _ptr(p), _stream(self.stream)))

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        y = torch.empty((x.shape[0], self.desc.n_vec * self.desc.n_in), dtype=torch.float32, device="cuda")
        msmg_net_forward(self.handle, x.contiguous(), y, self.stream)
        return y

    def gradients(self, x: torch.Tensor, target: torch.Tensor):
        g = torch.empty(self.n_param, dtype=torch.float32, device="cuda")
        loss = msmg_net_gradients(self.handle, x.contiguous(), target.contiguous(), g, self.stream)
        return loss, g

    def train_step(self, x: torch.Tensor, target: torch.Tensor, lr: float) -> float:
        return msmg_net_train_step(self.handle, x.contiguous(), target.contiguous(), lr, self.stream)

    def close(self):
        if getattr(self, "handle", None):
            load_library().msmg_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- convenience
def _read_cache(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


class Solver:
    """setup(permeability, grid, block sizes, eigenvectors per element, levels)
    then solve(rhs, rtol), on the current CUDA device and stream."""

    def __init__(self, kappa, opts: Options, h=None, n_rhs: int = 1, stream=None, tuning_cache: str | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("msmg needs a CUDA device (no CPU fallback)")
        k = torch.as_tensor(kappa)
        if not k.is_cuda:
            k = k.to("cuda")
        if k.dtype not in (torch.float64, torch.float32):
            k = k.to(torch.float64)
        k = k.contiguous()
        shape = tuple(k.shape[-3:])
        self.shape = shape
        self.n = shape[0] * shape[1] * shape[2]
        self.opts = opts
        self.grid = make_grid(shape, h)
        # autotune cache: a JSON file of tunings keyed by the problem's shape; a hit
        # applies the stored variants instead of timing them again
        key = None
        cached = None
        if tuning_cache:
            key = json.dumps([list(shape), list(opts.block), list(opts.n_eig[:opts.n_levels - 1]), opts.n_levels,
                              opts.precision, n_rhs])
            cached = _read_cache(tuning_cache).get(key)
        copts_opts = opts
        if cached is not None and opts.autotune:
            copts_opts = dataclasses.replace(opts, autotune=False)
        self.copts = copts_opts.to_c()
        self.n_rhs = n_rhs
        nbytes = msmg_workspace_size(self.grid, self.copts, n_rhs)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=k.device)
        self.ctx, self.setup_status = msmg_setup(self.grid, k, self.copts, self.workspace, stream)
        self.stream = stream
        if cached is not None:
            msmg_set_tuning(self.ctx, cached)
        elif tuning_cache and opts.autotune:
            c = _read_cache(tuning_cache)
            c[key] = self.info["tuning"]
            with open(tuning_cache, "w") as fh:
                json.dump(c, fh)

    def refresh(self, kappa, cell_diag: torch.Tensor | None = None):
        """Set up again for new coefficients on the same grid and hierarchy (new
        permeability, new cell term), in the workspace already held: the step of a
        time loop such as IMPES, where the operator changes every step."""
        k = torch.as_tensor(kappa)
        if not k.is_cuda:
            k = k.to("cuda")
        if k.dtype not in (torch.float64, torch.float32):
            k = k.to(torch.float64)
        k = k.contiguous()
        if tuple(k.shape[-3:]) != self.shape:
            raise ValueError("refresh keeps the grid: the permeability's shape differs")
        if (cell_diag is None) != (self.opts.cell_diag is None):
            raise ValueError("refresh keeps the options: a cell term must stay present or absent")
        opts = dataclasses.replace(self.opts, cell_diag=cell_diag)
        copts = opts.to_c()
        if msmg_workspace_size(self.grid, copts, self.n_rhs) > self.workspace.numel():
            raise ValueError("refresh needs a larger workspace than the solver holds")
        self.close()
        self.opts = opts            # keeps the cell term alive while the context uses it
        self.copts = copts
        self.ctx, self.setup_status = msmg_setup(self.grid, k, self.copts, self.workspace, self.stream)

    def close(self):
        if getattr(self, "ctx", None):
            msmg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        return msmg_get_setup_info(self.ctx)

    def solve(self, rhs: torch.Tensor, rtol: float = 1e-8, max_iter: int = 1000, x0: torch.Tensor | None = None):
        rhs = rhs.to(torch.float64).contiguous()
        x = torch.zeros_like(rhs) if x0 is None else x0.to(torch.float64).clone().contiguous()
        flags = FLAG_X0 if x0 is not None else 0
        if not rhs.is_cuda:
            flags |= FLAG_HOST_IO
        st, info = msmg_solve(self.ctx, rhs, x, rtol, max_iter, flags, self.stream)
        return x, (info[0] if len(info) == 1 else info), st

    def apply_A(self, p: torch.Tensor) -> torch.Tensor:
        q = torch.empty_like(p)
        msmg_apply_A(self.ctx, p.contiguous(), q, self.stream)
        return q

    def apply_precond(self, r: torch.Tensor) -> torch.Tensor:
        z = torch.empty_like(r)
        msmg_apply_precond(self.ctx, r.contiguous(), z, self.stream)
        return z

    def export_basis(self, level: int):
        info = self.info
        m = info["elements"][level - 1]
        L = self.opts.n_eig[level - 1]
        if level == 1:
            per = self.opts.block[0] * self.opts.block[1] * self.opts.block[2]
        else:
            r = self.opts.ratio[level - 2]
            per = r[0] * r[1] * r[2] * self.opts.n_eig[level - 2]
        basis = torch.empty((m, L, per), dtype=torch.float64, device="cuda")
        lam = torch.empty((m, L), dtype=torch.float64, device="cuda")
        msmg_export_basis(self.ctx, level, basis, lam, self.stream)
        return basis, lam

    def import_bases(self, bases: list) -> int:
        bs = [torch.as_tensor(b, dtype=torch.float64).to("cuda").contiguous() for b in bases]
        st = msmg_import_bases(self.ctx, bs, self.stream)
        torch.cuda.synchronize()
        return st

    def export_operator(self, level: int) -> torch.Tensor:
        n = self.info["dims"][level - 1]
        out = torch.empty((n, n), dtype=torch.float64, device="cuda")
        msmg_export_operator(self.ctx, level, out, self.stream)
        return out

    @property
    def max_batch_rhs(self) -> int:
        return msmg_max_batch_rhs(self.ctx)

    def time_kernels(self, reps: int = 20, n_rhs: int = 1) -> dict:
        v = msmg_time_kernels(self.ctx, reps, self.stream, n_rhs)
        keys = ["pre", "restrict", "prolong", "post", "coarse_levels", "pmatvec", "vcycle"]
        return dict(zip(keys, v))

    def learning_data(self):
        """(x [m, nb], y [m, L-1, nb]) training pairs of this context's level-1 elements."""
        m = self.info["elements"][0]
        nb = self.opts.block[0] * self.opts.block[1] * self.opts.block[2]
        L = self.opts.n_eig[0]
        x = torch.empty((m, nb), dtype=torch.float32, device="cuda")
        y = torch.empty((m, L - 1, nb), dtype=torch.float32, device="cuda")
        msmg_learning_data(self.ctx, x, y, self.stream)
        return x, y

    def velocity(self, p: torch.Tensor, f: torch.Tensor):
        """(v [3, nz, ny, nx], mass balance (||div v - b||, ||b||)) of a pressure field."""
        v = torch.empty((3,) + self.shape, dtype=torch.float64, device="cuda")
        bal = msmg_velocity(self.ctx, p.to(torch.float64).contiguous(), f.to(torch.float64).contiguous(), v,
                            self.stream)
        return v, bal

    def export_faces(self) -> torch.Tensor:
        out = torch.empty((3,) + self.shape, dtype=torch.float64, device="cuda")
        msmg_export_faces(self.ctx, out, self.stream)
        return out
