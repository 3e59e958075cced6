"""The two largest workloads at their full sizes, in the launch configuration
bench.py times (mixed form): the 512^3 layered channel field (12 eigenvectors,
6 levels) and the 1024^3 lognormal field (4 eigenvectors, 7 levels).

Neither fits the oracle whole, so the oracle is applied where it can be: at
sampled cells it recomputes, from 3x3x3 patches of the permeability and of the
solution, the face coefficients (Fig. (kappa edge)) and the flux balance
(A x)_i (Eq. (discrete varia)); these must match the library's exported
coefficients and a face-by-face evaluation of A x on the GPU at the same cells.
That evaluation, checked at the samples, then gives the global residual
||b - A x|| / ||b||, which must meet the solve's tolerance."""
import numpy as np
import pytest
import torch

import bench
import fields
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_19342_gb300 as p
    return p


def face_flux_balance(T, x, absolute=False):
    """(A x) face by face on the GPU: every internal face adds T (x_i - x_j) to
    cell i and subtracts it from its +d neighbour j.  absolute: (|A| |x|)_i =
    sum over the cell's faces of T (|x_i| + |x_j|), the scale of the rounding
    error of any evaluation of (A x)_i."""
    q = torch.zeros_like(x)
    if absolute:
        x = x.abs()
    for d, (lo, hi) in enumerate(((np.s_[:, :, :-1], np.s_[:, :, 1:]), (np.s_[:, :-1, :], np.s_[:, 1:, :]),
                                  (np.s_[:-1, :, :], np.s_[1:, :, :]))):
        f = T[d][lo] * ((x[lo] + x[hi]) if absolute else (x[lo] - x[hi]))
        q[lo] += f
        if absolute:
            q[hi] += f
        else:
            q[hi] -= f
        del f
    return q


def sample_cells(N, rng, count=2048):
    cells = rng.integers(0, N, size=(count, 3))
    corners = np.array([[0, 0, 0], [N - 1, N - 1, N - 1], [0, N - 1, 0], [N - 1, 0, N - 1]])
    return np.concatenate([corners, cells])


def check_against_oracle(kappa, x, T, q, cells, N):
    """kappa, x, T, q on the GPU (natural order, (z, y, x)); cells as (k, j, i)."""
    h = (1.0 / N,) * 3
    worst_T, worst_q = 0.0, 0.0
    for k, j, i in cells:
        sl = (slice(max(k - 1, 0), min(k + 2, N)), slice(max(j - 1, 0), min(j + 2, N)),
              slice(max(i - 1, 0), min(i + 2, N)))
        kp = kappa[sl].double().cpu().numpy()
        xp = x[sl].cpu().numpy()
        Tp = oracle.face_transmissibilities(kp, h)
        c = (k - sl[0].start, j - sl[1].start, i - sl[2].start)
        # the faces of the centre cell: to its +d neighbour and from its -d neighbour
        for d in range(3):
            for off in (0, -1):
                cc = list(c)
                cc[2 - d] += off
                if min(cc) < 0 or cc[2 - d] + 1 >= Tp.shape[3 - d]:
                    continue
                g = [k, j, i]
                g[2 - d] += off
                ref = Tp[d][tuple(cc)]
                got = float(T[d][tuple(g)])
                worst_T = max(worst_T, abs(got - ref) / abs(ref))
        qo = oracle.apply_A(Tp, xp).reshape(xp.shape)[c]
        scale = sum(abs(Tp[d]).sum() for d in range(3)) * np.abs(xp).max() + 1e-300
        worst_q = max(worst_q, abs(float(q[k, j, i]) - qo) / scale)
    return worst_T, worst_q


def solve_and_check(pkg, kappa, opts, N, rtol=1e-8, max_iter=3000):
    f = torch.zeros((N, N, N), dtype=torch.float64, device="cuda")
    f.view(-1)[0] = 1.0
    f.view(-1)[-1] = -1.0
    S = pkg.Solver(kappa, opts)
    assert S.setup_status == 0
    x, info, st = S.solve(f, rtol=rtol, max_iter=max_iter)
    assert st == 0 and info["converged"], info
    T = S.export_faces()
    S.close()
    del S
    torch.cuda.synchronize()
    assert abs(float(x.mean())) <= 1e-12 * float(x.abs().max())
    b = f - f.mean()
    nb = float(torch.linalg.norm(b))
    # the library's stopping test evaluated b - A x with its own rounding: allow
    # 32 eps ||(|A| |x|)|| on top of the tolerance
    slack = 32 * np.finfo(np.float64).eps * float(torch.linalg.norm(face_flux_balance(T, x, absolute=True))) / nb
    q = face_flux_balance(T, x)
    res = float(torch.linalg.norm(b - q)) / nb
    worst_T, worst_q = check_against_oracle(kappa, x, T, q, sample_cells(N, np.random.default_rng(0)), N)
    print(f"N={N}: iterations {info['iterations']}, residual {res:.3e} (library {info['true_rel_residual']:.3e}, "
          f"rounding slack {slack:.1e}), sampled face coefficients {worst_T:.1e}, sampled A x {worst_q:.1e}")
    assert worst_T <= 1e-14
    assert worst_q <= 1e-14
    assert res <= rtol + slack, (res, slack)
    del T, q, x, b, f
    torch.cuda.empty_cache()
    return info


def test_layered_512_full_size(pkg):
    N = bench.LAYERED_N
    kappa = torch.tensor(fields.layered_channels((N,) * 3, seed=100), device="cuda")
    opts = pkg.Options(n_levels=6, block=(8, 8, 8), ratio=[(2, 2, 2)] * 4, n_eig=[12] * 5, precision=pkg.MIXED,
                       eig_tol=1e-8)
    solve_and_check(pkg, kappa, opts, N)


def test_lognormal_1024_full_size(pkg):
    N = bench.SCALE_N
    opts = pkg.Options(n_levels=7, block=(8, 8, 8), ratio=[(2, 2, 2)] * 5, n_eig=[4] * 6, precision=pkg.MIXED,
                       eig_tol=1e-8)
    need = pkg.msmg_workspace_size(pkg.make_grid((N, N, N)), opts.to_c(), 1)
    torch.cuda.empty_cache()            # blocks cached for earlier tests count as used
    free, _ = torch.cuda.mem_get_info()
    extra = (4 + 8 * 3 + 8 * 3) * N ** 3          # kappa (FP32), x, b, q and face temporaries
    if need + extra + (4 << 30) > free:
        pytest.skip(f"needs {(need + extra) / 2**30:.0f} GiB of device memory, {free / 2**30:.0f} GiB free")
    kappa = fields.grf_lognormal_device((N, N, N), seed=5, contrast=1e6, device="cuda")
    solve_and_check(pkg, kappa, opts, N, max_iter=2000)
