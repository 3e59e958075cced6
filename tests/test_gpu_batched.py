"""Batched solves through the C-ABI: several right-hand sides of one context in
lockstep (msmg_solve with n_rhs > 1) and several contexts at once
(msmg_solve_batched).  Each system of a batch runs the same arithmetic as its
single solve (own scalars, own reduction slice with the same CTA partition),
so batched and single results must agree bit for bit; one batch is also
checked against the FP64 oracle."""
import numpy as np
import pytest
import torch

import fields
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_19342_gb300 as p
    return p


def h_of(shape):
    nz, ny, nx = shape
    return (1.0 / nx, 1.0 / ny, 1.0 / nz)


def make(pkg, kappa, precision=0, n_rhs=4, n_eig=(4, 4)):
    opts = pkg.Options(n_levels=3, block=(4, 4, 4), ratio=[(2, 2, 2)], n_eig=list(n_eig), precision=precision,
                       eig_tol=1e-12)
    return pkg.Solver(torch.tensor(kappa, device="cuda"), opts, n_rhs=n_rhs)


def abs_apply(T, x):
    """|A| |x| for the rounding bound of a residual evaluation: per face, T (|x_i| + |x_j|)
    added to both cells."""
    ax = np.abs(x)
    q = np.zeros_like(ax)
    f = T[0][:, :, :-1] * (ax[:, :, :-1] + ax[:, :, 1:])
    q[:, :, :-1] += f
    q[:, :, 1:] += f
    f = T[1][:, :-1, :] * (ax[:, :-1, :] + ax[:, 1:, :])
    q[:, :-1, :] += f
    q[:, 1:, :] += f
    f = T[2][:-1, :, :] * (ax[:-1, :, :] + ax[1:, :, :])
    q[:-1, :, :] += f
    q[1:, :, :] += f
    return q


def rhs_set(shape, k, seed=0):
    """k right-hand sides of different character: corner source/sink, line sources,
    then seeded random fields (mean removed by the solver)."""
    out = [fields.rhs_corners(shape), fields.rhs_line_sources(shape)]
    for j in range(k - 2):
        out.append(fields.rhs_random(shape, 1, seed=seed + j)[0])
    return np.stack(out[:k])


@pytest.fixture(scope="module")
def grf32():
    return fields.grf_lognormal((32, 32, 32), seed=0, contrast=1e3)


@pytest.fixture(scope="module")
def solver_fp64(pkg, grf32):
    S = make(pkg, grf32, precision=0, n_rhs=4)
    yield S
    S.close()


@pytest.fixture(scope="module")
def solver_mixed(pkg, grf32):
    S = make(pkg, grf32, precision=1, n_rhs=4)
    yield S
    S.close()


def single_solves(S, F, **kw):
    xs, infos = [], []
    for f in F:
        x, info, _ = S.solve(torch.tensor(f, device="cuda"), **kw)
        xs.append(x)
        infos.append(info)
    return torch.stack(xs), infos


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_batch_equals_single_solves(form, solver_fp64, solver_mixed):
    S = solver_fp64 if form == "fp64" else solver_mixed
    assert S.max_batch_rhs == 4
    F = rhs_set(S.shape, 4)
    X, infos, st = S.solve(torch.tensor(F, device="cuda"), rtol=1e-8)
    assert st == 0 and len(infos) == 4
    Xs, infos1 = single_solves(S, F, rtol=1e-8)
    for j in range(4):
        assert infos[j]["converged"]
        assert infos[j]["iterations"] == infos1[j]["iterations"]
        assert infos[j]["true_rel_residual"] <= 1.1e-8
    assert torch.equal(X, Xs)


def test_batch_against_oracle(pkg, grf32, solver_fp64):
    S = solver_fp64
    H = oracle.setup(grf32, h_of(S.shape), oracle.Options(n_levels=3, block=(4, 4, 4), ratio=[(2, 2, 2)],
                                                          n_eig=[4, 4], nu=[1, 1]))
    assert S.import_bases([H.basis[0], H.basis[1]]) == 0
    F = rhs_set(S.shape, 4, seed=7)
    k = 12
    X, infos, _ = S.solve(torch.tensor(F, device="cuda"), rtol=0.0, max_iter=k)
    for j in range(4):
        ref = oracle.solve(H, F[j].ravel(), rtol=0.0, max_iter=k)
        assert infos[j]["iterations"] == k == ref.iterations
        err = np.linalg.norm(X[j].cpu().numpy().ravel() - ref.x) / np.linalg.norm(ref.x)
        assert err < 1e-10, (j, err)


def test_heterogeneous_batch(solver_fp64):
    S = solver_fp64
    shape = S.shape
    F = np.stack([np.zeros(shape), np.full(shape, 2.5), fields.rhs_corners(shape),
                  fields.rhs_random(shape, 1, seed=3)[0]])
    X, infos, st = S.solve(torch.tensor(F, device="cuda"), rtol=1e-8)
    assert st == 0
    assert infos[0]["iterations"] == 0 and float(X[0].abs().max()) == 0.0
    assert infos[1]["iterations"] == 0 and infos[1]["rhs_mean"] == pytest.approx(2.5)
    assert float(X[1].abs().max()) == 0.0
    Xs, infos1 = single_solves(S, F[2:], rtol=1e-8)
    assert [i["iterations"] for i in infos[2:]] == [i["iterations"] for i in infos1]
    assert torch.equal(X[2:], Xs)


def test_more_systems_than_batch_width(pkg, grf32):
    S = make(pkg, grf32, n_rhs=2)
    assert S.max_batch_rhs == 2
    F = rhs_set(S.shape, 5, seed=11)
    X, infos, st = S.solve(torch.tensor(F, device="cuda"), rtol=1e-8)
    assert st == 0 and len(infos) == 5
    Xs, infos1 = single_solves(S, F, rtol=1e-8)
    assert [i["iterations"] for i in infos] == [i["iterations"] for i in infos1]
    assert torch.equal(X, Xs)
    S.close()


def test_batched_host_io_and_no_graph(pkg, solver_fp64):
    S = solver_fp64
    F = rhs_set(S.shape, 3, seed=5)
    Fd = torch.tensor(F, device="cuda")
    Xd, infd, _ = S.solve(Fd, rtol=1e-8)
    # host buffers: the copies run inside the call
    Fh = torch.tensor(F).pin_memory()
    Xh, infh, _ = S.solve(Fh, rtol=1e-8)
    assert torch.equal(Xd.cpu(), Xh)
    # kernel-by-kernel launches instead of the captured graph
    Xn = torch.zeros_like(Fd)
    st, infn = pkg.msmg_solve(S.ctx, Fd, Xn, 1e-8, 1000, pkg.FLAG_NO_GRAPH)
    assert [i["iterations"] for i in infn] == [i["iterations"] for i in infd]
    assert torch.equal(Xd, Xn)


def test_batched_warm_start(solver_fp64):
    S = solver_fp64
    F = torch.tensor(rhs_set(S.shape, 4, seed=9), device="cuda")
    X, infos, _ = S.solve(F, rtol=1e-10)
    X2, infos2, _ = S.solve(F, rtol=1e-8, x0=X)
    assert all(i["iterations"] == 0 for i in infos2)
    assert torch.allclose(X2, X, rtol=0, atol=1e-12 * float(X.abs().max()))


def test_solve_batched_contexts(pkg, grf32, solver_fp64):
    # three independent problems of different sizes and fields, 1 / 3 / 2 systems
    k16 = fields.grf_lognormal((16, 16, 16), seed=21, contrast=1e2)
    k24 = fields.grf_lognormal((24, 24, 24), seed=22, contrast=1e4)
    S16 = make(pkg, k16, n_rhs=1)
    S24 = make(pkg, k24, n_rhs=2, n_eig=(5, 4))
    S32 = solver_fp64
    F16 = rhs_set(S16.shape, 1, seed=1)
    F32 = rhs_set(S32.shape, 3, seed=2)
    F24 = rhs_set(S24.shape, 2, seed=3)
    rhs = [torch.tensor(F16, device="cuda"), torch.tensor(F32, device="cuda"), torch.tensor(F24, device="cuda")]
    xs = [torch.zeros_like(r) for r in rhs]
    st, infos = pkg.msmg_solve_batched([S16.ctx, S32.ctx, S24.ctx], rhs, xs, 1e-8, 1000)
    assert st == 0 and [len(i) for i in infos] == [1, 3, 2]
    for S, F, X, inf in ((S16, F16, xs[0], infos[0]), (S32, F32, xs[1], infos[1]), (S24, F24, xs[2], infos[2])):
        Xs, inf1 = single_solves(S, F, rtol=1e-8)
        assert [i["iterations"] for i in inf] == [i["iterations"] for i in inf1]
        assert all(i["converged"] for i in inf)
        assert torch.equal(X, Xs)
    # a context may appear once per call
    with pytest.raises(pkg.MsmgError):
        pkg.msmg_solve_batched([S16.ctx, S16.ctx], rhs[:1] * 2, xs[:1] * 2, 1e-8, 1000)
    S16.close()
    S24.close()


def test_time_kernels_batched(pkg, solver_mixed):
    t1 = solver_mixed.time_kernels(reps=3, n_rhs=1)
    t4 = solver_mixed.time_kernels(reps=3, n_rhs=4)
    assert all(v > 0 for v in t1.values()) and all(v > 0 for v in t4.values())
    with pytest.raises(pkg.MsmgError):
        solver_mixed.time_kernels(reps=1, n_rhs=5)


def test_batched_workload_full_size(pkg):
    # the batched workload at full size, in the launch configuration bench.py times
    # (8 contexts of 64^3..192^3, 16 right-hand sides each, one msmg_solve_batched call,
    # mixed form); checked through properties that hold at any size: every residual
    # b - A x recomputed with the oracle's operator is below rtol, x has zero mean,
    # and a batched system equals its single solve bit for bit
    solvers, F, X, data = [], [], [], []
    for kappa, f in fields.lognormal_batch(16, device="cuda"):
        opts = pkg.Options(n_levels=4, block=(8, 8, 8), ratio=[(2, 2, 2), (2, 2, 2)], n_eig=[4, 4, 4],
                           precision=pkg.MIXED, eig_tol=1e-8)
        solvers.append(pkg.Solver(torch.tensor(kappa, device="cuda"), opts, n_rhs=16))
        F.append(torch.tensor(f, device="cuda"))
        X.append(torch.zeros_like(F[-1]))
        data.append((kappa, f))
    st, infos = pkg.msmg_solve_batched([S.ctx for S in solvers], F, X, 1e-8, 2000)
    assert st == 0
    for (kappa, f), Xk, inf, S in zip(data, X, infos, solvers):
        assert all(i["converged"] for i in inf)
        T = oracle.face_transmissibilities(kappa, h_of(kappa.shape))
        for j in (0, 15):
            x = Xk[j].cpu().numpy()
            b = f[j] - f[j].mean()
            res = np.linalg.norm(b - oracle.apply_A(T, x)) / np.linalg.norm(b)
            # the two FP64 residual evaluations (library, oracle) differ by rounding of
            # order eps |A| |x|: allow a few units of it on top of rtol
            slack = 32 * np.finfo(np.float64).eps * np.linalg.norm(abs_apply(T, x)) / np.linalg.norm(b)
            assert res <= 1e-8 + slack, (kappa.shape, j, res, slack, inf[j])
            assert abs(x.mean()) <= 1e-13 * np.abs(x).max()
    x1, info1, _ = solvers[0].solve(F[0][3], rtol=1e-8, max_iter=2000)
    assert info1["iterations"] == infos[0][3]["iterations"]
    assert torch.equal(x1, X[0][3])
    for S in solvers:
        S.close()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_tuned_variants_give_the_same_bits(pkg, form, solver_fp64, solver_mixed):
    # the autotuner's variants (prolongation fused into post-smoothing or apart) change
    # only the time: single and batched solves agree bit for bit across them
    S = solver_fp64 if form == "fp64" else solver_mixed
    F = torch.tensor(rhs_set(S.shape, 4, seed=13), device="cuda")
    out = []
    forms = [0]
    for form in (1, 2, 3):
        try:
            pkg.msmg_set_tuning(S.ctx, (0, 0, form, form))
            forms.append(form)
        except pkg.MsmgError:
            pass
    assert 2 in forms                     # the cooperative coarse cycle is available here
    tunes = [(0, 0, 0, 0), (1, 1, 0, 0)] + [(f % 2, (f + 1) % 2, f, f) for f in forms[1:]]
    for tune in tunes:
        pkg.msmg_set_tuning(S.ctx, tune)
        X, infos, _ = S.solve(F, rtol=1e-8)
        x1, info1, _ = S.solve(F[1], rtol=1e-8)
        out.append((X, [i["iterations"] for i in infos], x1))
    for o in out[1:]:
        assert torch.equal(out[0][0], o[0]) and out[0][1] == o[1]
        assert torch.equal(out[0][2], o[2])
    pkg.msmg_autotune(S.ctx, 1, 2)
    pkg.msmg_autotune(S.ctx, 4, 2)
    tuning = S.info["tuning"]
    assert tuning[0] in (0, 1) and tuning[1] in (0, 1) and tuning[2] in forms and tuning[3] in forms
    X2, _, _ = S.solve(F, rtol=1e-8)
    assert torch.equal(X2, out[0][0])
