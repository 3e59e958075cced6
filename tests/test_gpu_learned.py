"""Learned warm start of the level-1 eigensolves through the C-ABI: the
network's forward pass, loss, gradients and Adam step against the FP64
oracle; the training pairs the library exports against the oracle's
eigenpairs; and the gain of a trained network over the cold start on a
held-out layered field, with the same final eigen-residual tolerance."""
import numpy as np
import pytest
import torch

import fields
import oracle
from oracle import learned

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_19342_gb300 as p
    return p


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_net(pkg, n_in=512, hidden=(256, 128), n_vec=5, batch_max=64, seed=3):
    return pkg.WarmStartNet(n_in=n_in, hidden=hidden, n_vec=n_vec, batch_max=batch_max, seed=seed)


def layout(net):
    w_off, b_off = net.offsets()
    d = net.desc
    return (d.n_in, d.hidden[0], d.hidden[1], d.n_vec * d.n_in), w_off, b_off


# Tolerances of the network against its oracle.  Both round every activation to
# BF16 before the product that reads it, the library after an FP32 accumulation,
# the oracle after an exact one; where the two straddle a BF16 rounding boundary
# (about 20 FP32 ulps in 2^16, a few activations in 10^4) the next product's
# operand differs by one BF16 ulp (2^-8 relative).  So outputs and loss agree to
# about 1e-3 relative and the gradients, which multiply two such factors, to 1e-2.
FWD_TOL, GRAD_TOL = 3e-3, 1e-2


@pytest.mark.parametrize("hidden,batch", [((256, 128), 64), ((512, 512), 300), ((192, 64), 64),
                                          ((512, 512), 4096), ((100, 60), 64)],
                         ids=["tensor_cores", "tensor_cores_ragged", "tensor_cores_tile64",
                              "tensor_cores_persistent", "cuda_cores"])
def test_forward_loss_gradients_match_oracle(pkg, hidden, batch):
    # widths multiples of 64 run the products on the tensor cores (tcgen05), others on
    # the CUDA cores; both read BF16 operands and accumulate in FP32.  Output tiles
    # 256, 128 and 64 wide all occur (192 and 64 take the 64-wide tile); at batch 4096
    # the last product has 320 tiles, more than the SMs, so CTAs take several tiles
    # and alternate their two accumulators.
    net = make_net(pkg, hidden=hidden, batch_max=batch)
    dims, w_off, b_off = layout(net)
    rng = np.random.default_rng(0)
    x = rng.normal(0, 0.5, size=(batch, 512)).astype(np.float32)
    t = rng.normal(size=(batch, 5, 512))
    t /= np.linalg.norm(t, axis=-1, keepdims=True)
    t = t.reshape(batch, -1).astype(np.float32)
    params = net.get_params().cpu().numpy()
    # forward: FP32 accumulation against FP64 with the same BF16 operands
    out = net.forward(torch.tensor(x, device="cuda")).cpu().numpy()
    Ws, bs = learned.unpack(params, dims, w_off, b_off)
    _, _, ref_out = learned.forward(Ws, bs, x)
    e_fwd = rel(out, ref_out)
    loss, g = net.gradients(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    ref_loss, ref_g = learned.gradients(params, dims, w_off, b_off, x, t, n_vec=5)
    g = g.cpu().numpy()
    e_g = max(rel(g[off:off + size], ref_g[off:off + size]) for l in range(3)
              for off, size in ((w_off[l], dims[l] * dims[l + 1]), (b_off[l], dims[l + 1])))
    print(f"hidden {hidden} batch {batch}: forward rel. error {e_fwd:.2e}, loss {loss:.6f} vs {ref_loss:.6f}, "
          f"worst gradient block {e_g:.2e}")
    assert e_fwd < FWD_TOL
    assert loss == pytest.approx(ref_loss, rel=FWD_TOL)
    assert e_g < GRAD_TOL
    net.close()


def test_train_step_is_adam(pkg):
    net = make_net(pkg, seed=5)
    rng = np.random.default_rng(1)
    x = torch.tensor(rng.normal(0, 0.5, size=(32, 512)), dtype=torch.float32, device="cuda")
    t = torch.tensor(rng.normal(size=(32, 5 * 512)), dtype=torch.float32, device="cuda")
    p0 = net.get_params().cpu().numpy().astype(np.float64)
    _, g = net.gradients(x, t)
    g = g.cpu().numpy().astype(np.float64)
    net.train_step(x, t, lr=1e-3)
    p1 = net.get_params().cpu().numpy()
    ref, _, _ = learned.adam_step(p0, g, np.zeros_like(p0), np.zeros_like(p0), step=1, lr=1e-3)
    np.testing.assert_allclose(p1, ref, rtol=1e-5, atol=1e-7)
    net.close()


def test_learning_data_against_oracle(pkg):
    # 32^3 GRF, 4^3 elements, L = 4: the exported pairs are the oracle's features and
    # the symmetric-form eigenvectors S^{1/2} phi_k, k = 1 .. 3 (compared as spans)
    N = 32
    kappa = fields.grf_lognormal((N, N, N), seed=0, contrast=1e3)
    opts = pkg.Options(n_levels=3, block=(4, 4, 4), ratio=[(2, 2, 2)], n_eig=[4, 4], eig_tol=1e-12)
    S = pkg.Solver(torch.tensor(kappa, device="cuda"), opts)
    x, y = S.learning_data()
    x, y = x.cpu().numpy(), y.cpu().numpy()
    h = (1.0 / N,) * 3
    Sw = oracle.trace_weight(kappa, h).ravel()
    cells = oracle.element_cells((N, N, N), (4, 4, 4))
    np.testing.assert_allclose(x, learned.features(Sw[cells]), atol=2e-6)
    H = oracle.setup(kappa, h, oracle.Options(n_levels=3, block=(4, 4, 4), ratio=[(2, 2, 2)], n_eig=[5, 4],
                                              nu=[1, 1]))
    lam = H.lam[0]
    for e in range(0, cells.shape[0], 11):
        Y = y[e].astype(np.float64)
        np.testing.assert_allclose(Y @ Y.T, np.eye(3), atol=1e-5)
        if lam[e, 4] - lam[e, 3] < 1e-3 * max(lam[e, 4], 1e-12):
            continue                                   # no gap at the cutoff: span not unique
        ref = np.sqrt(Sw[cells[e]])[None, :] * H.basis[0][e, 1:4]
        np.testing.assert_allclose(Y.T @ Y, ref.T @ ref, atol=1e-5)
    S.close()


def layered(N, seed):
    return fields.layered_channels((N, N, N), seed=seed)


def test_warm_start_gain_on_held_out_field(pkg):
    # Train on eight layered fields (seeds 101-108), set up a held-out one (seed 100)
    # cold and warm-started, and report what the network gains.  The warm start only
    # seeds the subspace iteration, which runs to the same eigen-residual tolerance,
    # so the preconditioner is as good as the cold one.  How much the
    # set-up gains depends on the accuracy of the guesses (only a small part of the
    # iterations at |cos| ~ 0.7); the test bounds any loss at 10% and prints the gain.
    N, L = 64, 6
    opts = dict(n_levels=3, block=(8, 8, 8), ratio=[(2, 2, 2)], n_eig=[L, 4], precision=pkg.MIXED, eig_tol=1e-8)
    xs, ys = [], []
    for seed in range(101, 109):
        S = pkg.Solver(torch.tensor(layered(N, seed), device="cuda"), pkg.Options(**opts))
        x, y = S.learning_data()
        xs.append(x)
        ys.append(y.reshape(y.shape[0], -1))
        S.close()
    X, Y = torch.cat(xs), torch.cat(ys)
    net = pkg.WarmStartNet(n_in=512, hidden=(512, 512), n_vec=L - 1, batch_max=256, seed=7)
    gen = torch.Generator(device="cuda").manual_seed(0)
    first = last = None
    for step in range(1500):
        idx = torch.randint(0, X.shape[0], (256,), device="cuda", generator=gen)
        loss = net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr=3e-4)
        first = loss if first is None else first
        last = loss
    assert last < 0.5 * first
    kappa = torch.tensor(layered(N, 100), device="cuda")
    cold = pkg.Solver(kappa, pkg.Options(**opts))
    warm = pkg.Solver(kappa, pkg.Options(**opts, warm_start=net))
    ic, iw = cold.info, warm.info
    assert iw["warm_started"] and not ic["warm_started"]
    assert ic["eig_residual_max"] <= 1e-8 and iw["eig_residual_max"] <= 1e-8
    gain = 1.0 - iw["eig_iterations_total"] / ic["eig_iterations_total"]
    print(f"training loss {first:.3f} -> {last:.3f}; subspace iterations cold {ic['eig_iterations_total']} "
          f"(max {ic['eig_iterations_max']}, {ic['eig_ms']:.1f} ms), warm {iw['eig_iterations_total']} "
          f"(max {iw['eig_iterations_max']}, {iw['eig_ms']:.1f} ms): gain {100 * gain:.1f}%")
    assert iw["eig_iterations_total"] <= 1.1 * ic["eig_iterations_total"]
    # both bases meet the same tolerance but agree only to it, and near-degenerate pairs
    # at the cutoff (common on layered fields) let the kept spans differ further: the
    # two preconditioners are equally valid, the PCG counts close
    f = torch.tensor(fields.rhs_corners((N, N, N)), device="cuda")
    _, infc, _ = cold.solve(f, rtol=1e-8)
    _, infw, _ = warm.solve(f, rtol=1e-8)
    assert infc["converged"] and infw["converged"]
    assert abs(infc["iterations"] - infw["iterations"]) <= 0.1 * infc["iterations"]
    cold.close()
    warm.close()
    net.close()
