"""The coarse IC(0) smoother (Section 5: incomplete Cholesky for M_c;
MSMG_BLOCK_IC0) through the C-ABI against the oracle's BlockIC0Dense, with the
oracle's bases imported so both sides factor the same coarse blocks: the
V-cycle element by element (FP64 rounding: 1e-10 of its norm, the factor and
its inverse being formed in different orders), a solve's iteration count
within one, and the fallback warning exactly when the oracle falls back."""
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


@pytest.mark.parametrize("contrast,seed", [(1e3, 0), (1e6, 2)])
def test_coarse_ic0_vcycle_and_solve(pkg, contrast, seed):
    N = 32
    kap = fields.grf_lognormal((N, N, N), seed=seed, contrast=contrast)
    oo = oracle.Options(n_levels=4, block=(4, 4, 4), ratio=[(2, 2, 2)] * 2, n_eig=[4, 4, 4], nu=[1] * 3,
                        coarse_smoother="ic0")
    H = oracle.setup(kap, (1 / N,) * 3, oo)
    go = pkg.Options(n_levels=4, block=(4, 4, 4), ratio=[(2, 2, 2)] * 2, n_eig=[4, 4, 4],
                     coarse_smoother=pkg.BLOCK_IC0)
    S = pkg.Solver(torch.tensor(kap, device="cuda"), go)
    st = S.import_bases(H.basis[:3])
    fell_back = any(getattr(M, "fallback", []) for M in H.M[1:])
    assert st == (2 if fell_back else 0), (st, [getattr(M, "fallback", None) for M in H.M[1:]])
    rng = np.random.default_rng(5)
    r = rng.standard_normal(H.dims[0])
    r -= r.mean()
    z = S.apply_precond(torch.tensor(r.reshape(H.shape), device="cuda")).cpu().numpy().ravel()
    ref = oracle.vcycle(H, r)
    assert np.linalg.norm(z - ref) <= 1e-10 * np.linalg.norm(ref)
    # IC(0) differs from the exact coarse blocks: the default smoother gives another result
    Hc = oracle.setup(kap, (1 / N,) * 3, oracle.Options(n_levels=4, block=(4, 4, 4), ratio=[(2, 2, 2)] * 2,
                                                        n_eig=[4, 4, 4], nu=[1] * 3))
    assert np.linalg.norm(oracle.vcycle(Hc, r) - ref) > 1e-6 * np.linalg.norm(ref)
    b = fields.rhs_corners(H.shape)
    res = oracle.solve(H, b.ravel(), rtol=1e-8)
    _, info, _ = S.solve(torch.tensor(b, device="cuda"), rtol=1e-8)
    print(f"contrast {contrast:g}: IC(0) coarse smoother iterations gpu {info['iterations']} "
          f"oracle {res.iterations}")
    assert abs(info["iterations"] - res.iterations) <= 1
