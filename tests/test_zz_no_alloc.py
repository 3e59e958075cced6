"""msmg_dot_noalloc: the dot product for callers that cannot allocate device
memory (its scratch is a fixed array inside the library).  Checked through the
C-ABI against msmg_dot, which uses a caller-provided scratch buffer, on two
calls in a row (the fixed array keeps the previous call's contents)."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_19342_gb300 as p
    return p


def test_noalloc_dot_matches_scratch_dot(pkg):
    rng = np.random.default_rng(12)
    for n in (1_000_003, 4097):                       # two calls in a row, different sizes
        a = rng.standard_normal(n)
        b = rng.standard_normal(n)
        ta, tb = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
        ref = pkg.msmg_dot(ta, tb)
        got = pkg.msmg_dot_noalloc(ta, tb)
        # the two launches differ only in how the sum is split across CTAs
        assert abs(got - ref) <= 1e-13 * float(np.abs(a * b).sum())
        assert abs(got - math.fsum(a * b)) <= 1e-13 * float(np.abs(a * b).sum())


def test_noalloc_dot_rejects_oversize(pkg):
    n = pkg.DOT_NOALLOC_MAX_N + 1
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.MsmgError) as e:
        pkg.msmg_dot_noalloc(a, a)
    assert e.value.status == -1
    assert pkg.msmg_dot_noalloc(a[:0], a[:0]) == 0.0


def test_noalloc_dot_rejects_mismatched_operands(pkg):
    # a shorter b would be read past its end: refused before any launch
    a = torch.zeros(1000, dtype=torch.float64, device="cuda")
    b = torch.zeros(999, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        pkg.msmg_dot_noalloc(a, b)
    with pytest.raises(ValueError):
        pkg.msmg_dot(a, b)
