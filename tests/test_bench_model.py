"""bench.py's algorithmic byte and flop model against the per-kernel table it is
built from: one PCG iteration of the mixed form on L eigenvectors per element
reads and writes, per fine cell, pre 72 B, restrict 20 + 4L, prolong 8 + 4L (or
nothing, inside k_post), post 48 B (+4L when the prolongation is fused),
pmatvec 64 B; the coefficient bytes are shared by the R right-hand sides of a
batched launch."""
import pytest

import bench


@pytest.mark.parametrize("L", [4, 6, 12])
def test_mixed_bytes_per_cell(L):
    kb = bench.kernel_bytes("mixed", L)
    assert kb == {"pre": 72, "restrict": 20 + 4 * L, "prolong": 8 + 4 * L, "post": 48, "pmatvec": 64}
    kf = bench.kernel_bytes("mixed", L, fused=True)
    assert kf["prolong"] == 0 and kf["post"] == 48 + 4 * L
    # fusing removes exactly the u read and write of the separate prolongation
    assert sum(kb.values()) - sum(kf.values()) == 8


def test_fp64_bytes_per_cell():
    kb = bench.kernel_bytes("fp64", 6)
    # no flexible beta in the FP64 form: post reads no q; its right-hand side is r
    # itself, read once (no V-precision copy)
    assert kb == {"pre": 96, "restrict": 40 + 48, "prolong": 16 + 48, "post": 56, "pmatvec": 64}


def test_batched_bytes_share_coefficients():
    one, many = bench.kernel_bytes("mixed", 6, 1), bench.kernel_bytes("mixed", 6, 16)
    # T, 1/d (pre), T and the basis (restrict), the basis (prolong), T and 1/d (post),
    # T and D (pmatvec) are read once for all 16 right-hand sides
    assert one["pre"] - many["pre"] == pytest.approx(16 * 15 / 16)
    assert one["restrict"] - many["restrict"] == pytest.approx((12 + 24) * 15 / 16)
    assert one["prolong"] - many["prolong"] == pytest.approx(24 * 15 / 16)
    assert one["post"] - many["post"] == pytest.approx(16 * 15 / 16)
    assert one["pmatvec"] - many["pmatvec"] == pytest.approx(32 * 15 / 16)


def test_fp64_flops_and_peak():
    assert bench.FP64_FLOPS_MIXED == {"pre": 6, "restrict": 0, "prolong": 0, "post": 4, "pmatvec": 17}
    # 152 SMs x 2 FP64 FMA per clock x 2 flops at 2070 MHz
    assert bench.fp64_peak_gflops(2070.0) == pytest.approx(152 * 2 * 2 * 2.07)
