"""The integer-pipe FP32 <-> FP64 conversions of the mixed-form V-cycle kernels
against the hardware conversions, bit for bit: normal values across the whole
range, exact halfway cases (ties to even), the binary32 subnormal range and its
rounding edges, overflow, signed zeros, infinities and NaNs, and every class of
binary32 input for the widening."""
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


def doubles_to_narrow(rng):
    parts = []
    # log-uniform magnitudes from far below the binary32 subnormals to far above its range
    parts.append(np.exp(rng.uniform(np.log(1e-50), np.log(1e45), 200000)) * rng.choice([-1.0, 1.0], 200000))
    # exact midpoints between neighbouring binary32 values (normal and subnormal), and
    # one double ulp either side of them
    f = np.concatenate([rng.normal(0, 1, 20000), np.exp(rng.uniform(-100, 85, 20000)),
                        rng.uniform(0, 1.2e-38, 20000)]).astype(np.float32)
    g = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + g.astype(np.float64)) / 2
    parts += [mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf), -mid]
    tiny = np.float64(np.finfo(np.float32).smallest_subnormal)
    fmax = np.float64(np.finfo(np.float32).max)
    ulp_top = fmax - np.float64(np.nextafter(np.float32(fmax), np.float32(0)))
    special = [0.0, -0.0, np.inf, -np.inf, np.nan, tiny, tiny / 2, np.nextafter(tiny / 2, 1.0),
               np.nextafter(tiny / 2, 0.0), tiny * 1.5, tiny * 2.5, 1e-310, -1e-310, 5e-324,
               np.float64(np.finfo(np.float32).tiny), np.float64(np.finfo(np.float32).tiny) * (1 - 2 ** -25),
               fmax, fmax + ulp_top / 2, np.nextafter(fmax + ulp_top / 2, 0.0), fmax * 2, 1e300, -1e300,
               1.0, -1.0, 1.0 + 2 ** -24, 1.0 + 3 * 2 ** -24, 1.0 + 2 ** -24 + 2 ** -50]
    parts.append(np.array(special, dtype=np.float64))
    return np.concatenate(parts)


def test_integer_conversions_match_hardware(pkg):
    rng = np.random.default_rng(7)
    d = torch.tensor(doubles_to_narrow(rng), device="cuda")
    bits = rng.integers(0, 2 ** 32, size=d.numel(), dtype=np.uint64).astype(np.uint32)
    bits[:8] = [0, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0x00000001, 0x807FFFFF, 0x7F7FFFFF]
    f = torch.tensor(bits.view(np.float32), device="cuda")
    out32, out64 = pkg.msmg_check_conversions(d, f)
    torch.cuda.synchronize()
    ref32, ref64 = d.to(torch.float32), f.to(torch.float64)
    nan32 = torch.isnan(ref32)
    assert torch.equal(torch.isnan(out32), nan32)
    assert torch.equal(out32[~nan32].view(torch.int32), ref32[~nan32].view(torch.int32))
    nan64 = torch.isnan(ref64)
    assert torch.equal(torch.isnan(out64), nan64)
    assert torch.equal(out64[~nan64].view(torch.int64), ref64[~nan64].view(torch.int64))
