"""The integer binary64 <-> binary32 conversions against the GPU's own
conversion instructions, bit for bit (sht_selftest_convert).

The FP32 and tensor-core paths convert every FP64 input and output value with
these helpers (round to nearest even, IEEE 754 subnormals, overflow to
infinity, NaN kept NaN), so a wrong rounding bit would bias every result.
Patterns: uniformly random bit patterns, random values with exponents around
the binary32 range (normal, subnormal and overflow boundaries), exact rounding
ties of both parities, and the special values.
"""
import numpy as np
import pytest

from paper_2004_11346_gb300 import _lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def patterns():
    rng = np.random.default_rng(2004)
    parts = [rng.integers(0, 2**63, size=1 << 22, dtype=np.uint64) | (rng.integers(0, 2, size=1 << 22, dtype=np.uint64) << np.uint64(63))]
    # exponents 1023-160 .. 1023+140: subnormal, normal and overflowing binary32 results
    n = 1 << 22
    e = rng.integers(1023 - 160, 1023 + 140, size=n, dtype=np.uint64)
    m = rng.integers(0, 1 << 52, size=n, dtype=np.uint64)
    s = rng.integers(0, 2, size=n, dtype=np.uint64)
    parts.append((s << np.uint64(63)) | (e << np.uint64(52)) | m)
    # exact ties at the 29-bit rounding position (normal results) and at the
    # subnormal rounding positions, both parities of the kept bit
    e = rng.integers(1023 - 160, 1023 + 128, size=n, dtype=np.uint64)
    hi = rng.integers(0, 1 << 23, size=n, dtype=np.uint64) << np.uint64(29)
    ties = []
    for sh in range(29, 53):
        ties.append((s << np.uint64(63)) | (e << np.uint64(52)) | ((hi >> np.uint64(sh)) << np.uint64(sh)) | (np.uint64(1) << np.uint64(sh - 1)))
    parts.append(np.concatenate(ties)[: 1 << 22])
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 3.4028234663852886e38,
                        3.4028235677973366e38, 3.4028235677973362e38, 1.1754943508222875e-38,
                        1.1754942106924411e-38, 1.401298464324817e-45, 7.006492321624085e-46,
                        7.006492321624087e-46, 2.1019476964872256e-45, 5e-324, -5e-324,
                        np.finfo(np.float64).max, np.finfo(np.float64).tiny], dtype=np.float64)
    parts.append(special.view(np.uint64))
    return np.concatenate(parts).view(np.float64)


def test_conversions_match_the_hardware_bit_for_bit():
    x = torch.from_numpy(patterns()).cuda()
    n = x.numel()
    f32 = torch.empty(n, dtype=torch.float32, device="cuda")
    back = torch.empty(n, dtype=torch.float64, device="cuda")
    _lib.sht_selftest_convert(x.data_ptr(), f32.data_ptr(), back.data_ptr(), n,
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ref32 = x.to(torch.float32)
    nan = torch.isnan(ref32)
    assert torch.equal(torch.isnan(f32), nan)
    assert torch.equal(f32[~nan].view(torch.int32), ref32[~nan].view(torch.int32))
    ref64 = f32.to(torch.float64)
    nan = torch.isnan(ref64)
    assert torch.equal(torch.isnan(back), nan)
    assert torch.equal(back[~nan].view(torch.int64), ref64[~nan].view(torch.int64))
    # the fast paths and the slow paths were both exercised
    a = ref32[~torch.isnan(ref32)].abs()
    assert int(((a > 0) & (a < 1.1754943508222875e-38)).sum()) > 1000  # binary32 subnormals
    assert int(torch.isinf(ref32).sum()) > 1000


def test_convert_arguments():
    with pytest.raises(_lib.ShtError):
        _lib.sht_selftest_convert(0, 0, 0, 5)
    _lib.sht_selftest_convert(0, 0, 0, 0)
