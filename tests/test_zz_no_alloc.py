"""alt_forward_m_noalloc: the forward single-order ALT with no allocation.

That entry point serves callers that cannot allocate device memory, such as
code inside a pool or arena that owns the device, or latency-critical loops
where cudaMalloc/cudaFree would synchronise the device.  It keeps its scratch
in a fixed array in the library's device image.  This test calls it through
the C ABI and checks, on two calls in a row, that it gives what
alt_forward_m gives, within the FP64 path's tolerance.  The file is named so
that pytest collects it last.
"""
import numpy as np
import pytest

import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("N,kw", [
    (64, dict(n0=16, n_leaf=8, flags=_lib.SHT_FLAG_FORCE_FACTOR)),
    (256, {}),
])
def test_noalloc_matches_alt_forward_m(N, kw):
    plan = sht.Plan(N, 1e-12, **kw)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(N)
    F = 3
    for call in range(2):
        for m in [0, 1, -6, N, -(2 * N - 1)]:
            bm = torch.from_numpy(rng.standard_normal((F, 2 * N - abs(m), 2))).cuda()
            ref = torch.empty((F, 2 * N, 2), dtype=torch.float64, device="cuda")
            got = torch.full((F, 2 * N, 2), float("nan"), dtype=torch.float64, device="cuda")
            _lib.alt_forward_m(plan.handle, m, bm.data_ptr(), ref.data_ptr(), F, stream)
            _lib.alt_forward_m_noalloc(plan.handle, m, bm.data_ptr(), got.data_ptr(), F, stream)
            torch.cuda.synchronize()
            r, g = ref.cpu().numpy(), got.cpu().numpy()
            err = np.linalg.norm((g - r).reshape(F, -1), axis=1) / np.linalg.norm(r.reshape(F, -1), axis=1)
            assert np.all(err <= TOL_FP64), (call, m, err)
    plan.sync()


def test_noalloc_rejects_bad_arguments():
    N = 16
    plan = sht.Plan(N, 1e-12)
    x = torch.zeros((1, 2 * N, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.ShtError):
        _lib.alt_forward_m_noalloc(plan.handle, 2 * N, x.data_ptr(), x.data_ptr(), 1, 0)
    with pytest.raises(_lib.ShtError):
        _lib.alt_forward_m_noalloc(plan.handle, 0, 0, x.data_ptr(), 1, 0)
    _lib.alt_forward_m_noalloc(plan.handle, 0, 0, 0, 0, 0)  # F = 0 is a no-op


def test_noalloc_needs_fp64_plan():
    """Mixed-precision plans keep no FP64 factor store on the device."""
    N = 16
    plan = sht.Plan(N, 1e-7, precision=_lib.SHT_MIXED)
    x = torch.zeros((1, 2 * N, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.ShtError) as ei:
        _lib.alt_forward_m_noalloc(plan.handle, 0, x.data_ptr(), x.data_ptr(), 1, 0)
    assert ei.value.status == _lib.SHT_ERR_UNSUPPORTED


def test_noalloc_launches_are_timed():
    """With SHT_FLAG_TIMING the entry point's launches are counted like the others."""
    N = 32
    plan = sht.Plan(N, 1e-12, flags=_lib.SHT_FLAG_TIMING)
    x = torch.from_numpy(np.random.default_rng(1).standard_normal((2, 2 * N - 3, 2))).cuda()
    y = torch.empty((2, 2 * N, 2), dtype=torch.float64, device="cuda")
    plan.kernel_time()
    _lib.alt_forward_m_noalloc(plan.handle, 3, x.data_ptr(), y.data_ptr(), 2, 0)
    t = plan.kernel_time()
    assert t["launches"] == 1 and t["apply_ms"] > 0
