"""Failure detection on the GPU without a fault.

- A bounded wait that runs out: the self-test launch of the tensor-core kernel
  publishes no work item, every other role's wait for it gives up after about
  a second, the host reads SHT_ERR_TIMEOUT, and the plan keeps working.
- An allocation failure during plan creation (injected on the host with
  SHT_FAIL_ALLOC): SHT_ERR_OOM, with everything allocated so far released.
"""
import gc
import os

import numpy as np
import pytest

import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def forward_err(p, N, F=3, seed=7):
    beta = inputs.coefficients(N, F, seed=seed)
    g = p.forward(torch.from_numpy(beta).cuda())
    torch.cuda.synchronize()
    p.sync()
    ref = oracle.alt_forward(N, beta)
    return np.max(np.linalg.norm((g.cpu().numpy() - ref).reshape(F, -1), axis=1)
                  / np.linalg.norm(ref.reshape(F, -1), axis=1))


def test_bounded_wait_reports_timeout_and_plan_recovers():
    N = 32
    p = sht.Plan(N, 1e-7, precision=_lib.SHT_MIXED, max_fields=8)
    assert forward_err(p, N) <= 1e-6
    _lib.sht_selftest_timeout(p.handle, torch.cuda.current_stream().cuda_stream)
    with pytest.raises(_lib.ShtError) as e:
        p.sync()
    assert e.value.status == _lib.SHT_ERR_TIMEOUT
    p.sync()  # the flag was read and cleared
    assert forward_err(p, N, seed=8) <= 1e-6


def test_selftest_needs_a_tensor_core_plan():
    p = sht.Plan(16, 1e-12)
    with pytest.raises(_lib.ShtError) as e:
        _lib.sht_selftest_timeout(p.handle, 0)
    assert e.value.status == _lib.SHT_ERR_UNSUPPORTED


@pytest.mark.parametrize("k", [1, 3, 7, 12])
def test_injected_allocation_failure(k):
    N = 32
    # plans of earlier tests can outlive them in reference cycles (an exception
    # kept by pytest.raises holds its frame): free them before measuring
    gc.collect()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    os.environ["SHT_FAIL_ALLOC"] = str(k)
    try:
        with pytest.raises(_lib.ShtError) as e:
            sht.Plan(N, 1e-7, precision=_lib.SHT_MIXED, max_fields=8)
        assert e.value.status == _lib.SHT_ERR_OOM
    finally:
        del os.environ["SHT_FAIL_ALLOC"]
    del e
    gc.collect()
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 64 << 20  # nothing of the failed plan stays allocated
    p = sht.Plan(N, 1e-7, precision=_lib.SHT_MIXED, max_fields=8)
    assert forward_err(p, N) <= 1e-6
    p.close()
