"""Plans created with SHT_FLAG_TIMING record CUDA events around their apply
kernels; the summed device times come back through sht_plan_kernel_time and
the results are those of the oracle as without the flag."""
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


@pytest.mark.parametrize("prec,eps,F,tol", [(_lib.SHT_FP64, 1e-12, 2, 1e-10), (_lib.SHT_MIXED, 1e-7, 40, 1e-6)])
def test_kernel_time(prec, eps, F, tol):
    N = 64
    p = sht.Plan(N, eps, precision=prec, flags=_lib.SHT_FLAG_TIMING)
    beta = inputs.coefficients(N, F, seed=2)
    b = torch.from_numpy(beta).cuda()
    g = p.forward(b)
    back = p.inverse(g)
    t = p.kernel_time()
    # default max_fields = 1: the 40-field tensor-core call runs as two 32-field batches
    per_call = 1 if prec == _lib.SHT_FP64 else 2
    assert t["launches"] == 2 * per_call
    assert t["apply_ms"] > 0
    assert (t["output_ms"] > 0) == (prec == _lib.SHT_MIXED)
    assert p.kernel_time()["launches"] == 0  # reset by the previous query
    ref = oracle.alt_forward(N, beta)
    e = np.linalg.norm((g.cpu().numpy() - ref).reshape(F, -1), axis=1) / np.linalg.norm(ref.reshape(F, -1), axis=1)
    assert np.all(e <= tol)
    e2 = np.linalg.norm((back.cpu().numpy() - oracle.alt_inverse(N, g.cpu().numpy())).reshape(F, -1), axis=1)
    assert np.all(e2 <= tol * np.linalg.norm(back.cpu().numpy().reshape(F, -1), axis=1))


def test_timing_can_be_paused():
    N, F = 32, 3
    p = sht.Plan(N, 1e-7, precision=_lib.SHT_MIXED, max_fields=F, flags=_lib.SHT_FLAG_TIMING)
    b = torch.from_numpy(inputs.coefficients(N, F, seed=3)).cuda()
    p.kernel_time()
    p.set_timing(False)
    g = p.forward(b)
    assert p.kernel_time()["launches"] == 0
    p.set_timing(True)
    g2 = p.forward(b)
    assert p.kernel_time()["launches"] == 1
    torch.cuda.synchronize()
    assert torch.equal(g, g2) or float((g - g2).norm() / g.norm()) < 1e-6
    q = sht.Plan(N, 1e-7, precision=_lib.SHT_MIXED)
    with pytest.raises(_lib.ShtError):
        q.set_timing(False)
