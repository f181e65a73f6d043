"""The autotuner on the GPU: it times its best-ranked candidates and returns
the fastest as a device plan, whose transform still matches the oracle."""
import numpy as np
import pytest

import oracle
from paper_2004_11346_gb300 import autotune, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_autotune_returns_fastest_measured_plan():
    N, F = 48, 8
    plan, rows = autotune.autotune(N, 1e-7, F, top=2, steps=2, cands=[(12, 6), (24, 6), (24, 12)])
    timed = [r for r in rows if "measured_ms" in r]
    assert len(timed) == 2
    best = min(timed, key=lambda r: r["measured_ms"])
    assert (plan.opts.n0, plan.opts.n_leaf) == (best["n0"], best["n_leaf"])
    beta = inputs.coefficients(N, F, seed=2)
    g = plan.forward(torch.from_numpy(beta).cuda())
    torch.cuda.synchronize()
    ref = oracle.alt_forward(N, beta)
    err = np.linalg.norm((g.cpu().numpy() - ref).reshape(F, -1), axis=1) / np.linalg.norm(ref.reshape(F, -1), axis=1)
    assert np.all(err <= 1e-6)
