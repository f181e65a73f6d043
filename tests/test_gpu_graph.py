"""The apply entry points can be captured in a CUDA graph and replayed.

The batched schedule (all orders x all fields in one launch per direction)
is meant to be replayed from a graph; this checks that capture works for the
FP64 and the tensor-core paths and that replays reproduce the eager result.
"""
import numpy as np
import pytest

import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("N,eps,prec,F,tol", [
    (64, 1e-12, _lib.SHT_FP64, 2, 1e-13),
    (128, 1e-7, _lib.SHT_MIXED, 40, 1e-6),
])
def test_graph_replay_matches_eager(N, eps, prec, F, tol):
    p = sht.Plan(N, eps, precision=prec)
    beta = torch.from_numpy(inputs.coefficients(N, F, seed=3)).cuda()
    g = torch.empty((F, 4 * N - 1, 2 * N, 2), dtype=torch.float64, device="cuda")
    back = torch.empty_like(beta)
    # eager reference
    p.forward(beta, out=g)
    p.inverse(g, out=back)
    torch.cuda.synchronize()
    g_ref, back_ref = g.clone(), back.clone()
    # capture (after a warm-up on a side stream, as torch requires)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        p.forward(beta, out=g)
        p.inverse(g, out=back)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        p.forward(beta, out=g)
        p.inverse(g, out=back)
    g.zero_()
    back.zero_()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    p.sync()
    eg = (g - g_ref).norm() / g_ref.norm()
    eb = (back - back_ref).norm() / back_ref.norm()
    assert float(eg) <= tol and float(eb) <= tol
