"""Batches of plans of different orders N in one launch (sht_batch_create).

Each plan's fields in a batch must give what the plan gives on its own: the
oracle's ALT within the mixed-precision tolerance, and the single-plan
tensor-core path to within the reordering of its FP32 accumulations.
"""
import numpy as np
import pytest

import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6


def rel_err(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


# uneven orders and field counts: one field group, a full group plus one
# field, a partial group; forced factorisation gives every op kind at small N
SIZES = [(24, 3, dict(n0=8, n_leaf=4, flags=_lib.SHT_FLAG_FORCE_FACTOR)), (40, 33, dict()),
         (64, 7, dict(n0=16, n_leaf=8))]


@pytest.fixture(scope="module")
def plans():
    return [sht.Plan(N, 1e-7, precision=_lib.SHT_MIXED, max_fields=40, **kw) for N, _, kw in SIZES]


@pytest.fixture(scope="module")
def batch(plans):
    return sht.Batch(plans, [F for _, F, _ in SIZES])


def test_forward_matches_oracle_and_single_plan(plans, batch):
    betas = [inputs.coefficients(N, F, seed=10 + N) for N, F, _ in SIZES]
    gs = batch.forward([dev(b) for b in betas])
    torch.cuda.synchronize()
    batch.sync()
    for p, (N, F, _), beta, g in zip(plans, SIZES, betas, gs):
        got = g.cpu().numpy()
        assert np.all(rel_err(got, oracle.alt_forward(N, beta)) <= TOL_MIXED), N
        alone = p.forward(dev(beta))
        torch.cuda.synchronize()
        assert np.all(rel_err(got, alone.cpu().numpy()) <= 1e-6), N


def test_inverse_matches_oracle(plans, batch):
    rng = np.random.default_rng(5)
    gs = [rng.standard_normal((F, 4 * N - 1, 2 * N, 2)) for N, F, _ in SIZES]
    bs = batch.inverse([dev(g) for g in gs])
    torch.cuda.synchronize()
    batch.sync()
    for (N, F, _), g, b in zip(SIZES, gs, bs):
        assert np.all(rel_err(b.cpu().numpy(), oracle.alt_inverse(N, g)) <= TOL_MIXED), N


def test_plan_without_fields(plans):
    b = sht.Batch(plans, [0, 2, 0])
    N = SIZES[1][0]
    beta = inputs.coefficients(N, 2, seed=4)
    out = b.forward([None, dev(beta), None])
    torch.cuda.synchronize()
    b.sync()
    assert out[0] is None and out[2] is None
    assert np.all(rel_err(out[1].cpu().numpy(), oracle.alt_forward(N, beta)) <= TOL_MIXED)


def test_sht_round_trip(plans, batch):
    betas = [inputs.coefficients(N, F, seed=20 + N) for N, F, _ in SIZES]
    fs = batch.sht_forward([dev(b) for b in betas])
    back = batch.sht_inverse(fs)
    torch.cuda.synchronize()
    batch.sync()
    for (N, F, _), beta, f, bb in zip(SIZES, betas, fs, back):
        assert np.all(rel_err(f.cpu().numpy(), oracle.sht_forward(N, beta)) <= TOL_MIXED), N
        assert np.all(rel_err(bb.cpu().numpy(), beta) <= 2 * TOL_MIXED), N


def test_graph_replay(plans, batch):
    betas = [dev(inputs.coefficients(N, F, seed=30 + N)) for N, F, _ in SIZES]
    ref = [g.clone() for g in batch.forward(betas)]
    torch.cuda.synchronize()
    ins = [b.data_ptr() for b in betas]
    outs = [torch.zeros_like(g) for g in ref]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        _lib.alt_forward_batch(batch.handle, ins, [o.data_ptr() for o in outs], s.cuda_stream)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        _lib.alt_forward_batch(batch.handle, ins, [o.data_ptr() for o in outs],
                               torch.cuda.current_stream().cuda_stream)
    for o in outs:
        o.zero_()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    batch.sync()
    for o, r in zip(outs, ref):
        assert float((o - r).norm() / r.norm()) <= 1e-6


def test_argument_errors(plans):
    with pytest.raises(_lib.ShtError) as e:
        _lib.sht_batch_create([plans[0].handle, plans[0].handle], [1, 1])
    assert e.value.status == _lib.SHT_ERR_ARG
    with pytest.raises(_lib.ShtError) as e:
        _lib.sht_batch_create([plans[0].handle], [41])  # above the plan's max_fields
    assert e.value.status == _lib.SHT_ERR_ARG
    p64 = sht.Plan(16, 1e-12)
    with pytest.raises(_lib.ShtError) as e:
        _lib.sht_batch_create([p64.handle], [1])
    assert e.value.status == _lib.SHT_ERR_UNSUPPORTED
