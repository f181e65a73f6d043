"""GPU parity of the FP64 IDBF ALT against the dense FP64 oracle.

Calls the library through its C ABI (ctypes binding) on device buffers and
compares element by element with the oracle on the same seeded inputs.
Tolerance: relative l2 error per field <= 1e-10 at eps = 1e-12 (the FP64
path's target), on the whole output of every field.
"""
import numpy as np
import pytest

import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, inputs
from parity import max_order_err, order_err_coefficients, order_err_values, weighted_input_norms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


def rel_err(a, b, axis=None):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


PLANS = {
    "N64_default": (64, {}),
    "N64_forced_idbf": (64, dict(n0=16, n_leaf=8, flags=_lib.SHT_FLAG_FORCE_FACTOR)),
    "N96_forced_idbf": (96, dict(n0=16, n_leaf=8, flags=_lib.SHT_FLAG_FORCE_FACTOR)),
}


@pytest.fixture(scope="module")
def plans():
    return {k: sht.Plan(N, 1e-12, **kw) for k, (N, kw) in PLANS.items()}


@pytest.mark.parametrize("name", list(PLANS))
def test_forward_all_orders(plans, name):
    p = plans[name]
    N = p.N
    F = 3
    beta = inputs.coefficients(N, F, seed=0, real_m0=True)
    g = p.forward(dev(beta))
    torch.cuda.synchronize()
    p.sync()
    ref = oracle.alt_forward(N, beta)
    got = g.cpu().numpy()
    err = rel_err(got, ref)
    assert np.all(err <= TOL_FP64), err
    # every (field, order) on its own, not only the field's norm
    eo = order_err_values(got, ref)
    assert max_order_err(eo) <= TOL_FP64, np.unravel_index(np.nanargmax(eo), eo.shape)


@pytest.mark.parametrize("name", list(PLANS))
def test_inverse_all_orders(plans, name):
    p = plans[name]
    N = p.N
    F = 2
    rng = np.random.default_rng(11)
    g = rng.standard_normal((F, 4 * N - 1, 2 * N, 2))
    beta = p.inverse(dev(g))
    torch.cuda.synchronize()
    ref = oracle.alt_inverse(N, g)
    got = beta.cpu().numpy()
    err = rel_err(got, ref)
    assert np.all(err <= TOL_FP64), err
    # random g lies outside the forward's range: per order, relative to the input's W-norm
    _, wts = oracle.gl_rule(2 * N)
    eo = order_err_coefficients(got, ref, N, denom=weighted_input_norms(g, wts))
    assert max_order_err(eo) <= TOL_FP64, np.unravel_index(np.nanargmax(eo), eo.shape)


def test_round_trip(plans):
    p = plans["N64_forced_idbf"]
    N = p.N
    beta = inputs.coefficients(N, 2, seed=5)
    back = p.inverse(p.forward(dev(beta)))
    torch.cuda.synchronize()
    assert np.all(rel_err(back.cpu().numpy(), beta) <= TOL_FP64)


@pytest.mark.parametrize("m", [0, 1, -1, 7, -8, 63, -64, 127, -127])
def test_single_order(plans, m):
    p = plans["N64_forced_idbf"]
    N = p.N
    F = 2
    rng = np.random.default_rng(abs(m) + 3)
    bm = rng.standard_normal((F, 2 * N - abs(m), 2))
    x, w = oracle.gl_rule(2 * N)
    gm = p.forward_m(m, dev(bm))
    torch.cuda.synchronize()
    ref = np.stack([oracle.alt_forward_m(N, m, bm[f], x) for f in range(F)])
    assert np.all(rel_err(gm.cpu().numpy(), ref) <= TOL_FP64)
    gin = rng.standard_normal((F, 2 * N, 2))
    bo = p.inverse_m(m, dev(gin))
    torch.cuda.synchronize()
    ref = np.stack([oracle.alt_inverse_m(N, m, gin[f], x, w) for f in range(F)])
    assert np.all(rel_err(bo.cpu().numpy(), ref) <= TOL_FP64)


def test_single_order_matches_batched(plans):
    p = plans["N96_forced_idbf"]
    N = p.N
    beta = inputs.coefficients(N, 1, seed=9)
    g = p.forward(dev(beta)).cpu().numpy()[0]
    for m in [0, 5, -5, 2 * N - 1, -(2 * N - 1)]:
        off = oracle.coef_offset(N, m)
        gm = p.forward_m(m, dev(beta[:, off: off + 2 * N - abs(m)])).cpu().numpy()[0]
        # output rows shared by several blocks are summed with atomics, whose
        # order (and so the last bit) varies between launches
        np.testing.assert_allclose(gm, g[oracle.order_slot(m)], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_tiny_orders(N):
    p = sht.Plan(N, 1e-12)
    beta = inputs.coefficients(N, 2, seed=N)
    g = p.forward(dev(beta)).cpu().numpy()
    assert np.all(rel_err(g, oracle.alt_forward(N, beta)) <= TOL_FP64)
    b = p.inverse(dev(g)).cpu().numpy()
    assert np.all(rel_err(b, oracle.alt_inverse(N, g)) <= TOL_FP64)


def test_empty_batch_and_bad_arguments(plans):
    p = plans["N64_default"]
    N = p.N
    z = torch.empty((0, 4 * N * N, 2), dtype=torch.float64, device="cuda")
    out = p.forward(z)
    assert out.shape[0] == 0
    with pytest.raises(_lib.ShtError):
        _lib.alt_forward_m(p.handle, 2 * N, z.data_ptr(), z.data_ptr(), 1, 0)
    with pytest.raises(_lib.ShtError):
        _lib.alt_forward(p.handle, 0, 0, 1, 0)
    with pytest.raises(_lib.ShtError):
        sht.Plan(0, 1e-12)
    with pytest.raises(_lib.ShtError):
        sht.Plan(16, 0.0)


def test_stream_ordering():
    # work queued on a side stream is ordered with that stream only
    p = sht.Plan(32, 1e-12)
    N = 32
    beta = inputs.coefficients(N, 4, seed=2)
    s = torch.cuda.Stream()
    b = dev(beta)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        g = p.forward(b)
        back = p.inverse(g)
    s.synchronize()
    assert np.all(rel_err(back.cpu().numpy(), beta) <= TOL_FP64)


@pytest.mark.slow
def test_N1024_fp64_sampled_orders():
    """Full-size FP64 workload: 1 field, coefficients N(0,1)(k+1)^-1, eps=1e-12.

    The whole forward and inverse run on the GPU; the oracle recomputes a
    sample of orders (all 2N nodes of each) one by one.
    """
    N = 1024
    p = sht.Plan(N, 1e-12)
    beta = inputs.workload_coefficients("fp64_N1024")
    g = p.forward(dev(beta)).cpu().numpy()[0]
    x, w = oracle.gl_rule(2 * N)
    for m in [0, 1, -2, 300, -511, 1024, -1500, 2046, -2047]:
        off = oracle.coef_offset(N, m)
        ref = oracle.alt_forward_m(N, m, beta[0, off: off + 2 * N - abs(m)], x)
        e = np.linalg.norm(g[oracle.order_slot(m)] - ref) / np.linalg.norm(ref)
        assert e <= TOL_FP64, (m, e)
    b = p.inverse(dev(g[None])).cpu().numpy()[0]
    for m in [0, 3, -700, 2047]:
        off = oracle.coef_offset(N, m)
        ref = oracle.alt_inverse_m(N, m, g[oracle.order_slot(m)], x, w)
        e = np.linalg.norm(b[off: off + 2 * N - abs(m)] - ref) / np.linalg.norm(ref)
        assert e <= TOL_FP64, (m, e)
