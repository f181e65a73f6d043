"""GPU parity of the dense ALT with the recurrence run on the fly
(SHT_FLAG_DIRECT plans) against the dense FP64 oracle.

Nothing is factored or stored: every call evaluates Pbar_k^{|m|} at the
positive nodes by the three-term recurrence, carried with a separate binary
exponent while the values are below the FP64 range, and contracts it with the
right-hand sides in FP64.  The result is the plain definition up to rounding,
so the bound is the FP64 one (1e-10 per field and per order, as for FP64
plans).  Orders near 2N-1 at N = 1024 start far below 2^-1074 at the outer
nodes: they exercise the extended exponent.
"""
import numpy as np
import pytest

import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, inputs
from parity import field_err, max_order_err, order_err_coefficients, order_err_values, weighted_input_norms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# N = 1 (two nodes, orders 0 and +-1), odd and even N, and a field count
# above max_fields (the calls run in chunks of max_fields fields)
@pytest.mark.parametrize("N", [1, 2, 5, 8, 33, 64])
def test_direct_forward_inverse_all_orders(N):
    F = 5
    p = sht.Plan(N, 1e-12, flags=_lib.SHT_FLAG_DIRECT, max_fields=2)
    beta = inputs.coefficients(N, F, seed=N)
    g = p.forward(dev(beta)).cpu().numpy()
    ref = oracle.alt_forward(N, beta)
    assert np.all(field_err(g, ref) <= TOL)
    assert max_order_err(order_err_values(g, ref)) <= TOL
    gin = np.random.default_rng(N + 1).standard_normal((F, 4 * N - 1, 2 * N, 2))
    b = p.inverse(dev(gin)).cpu().numpy()
    x, w = oracle.gl_rule(2 * N)
    refb = oracle.alt_inverse(N, gin, x, w)
    assert np.all(field_err(b, refb) <= TOL)
    # per order against the weighted input norm: random g is not in the range of the forward map
    assert max_order_err(order_err_coefficients(b, refb, N, denom=weighted_input_norms(gin, w))) <= TOL


def test_direct_headline_order_sampled_orders():
    """N = 1024, two fields, sampled orders across the range, both directions."""
    N, F = 1024, 2
    p = sht.Plan(N, 1e-12, flags=_lib.SHT_FLAG_DIRECT, max_fields=F)
    beta = inputs.coefficients(N, F, seed=11)
    g = p.forward(dev(beta))
    torch.cuda.synchronize()
    x, w = oracle.gl_rule(2 * N)
    ms = [0, 1, -1, 7, -300, 511, 1023, -1024, 1500, -1800, 2000, 2 * N - 2, -(2 * N - 1)]
    gin = torch.zeros_like(g)
    grefs = {}
    for m in ms:
        off = oracle.coef_offset(N, m)
        ref = oracle.alt_forward_m_fields(N, m, beta[:, off: off + 2 * N - abs(m)], x)
        got = g[:, oracle.order_slot(m)].cpu().numpy()
        e = np.linalg.norm((got - ref).reshape(F, -1), axis=1) / np.linalg.norm(ref.reshape(F, -1), axis=1)
        assert np.all(e <= TOL), (m, e)
        grefs[m] = ref
        gin[:, oracle.order_slot(m)] = torch.from_numpy(ref).cuda()
    b = p.inverse(gin).cpu().numpy()
    for m in ms:
        off = oracle.coef_offset(N, m)
        ref = oracle.alt_inverse_m_fields(N, m, grefs[m], x, w)
        got = b[:, off: off + 2 * N - abs(m)]
        e = np.linalg.norm((got - ref).reshape(F, -1), axis=1) / np.linalg.norm(ref.reshape(F, -1), axis=1)
        assert np.all(e <= TOL), (m, e)
        # and the inverse of the forward values gives beta back
        np.testing.assert_allclose(got, beta[:, off: off + 2 * N - abs(m)], rtol=0, atol=1e-10)


def test_direct_full_sht():
    N, F = 32, 3
    p = sht.Plan(N, 1e-12, flags=_lib.SHT_FLAG_DIRECT, max_fields=2)
    beta = inputs.coefficients(N, F, seed=4, real_m0=True)
    f = p.sht_forward(dev(beta)).cpu().numpy()
    assert np.all(field_err(f, oracle.sht_forward(N, beta)) <= TOL)
    b = p.sht_inverse(dev(f)).cpu().numpy()
    assert np.all(field_err(b, beta) <= TOL)
