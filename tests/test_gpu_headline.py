"""GPU parity of the benchmarked configuration against the dense FP64 oracle.

The plan is exactly the one bench.py times by default: N = 1024, eps = 1e-7,
the tensor-core path (SHT_MIXED) with the partition stop size and leaf size
of the workload ``mixed_N1024_F64`` (n0 = n_leaf = 256), workspace for 64
fields, and that workload's 64 seeded N(0,1) fields.

The oracle cannot afford all 4095 orders x 64 fields here, so every field is
checked at a set of orders that spans the transform: m = 0, +-1, the last
order +-(2N-1), and orders on both sides of and across the turning-point
region of the partition (Eq. new5).  At each (field, order) the relative l2
error must be <= 1e-6, forward (beta -> g, Eq. sht_lt) and inverse
(g -> beta, Sec. 3.1.1).  The inverse is fed the oracle's own forward values
at the sampled orders (zero elsewhere: an order's output depends only on its
own input row).
"""
import numpy as np
import pytest

import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6
WORKLOAD = "mixed_N1024_F64"


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def sampled_orders(N):
    a = [0, 1, 7, 100, 300, N // 2 - 1, N // 2, 700, N - 1, N, N + 1, 1500, 1800, 2 * N - 2, 2 * N - 1]
    ms = []
    for v in a:
        ms += [v, -v] if v else [0]
    return ms


def per_order_err(got, ref):
    """(F,) relative l2 error of each field at one order."""
    d = (got - ref).reshape(got.shape[0], -1)
    return np.linalg.norm(d, axis=1) / np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1)


@pytest.fixture(scope="module")
def headline():
    w = inputs.WORKLOADS[WORKLOAD]
    N, F = w["N"], w["F"]
    plan = sht.Plan(N, w["eps"], precision=_lib.SHT_MIXED, max_fields=F, **w["plan"])
    beta = inputs.workload_coefficients(WORKLOAD)
    x, wts = oracle.gl_rule(2 * N)
    return plan, beta, x, wts


def test_forward_every_field_sampled_orders(headline):
    plan, beta, x, _ = headline
    N, F = plan.N, beta.shape[0]
    g = plan.forward(torch.from_numpy(beta).cuda())
    torch.cuda.synchronize()
    plan.sync()
    worst = 0.0
    for m in sampled_orders(N):
        off = oracle.coef_offset(N, m)
        ref = oracle.alt_forward_m_fields(N, m, beta[:, off: off + 2 * N - abs(m)], x)
        got = g[:, oracle.order_slot(m)].cpu().numpy()
        err = per_order_err(got, ref)
        worst = max(worst, float(err.max()))
        assert np.all(err <= TOL_MIXED), (m, err.max(), int(err.argmax()))
    print(f"forward: max per-(field, order) rel err {worst:.3e} over {len(sampled_orders(N))} orders x {F} fields")


def test_inverse_every_field_sampled_orders(headline):
    plan, beta, x, wts = headline
    N, F = plan.N, beta.shape[0]
    ms = sampled_orders(N)
    g = torch.zeros((F, 4 * N - 1, 2 * N, 2), dtype=torch.float64, device="cuda")
    gref = {}
    for m in ms:
        off = oracle.coef_offset(N, m)
        gref[m] = oracle.alt_forward_m_fields(N, m, beta[:, off: off + 2 * N - abs(m)], x)
        g[:, oracle.order_slot(m)] = torch.from_numpy(gref[m]).cuda()
    b = plan.inverse(g)
    torch.cuda.synchronize()
    plan.sync()
    worst = 0.0
    for m in ms:
        off = oracle.coef_offset(N, m)
        ref = oracle.alt_inverse_m_fields(N, m, gref[m], x, wts)
        got = b[:, off: off + 2 * N - abs(m)].cpu().numpy()
        err = per_order_err(got, ref)
        worst = max(worst, float(err.max()))
        assert np.all(err <= TOL_MIXED), (m, err.max(), int(err.argmax()))
        # and the oracle's inverse of its own forward values gives back beta
        # (FP64 sums over 2N = 2048 nodes: round-off of order 1e-11)
        np.testing.assert_allclose(ref, beta[:, off: off + 2 * N - abs(m)], rtol=0, atol=1e-10)
    print(f"inverse: max per-(field, order) rel err {worst:.3e} over {len(ms)} orders x {F} fields")
