"""GPU parity of the many-field FP32 path against the dense FP64 oracle.

Plans at eps = 1e-7 with FP32 factors and FP32 arithmetic (FP64 inputs and
outputs).  Tolerance: relative l2 error per field <= 1e-6.  The gpu-marked
dense-plan test covers the unfactored baseline with both kernels.
"""
import numpy as np
import pytest

import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, inputs
from parity import max_order_err, order_err_coefficients, order_err_values, weighted_input_norms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6
TOL_FP64 = 1e-10


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


PLANS = {
    "N64_fp32": (64, dict(precision=_lib.SHT_FP32)),
    "N96_fp32_forced": (96, dict(precision=_lib.SHT_FP32, n0=16, n_leaf=8, flags=_lib.SHT_FLAG_FORCE_FACTOR)),
    "N128_mixed": (128, dict(precision=_lib.SHT_MIXED, n0=32, n_leaf=16)),
    "N96_mixed_forced": (96, dict(precision=_lib.SHT_MIXED, n0=16, n_leaf=8, flags=_lib.SHT_FLAG_FORCE_FACTOR)),
    "N200_mixed": (200, dict(precision=_lib.SHT_MIXED)),
}


@pytest.fixture(scope="module")
def plans():
    return {k: sht.Plan(N, 1e-7, **kw) for k, (N, kw) in PLANS.items()}


@pytest.mark.parametrize("name", list(PLANS))
@pytest.mark.parametrize("F", [1, 8, 11, 40])
def test_forward(plans, name, F):
    p = plans[name]
    N = p.N
    beta = inputs.coefficients(N, F, seed=F)
    g = p.forward(dev(beta))
    torch.cuda.synchronize()
    p.sync()
    got, ref = g.cpu().numpy(), oracle.alt_forward(N, beta)
    err = rel_err(got, ref)
    assert np.all(err <= TOL_MIXED), err
    # every (field, order) on its own, not only the field's norm
    eo = order_err_values(got, ref)
    assert max_order_err(eo) <= TOL_MIXED, np.unravel_index(np.nanargmax(eo), eo.shape)


@pytest.mark.parametrize("name", list(PLANS))
def test_inverse(plans, name):
    p = plans[name]
    N = p.N
    F = 9
    g = np.random.default_rng(3).standard_normal((F, 4 * N - 1, 2 * N, 2))
    b = p.inverse(dev(g))
    torch.cuda.synchronize()
    got, ref = b.cpu().numpy(), oracle.alt_inverse(N, g)
    err = rel_err(got, ref)
    assert np.all(err <= TOL_MIXED), err
    # random g lies outside the forward's range: per order, relative to the input's W-norm
    _, wts = oracle.gl_rule(2 * N)
    eo = order_err_coefficients(got, ref, N, denom=weighted_input_norms(g, wts))
    assert max_order_err(eo) <= TOL_MIXED, np.unravel_index(np.nanargmax(eo), eo.shape)


@pytest.mark.parametrize("m", [0, 3, -3, 191, -191])
@pytest.mark.parametrize("name", ["N96_fp32_forced", "N96_mixed_forced"])
def test_single_order(plans, m, name):
    p = plans[name]
    N = p.N
    F = 10
    rng = np.random.default_rng(abs(m))
    x, w = oracle.gl_rule(2 * N)
    bm = rng.standard_normal((F, 2 * N - abs(m), 2))
    gm = p.forward_m(m, dev(bm))
    torch.cuda.synchronize()
    ref = np.stack([oracle.alt_forward_m(N, m, bm[f], x) for f in range(F)])
    assert np.all(rel_err(gm.cpu().numpy(), ref) <= TOL_MIXED)
    gi = rng.standard_normal((F, 2 * N, 2))
    bo = p.inverse_m(m, dev(gi))
    torch.cuda.synchronize()
    ref = np.stack([oracle.alt_inverse_m(N, m, gi[f], x, w) for f in range(F)])
    assert np.all(rel_err(bo.cpu().numpy(), ref) <= TOL_MIXED)


@pytest.mark.parametrize("prec,tol", [(_lib.SHT_FP64, TOL_FP64), (_lib.SHT_FP32, TOL_MIXED),
                                      (_lib.SHT_MIXED, TOL_MIXED)])
def test_dense_plan(prec, tol):
    N = 48
    p = sht.Plan(N, 1e-12, precision=prec, flags=_lib.SHT_FLAG_DENSE)
    st = p.stats()
    assert st["entries_total"] == st["entries_matrix"] and st["n_blocks_idbf"] == 0
    beta = inputs.coefficients(N, 3, seed=1)
    g = p.forward(dev(beta))
    b = p.inverse(g)
    torch.cuda.synchronize()
    assert np.all(rel_err(g.cpu().numpy(), oracle.alt_forward(N, beta)) <= tol)
    assert np.all(rel_err(b.cpu().numpy(), beta) <= tol)


@pytest.mark.slow
def test_N1024_mixed_64_fields_sampled():
    """Headline workload: N=1024, eps=1e-7, 64 fields N(0,1), FP32 path.

    Every field's output at a sample of orders is recomputed by the oracle."""
    N, F = 1024, 64
    p = sht.Plan(N, 1e-7, precision=_lib.SHT_MIXED)
    beta = inputs.workload_coefficients("mixed_N1024_F64")
    g = p.forward(dev(beta)).cpu().numpy()
    x, _ = oracle.gl_rule(2 * N)
    for m in [0, 7, -300, 1024, -2047]:
        off = oracle.coef_offset(N, m)
        for f in range(0, F, 9):
            ref = oracle.alt_forward_m(N, m, beta[f, off: off + 2 * N - abs(m)], x)
            e = np.linalg.norm(g[f, oracle.order_slot(m)] - ref) / np.linalg.norm(ref)
            assert e <= TOL_MIXED, (m, f, e)
