"""The device Legendre recurrence (sht_legendre) against the oracle's table,
and plans whose builder takes its Legendre matrices from the device
(SHT_FLAG_GPU_LEGENDRE) against the oracle's transform.

The device writes values below 2^-760 as 0, so the comparison bounds the
absolute error against the largest value of each order's table and the
relative error of every value above 1e-200 of that largest value.
"""
import numpy as np
import pytest

import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, inputs
from parity import field_err, max_order_err, order_err_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("N,orders", [(8, list(range(16))), (64, [0, 1, 2, 31, 63, 64, 100, 127]),
                                      (1024, [0, 1, 513, 1024, 1500, 1900, 2046, 2047])])
def test_device_table_matches_the_oracle(N, orders):
    p = sht.Plan(N, 1e-12, flags=_lib.SHT_FLAG_DIRECT)
    x, _ = oracle.gl_rule(2 * N)
    xp = x[N:]
    for am in orders:
        got = p.legendre(am).cpu().numpy()          # (2N - am, N): degree-major
        ref = oracle.alf_table(am, 2 * N - 1, xp).T  # (2N - am, N)
        big = np.abs(ref).max()
        # two FP64 forward recurrences with different rounding (the oracle's
        # plain sequence, the device's fused multiply-adds and coefficient
        # table) drift apart by up to a small multiple of k eps max|Pbar| in
        # absolute terms after k steps: bounds proportional to the 2N steps
        steps = 2 * N
        assert np.abs(got - ref).max() <= steps * 2e-14 * big, am
        a = np.abs(ref)
        large = a >= 0.05 * big
        assert np.max(np.abs(got[large] - ref[large]) / a[large]) <= steps * 4e-13, am
        # before the turning point the values grow monotonically from far below
        # the FP64 range (the separate exponent's region): there the error
        # stays relative to each value
        tiny = (a > 1e-200 * big) & (a < 1e-12 * big)
        if np.any(tiny):
            assert np.max(np.abs(got[tiny] - ref[tiny]) / a[tiny]) <= steps * 1e-13, am


def test_plan_built_from_device_legendre_fp64():
    N, F = 64, 3
    host = sht.Plan(N, 1e-12, n0=16, n_leaf=8)
    dev = sht.Plan(N, 1e-12, n0=16, n_leaf=8, flags=_lib.SHT_FLAG_GPU_LEGENDRE)
    sh, sd = host.stats(), dev.stats()
    # the same partition and nearly the same factorisation (values agree to rounding)
    assert abs(sd["entries_total"] - sh["entries_total"]) <= 0.01 * sh["entries_total"]
    assert sd["n_blocks_idbf"] + sd["n_blocks_dense"] > 0
    beta = inputs.coefficients(N, F, seed=9)
    g = dev.forward(torch.from_numpy(beta).cuda()).cpu().numpy()
    ref = oracle.alt_forward(N, beta)
    assert np.all(field_err(g, ref) <= 1e-10)
    assert max_order_err(order_err_values(g, ref)) <= 1e-10
    b = dev.inverse(torch.from_numpy(ref).cuda()).cpu().numpy()
    assert np.all(field_err(b, beta) <= 1e-10)


def test_plan_built_from_device_legendre_mixed():
    N, F = 256, 8
    p = sht.Plan(N, 1e-7, precision=_lib.SHT_MIXED, max_fields=F, flags=_lib.SHT_FLAG_GPU_LEGENDRE)
    beta = inputs.coefficients(N, F, seed=10)
    g = p.forward(torch.from_numpy(beta).cuda())
    torch.cuda.synchronize()
    p.sync()
    ref = oracle.alt_forward(N, beta)
    assert np.all(field_err(g.cpu().numpy(), ref) <= 1e-6)


def test_legendre_arguments():
    p = sht.Plan(8, 1e-12, flags=_lib.SHT_FLAG_DIRECT)
    buf = torch.empty(16 * 8, dtype=torch.float64, device="cuda")
    for am in (-1, 16):
        with pytest.raises(_lib.ShtError) as e:
            _lib.sht_legendre(p.handle, am, buf.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert e.value.status == _lib.SHT_ERR_ARG
