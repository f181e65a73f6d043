"""The per-order error measures of the GPU parity tests (CPU)."""
import numpy as np

from parity import field_err, order_err_coefficients, order_err_values
from paper_2004_11346_gb300 import inputs


def test_order_err_values_finds_one_bad_order():
    rng = np.random.default_rng(0)
    N, F = 8, 3
    ref = rng.standard_normal((F, 4 * N - 1, 2 * N, 2))
    ref[:, -1] *= 1e-8  # a tiny high-|m| order
    got = ref.copy()
    got[1, -1] *= 1 + 1e-3  # wrong by 1e-3 of its own size, ~1e-11 of the field's
    assert field_err(got, ref).max() < 1e-9
    e = order_err_values(got, ref)
    assert e.shape == (F, 4 * N - 1)
    assert np.nanargmax(e) == np.ravel_multi_index((1, 4 * N - 2), e.shape)
    np.testing.assert_allclose(e[1, -1], 1e-3, rtol=1e-9)
    assert np.nanmax(np.delete(e.ravel(), np.nanargmax(e))) == 0.0


def test_order_err_coefficients_follows_the_storage_order():
    N, F = 6, 2
    beta = inputs.coefficients(N, F, seed=1)
    k, m = inputs.degree_index(N)
    got = beta.copy()
    sel = m == -(2 * N - 3)
    got[0, sel] *= 1 + 1e-4
    e = order_err_coefficients(got, beta, N)
    # storage sequence 0, 1, -1, 2, -2, ...: order -a sits at position 2a
    pos = 2 * (2 * N - 3)
    np.testing.assert_allclose(e[0, pos], 1e-4, rtol=1e-9)
    e[0, pos] = 0
    assert np.nanmax(e) == 0.0
