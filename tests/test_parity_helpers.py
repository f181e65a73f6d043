"""The per-order error measures of the GPU parity tests (CPU)."""
import numpy as np

from parity import field_err, order_err_coefficients, order_err_values, weighted_input_norms
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


def test_weighted_input_norms_bound_the_inverse():
    # |A_m^T W g| <= |W^(1/2) g| for every order (A^T W A = I): the denominator
    # the inverse tests use is never below the reference output
    import oracle
    N = 8
    rng = np.random.default_rng(3)
    g = rng.standard_normal((2, 4 * N - 1, 2 * N, 2))
    x, w = oracle.gl_rule(2 * N)
    beta = oracle.alt_inverse(N, g, x, w)
    wn = weighted_input_norms(g, w)
    e = order_err_coefficients(np.zeros_like(beta), beta, N, denom=wn)
    assert e.shape == (2, 4 * N - 1) and np.all(e <= 1 + 1e-12)
    # and the plain relative error of zero output is exactly one
    np.testing.assert_allclose(order_err_coefficients(np.zeros_like(beta), beta, N), 1.0)
