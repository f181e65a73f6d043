"""Pins of the dense FP64 oracle to facts outside itself (CPU only).

Each test checks the oracle against something the mathematics fixes:
library routines (numpy's Gauss-Legendre rule and FFT), closed forms, exact
rational evaluation of the Rodrigues formula, the addition theorem, discrete
orthonormality under the Gauss-Legendre rule (Sec. 3.1.1), the parity
symmetry of Sec. 3.1.2, and brute force in high precision on tiny N.
"""
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest

import oracle
from paper_2004_11346_gb300 import inputs

mp = pytest.importorskip("mpmath")


def pbar_exact(k: int, m: int, x: Fraction, dps: int = 60):
    """Pbar_k^m(x) from the Rodrigues formula with exact rational arithmetic.

    P_k(x) = 2^-k sum_j (-1)^j C(k,j) C(2k-2j,k) x^(k-2j) is differentiated
    m times term by term (exact integers), multiplied by (1-x^2)^(m/2) and by
    sqrt((2k+1)/2 (k-m)!/(k+m)!); no Condon-Shortley phase.
    """
    mp.mp.dps = dps
    s = Fraction(0)
    for j in range(0, (k - m) // 2 + 1):
        n = k - 2 * j
        s += (-1) ** j * comb(k, j) * comb(2 * k - 2 * j, k) * (factorial(n) // factorial(n - m)) * x ** (n - m)
    v = mp.mpf(s.numerator) / mp.mpf(s.denominator) / mp.mpf(2) ** k
    one = 1 - x * x
    v *= mp.sqrt(mp.mpf(one.numerator) / one.denominator) ** m
    v *= mp.sqrt(mp.mpf(2 * k + 1) / 2 * mp.factorial(k - m) / mp.factorial(k + m))
    return v


# ---------------------------------------------------------------- GL rule
@pytest.mark.parametrize("n", [1, 2, 3, 8, 64, 128, 255, 256])
def test_gl_rule_matches_numpy(n):
    x, w = oracle.gl_rule(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.all(np.diff(x) > 0)
    np.testing.assert_allclose(x, xr, rtol=0, atol=2e-15)
    # numpy's end weights carry up to ~1e-11 relative error of their own
    np.testing.assert_allclose(w, wr, rtol=1e-10, atol=0)


@pytest.mark.parametrize("n", [5, 64])
def test_gl_weights_high_precision(n):
    # w_i = 2 (1 - x_i^2) / (n P_{n-1}(x_i))^2 at the 40-digit roots of P_n
    mp.mp.dps = 40
    x, w = oracle.gl_rule(n)
    for i in range(n):
        z = mp.mpf(x[i])
        for _ in range(6):
            p0, p1 = mp.mpf(1), z
            for k in range(2, n + 1):
                p0, p1 = p1, ((2 * k - 1) * z * p1 - (k - 1) * p0) / k
            z -= p1 * (z * z - 1) / (n * (z * p1 - p0))
        p0, p1 = mp.mpf(1), z
        for k in range(2, n + 1):
            p0, p1 = p1, ((2 * k - 1) * z * p1 - (k - 1) * p0) / k
        wt = 2 * (1 - z * z) / (n * p0) ** 2
        assert abs(x[i] - z) < 1e-16
        assert abs(w[i] - wt) < 2e-13 * wt


@pytest.mark.parametrize("n", [128, 2048])
def test_gl_rule_moments_and_symmetry(n):
    x, w = oracle.gl_rule(n)
    assert abs(w.sum() - 2.0) < 1e-13
    np.testing.assert_allclose(x, -x[::-1], atol=1e-15)
    np.testing.assert_allclose(w, w[::-1], rtol=1e-12)
    # exact for polynomials of degree <= 2n-1: int x^{2j} = 2/(2j+1)
    for j in [1, 2, 5, 17, n // 2, n - 1]:
        assert abs(np.dot(w, x ** (2 * j)) - 2.0 / (2 * j + 1)) < 2e-13


# ---------------------------------------------------------------- Legendre functions
def test_alf_closed_forms():
    xs = np.array([-0.9, -0.3, 0.0, 0.5, 0.99])
    u = np.sqrt(1 - xs ** 2)
    ref = {
        (0, 0): np.full_like(xs, 1 / np.sqrt(2)),
        (1, 0): np.sqrt(1.5) * xs,
        (1, 1): np.sqrt(3) / 2 * u,
        (2, 0): np.sqrt(2.5) * (3 * xs ** 2 - 1) / 2,
        (2, 1): np.sqrt(15) / 2 * xs * u,
        (2, 2): np.sqrt(15) / 4 * u ** 2,
    }
    for m in range(3):
        t = oracle.alf_table(m, 2, xs)
        for k in range(m, 3):
            np.testing.assert_allclose(t[:, k - m], ref[(k, m)], rtol=1e-15, atol=1e-16)


@pytest.mark.parametrize("k,m,x", [
    (17, 5, Fraction(1, 3)),
    (300, 200, Fraction(7, 8)),
    (1000, 0, Fraction(5, 8)),
    (2047, 1, Fraction(-3, 4)),
    (2047, 1500, Fraction(3, 4)),
    (2047, 2000, Fraction(1, 2)),
    # sectoral start Pbar_700^700(15/16) ~ 4.8e-321 is below the FP64 normal
    # range; the value at k = 2047 is O(1): needs the extended exponent
    (2047, 700, Fraction(15, 16)),
    (2047, 1200, Fraction(31, 32)),
    # degrees of an N = 4096 transform: start Pbar_7000^7000(1/2) ~ 1e-437, far
    # outside FP64, value O(1); a value near the turning point; and one whose
    # exact size (~5e-2547) has no FP64 representation, so the oracle gives 0
    (8191, 7000, Fraction(1, 2)),
    (8191, 7800, Fraction(1, 3)),
    (8191, 7900, Fraction(9, 10)),
])
def test_alf_against_exact_rational(k, m, x):
    ref = pbar_exact(k, m, x)
    got = oracle.alf_table(m, k, [float(x)])[0, -1]
    assert abs(mp.mpf(got) - ref) <= 1e-12 * abs(ref) + 1e-300


def test_alf_extended_exponent_whole_column():
    # every degree of an order whose start underflows, against exact values
    m, x = 700, Fraction(15, 16)
    col = oracle.alf_table(m, 2047, [float(x)])[0]
    for k in [701, 760, 900, 1300, 1700, 2000]:
        ref = pbar_exact(k, m, x)
        # outputs below 2^-1022 are FP64 subnormals: one subnormal step of slack
        assert abs(mp.mpf(col[k - m]) - ref) <= 1e-12 * abs(ref) + 5e-324


@pytest.mark.parametrize("N", [8, 64])
def test_addition_theorem(N):
    # sum_{m=-k}^{k} Pbar_k^{|m|}(x)^2 = (2k+1)/2 at every node
    x, _ = oracle.gl_rule(2 * N)
    K = 2 * N
    acc = np.zeros((x.size, K))
    for m in range(K):
        t = oracle.alf_table(m, K - 1, x)
        acc[:, m:] += (1.0 if m == 0 else 2.0) * t ** 2
    ref = (2 * np.arange(K) + 1) / 2.0
    np.testing.assert_allclose(acc, np.broadcast_to(ref, acc.shape), rtol=1e-13)


@pytest.mark.parametrize("N", [4, 16, 64])
def test_discrete_orthonormality(N):
    # A_m^T W A_m = I: the 2N-point rule integrates the products exactly (Sec. 3.1.1)
    x, w = oracle.gl_rule(2 * N)
    for m in list(range(0, 2 * N, max(1, N // 8))) + [2 * N - 1]:
        A = oracle.alf_table(m, 2 * N - 1, x)
        G = A.T @ (w[:, None] * A)
        np.testing.assert_allclose(G, np.eye(G.shape[0]), atol=5e-14)


# ---------------------------------------------------------------- ALT
def test_alt_forward_bruteforce_high_precision():
    # tiny N: the definition evaluated in 40-digit arithmetic from exact Pbar
    N = 3
    beta = inputs.coefficients(N, 1, seed=3)
    x, _ = oracle.gl_rule(2 * N)
    g = oracle.alt_forward(N, beta, x)
    for m in range(-(2 * N - 1), 2 * N):
        off = oracle.coef_offset(N, m)
        slot = oracle.order_slot(m)
        for l in range(2 * N):
            xl = Fraction(x[l])
            re = mp.mpf(0)
            im = mp.mpf(0)
            for k in range(abs(m), 2 * N):
                p = pbar_exact(k, abs(m), xl, dps=40)
                re += mp.mpf(beta[0, off + k - abs(m), 0]) * p
                im += mp.mpf(beta[0, off + k - abs(m), 1]) * p
            assert abs(g[0, slot, l, 0] - float(re)) < 1e-14
            assert abs(g[0, slot, l, 1] - float(im)) < 1e-14


def test_layout_offsets():
    N = 5
    k, m = inputs.degree_index(N)
    assert k.size == 4 * N * N
    for mm in range(-(2 * N - 1), 2 * N):
        off = oracle.coef_offset(N, mm)
        assert m[off] == mm and k[off] == abs(mm)
        assert oracle.order_slot(mm) == list(inputs.order_sequence(N)).index(mm)


@pytest.mark.parametrize("N", [4, 32])
def test_alt_round_trip(N):
    beta = inputs.coefficients(N, 2, seed=1)
    g = oracle.alt_forward(N, beta)
    back = oracle.alt_inverse(N, g)
    np.testing.assert_allclose(back, beta, atol=2e-13)


def test_alt_inverse_is_weighted_transpose():
    # <inv(g), b> = sum_l w_l <g_l, (A b)_l>  for real b and g (B = A^T W)
    N = 16
    rng = np.random.default_rng(7)
    x, w = oracle.gl_rule(2 * N)
    b = rng.standard_normal((1, 4 * N * N, 2))
    g = rng.standard_normal((1, 4 * N - 1, 2 * N, 2))
    lhs = np.sum(oracle.alt_inverse(N, g) * b)
    rhs = np.sum(w[None, None, :, None] * g * oracle.alt_forward(N, b))
    assert abs(lhs - rhs) < 1e-11 * abs(rhs)


def test_alt_single_order_matches_batched():
    N = 16
    beta = inputs.coefficients(N, 1, seed=2)
    x, w = oracle.gl_rule(2 * N)
    g = oracle.alt_forward(N, beta, x)
    for m in [0, 3, -3, 31, -31]:
        off = oracle.coef_offset(N, m)
        gm = oracle.alt_forward_m(N, m, beta[0, off: off + 2 * N - abs(m)], x)
        np.testing.assert_array_equal(gm, g[0, oracle.order_slot(m)])
        bm = oracle.alt_inverse_m(N, m, gm, x, w)
        np.testing.assert_allclose(bm, beta[0, off: off + 2 * N - abs(m)], atol=1e-13)


def test_alt_m_fields_match_single_field_calls():
    # the many-field helpers are the same sums as the per-field definitions
    N = 24
    x, w = oracle.gl_rule(2 * N)
    rng = np.random.default_rng(12)
    for m in [0, 5, -5, 2 * N - 1, -(2 * N - 1)]:
        bm = rng.standard_normal((3, 2 * N - abs(m), 2))
        got = oracle.alt_forward_m_fields(N, m, bm, x)
        ref = np.stack([oracle.alt_forward_m(N, m, bm[f], x) for f in range(3)])
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
        gm = rng.standard_normal((3, 2 * N, 2))
        got = oracle.alt_inverse_m_fields(N, m, gm, x, w)
        ref = np.stack([oracle.alt_inverse_m(N, m, gm[f], x, w) for f in range(3)])
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_parity_symmetry():
    # Sec. 3.1.2: terms with k-|m| even are even in x, odd ones odd in x
    N = 16
    beta = inputs.coefficients(N, 1, seed=4)
    k, m = inputs.degree_index(N)
    even = beta.copy()
    even[0, (k - np.abs(m)) % 2 == 1] = 0
    odd = beta - even
    ge = oracle.alt_forward(N, even)
    go = oracle.alt_forward(N, odd)
    np.testing.assert_allclose(ge, ge[:, :, ::-1], atol=1e-13)
    np.testing.assert_allclose(go, -go[:, :, ::-1], atol=1e-13)


# ---------------------------------------------------------------- phi direction
def _phi_synthesis_fft(N, g):
    M = 4 * N - 1
    f = np.zeros((g.shape[0], 2 * N, M), dtype=complex)
    gc = g[..., 0] + 1j * g[..., 1]
    for mm in range(-(2 * N - 1), 2 * N):
        c = gc[:, oracle.order_slot(mm), :] * np.exp(1j * np.pi * mm / M)
        spec = np.zeros((g.shape[0], 2 * N, M), dtype=complex)
        spec[:, :, mm % M] = c
        f += np.fft.ifft(spec, axis=-1) * M
    return np.stack([f.real, f.imag], axis=-1)


def test_phi_synthesis_matches_fft():
    N = 6
    rng = np.random.default_rng(5)
    g = rng.standard_normal((2, 4 * N - 1, 2 * N, 2))
    f = oracle.phi_synthesis(N, g)
    np.testing.assert_allclose(f, _phi_synthesis_fft(N, g), atol=1e-12)


def test_phi_round_trip():
    N = 8
    rng = np.random.default_rng(6)
    g = rng.standard_normal((1, 4 * N - 1, 2 * N, 2))
    np.testing.assert_allclose(oracle.phi_analysis(N, oracle.phi_synthesis(N, g)), g, atol=1e-13)


def _phi_analysis_fft(N, f):
    """(1/M) sum_j f e^{-i m phi_j} = e^{-i pi m / M} FFT(f)[m mod M] / M."""
    M = 4 * N - 1
    F = np.fft.fft(f[..., 0] + 1j * f[..., 1], axis=-1) / M  # (F, rows, M)
    g = np.zeros((f.shape[0], M, f.shape[1]), dtype=complex)
    for mm in range(-(2 * N - 1), 2 * N):
        g[:, oracle.order_slot(mm), :] = F[:, :, mm % M] * np.exp(-1j * np.pi * mm / M)
    return np.stack([g.real, g.imag], axis=-1)


def test_phi_nodes_match_fft():
    # the node-subset sums against numpy's FFT at chosen nodes, both directions
    N = 7
    rng = np.random.default_rng(8)
    g = rng.standard_normal((2, 4 * N - 1, 2 * N, 2))
    nodes = [0, 3, 13]
    f = oracle.phi_synthesis_nodes(N, g[:, :, nodes])
    np.testing.assert_allclose(f, _phi_synthesis_fft(N, g)[:, nodes], atol=1e-12)
    frows = rng.standard_normal((2, 3, 4 * N - 1, 2))
    np.testing.assert_allclose(oracle.phi_analysis_nodes(N, frows), _phi_analysis_fft(N, frows), atol=1e-13)
    # and a subset of the full sums is the node-subset sum (same arithmetic)
    np.testing.assert_array_equal(f, oracle.phi_synthesis(N, g)[:, nodes])


def test_sht_round_trip():
    N = 8
    beta = inputs.coefficients(N, 1, seed=0, real_m0=True)
    f = oracle.sht_forward(N, beta)
    np.testing.assert_allclose(oracle.sht_inverse(N, f), beta, atol=1e-12)
