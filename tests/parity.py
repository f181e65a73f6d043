"""Error measures shared by the GPU parity tests.

Whole-field relative l2 errors are dominated by the large low-|m| orders, so
the all-order tests also take the relative error of every (field, order)
separately and bound its maximum: a wrong high-|m| order, whose values near
the poles are tiny, cannot hide inside the field's norm.
"""
import numpy as np


def field_err(a, b):
    """(F,) relative l2 error of each field over its whole output."""
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def order_err_values(a, b):
    """(F, 4N-1) relative l2 error of every (field, order) of ALT values
    shaped (F, 4N-1, 2N, 2); orders whose reference is zero are NaN."""
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.linalg.norm((a - b).reshape(a.shape[0], a.shape[1], -1), axis=2)
    r = np.linalg.norm(b.reshape(b.shape[0], b.shape[1], -1), axis=2)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(r > 0, d / r, np.nan)


def order_err_coefficients(a, b, N, denom=None):
    """(F, 4N-1) relative l2 error of every (field, order) of coefficients
    shaped (F, 4N^2, 2), orders in the storage sequence 0, 1, -1, 2, -2, ...
    (2N-|m| degrees each); orders whose reference is zero are NaN.  With
    `denom` ((F, 4N-1)), the error of each order is taken relative to it
    instead of the reference's norm."""
    a = np.asarray(a)
    b = np.asarray(b)
    lens = [2 * N] + [2 * N - am for am in range(1, 2 * N) for _ in (0, 1)]
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    dd = np.sum((a - b) ** 2, axis=2)
    d = np.sqrt(np.add.reduceat(dd, starts, axis=1))
    r = np.sqrt(np.add.reduceat(np.sum(b ** 2, axis=2), starts, axis=1)) if denom is None else np.asarray(denom)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(r > 0, d / r, np.nan)


def weighted_input_norms(g, w):
    """(F, 4N-1) norm sqrt(sum_l w_l |g(m, theta_l)|^2) of every (field, order)
    of ALT values g shaped (F, 4N-1, 2N, 2).  The inverse ALT of one order is
    the projection beta = A^T W g with A^T W A = I, so |beta| is at most this
    norm: for inputs outside the range of the forward transform (random g) the
    per-order error of the inverse is measured against it, since the output
    itself can be far smaller than its input."""
    g = np.asarray(g)
    return np.sqrt(np.einsum("fmlc,l->fm", g * g, np.asarray(w)))


def max_order_err(e):
    return float(np.nanmax(e))
