"""Dense FP64 CPU oracle for the ALT / SHT (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The library's product path never does:
the oracle shares no code, headers or tables with the CUDA path.

Every function here is the plain definition of the map it computes
(arXiv:2004.11346, Eq. sht_re, Eq. sht_lt, Eq. sht_fft, Sec. 3.1.1), in FP64,
with no parity folding, blocking or factorisation.  The C source is
``oracle/oracle.c``; it is compiled with ``-ffp-contract=off`` so that every
product is rounded on its own.

Array layouts (complex numbers as trailing axis of size 2, float64):
  beta : (F, 4N^2, 2)   orders 0, 1, -1, 2, -2, ..., degrees |m|..2N-1 each
  g    : (F, 4N-1, 2N, 2) orders in the same sequence, nodes ascending in x
  f    : (F, 2N, 4N-1, 2) theta-major grid values
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so with gcc + OpenMP."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        d = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        lib.oracle_gl_rule.argtypes = [i, d, d]
        lib.oracle_alf_table.argtypes = [i, i, d, i, d]
        lib.oracle_alt_forward.argtypes = [i, d, d, d, i]
        lib.oracle_alt_inverse.argtypes = [i, d, d, d, d, i]
        lib.oracle_alt_forward_m.argtypes = [i, i, d, i, d, d]
        lib.oracle_alt_inverse_m.argtypes = [i, i, d, d, d, d]
        lib.oracle_phi_synthesis.argtypes = [i, d, d, i]
        lib.oracle_phi_analysis.argtypes = [i, d, d, i]
        lib.oracle_phi_synthesis_nodes.argtypes = [i, i, d, d, i]
        lib.oracle_phi_analysis_nodes.argtypes = [i, i, d, d, i]
        lib.oracle_coef_offset.argtypes = [ctypes.c_long, ctypes.c_long]
        lib.oracle_coef_offset.restype = ctypes.c_long
        lib.oracle_order_slot.argtypes = [ctypes.c_long]
        lib.oracle_order_slot.restype = ctypes.c_long
        for name in ["oracle_gl_rule", "oracle_alf_table", "oracle_alt_forward",
                     "oracle_alt_inverse", "oracle_alt_forward_m", "oracle_alt_inverse_m",
                     "oracle_phi_synthesis", "oracle_phi_analysis", "oracle_phi_synthesis_nodes",
                     "oracle_phi_analysis_nodes", "oracle_num_threads"]:
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def coef_offset(N: int, m: int) -> int:
    """Index of beta_{|m|,m} in the packed coefficient array."""
    return int(_load().oracle_coef_offset(N, m))


def order_slot(m: int) -> int:
    """Row of order m in the ALT value array (sequence 0, 1, -1, 2, -2, ...)."""
    return int(_load().oracle_order_slot(m))


def gl_rule(n: int):
    """n-point Gauss-Legendre nodes (ascending) and weights."""
    x = np.empty(n)
    w = np.empty(n)
    _check(_load().oracle_gl_rule(n, _p(x), _p(w)), "gl_rule")
    return x, w


def alf_table(m: int, kmax: int, x) -> np.ndarray:
    """T[i, k-m] = Pbar_k^m(x_i), k = m..kmax (L2-normalised, no CS phase)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    out = np.empty((x.size, kmax - m + 1))
    _check(_load().oracle_alf_table(m, kmax, _p(x), x.size, _p(out)), "alf_table")
    return out


def alt_forward(N: int, beta: np.ndarray, x=None) -> np.ndarray:
    """Forward ALT of F fields: beta (F, 4N^2, 2) -> g (F, 4N-1, 2N, 2)."""
    if x is None:
        x, _ = gl_rule(2 * N)
    beta = np.ascontiguousarray(beta, dtype=np.float64).reshape(-1, 4 * N * N, 2)
    F = beta.shape[0]
    g = np.empty((F, 4 * N - 1, 2 * N, 2))
    _check(_load().oracle_alt_forward(N, _p(np.ascontiguousarray(x)), _p(beta), _p(g), F), "alt_forward")
    return g


def alt_inverse(N: int, g: np.ndarray, x=None, w=None) -> np.ndarray:
    """Inverse ALT of F fields: g (F, 4N-1, 2N, 2) -> beta (F, 4N^2, 2)."""
    if x is None or w is None:
        x, w = gl_rule(2 * N)
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1, 4 * N - 1, 2 * N, 2)
    F = g.shape[0]
    beta = np.empty((F, 4 * N * N, 2))
    _check(_load().oracle_alt_inverse(N, _p(np.ascontiguousarray(x)), _p(np.ascontiguousarray(w)),
                                      _p(g), _p(beta), F), "alt_inverse")
    return beta


def alt_forward_m(N: int, m: int, beta_m: np.ndarray, x_nodes) -> np.ndarray:
    """g(m, .) at arbitrary nodes from the 2N-|m| coefficients of order m."""
    beta_m = np.ascontiguousarray(beta_m, dtype=np.float64).reshape(-1, 2)
    assert beta_m.shape[0] == 2 * N - abs(m)
    xs = np.ascontiguousarray(np.asarray(x_nodes, dtype=np.float64).ravel())
    out = np.empty((xs.size, 2))
    _check(_load().oracle_alt_forward_m(N, m, _p(xs), xs.size, _p(beta_m), _p(out)), "alt_forward_m")
    return out


def alt_inverse_m(N: int, m: int, g_m: np.ndarray, x=None, w=None) -> np.ndarray:
    """beta_{k,m}, k = |m|..2N-1, from g(m, theta_l) at all 2N nodes."""
    if x is None or w is None:
        x, w = gl_rule(2 * N)
    g_m = np.ascontiguousarray(g_m, dtype=np.float64).reshape(2 * N, 2)
    out = np.empty((2 * N - abs(m), 2))
    _check(_load().oracle_alt_inverse_m(N, m, _p(np.ascontiguousarray(x)), _p(np.ascontiguousarray(w)),
                                        _p(g_m), _p(out)), "alt_inverse_m")
    return out


def alt_forward_m_fields(N: int, m: int, beta_m: np.ndarray, x_nodes) -> np.ndarray:
    """g(m, .) of F fields of order m at arbitrary nodes (Eq. sht_lt).

    beta_m: (F, 2N-|m|, 2).  The sum over degrees is one matrix product of the
    table T[i, k-|m|] = Pbar_k^{|m|}(x_i) (``alf_table``) with the coefficients:
    the same definition as ``alt_forward_m``, for many fields at once.
    """
    beta_m = np.asarray(beta_m, dtype=np.float64)
    assert beta_m.ndim == 3 and beta_m.shape[1] == 2 * N - abs(m)
    T = alf_table(abs(m), 2 * N - 1, x_nodes)
    return np.einsum("ik,fkc->fic", T, beta_m)


def alt_inverse_m_fields(N: int, m: int, g_m: np.ndarray, x=None, w=None) -> np.ndarray:
    """beta_{k,m}, k = |m|..2N-1, of F fields from g(m, theta_l) (Sec. 3.1.1).

    g_m: (F, 2N, 2).  beta_k = sum_l w_l Pbar_k^{|m|}(x_l) g_l as one matrix
    product of the transposed table with the weighted values.
    """
    if x is None or w is None:
        x, w = gl_rule(2 * N)
    g_m = np.asarray(g_m, dtype=np.float64)
    assert g_m.ndim == 3 and g_m.shape[1] == 2 * N
    T = alf_table(abs(m), 2 * N - 1, x)
    return np.einsum("ik,fic->fkc", T, np.asarray(w)[None, :, None] * g_m)


def phi_synthesis(N: int, g: np.ndarray) -> np.ndarray:
    """f(theta_l, phi_j) = sum_m g(m, theta_l) e^{i m phi_j}: (F,4N-1,2N,2) -> (F,2N,4N-1,2)."""
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1, 4 * N - 1, 2 * N, 2)
    F = g.shape[0]
    f = np.empty((F, 2 * N, 4 * N - 1, 2))
    _check(_load().oracle_phi_synthesis(N, _p(g), _p(f), F), "phi_synthesis")
    return f


def phi_analysis(N: int, f: np.ndarray) -> np.ndarray:
    """g(m, theta_l) = (1/M) sum_j f e^{-i m phi_j}: (F,2N,4N-1,2) -> (F,4N-1,2N,2)."""
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1, 2 * N, 4 * N - 1, 2)
    F = f.shape[0]
    g = np.empty((F, 4 * N - 1, 2 * N, 2))
    _check(_load().oracle_phi_analysis(N, _p(f), _p(g), F), "phi_analysis")
    return g


def phi_synthesis_nodes(N: int, g_nodes: np.ndarray) -> np.ndarray:
    """phi_synthesis at a subset of nodes: g_nodes (F,4N-1,nl,2), the chosen node
    columns of g (orders in the storage sequence) -> their grid rows (F,nl,4N-1,2)."""
    g_nodes = np.ascontiguousarray(g_nodes, dtype=np.float64)
    F, M, nl = g_nodes.shape[0], g_nodes.shape[1], g_nodes.shape[2]
    assert M == 4 * N - 1 and g_nodes.shape[3] == 2
    f = np.empty((F, nl, M, 2))
    _check(_load().oracle_phi_synthesis_nodes(N, nl, _p(g_nodes), _p(f), F), "phi_synthesis_nodes")
    return f


def phi_analysis_nodes(N: int, f_rows: np.ndarray) -> np.ndarray:
    """phi_analysis at a subset of nodes: grid rows f_rows (F,nl,4N-1,2) -> the
    nodes' ALT values (F,4N-1,nl,2)."""
    f_rows = np.ascontiguousarray(f_rows, dtype=np.float64)
    F, nl, M = f_rows.shape[0], f_rows.shape[1], f_rows.shape[2]
    assert M == 4 * N - 1 and f_rows.shape[3] == 2
    g = np.empty((F, M, nl, 2))
    _check(_load().oracle_phi_analysis_nodes(N, nl, _p(f_rows), _p(g), F), "phi_analysis_nodes")
    return g


def sht_forward(N: int, beta: np.ndarray) -> np.ndarray:
    """Full forward SHT (Eq. sht_re): coefficients -> grid values."""
    return phi_synthesis(N, alt_forward(N, beta))


def sht_inverse(N: int, f: np.ndarray) -> np.ndarray:
    """Full inverse SHT: grid values -> coefficients."""
    return alt_inverse(N, phi_analysis(N, f))
