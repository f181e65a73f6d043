"""Test-only host evaluation of an exported apply program (numpy, FP64).

Runs the plan's dense block products in phase order exactly as the kernels
are specified to (program.hpp), so that factorisation error can be told apart
from kernel error.  Never used by the library.
"""
import numpy as np


def _coef_offset(N, m):
    a = abs(m)
    if a == 0:
        return 0
    pos = 2 * N * (2 * a - 1) - a * (a - 1)
    return pos if m > 0 else pos + (2 * N - a)


def _slot(m):
    return 0 if m == 0 else (2 * m - 1 if m > 0 else -2 * m)


def _block(prog, op):
    f = prog["factors"]
    B = f[op["b_off"]: op["b_off"] + op["ld"] * op["ni"]].reshape(op["ni"], op["ld"]).T
    return B[: op["mo"]]


def _rows(off, ln):
    return np.concatenate([np.arange(off[0], off[0] + ln[0]), np.arange(off[1], off[1] + ln[1])]).astype(np.int64)


def forward(prog, N, beta):
    """beta (4N^2, 2) -> g (4N-1, 2N, 2) by the program."""
    K = 2 * N
    g = np.zeros((4 * N - 1, K, 2))
    ops, phases = prog["ops"], prog["phases"]
    for u in prog["units"]:
        am = int(u["am"])
        vec = np.zeros((u["nrows"], 4))
        bp = beta[_coef_offset(N, am): _coef_offset(N, am) + K - am]
        bn = beta[_coef_offset(N, -am): _coef_offset(N, -am) + K - am] if am else np.zeros_like(bp)
        nce = int(u["nce"])
        vec[: nce, :2] = bp[0::2]
        vec[: nce, 2:] = bn[0::2]
        vec[nce: nce + int(u["nco"]), :2] = bp[1::2]
        vec[nce: nce + int(u["nco"]), 2:] = bn[1::2]
        for ph in range(u["nphase"]):
            for oi in range(phases[u["ph_begin"] + ph], phases[u["ph_begin"] + ph + 1]):
                op = ops[oi]
                y = _block(prog, op) @ vec[_rows(op["in_off"], op["in_len"])]
                rows = _rows(op["out_off"], op["out_len"])
                if op["flags"] & 1:
                    vec[rows] += y
                else:
                    vec[rows] = y
        ye = vec[u["ye"]: u["ye"] + N]
        yo = vec[u["yo"]: u["yo"] + N]
        for s, m in enumerate([am, -am] if am else [0]):
            e, o = ye[:, 2 * s: 2 * s + 2], yo[:, 2 * s: 2 * s + 2]
            g[_slot(m), N:] = e + o
            g[_slot(m), :N] = (e - o)[::-1]
    return g


def inverse(prog, N, g, w):
    """g (4N-1, 2N, 2) -> beta (4N^2, 2) by the transposed program."""
    K = 2 * N
    beta = np.zeros((4 * N * N, 2))
    ops, phases = prog["ops"], prog["phases"]
    wp = w[N:][:, None]
    for u in prog["units"]:
        am = int(u["am"])
        vec = np.zeros((u["nrows"], 4))
        for s, m in enumerate([am, -am] if am else [0]):
            a = g[_slot(m), N:]
            b = g[_slot(m), :N][::-1]
            vec[u["ye"]: u["ye"] + N, 2 * s: 2 * s + 2] = wp * (a + b)
            vec[u["yo"]: u["yo"] + N, 2 * s: 2 * s + 2] = wp * (a - b)
        for ph in range(u["nphase"] - 1, -1, -1):
            for oi in range(phases[u["ph_begin"] + ph], phases[u["ph_begin"] + ph + 1]):
                op = ops[oi]
                y = _block(prog, op).T @ vec[_rows(op["out_off"], op["out_len"])]
                rows = _rows(op["in_off"], op["in_len"])
                if op["flags"] & 2:
                    vec[rows] += y
                else:
                    vec[rows] = y
        nce, nco = int(u["nce"]), int(u["nco"])
        for s, m in enumerate([am, -am] if am else [0]):
            off = _coef_offset(N, m)
            seg = beta[off: off + K - am]
            seg[0::2] = vec[:nce, 2 * s: 2 * s + 2]
            seg[1::2] = vec[nce: nce + nco, 2 * s: 2 * s + 2]
    return beta
