"""Seeded synthetic inputs for the ALT / SHT workloads.

This module holds no arithmetic of the transform itself: it only draws
coefficient arrays in the packed layout the library and the oracle both take.
Both sides of every parity check receive the arrays made here.

Coefficient layout (per field, complex as a trailing axis of 2 doubles):
orders in the sequence m = 0, 1, -1, 2, -2, ..., 2N-1, -(2N-1); for each
order the degrees k = |m|..2N-1 are contiguous, 4N^2 complex values in all.
"""
from __future__ import annotations

import numpy as np


def order_sequence(N: int) -> np.ndarray:
    """Orders in storage order: 0, 1, -1, 2, -2, ..., 2N-1, -(2N-1)."""
    ms = [0]
    for a in range(1, 2 * N):
        ms += [a, -a]
    return np.array(ms, dtype=np.int64)


def degree_index(N: int) -> tuple[np.ndarray, np.ndarray]:
    """(k, m) of every packed coefficient position, length 4N^2."""
    ks, ms = [], []
    for m in order_sequence(N):
        a = abs(int(m))
        ks.append(np.arange(a, 2 * N, dtype=np.int64))
        ms.append(np.full(2 * N - a, m, dtype=np.int64))
    return np.concatenate(ks), np.concatenate(ms)


def coefficients(N: int, F: int, seed: int, *, decay: float = 0.0,
                 real_m0: bool = False, field_offset: int = 0) -> np.ndarray:
    """(F, 4N^2, 2) float64: Re and Im i.i.d. N(0,1) times (k+1)^-decay.

    Fields are drawn one after another from ``numpy.random.default_rng(seed)``
    (PCG64); ``field_offset`` skips that many fields so that a sample of a
    batch reproduces the same numbers as the full batch.  ``real_m0`` zeroes
    the imaginary part of the m = 0 coefficients.
    """
    n = 4 * N * N
    rng = np.random.default_rng(seed)
    if field_offset:
        rng.standard_normal((field_offset, n, 2))
    beta = rng.standard_normal((F, n, 2))
    if decay:
        k, _ = degree_index(N)
        beta *= ((k + 1.0) ** (-decay))[None, :, None]
    if real_m0:
        beta[:, : 2 * N, 1] = 0.0
    return beta


# Workloads named by what they are (the paper's settings: eps, N, fields).
WORKLOADS = {
    # FP64 IDBF ALT + SHT at N=64, one field, eps=1e-12, beta_{k,0} real
    "fp64_N64": dict(N=64, F=1, seed=0, decay=0.0, real_m0=True, eps=1e-12, precision="fp64"),
    # FP64 IDBF ALT at N=1024, one field, coefficients scaled by (k+1)^-1
    "fp64_N1024": dict(N=1024, F=1, seed=0, decay=1.0, real_m0=False, eps=1e-12, precision="fp64"),
    # mixed-precision IDBF at N=1024, 64 fields, eps=1e-7; partition stop size
    # and leaf size picked by paper_2004_11346_gb300.autotune (measured on GB300)
    "mixed_N1024_F64": dict(N=1024, F=64, seed=0, decay=0.0, real_m0=False, eps=1e-7, precision="mixed",
                            plan=dict(n0=256, n_leaf=256)),
    # N=4096, 16 fields, spectrum N(0,(k+1)^-2), eps=1e-10
    "N4096_F16": dict(N=4096, F=16, seed=0, decay=1.0, real_m0=False, eps=1e-10, precision="fp64"),
}


def workload_coefficients(name: str, F: int | None = None, field_offset: int = 0) -> np.ndarray:
    w = WORKLOADS[name]
    return coefficients(w["N"], w["F"] if F is None else F, w["seed"], decay=w["decay"],
                        real_m0=w["real_m0"], field_offset=field_offset)


# Uneven batch: fields of mixed orders N, the sizes and then the coefficients
# drawn from one generator (default_rng(seed)): size index per field uniform
# over `sizes`, then for each size in increasing order its fields' Re and Im
# i.i.d. N(0,1).
UNEVEN_SIZES = (128, 256, 512, 1024, 2048)


def uneven_batch(F: int = 256, seed: int = 1, sizes=UNEVEN_SIZES):
    """(size of each field, {N: (count_N, 4N^2, 2) float64 coefficients})."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, len(sizes), F)
    per_field = np.asarray(sizes, dtype=np.int64)[idx]
    coeffs = {}
    for N in sorted(sizes):
        count = int((per_field == N).sum())
        if count:
            coeffs[N] = rng.standard_normal((count, 4 * N * N, 2))
    return per_field, coeffs
