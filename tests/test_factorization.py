"""The factorisation against its tolerance, matrix by matrix.

For every order |m| and parity, the matrix the plan represents -- all of its
blocks' factors (IDBF, randomized-SVD low-rank, trimmed dense) applied to the
identity by the test-only host evaluation -- is compared with the oracle's
dense matrix of normalised Legendre values at the positive nodes (Sec. 3.1.2).
The IDs and the SVD truncate at an absolute tolerance eps on the scale of the
matrix's largest entry (Sec. 2.1, 2.3), and trimming drops entries a thousand
times smaller.  The randomized SVD accepts a block once its residual is below
10 eps (its rank is doubled until then), so with low-rank blocks every entry
must be within 10 eps * max|A|, and within 2 eps * max|A| when only IDs and
trimming are involved; the two parities never mix.
"""
import numpy as np
import pytest

import host_apply
import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib

HOST = _lib.SHT_FLAG_HOST_ONLY
FORCE = _lib.SHT_FLAG_FORCE_FACTOR


def represented(prog, u):
    """(even, odd, even-from-odd, odd-from-even) matrices of unit u."""
    ops, phases = prog["ops"], prog["phases"]
    nce, nco = int(u["nce"]), int(u["nco"])
    nx = nce + nco
    N = int(u["yo"] - u["ye"])
    vec = np.zeros((int(u["nrows"]), nx))
    vec[:nx] = np.eye(nx)  # X_e then X_o rows: the identity on the coefficients
    for ph in range(int(u["nphase"])):
        for oi in range(phases[u["ph_begin"] + ph], phases[u["ph_begin"] + ph + 1]):
            op = ops[oi]
            y = host_apply._block(prog, op) @ vec[host_apply._rows(op["in_off"], op["in_len"])]
            rows = host_apply._rows(op["out_off"], op["out_len"])
            if op["flags"] & 1:
                vec[rows] += y
            else:
                vec[rows] = y
    ye = vec[u["ye"]: u["ye"] + N]
    yo = vec[u["yo"]: u["yo"] + N]
    return ye[:, :nce], yo[:, nce:], ye[:, nce:], yo[:, :nce]


def worst_error(p, N):
    """max over orders and parities of max|A_plan - A| / max|A|; and the largest cross-parity entry."""
    prog = p.program()
    x, _ = oracle.gl_rule(2 * N)
    worst, cross = 0.0, 0.0
    for u in prog["units"]:
        am = int(u["am"])
        T = oracle.alf_table(am, 2 * N - 1, x[N:])  # T[i, k - am] at the positive nodes
        ae, ao, c1, c2 = represented(prog, u)
        for plan_m, ref in ((ae, T[:, 0::2]), (ao, T[:, 1::2])):
            if ref.size:
                worst = max(worst, float(np.abs(plan_m - ref).max() / np.abs(ref).max()))
        for c in (c1, c2):
            if c.size:
                cross = max(cross, float(np.abs(c).max()))
    return worst, cross


N = 32
KW = dict(flags=HOST | FORCE, n0=8, n_leaf=4, rsvd_r=2)


@pytest.mark.parametrize("eps", [1e-4, 1e-7, 1e-10])
def test_every_matrix_within_tolerance(eps):
    p = sht.Plan(N, eps, **KW)
    st = p.stats()
    # all three block kinds of Sec. 3.3 take part
    assert st["n_blocks_idbf"] > 0 and st["n_blocks_lowrank"] > 0 and st["n_blocks_dense"] > 0
    worst, cross = worst_error(p, N)
    assert worst <= 10 * eps, worst
    assert cross == 0.0


@pytest.mark.parametrize("eps", [1e-4, 1e-7, 1e-10])
def test_ids_and_trimming_within_tolerance(eps):
    # the default starting rank of the randomized SVD (Sec. 5: 30) leaves these
    # small non-oscillatory blocks dense: IDBF blocks and trimmed dense blocks only
    p = sht.Plan(N, eps, flags=HOST | FORCE, n0=8, n_leaf=4)
    st = p.stats()
    assert st["n_blocks_idbf"] > 0 and st["n_blocks_lowrank"] == 0
    worst, cross = worst_error(p, N)
    assert worst <= 2 * eps, worst
    assert cross == 0.0


def test_error_follows_the_tolerance():
    errs = [worst_error(sht.Plan(N, eps, **KW), N)[0] for eps in (1e-4, 1e-7, 1e-10)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 1e-2 * errs[0] and errs[2] < 1e-2 * errs[1]


@pytest.mark.parametrize("sampling", [0, 1])
def test_sampling_modes(sampling):
    # mock-Chebyshev (0) and random (1) row samples of the ID (Sec. 2.1)
    worst, _ = worst_error(sht.Plan(N, 1e-7, sampling=sampling, **KW), N)
    assert worst <= 1e-6, worst


def test_large_leaf_plan_shape():
    # the shape the autotuner picks for the tensor-core apply: n0 = N/4, leaves
    # four times the default
    d = _lib.sht_opts_default(N, 1e-7)
    p = sht.Plan(N, 1e-7, flags=HOST, n0=N // 4, n_leaf=4 * d.n_leaf)
    worst, cross = worst_error(p, N)
    assert worst <= 2e-7 and cross == 0.0
