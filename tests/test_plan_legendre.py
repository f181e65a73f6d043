"""The library's own Legendre matrices against the oracle's, entry by entry (CPU).

The plan builder evaluates Pbar_k^|m| at the positive Gauss-Legendre nodes
with its own recurrence (a binary exponent carried with the recurrence pair),
separate from the oracle's (extended-exponent numbers), which the oracle tests
pin to exact rational values.  A dense plan (SHT_FLAG_DENSE: no partition,
trimming or factorisation) stores every entry of every parity matrix, so its
factors are those matrices.  At N = 160 the sectoral starts near the poles
fall far below the FP64 range (1 - x^2 ~ 6e-5 at the outermost node, to the
power m/2 up to 160), so the comparison covers the underflow region too.
"""
import numpy as np

import host_apply
import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib


def test_dense_plan_holds_the_legendre_matrices():
    N = 160
    p = sht.Plan(N, 1e-12, flags=_lib.SHT_FLAG_HOST_ONLY | _lib.SHT_FLAG_DENSE)
    prog = p.program(("units", "ops", "factors"))
    # the plan's own nodes: the two Gauss-Legendre rules differ by an ulp here
    # and there, which the sectoral start raises to the power m/2
    x, _ = p.nodes()
    tiny = subnormal = 0
    for u in prog["units"]:
        am = int(u["am"])
        T = oracle.alf_table(am, 2 * N - 1, x[N:])  # T[i, k - am] at the positive nodes
        M = np.full(T.shape, np.nan)
        for op in prog["ops"][u["op_begin"]: u["op_end"]]:
            B = host_apply._block(prog, op)
            orow = host_apply._rows(op["out_off"], op["out_len"])
            irow = host_apply._rows(op["in_off"], op["in_len"])
            # output rows are nodes of Y_e / Y_o, input rows degrees of X_e / X_o,
            # and a product never mixes the parities (Sec. 3.1.2)
            assert np.all((orow >= u["yo"])[:, None] == (irow >= u["xo"])[None, :])
            i = np.where(orow < u["yo"], orow - u["ye"], orow - u["yo"])
            k = np.where(irow < u["xo"], am + 2 * (irow - u["xe"]), am + 1 + 2 * (irow - u["xo"]))
            assert np.all(np.isnan(M[i[:, None], k[None, :] - am]))  # each entry stored once
            M[i[:, None], k[None, :] - am] = B
        assert not np.any(np.isnan(M)), am  # and every entry stored
        # the two evaluate the same recurrence, so they agree to rounding (on
        # x86-64 without FMA contraction, bit for bit); rounding differences
        # grow relative to the magnitude of the neighbouring degrees (near a
        # root of Pbar the value is small, not its error): bound the
        # difference by that local scale
        A = np.abs(T)
        pad = np.pad(A, ((0, 0), (3, 3)))
        local = np.max([pad[:, s: s + A.shape[1]] for s in range(7)], axis=0)
        d = np.abs(M - T)
        big = A > 1e-290
        assert np.all(d[big] <= 2e-12 * local[big]), am
        # entries the extended exponents carry down to (and below) the FP64
        # range agree to within a few subnormal steps, and zeros are zeros
        assert np.all(d[~big] <= 1e-300), am
        assert np.array_equal(T == 0, M == 0), am
        tiny += int((~big).sum())
        subnormal += int(((A < 2.2250738585072014e-308) & (A > 0)).sum())
    assert tiny > 10000 and subnormal > 1000  # the underflow region was exercised
