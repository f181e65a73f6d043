"""Randomised plan options against the oracle (CPU, hypothesis).

For small orders N and random partition, leaf, rank, sampling, trimming and
seed options, a host-only plan must be built (its program passes the
library's consistency check on creation) and reproduce the oracle's forward
and inverse ALT to the scale of its tolerance: the IDs, the randomized SVD
(accepted at 10 eps) and trimming all truncate relative to the largest entry,
so the transform of N(0,1) coefficients stays at the scale of eps: bounded
here by 10 eps (over 250 random option sets the largest relative error seen
was 0.8 eps), far below what a dropped block or a misplaced product would
cause.  Plans with the same options and seed are identical, and single
orders built on their own (sht_order_stats) match the plan's units.
"""
import numpy as np
import pytest

import host_apply
import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, inputs

hyp = pytest.importorskip("hypothesis")
st = hyp.strategies

HOST = _lib.SHT_FLAG_HOST_ONLY
FORCE = _lib.SHT_FLAG_FORCE_FACTOR


@st.composite
def plan_options(draw):
    N = draw(st.integers(1, 40))
    eps = draw(st.sampled_from([1e-4, 1e-7, 1e-10]))
    kw = dict(
        n0=draw(st.integers(1, max(1, N))),
        n_leaf=draw(st.integers(1, 16)),
        r_k=draw(st.integers(1, 40)),
        oversample=draw(st.sampled_from([1.0, 1.5, 2.0, 3.0])),
        rsvd_r=draw(st.integers(1, 8)),
        rsvd_q=draw(st.integers(1, 3)),
        sampling=draw(st.integers(0, 1)),
        seed=draw(st.integers(0, 2 ** 32)),
        flags=HOST | draw(st.sampled_from([0, FORCE])),
    )
    return N, eps, kw


@hyp.settings(max_examples=60, deadline=None, derandomize=True)
@hyp.given(plan_options())
def test_random_plans_reproduce_the_oracle(case):
    N, eps, kw = case
    p = sht.Plan(N, eps, **kw)
    prog = p.program()
    x, w = p.nodes()
    beta = inputs.coefficients(N, 1, seed=3, real_m0=True)
    g_ref = oracle.alt_forward(N, beta)[0]
    g = host_apply.forward(prog, N, beta[0])
    assert np.linalg.norm(g - g_ref) <= 10 * eps * np.linalg.norm(g_ref)
    b_ref = oracle.alt_inverse(N, g_ref[None])[0]
    b = host_apply.inverse(prog, N, g_ref, w)
    assert np.linalg.norm(b - b_ref) <= 10 * eps * np.linalg.norm(b_ref)
    # deterministic given the options and the seed
    q = sht.Plan(N, eps, **kw).program()
    for part in ("units", "ops", "factors"):
        assert prog[part].tobytes() == q[part].tobytes()
    # an order built on its own is the plan's unit at that order
    units = prog["units"]
    blocks = p.program(("unit_blocks",))["unit_blocks"].reshape(-1, 4)
    ms = sorted({0, N, 2 * N - 1, N // 2})
    for r in _lib.sht_order_stats(N, eps, ms, sht.opts(N, eps, **kw)):
        u = units[r["am"]]
        assert (r["n_ops"], r["rows"], r["n_phases"]) == (u["op_end"] - u["op_begin"], u["nrows"], u["nphase"])
        assert r["flops_per_rhs"] == float(u["cost"])
        assert (r["n_blocks_idbf"], r["n_blocks_lowrank"], r["n_blocks_dense"], r["n_blocks_dropped"]) == \
            tuple(int(v) for v in blocks[r["am"]])
