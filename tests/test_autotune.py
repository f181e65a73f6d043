"""The autotuner's host side: candidate parameters and the work model.

The model counts what the tensor-core kernel streams per 32-field group:
pipeline stages (128-row tiles x 32-wide K chunks of row groups), operand-image
bytes and activation bytes.  Checked here against invariants that hold for any
plan; the GPU test times the ranked candidates.
"""
import numpy as np

import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, autotune

HOST = _lib.SHT_FLAG_HOST_ONLY


def test_candidates_include_defaults_and_are_valid():
    for N in (32, 256, 1024, 2048):
        d = _lib.sht_opts_default(N, 1e-7)
        c = autotune.candidates(N, 1e-7)
        assert (d.n0, d.n_leaf) in c
        assert len(set(c)) == len(c)
        assert all(n0 >= 8 and 4 <= nl <= n0 for n0, nl in c)


def test_work_model_invariants():
    p = sht.Plan(48, 1e-7, flags=HOST, precision=_lib.SHT_MIXED, n0=16, n_leaf=8)
    prog = p.program(("ops", "units"))
    ops = prog["ops"]
    w = autotune.work_model(ops, prog["units"], 48)
    live = ops[ops["ni"] > 0]
    # every product is at least one tile and one stage
    assert w["tiles"] >= len(live) and w["stages"] >= w["tiles"]
    # three 2-byte pieces per stored entry, before padding
    assert w["image_bytes"] >= 6 * int((live["mo"].astype(np.int64) * live["ni"]).sum())
    # every stage moves at least one row group of activations
    assert w["activation_bytes"] >= autotune.GROUP_BYTES * w["tiles"]


def test_dense_plan_counts():
    # one dense product per (order, parity) at N=8: every product is a single
    # tile, so the stage count is the number of K chunks of each product
    N = 8
    p = sht.Plan(N, 1e-7, flags=HOST | _lib.SHT_FLAG_DENSE, precision=_lib.SHT_MIXED)
    prog = p.program(("ops", "units"))
    ops = prog["ops"]
    w = autotune.work_model(ops, prog["units"], N)
    assert np.all(ops["mo"] <= 128)
    assert w["tiles"] == int((ops["ni"] > 0).sum())
    assert w["stages"] >= w["tiles"]


def test_rank_is_sorted_by_model():
    rows = autotune.rank(64, 1e-7, [(16, 8), (32, 8), (32, 16)])
    assert [(r["n0"], r["n_leaf"]) for r in rows] != []
    costs = [r["model_us"] for r in rows]
    assert costs == sorted(costs)
    assert all(r["entries"] > 0 and r["stages"] > 0 for r in rows)


def test_sampled_work_model_is_exact_with_every_order():
    N, kw = 64, dict(n0=16, n_leaf=8)
    p = sht.Plan(N, 1e-7, flags=HOST, precision=_lib.SHT_MIXED, **kw)
    prog = p.program(("ops", "units"))
    full = autotune.work_model(prog["ops"], prog["units"], N)
    w, entries = autotune.sampled_work_model(N, 1e-7, 2 * N, **kw)
    assert w == full
    assert entries == p.stats()["entries_total"]


def test_sampled_work_model_is_close_with_a_sample():
    N = 256
    p = sht.Plan(N, 1e-7, flags=HOST, precision=_lib.SHT_MIXED)
    prog = p.program(("ops", "units"))
    full = autotune.work_model(prog["ops"], prog["units"], N)
    w, _ = autotune.sampled_work_model(N, 1e-7, 32)
    for k in full:
        assert abs(w[k] / full[k] - 1) < 0.05, (k, w[k], full[k])


def test_rank_from_samples(capsys):
    import json
    cands = [(16, 8), (32, 8), (32, 16)]
    rows = autotune.rank(64, 1e-7, cands, sample=128)
    assert rows == autotune.rank(64, 1e-7, cands)  # 128 = 2N: every order
    autotune.main(["--N", "64", "--eps", "1e-7", "--cands", "16:8,32:16", "--sample", "16", "--rank-only"])
    out = [json.loads(l) for l in capsys.readouterr().out.strip().splitlines()]
    assert len(out) == 2 and out[0]["model_us"] <= out[1]["model_us"]


def test_schedules_are_permutations_and_set_on_the_plan():
    N = 24
    p = sht.Plan(N, 1e-7, flags=HOST, precision=_lib.SHT_MIXED, n0=12, n_leaf=6)
    units = p.program(("units",))["units"]
    cost = {int(u["am"]): float(u["cost"]) for u in units}
    for kind in autotune.SCHEDULES:
        o = autotune.schedule(units, kind)
        assert sorted(o.tolist()) == list(range(2 * N))
        p.set_order(o)
        assert np.array_equal(p.order(), o)
    lpt = autotune.schedule(units, "lpt")
    assert all(cost[int(a)] >= cost[int(b)] for a, b in zip(lpt[:-1], lpt[1:]))
    # the plan starts in LPT order
    q = sht.Plan(N, 1e-7, flags=HOST, precision=_lib.SHT_MIXED, n0=12, n_leaf=6)
    assert np.array_equal(q.order(), lpt)
    pairs = autotune.schedule(units, "pairs")
    assert pairs[0] == lpt[0] and pairs[1] == lpt[-1] and pairs[2] == lpt[1]
    assert np.array_equal(autotune.schedule(units, "ascending"), np.arange(2 * N))


def test_set_order_refuses_what_is_not_a_permutation():
    import pytest
    N = 8
    p = sht.Plan(N, 1e-7, flags=HOST, precision=_lib.SHT_MIXED)
    before = p.order()
    for bad in ([0] * (2 * N), list(range(2 * N - 1)), list(range(1, 2 * N + 1)), [-1] + list(range(1, 2 * N))):
        with pytest.raises(_lib.ShtError) as e:
            p.set_order(bad)
        assert e.value.status == _lib.SHT_ERR_ARG
    assert np.array_equal(p.order(), before)
