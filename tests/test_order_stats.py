"""One order built on its own (sht_order_stats) against the full plan (CPU).

The per-order build is what the paper's experiments of Sec. 5 time order by
order, and what sizes a large plan from a sample of its orders.  It must
describe exactly what sht_plan_create builds at that order: the same blocks
and block products, the same vector space, cost estimate and factor store
size, and tensor-core images of the sizes sht_plan_op_image reports.
"""
import numpy as np
import pytest

import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib

HOST = _lib.SHT_FLAG_HOST_ONLY
FORCE = _lib.SHT_FLAG_FORCE_FACTOR


@pytest.fixture(scope="module", params=["forced", "default"])
def case(request):
    # forced factorisation with a small starting rSVD rank (IDBF, low-rank and
    # dense blocks all present), and a default mixed-precision plan
    if request.param == "forced":
        N, eps, kw = 48, 1e-7, dict(flags=HOST | FORCE, n0=12, n_leaf=4, rsvd_r=2)
    else:
        N, eps, kw = 96, 1e-7, dict(flags=HOST, precision=_lib.SHT_MIXED)
    p = sht.Plan(N, eps, **kw)
    prog = p.program(("units", "ops", "factors", "unit_blocks"))
    rows = _lib.sht_order_stats(N, eps, range(2 * N), sht.opts(N, eps, **kw))
    return p, prog, rows, request.param


def test_every_order_matches_the_plan(case):
    p, prog, rows, kind = case
    N = p.N
    units, ops, blocks = prog["units"], prog["ops"], prog["unit_blocks"].reshape(-1, 4)
    for am, r in enumerate(rows):
        u = units[am]
        assert r["N"] == N and r["am"] == am
        assert (r["cols_even"], r["cols_odd"]) == (u["nce"], u["nco"])
        assert r["rows"] == u["nrows"] and r["n_phases"] == u["nphase"]
        assert r["flops_per_rhs"] == float(u["cost"])
        assert r["n_ops"] == u["op_end"] - u["op_begin"]
        got = (r["n_blocks_idbf"], r["n_blocks_lowrank"], r["n_blocks_dense"], r["n_blocks_dropped"])
        assert got == tuple(int(v) for v in blocks[am])
        assert r["entries_total"] == r["entries_idbf"] + r["entries_lowrank"] + r["entries_dense"]
        assert r["entries_matrix"] == N * (u["nce"] + u["nco"])
        assert r["t_mat_s"] >= 0.0 and r["t_fac_s"] >= 0.0
    st = p.stats()
    for k in ("n_blocks_idbf", "n_blocks_lowrank", "n_blocks_dense", "n_blocks_dropped", "entries_idbf",
              "entries_lowrank", "entries_dense", "entries_total", "entries_matrix", "n_ops"):
        assert sum(r[k] for r in rows) == st[k], k
    assert max(r["max_rank"] for r in rows) == st["max_rank"]
    assert max(r["n_phases"] for r in rows) == st["max_phases"]
    # the units' factor stores are concatenated in order of |m|
    assert sum(r["factor_doubles"] for r in rows) == len(prog["factors"])
    if kind == "forced":
        assert st["n_blocks_idbf"] > 0 and st["n_blocks_lowrank"] > 0 and st["n_blocks_dense"] > 0


def test_factor_stores_line_up(case):
    # every unit's block products read only its own stretch of the plan's
    # factor store, whose length is the order's factor_doubles
    p, prog, rows, _ = case
    units, ops = prog["units"], prog["ops"]
    start = 0
    for am, r in enumerate(rows):
        u = units[am]
        uops = ops[u["op_begin"]: u["op_end"]]
        # each unit's factor offsets are relative to its own store
        if len(uops):
            assert uops["b_off"].min() >= start
            assert (uops["b_off"] + uops["ld"].astype(np.int64) * uops["ni"]).max() <= start + r["factor_doubles"]
        start += r["factor_doubles"]


def test_image_sizes_match_the_op_images(case):
    p, prog, rows, _ = case
    units = prog["units"]
    for am in range(0, len(rows), max(1, len(rows) // 12)):
        u = units[am]
        n = sum(len(_lib.sht_plan_op_image(p.handle, k, t)) for k in range(u["op_begin"], u["op_end"])
                for t in (False, True))
        assert rows[am]["image_elems"] == n, am


def untimed(r):
    return {k: v for k, v in r.items() if not k.startswith("t_")}


def test_signed_orders_and_defaults():
    N, eps = 40, 1e-7
    a, b = _lib.sht_order_stats(N, eps, [7, -7])
    assert untimed(a) == untimed(b)
    # NULL options are the defaults
    c = _lib.sht_order_stats(N, eps, [7], _lib.sht_opts_default(N, eps))[0]
    assert untimed(c) == untimed(a)
    # the extreme orders: |m| = 2N - 1 has one even degree and no odd one
    e = _lib.sht_order_stats(N, eps, [-(2 * N - 1), 0])
    assert (e[0]["cols_even"], e[0]["cols_odd"]) == (1, 0)
    assert (e[1]["cols_even"], e[1]["cols_odd"]) == (N, N)
    assert _lib.sht_order_stats(N, eps, []) == []


def test_argument_errors():
    N, eps = 40, 1e-7
    for bad in ([2 * N], [-2 * N], [0, 2 * N + 5]):
        with pytest.raises(_lib.ShtError) as e:
            _lib.sht_order_stats(N, eps, bad)
        assert e.value.status == _lib.SHT_ERR_ARG
    for n, tol in ((0, eps), (N, 0.0), (N, 1.0), (1 << 15, eps)):
        with pytest.raises(_lib.ShtError):
            _lib.sht_order_stats(n, tol, [0])
    with pytest.raises(_lib.ShtError):
        _lib.sht_order_stats(N, eps, [0], sht.opts(N, eps, n0=0))
    lib = _lib.load()
    assert lib.sht_order_stats(N, eps, None, -1, None, None) == _lib.SHT_ERR_ARG
    assert lib.sht_order_stats(N, eps, None, 1, None, None) == _lib.SHT_ERR_ARG
    assert lib.sht_order_stats(N, eps, None, 0, None, None) == _lib.SHT_OK


def test_stratified_sample_covers_every_order_once():
    from paper_2004_11346_gb300 import orders
    for N, count in ((40, 7), (40, 80), (40, 500), (1024, 64), (5, 3)):
        ms, ws = orders.sample_orders(N, count)
        assert sum(ws) == 2 * N and len(ms) == min(count, 2 * N)
        lo = 0
        for m, w in zip(ms, ws):
            assert lo <= m < lo + w  # the order lies inside its own stratum
            lo += w


def test_estimate_is_exact_with_every_order_and_close_with_a_sample():
    from paper_2004_11346_gb300 import orders
    N, eps = 128, 1e-7
    o = sht.opts(N, eps, flags=HOST, precision=_lib.SHT_MIXED)
    st = sht.Plan(N, eps, flags=HOST, precision=_lib.SHT_MIXED).stats()
    full = orders.estimate(N, eps, 2 * N, o)
    assert full["exact"]
    for k in ("entries_total", "entries_matrix", "n_ops", "n_blocks_dense", "n_blocks_idbf"):
        assert full["totals"][k] == st[k], k
    part = orders.estimate(N, eps, 32, o)
    assert not part["exact"] and part["orders_sampled"] == 32
    for k in ("entries_total", "entries_matrix", "factor_doubles", "image_elems"):
        assert abs(part["totals"][k] / full["totals"][k] - 1) < 0.05, k


def test_command_line(capsys):
    import json
    from paper_2004_11346_gb300 import orders
    orders.main(["--N", "32", "--eps", "1e-7", "--sample", "8"])
    d = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert d["N"] == 32 and d["orders_sampled"] == 8 and 0 < d["stored_over_matrix"] <= 1.5
    assert d["factor_bytes"]["fp64"] == 2 * d["factor_bytes"]["fp32"]
    orders.main(["--N", "32", "--eps", "1e-7", "--at", "0,0.5,1,1.5,2"])
    rows = [json.loads(l) for l in capsys.readouterr().out.strip().splitlines()]
    assert [r["am"] for r in rows] == [0, 16, 32, 48, 63]
