"""Per-order plan statistics: the paper's order-by-order experiments, and plan sizing.

sht_order_stats builds single orders of a plan on the host, one thread per
order, with no device.  Each order gets exactly the blocks, products and
factors that the full plan would hold there.

Sec. 5 of the paper measures block counts, matrix-construction time (T_mat)
and factorisation time (T_fac) order by order, at m = 0, N/2, N and 3N/2.
The same builds, taken at a stratified sample of orders, estimate a plan that
is too large to build casually: its stored entries, its factor store in each
precision, and its precomputation time.

    python -m paper_2004_11346_gb300.orders --N 4096 --eps 1e-10 --sample 64
    python -m paper_2004_11346_gb300.orders --N 2048 --eps 1e-10 --at 0,0.5,1,1.5
"""
from __future__ import annotations

import argparse
import json
import os

from . import _lib

SUMMED = ("n_blocks_idbf", "n_blocks_lowrank", "n_blocks_dense", "n_blocks_dropped", "entries_idbf",
          "entries_lowrank", "entries_dense", "entries_total", "entries_matrix", "factor_doubles", "image_elems",
          "tc_stages", "tc_tiles", "tc_image_fwd_bytes", "tc_act_bytes", "n_ops", "t_mat_s", "t_fac_s")


def sample_orders(N: int, count: int):
    """Orders |m| standing for all 2N: the middle order of each of `count`
    nearly equal strata of 0..2N-1, with the stratum's size as its weight.
    With count >= 2N every order stands for itself."""
    K = 2 * N
    count = max(1, min(count, K))
    orders, weights = [], []
    for s in range(count):
        lo, hi = s * K // count, (s + 1) * K // count
        orders.append((lo + hi - 1) // 2)
        weights.append(hi - lo)
    return orders, weights


def estimate(N: int, eps: float, count: int, opts: _lib.sht_opts | None = None) -> dict:
    """Totals of the plan sht_plan_create(N, eps, opts) from a stratified
    sample of `count` orders (exact when count >= 2N)."""
    orders, weights = sample_orders(N, count)
    rows = _lib.sht_order_stats(N, eps, orders, opts)
    tot = {k: sum(w * r[k] for w, r in zip(weights, rows)) for k in SUMMED}
    for k in SUMMED:
        if not k.startswith("t_"):
            tot[k] = int(round(tot[k]))
    tot["max_rank"] = max(r["max_rank"] for r in rows)
    tot["max_rows"] = max(r["rows"] for r in rows)
    return {
        "N": N, "eps": eps, "orders_sampled": len(orders), "exact": len(orders) == 2 * N,
        "totals": tot,
        "stored_over_matrix": tot["entries_total"] / max(1, tot["entries_matrix"]),
        "factor_bytes": {"fp64": 8 * tot["factor_doubles"], "fp32": 4 * tot["factor_doubles"],
                         "mixed_images": 2 * tot["image_elems"]},
        "io_bytes_per_field": {"beta": 16 * 4 * N * N, "g": 16 * (4 * N - 1) * 2 * N},
        "precompute_thread_s": tot["t_mat_s"] + tot["t_fac_s"],
        "per_order": [dict(r, weight=w) for r, w in zip(rows, weights)],
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--N", type=int, required=True)
    ap.add_argument("--eps", type=float, default=1e-10)
    ap.add_argument("--sample", type=int, default=64, help="orders in the stratified sample")
    ap.add_argument("--at", default=None,
                    help="comma-separated orders as multiples of N (e.g. 0,0.5,1,1.5): per-order rows only")
    ap.add_argument("--n0", type=int, default=None)
    ap.add_argument("--n-leaf", type=int, default=None)
    ap.add_argument("--per-order", action="store_true", help="print the sampled orders' rows too")
    a = ap.parse_args(argv)
    o = _lib.sht_opts_default(a.N, a.eps)
    if a.n0:
        o.n0 = a.n0
    if a.n_leaf:
        o.n_leaf = a.n_leaf
    head = {"N": a.N, "eps": a.eps, "n0": o.n0, "n_leaf": o.n_leaf, "r_k": o.r_k, "threads": os.cpu_count()}
    if a.at:
        ms = [min(2 * a.N - 1, int(round(float(v) * a.N))) for v in a.at.split(",")]
        for r in _lib.sht_order_stats(a.N, a.eps, ms, o):
            print(json.dumps(dict(head, **r)))
        return
    est = estimate(a.N, a.eps, a.sample, o)
    rows = est.pop("per_order")
    if a.per_order:
        for r in rows:
            print(json.dumps(r))
    print(json.dumps(dict(head, **est)))


if __name__ == "__main__":
    main()
