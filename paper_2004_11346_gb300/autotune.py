"""Autotuning of the plan parameters for the tensor-core apply.

The factorisation has two free size parameters: the partition stops splitting
turning-point blocks below n0 rows or columns (Sec. 3.2), and the IDBF leaves
hold n_leaf rows (Sec. 2.2, the depth L follows from it).  They trade stored
factor entries against the shapes of the block products.  For the split-BF16
tensor-core apply the time follows the pipeline stages, one per 128-row tile
and 32-wide K chunk of every product, and the bytes those stages move. Entries
alone are a poor guide: smaller leaves store fewer entries in more, skinnier
products.

autotune() ranks candidate (n0, n_leaf) pairs by that work model on host-only
plans (no GPU needed), then builds the best few on the device, times a forward
and an inverse apply of the requested batch with CUDA events, and keeps the
fastest; on it, it then times the queue orders of the persistent kernel (the
m-to-CTA schedule, schedule()) and keeps the fastest of those too.  The model's counts mirror how the kernel cuts the work: segments
moved to the kernel's scratch rows (X_o, Y_e and Y_o start on whole groups),
K sides widened to whole 8-row groups, chunks of 4 groups (the last rounded
to an even number), the outputs of products that write intermediate rows
widened to whole groups too, N tiles of 128 rows padded to 16.
"""
from __future__ import annotations

import numpy as np

from . import _lib

TILE_N = 128       # rows of one tensor-core tile
GROUP_ROWS = 8     # rows of one activation group
GROUP_BYTES = 6144  # one group: 8 rows x 3 BF16 pieces x 128 right-hand sides
CHUNK_GROUPS = 4   # groups of one K chunk (32 rows)
FWD_ACCUM = 1      # op flag: forward outputs accumulate (Y rows)


def _r8(v):
    return (v + 7) & ~7


def scratch_rows(nce, nco, N):
    """(xo, ye, yo, shift) of the tensor-core scratch layout of one order:
    X_o, Y_e and Y_o start on whole groups, intermediates move by `shift`."""
    xo = _r8(nce)
    ye = _r8(xo + nco)
    yo = ye + _r8(N)
    return xo, ye, yo, _r8(yo + N) - _r8(nce + nco + 2 * N)


def _seg_row(off, nce, nco, N, rows):
    xo, ye, yo, shift = rows
    if off < nce:
        return off
    if off < nce + nco:
        return off - nce + xo
    if off < nce + nco + N:
        return off - nce - nco + ye
    if off < nce + nco + 2 * N:
        return off - nce - nco - N + yo
    return off + shift


def _groups(off0, len0, off1, len1):
    """Groups of one side of a product (two row segments) widened to whole groups."""
    ng0 = (off0 + len0 + GROUP_ROWS - 1) // GROUP_ROWS - off0 // GROUP_ROWS if len0 > 0 else 0
    ng1 = (off1 + len1 + GROUP_ROWS - 1) // GROUP_ROWS - off1 // GROUP_ROWS if len1 > 0 else 0
    return ng0 + ng1


def _kside(ngt):
    """K chunks and padded K columns of a side of ngt groups."""
    nk = (ngt + CHUNK_GROUPS - 1) // CHUNK_GROUPS
    kp = 32 * (nk - 1) + 16 * ((ngt - CHUNK_GROUPS * (nk - 1) + 1) // 2) if nk > 0 else 0
    return nk, kp


def work_model(ops, units, N) -> dict:
    """Stages, tiles, operand-image and activation bytes of one forward apply
    of one 32-field group, from a plan's op and unit records (Plan.program()):
    segments moved to the scratch rows, K sides widened to whole groups, the
    outputs of non-accumulating products widened likewise, tiles of TILE_N."""
    stages = tiles = img = act = 0
    for u in units:
        nce, nco = int(u["nce"]), int(u["nco"])
        rows = scratch_rows(nce, nco, N)
        for k in range(int(u["op_begin"]), int(u["op_end"])):
            op = ops[k]
            if op["ni"] <= 0:
                continue

            def segs(offs, lens):
                return [_seg_row(int(o), nce, nco, N, rows) if int(l) > 0 else 0 for o, l in zip(offs, lens)]
            io, il = segs(op["in_off"], op["in_len"]), [int(v) for v in op["in_len"]]
            ngt = _groups(io[0], il[0], io[1], il[1])
            nk, kp = _kside(ngt)
            if int(op["flags"]) & FWD_ACCUM:
                nn = int(op["mo"])
            else:
                oo, ol = segs(op["out_off"], op["out_len"]), [int(v) for v in op["out_len"]]
                nn = GROUP_ROWS * _groups(oo[0], ol[0], oo[1], ol[1])
            nt = (nn + TILE_N - 1) // TILE_N
            np_tot = TILE_N * (nt - 1) + ((nn - TILE_N * (nt - 1) + 15) & ~15)
            stages += nt * nk
            tiles += nt
            img += 2 * 3 * np_tot * kp
            act += nt * ngt * GROUP_BYTES
    return {"stages": int(stages), "tiles": int(tiles), "image_bytes": int(img), "activation_bytes": int(act)}


def model_cost(w: dict, stage_us: float = 1.2, sms: int = 152, gbps: float = 4000.0) -> float:
    """Predicted microseconds of one forward launch per field group: the larger
    of the stage pipeline (stage_us per stage per SM, the measured rate of the
    kernel) and the bytes at gbps."""
    return max(w["stages"] * stage_us / sms, (w["image_bytes"] + w["activation_bytes"]) / (gbps * 1e3))


def candidates(N: int, eps: float):
    """(n0, n_leaf) pairs around the defaults of sht_opts_default: n0 halved
    and doubled, n_leaf from half to four times the default (larger leaves make
    fewer, fuller tensor-core products)."""
    d = _lib.sht_opts_default(N, eps)
    out = []
    for n0 in (d.n0 // 2, d.n0, d.n0 * 2):
        for nl in (d.n_leaf // 2, d.n_leaf, d.n_leaf * 2, d.n_leaf * 4):
            if n0 >= 8 and 4 <= nl <= n0 and (n0, nl) not in out:
                out.append((n0, nl))
    return out


def sampled_work_model(N: int, eps: float, sample: int, **plan_kw):
    """work_model and stored entries of the plan with these options, summed
    over a stratified sample of `sample` orders built one by one on the host
    (sht_order_stats; exact when sample >= 2N).  A full host plan at large N
    holds its whole FP64 factor store in memory; a sample holds a few orders."""
    from . import opts, orders
    est = orders.estimate(N, eps, sample, opts(N, eps, precision=_lib.SHT_MIXED, **plan_kw))
    t = est["totals"]
    w = {"stages": t["tc_stages"], "tiles": t["tc_tiles"], "image_bytes": t["tc_image_fwd_bytes"],
         "activation_bytes": t["tc_act_bytes"]}
    return w, t["entries_total"]


def rank(N: int, eps: float, cands=None, sample: int | None = None, **plan_kw):
    """Every candidate ranked by model_cost (best first): from a host-only
    plan of each, or, with `sample`, from that many sampled orders."""
    from . import Plan
    rows = []
    for n0, nl in cands or candidates(N, eps):
        if sample:
            w, entries = sampled_work_model(N, eps, sample, n0=n0, n_leaf=nl, **plan_kw)
        else:
            p = Plan(N, eps, flags=_lib.SHT_FLAG_HOST_ONLY, precision=_lib.SHT_MIXED, n0=n0, n_leaf=nl, **plan_kw)
            prog = p.program(("ops", "units"))
            w = work_model(prog["ops"], prog["units"], N)
            entries = int(p.stats()["entries_total"])
            p.close()
        rows.append({"n0": n0, "n_leaf": nl, "entries": int(entries), **w, "model_us": model_cost(w)})
    rows.sort(key=lambda r: r["model_us"])
    return rows


SCHEDULES = ("lpt", "pairs", "ascending")


def schedule(units, kind: str) -> np.ndarray:
    """A queue order of the units (the m-to-CTA schedule) from a plan's unit
    records: "lpt", decreasing modelled cost (the order plans start with);
    "pairs", the costliest and the cheapest remaining units alternately, so
    that the CTAs in flight mix large and small working sets; "ascending",
    |m| = 0, 1, ... (an order's work falls with |m|)."""
    cost = np.asarray(units["cost"], dtype=np.float64)
    am = np.asarray(units["am"], dtype=np.int32)
    lpt = am[np.argsort(-cost, kind="stable")]
    if kind == "lpt":
        return lpt
    if kind == "pairs":
        out = np.empty_like(lpt)
        out[0::2] = lpt[: (len(lpt) + 1) // 2]
        out[1::2] = lpt[::-1][: len(lpt) // 2]
        return out
    if kind == "ascending":
        return np.sort(am)
    raise ValueError(kind)


def _time_round_trip(torch, p, beta, gv, back, steps):
    p.forward(beta, out=gv)
    p.inverse(gv, out=back)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        p.forward(beta, out=gv)
        p.inverse(gv, out=back)
    e1.record()
    torch.cuda.synchronize()
    p.sync()
    return e0.elapsed_time(e1) / steps


def tune_schedule(p, beta, gv, back, steps: int = 3):
    """Time every schedule of SCHEDULES on plan p (forward + inverse of the
    given batch), leave the fastest set on the plan and return one row per
    schedule."""
    import torch
    units = p.program(("units",))["units"]
    rows = []
    for kind in SCHEDULES:
        p.set_order(schedule(units, kind))
        rows.append({"schedule": kind, "measured_ms": _time_round_trip(torch, p, beta, gv, back, steps)})
    best = min(rows, key=lambda r: r["measured_ms"])
    p.set_order(schedule(units, best["schedule"]))
    return rows


def autotune(N: int, eps: float, fields: int, top: int = 3, steps: int = 3, cands=None, seed: int = 0,
             sample: int | None = None, schedules: bool = True):
    """Rank the candidates by the work model (from sampled orders when
    `sample` is given), time the best `top` of them on the current CUDA
    device (forward + inverse ALT of `fields` random fields, CUDA events,
    after a warm-up), then, on the fastest, time the queue orders of
    SCHEDULES, and return (best Plan, table of all rows).  The returned plan
    is built on the device with the winning parameters and schedule."""
    import torch
    from . import Plan
    rows = rank(N, eps, cands, sample=sample, max_fields=fields)
    g = torch.Generator(device="cuda").manual_seed(seed)
    beta = torch.randn((fields, 4 * N * N, 2), dtype=torch.float64, device="cuda", generator=g)
    gv = torch.empty((fields, 4 * N - 1, 2 * N, 2), dtype=torch.float64, device="cuda")
    back = torch.empty_like(beta)
    best, best_ms = None, float("inf")
    for r in rows[:top]:
        p = Plan(N, eps, precision=_lib.SHT_MIXED, n0=r["n0"], n_leaf=r["n_leaf"], max_fields=fields)
        r["measured_ms"] = _time_round_trip(torch, p, beta, gv, back, steps)
        if r["measured_ms"] < best_ms:
            if best is not None:
                best.close()
            best, best_ms = p, r["measured_ms"]
        else:
            p.close()
    if schedules:
        for s in tune_schedule(best, beta, gv, back, steps):
            rows.append({"n0": int(best.opts.n0), "n_leaf": int(best.opts.n_leaf), **s})
    return best, rows


def main(argv=None):
    """python -m paper_2004_11346_gb300.autotune --N 1024 --eps 1e-7 --fields 64:
    prints one JSON line per candidate (model counts, and the measured ms of the
    timed ones) and a last line with the winner."""
    import argparse
    import json
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--N", type=int, required=True)
    ap.add_argument("--eps", type=float, default=1e-7)
    ap.add_argument("--fields", type=int, default=32)
    ap.add_argument("--top", type=int, default=3)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--cands", default=None, help="n0:n_leaf,... to rank instead of the default grid")
    ap.add_argument("--sample", type=int, default=None,
                    help="rank from this many sampled orders instead of full host-only plans")
    ap.add_argument("--rank-only", action="store_true", help="print the model's ranking only (no GPU)")
    a = ap.parse_args(argv)
    cands = [tuple(int(v) for v in c.split(":")) for c in a.cands.split(",")] if a.cands else None
    if a.rank_only:
        for r in rank(a.N, a.eps, cands, sample=a.sample, max_fields=a.fields):
            print(json.dumps(r), flush=True)
        return
    plan, rows = autotune(a.N, a.eps, a.fields, top=a.top, steps=a.steps, cands=cands, sample=a.sample)
    for r in rows:
        print(json.dumps(r), flush=True)
    sched = [r for r in rows if "schedule" in r]
    best_sched = min(sched, key=lambda r: r["measured_ms"])["schedule"] if sched else "lpt"
    print(json.dumps({"best": {"n0": int(plan.opts.n0), "n_leaf": int(plan.opts.n_leaf), "schedule": best_sched},
                      "N": a.N, "eps": a.eps, "fields": a.fields}), flush=True)


if __name__ == "__main__":
    main()
