"""The paper's plan experiments of Sec. 5 that need no timing, CPU.

Block counts: after the blocks that hold no non-negligible entry are dropped,
the number of remaining blocks of one order grows nearly linearly with N, for
m = N/2, N and 3N/2 (the paper's figure of block counts; its data is not
printed).  Here with the partition's stop size fixed (n0 = 32) as in the paper
(n0 = 512 over its larger N), so that deeper partitions come from N alone.

Error against the order: the paper's relative errors of the forward and
inverse ALT of one order, over 256 sampled rows (nodes, resp. degrees) of the
even or odd matrix (its eps^fwd and eps^inv), are not affected by m: every
order stays within the tolerance, and none is less accurate than m = 0.
order_errors computes them for the matrices a plan represents, against the
oracle's.
"""
import numpy as np

import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib
from test_factorization import represented

HOST = _lib.SHT_FLAG_HOST_ONLY


def remaining(N, **kw):
    p = sht.Plan(N, 1e-10, flags=HOST, n0=32, n_leaf=8, **kw)
    ub = p.program(("unit_blocks",))["unit_blocks"].reshape(-1, 4)
    st = p.stats()
    # the per-order counts add up to the plan's totals
    assert ub.shape[0] == 2 * N
    assert ub[:, 0].sum() == st["n_blocks_idbf"] and ub[:, 1].sum() == st["n_blocks_lowrank"]
    assert ub[:, 2].sum() == st["n_blocks_dense"] and ub[:, 3].sum() == st["n_blocks_dropped"]
    return {f: int(ub[int(f * N), :3].sum()) for f in (0.5, 1.0, 1.5)}


def test_remaining_blocks_grow_nearly_linearly():
    counts = {N: remaining(N) for N in (64, 128, 256, 512)}
    for f in (0.5, 1.0, 1.5):
        seq = [counts[N][f] for N in (64, 128, 256, 512)]
        assert all(a < b for a, b in zip(seq, seq[1:])), (f, seq)
        # doubling N at the largest sizes: about 2 (linear) to 2.25 (N log N),
        # far from the 4 of a quadratic growth
        assert 1.6 <= seq[-1] / seq[-2] <= 2.6, (f, seq)


def test_loaded_plans_have_no_block_counts(tmp_path):
    p = sht.Plan(16, 1e-10, flags=HOST)
    path = str(tmp_path / "p.plan")
    p.save(path)
    q = sht.Plan.load(path)
    assert q.program(("unit_blocks",))["unit_blocks"].size == 0


def order_errors(p, prog, am, rng):
    """[(eps_fwd, eps_inv)] of the even and odd matrix of order |m| = am:
    random N(0,1) right-hand sides (Re, Im), 256 sampled rows (or all)."""
    N = p.N
    x, w = p.nodes()
    xp, wp = x[N:], w[N:]
    T = oracle.alf_table(am, 2 * N - 1, xp)
    ae, ao, _, _ = represented(prog, prog["units"][am])
    out = []
    for pm, ref in ((ae, T[:, 0::2]), (ao, T[:, 1::2])):
        if ref.size == 0:
            continue
        xv = rng.standard_normal((ref.shape[1], 2))
        s1 = rng.choice(N, min(256, N), replace=False)
        gb, gd = (pm @ xv)[s1], (ref @ xv)[s1]
        gv = rng.standard_normal((N, 2)) * wp[:, None]
        s2 = rng.choice(ref.shape[1], min(256, ref.shape[1]), replace=False)
        ab, ad = (pm.T @ gv)[s2], (ref.T @ gv)[s2]
        out.append((float(np.sqrt(((gb - gd) ** 2).sum() / (gd ** 2).sum())),
                    float(np.sqrt(((ab - ad) ** 2).sum() / (ad ** 2).sum()))))
    return out


def test_error_does_not_depend_on_the_order():
    # factored blocks kept even where they are larger than dense, so that
    # every order has IDBF blocks at this small N
    N, eps = 128, 1e-10
    p = sht.Plan(N, eps, flags=HOST | _lib.SHT_FLAG_FORCE_FACTOR)
    prog = p.program()
    rng = np.random.default_rng(0)
    ams = [min(2 * N - 1, int(f * N)) for f in (0, 0.5, 1.0, 1.5)]
    errs = {am: order_errors(p, prog, am, rng) for am in ams}
    flat = [e for v in errs.values() for pair in v for e in pair]
    assert max(flat) <= 2 * eps, errs
    # no order is less accurate than m = 0, whose matrices are single
    # butterflies of the greatest depth (larger orders hold smaller, shallower
    # ones next to trimmed turning-point blocks)
    worst = [max(e for pair in errs[am] for e in pair) for am in ams]
    assert max(worst[1:]) <= 1.5 * worst[0], errs
