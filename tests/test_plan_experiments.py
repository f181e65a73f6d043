"""The paper's plan experiment on block counts (Sec. 5, first experiment), CPU.

After the blocks that hold no non-negligible entry are dropped, the number of
remaining blocks of one order grows nearly linearly with N, for m = N/2, N and
3N/2 (the paper's figure of block counts; its data is not printed).  Here with
the partition's stop size fixed (n0 = 32) as in the paper (n0 = 512 over its
larger N), so that deeper partitions come from N alone.
"""
import numpy as np

import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib

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
