"""The tensor-core operand images against the factors they encode (CPU).

Every op's image (sht_plan_op_image) is decoded here with the layout the
kernel uses, restated independently:
  - segments move to the kernel's scratch rows: X_e at 0, X_o, Y_e and Y_o
    each at the next multiple of 8 after the previous region (Y_o r8(N) rows
    after Y_e), intermediate segments shifted by a multiple of 8;
  - the K side (the op's inputs in that direction) is widened to whole 8-row
    groups of scratch rows; so is the N side (its outputs) unless they
    accumulate into the item's FP32 rows (Y forward, X transposed);
  - tiles of 128 N positions padded to 16, K chunks of 32 (the last one
    rounded to an even number of groups), each chunk piece by piece in 8 x 8
    core matrices, K-outer.
Checked: the three BF16 pieces of every position sum to the FP64 factor entry
(or its transpose) to within the 24 bits three pieces carry (values far below
FP32's normal range, where the lower pieces are subnormal, within 2^-126
absolute), every widened or padded position is zero in all pieces, and the
image has exactly the size the layout implies.
"""
import numpy as np
import pytest

import host_apply
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib

HOST = _lib.SHT_FLAG_HOST_ONLY
TILE = 128


def r16(v):
    return (v + 15) // 16 * 16


def r8(v):
    return (v + 7) // 8 * 8


def scratch_row(off, nce, nco, N):
    xo = r8(nce)
    ye = r8(xo + nco)
    yo = ye + r8(N)
    if off < nce:
        return off
    if off < nce + nco:
        return off - nce + xo
    if off < nce + nco + N:
        return off - nce - nco + ye
    if off < nce + nco + 2 * N:
        return off - nce - nco - N + yo
    return off + r8(yo + N) - r8(nce + nco + 2 * N)


def widened(off0, len0, off1, len1):
    """Index into the unwidened side behind each widened position (-1 where the
    position only pads) and the number of whole groups."""
    g0, n0 = off0 // 8, ((off0 + len0 + 7) // 8 - off0 // 8) if len0 > 0 else 0
    g1, n1 = off1 // 8, ((off1 + len1 + 7) // 8 - off1 // 8) if len1 > 0 else 0
    idx = []
    for j in range(n0 + n1):
        for e in range(8):
            if j < n0:
                r = (g0 + j) * 8 + e
                idx.append(r - off0 if off0 <= r < off0 + len0 else -1)
            else:
                r = (g1 + j - n0) * 8 + e
                idx.append(len0 + r - off1 if off1 <= r < off1 + len1 else -1)
    return np.array(idx, dtype=np.int64), n0 + n1


def kside(off0, len0, off1, len1):
    korig, ngt = widened(off0, len0, off1, len1)
    nk = (ngt + 3) // 4
    kp_tot = 32 * (nk - 1) + 16 * ((ngt - 4 * (nk - 1) + 1) // 2) if nk else 0
    korig = np.concatenate([korig, -np.ones(kp_tot - len(korig), dtype=np.int64)])
    return korig, nk, kp_tot


def bf16_to_f64(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def decode(img, NN, kp_tot):
    """(3, NN_pad, kp_tot) piece values and the total length the layout implies."""
    nt = (NN + TILE - 1) // TILE
    np_tot = TILE * (nt - 1) + r16(NN - TILE * (nt - 1))
    out = np.zeros((3, np_tot, kp_tot))
    o = 0
    for t in range(nt):
        Np = r16(min(TILE, NN - TILE * t))
        for c in range((kp_tot + 31) // 32):
            Kp = min(32, kp_tot - 32 * c)
            for p in range(3):
                blk = bf16_to_f64(img[o: o + Np * Kp]).reshape(Kp // 8, Np // 8, 8, 8)  # (ki, mi, rr, kk)
                out[p, TILE * t: TILE * t + Np, 32 * c: 32 * c + Kp] = blk.transpose(1, 2, 0, 3).reshape(Np, Kp)
                o += Np * Kp
    return out, o


@pytest.fixture(scope="module", params=["butterflies", "wide_blocks"])
def plan(request):
    # forced butterflies at N=40 (two-segment K sides), and a plan with wide
    # dense blocks whose transposed images span several 128-row tiles
    if request.param == "butterflies":
        p = sht.Plan(40, 1e-7, flags=HOST | _lib.SHT_FLAG_FORCE_FACTOR, precision=_lib.SHT_MIXED, n0=12, n_leaf=6)
    else:
        p = sht.Plan(160, 1e-7, flags=HOST, precision=_lib.SHT_MIXED, n0=80, n_leaf=64)
    return p, p.program(), request.param


def test_images_encode_the_factors(plan):
    p, prog, kind = plan
    ops, units = prog["ops"], prog["units"]
    N = p.N
    unit_of = np.zeros(len(ops), dtype=np.int64)
    for ui, u in enumerate(units):
        unit_of[u["op_begin"]: u["op_end"]] = ui
    two_segment = multi_tile = widened_out = 0
    for k in range(len(ops)):
        op = ops[k]
        if op["ni"] == 0:
            continue
        u = units[unit_of[k]]
        nce, nco = int(u["nce"]), int(u["nco"])

        def segs(offs, lens):
            return [scratch_row(int(o), nce, nco, N) if int(l) > 0 else 0 for o, l in zip(offs, lens)], \
                   [int(v) for v in lens]
        ins, outs = segs(op["in_off"], op["in_len"]), segs(op["out_off"], op["out_len"])
        B = host_apply._block(prog, op)  # mo x ni
        for transposed in (False, True):
            M = B.T if transposed else B
            ks, ns = (outs, ins) if transposed else (ins, outs)
            accum = bool(int(op["flags"]) & (2 if transposed else 1))
            two_segment += int(ks[1][1] > 0)
            korig, nk, kp_tot = kside(ks[0][0], ks[1][0], ks[0][1], ks[1][1])
            if accum:
                norig = np.arange(M.shape[0])
            else:
                norig, _ = widened(ns[0][0], ns[1][0], ns[0][1], ns[1][1])
                widened_out += int(len(norig) > M.shape[0])
            NN = len(norig)
            img = _lib.sht_plan_op_image(p.handle, k, transposed)
            pieces, length = decode(img, NN, kp_tot)
            multi_tile += int(NN > TILE)
            assert length == len(img)
            want = np.zeros(pieces.shape[1:])
            cols, rows = korig >= 0, np.nonzero(norig >= 0)[0]
            want[np.ix_(rows, np.nonzero(cols)[0])] = M[np.ix_(norig[rows], korig[cols])]
            got = pieces.sum(axis=0)
            assert np.all(np.abs(got - want) <= 2.0 ** -23 * np.abs(want) + 2.0 ** -126), (k, transposed)
            # widened and padded positions are zero in every piece
            assert not np.any(pieces[:, :, ~cols]) and not np.any(pieces[:, NN:, :])
            assert not np.any(pieces[:, np.nonzero(norig < 0)[0], :])
            # piece p + 1 is what piece p leaves: at most half an ulp of BF16 below it
            assert np.all(np.abs(pieces[1]) <= 2.0 ** -8 * np.abs(pieces[0]) + 2.0 ** -126)
    if kind == "butterflies":
        assert two_segment > 0  # products whose K side is two segments (butterfly levels)
        assert widened_out > 0  # intermediate outputs widened to whole groups
    else:
        assert multi_tile > 0  # images of more than one 128-row tile


def test_argument_errors(plan):
    p, prog, _ = plan
    with pytest.raises(_lib.ShtError):
        _lib.sht_plan_op_image(p.handle, len(prog["ops"]), False)
    with pytest.raises(_lib.ShtError):
        _lib.sht_plan_op_image(p.handle, -1, True)
