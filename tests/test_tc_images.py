"""The tensor-core operand images against the factors they encode (CPU).

Every op's image (sht_plan_op_image) is decoded here with the layout the
header documents: tiles of 128 rows padded to 16, K chunks of 32 (the last one
rounded to an even number of 8-row groups), each chunk piece by piece in 8 x 8
core matrices, K-outer.  The K side is the op's input segments widened to whole
8-row groups of the vector space.  Checked: the three BF16 pieces of every
position sum to the FP64 factor entry (or its transpose) to within the 24 bits
three pieces carry (values far below FP32's normal range, where the lower
pieces are subnormal, within 2^-126 absolute), every widened or padded
position is zero in all pieces,
and the image has exactly the size the layout implies.
"""
import numpy as np
import pytest

import host_apply
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib

HOST = _lib.SHT_FLAG_HOST_ONLY


def r16(v):
    return (v + 15) // 16 * 16


def widened(off0, len0, off1, len1):
    """Rows of the vector space behind each widened K position, and the K index
    of the unwidened side there (-1 where the position only pads)."""
    g0, n0 = off0 // 8, ((off0 + len0 + 7) // 8 - off0 // 8) if len0 > 0 else 0
    g1, n1 = off1 // 8, ((off1 + len1 + 7) // 8 - off1 // 8) if len1 > 0 else 0
    korig = []
    for j in range(n0 + n1):
        for e in range(8):
            if j < n0:
                r = (g0 + j) * 8 + e
                korig.append(r - off0 if off0 <= r < off0 + len0 else -1)
            else:
                r = (g1 + j - n0) * 8 + e
                korig.append(len0 + r - off1 if off1 <= r < off1 + len1 else -1)
    ngt = n0 + n1
    nk = (ngt + 3) // 4
    kp_tot = 32 * (nk - 1) + 16 * ((ngt - 4 * (nk - 1) + 1) // 2) if nk else 0
    korig += [-1] * (kp_tot - len(korig))
    return np.array(korig, dtype=np.int64), nk, kp_tot


def bf16_to_f64(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def decode(img, NN, kp_tot):
    """(3, NN_pad, kp_tot) piece values and the total length the layout implies."""
    nt = (NN + 127) // 128
    np_tot = 128 * (nt - 1) + r16(NN - 128 * (nt - 1))
    out = np.zeros((3, np_tot, kp_tot))
    o = 0
    for t in range(nt):
        Np = r16(min(128, NN - 128 * t))
        for c in range((kp_tot + 31) // 32):
            Kp = min(32, kp_tot - 32 * c)
            for p in range(3):
                blk = bf16_to_f64(img[o: o + Np * Kp]).reshape(Kp // 8, Np // 8, 8, 8)  # (ki, mi, rr, kk)
                out[p, 128 * t: 128 * t + Np, 32 * c: 32 * c + Kp] = blk.transpose(1, 2, 0, 3).reshape(Np, Kp)
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
    ops = prog["ops"]
    two_segment = multi_tile = 0
    for k in range(len(ops)):
        op = ops[k]
        if op["ni"] == 0:
            continue
        B = host_apply._block(prog, op)  # mo x ni
        for transposed in (False, True):
            M = B.T if transposed else B
            segs = (op["out_off"][0], op["out_len"][0], op["out_off"][1], op["out_len"][1]) if transposed else \
                   (op["in_off"][0], op["in_len"][0], op["in_off"][1], op["in_len"][1])
            two_segment += int(segs[3] > 0)
            korig, nk, kp_tot = widened(*(int(v) for v in segs))
            img = _lib.sht_plan_op_image(p.handle, k, transposed)
            pieces, length = decode(img, M.shape[0], kp_tot)
            multi_tile += int(M.shape[0] > 128)
            assert length == len(img)
            want = np.zeros(pieces.shape[1:])
            cols = korig >= 0
            want[: M.shape[0], cols] = M[:, korig[cols]]
            got = pieces.sum(axis=0)
            assert np.all(np.abs(got - want) <= 2.0 ** -23 * np.abs(want) + 2.0 ** -126), (k, transposed)
            # widened and padded positions are zero in every piece
            assert not np.any(pieces[:, :, ~cols]) and not np.any(pieces[:, M.shape[0]:, :])
            # piece p + 1 is what piece p leaves: at most half an ulp of BF16 below it
            assert np.all(np.abs(pieces[1]) <= 2.0 ** -8 * np.abs(pieces[0]) + 2.0 ** -126)
    if kind == "butterflies":
        assert two_segment > 0  # products whose K side is two segments (butterfly levels)
    else:
        assert multi_tile > 0  # images of more than one 128-row tile


def test_argument_errors(plan):
    p, prog, _ = plan
    with pytest.raises(_lib.ShtError):
        _lib.sht_plan_op_image(p.handle, len(prog["ops"]), False)
    with pytest.raises(_lib.ShtError):
        _lib.sht_plan_op_image(p.handle, -1, True)
