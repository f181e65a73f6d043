"""Plan files (sht_plan_save / sht_plan_load).

Host-side: a saved and reloaded plan exports the same program byte for byte
and still reproduces the oracle through the test-only numpy apply; missing,
truncated, damaged and foreign files are refused with SHT_ERR_IO, including a
file whose checksum was recomputed over a program that addresses factors past
the end of the store (the consistency check, not the checksum, catches it),
statistics that name another N than the program, and element counts larger
than the rest of the file (refused before allocating).  Random forgeries of
the metadata with matching checksums are refused or load a program that
passes an independent bounds check.
GPU: a loaded plan of each precision gives the original plan's results.
"""
import struct

import numpy as np
import pytest

import host_apply
import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, inputs

HOST = _lib.SHT_FLAG_HOST_ONLY
PARTS = ("units", "ops", "phases", "factors", "order")
HEADER = 8 + 5 * 4 + 2 * 4  # magic, version and struct sizes, N and max_rows


def fnv1a(data: bytes) -> int:
    h = 0xcbf29ce484222325
    for b in data:
        h = ((h ^ b) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


@pytest.fixture(scope="module")
def saved(tmp_path_factory):
    p = sht.Plan(40, 1e-10, flags=HOST, n0=12, n_leaf=6)
    path = str(tmp_path_factory.mktemp("plans") / "n40.plan")
    p.save(path)
    return p, path


def test_round_trip_is_exact(saved):
    p, path = saved
    q = sht.Plan.load(path)
    assert q.host_only and q.N == p.N and q.eps == p.eps
    a, b = p.program(PARTS), q.program(PARTS)
    for k in PARTS:
        assert a[k].tobytes() == b[k].tobytes(), k
    sa, sb = p.stats(), q.stats()
    for k in ("entries_total", "n_ops", "n_blocks_idbf", "n_blocks_lowrank", "n_blocks_dense", "max_rank"):
        assert sa[k] == sb[k], k
    xa, wa = p.nodes()
    xb, wb = q.nodes()
    assert np.array_equal(xa, xb) and np.array_equal(wa, wb)


def test_loaded_program_reproduces_oracle(saved):
    _, path = saved
    q = sht.Plan.load(path)
    N = q.N
    beta = inputs.coefficients(N, 1, seed=5)
    g = host_apply.forward(q.program(), N, beta[0])
    ref = oracle.alt_forward(N, beta)[0]
    assert np.linalg.norm(g - ref) <= 1e-9 * np.linalg.norm(ref)


def expect_io(path):
    with pytest.raises(_lib.ShtError) as ei:
        sht.Plan.load(str(path))
    assert ei.value.status == _lib.SHT_ERR_IO


def test_missing_file(tmp_path):
    expect_io(tmp_path / "nothing.plan")


def test_foreign_and_damaged_files(saved, tmp_path):
    _, path = saved
    raw = open(path, "rb").read()
    cases = {
        "empty": b"",
        "text": b"not a plan file\n" * 8,
        "truncated": raw[: len(raw) // 2],
        "no_checksum": raw[:-8],
        "bad_magic": b"X" + raw[1:],
        "bad_version": raw[:8] + struct.pack("<I", 99) + raw[12:],
    }
    # one flipped bit in the middle of the factor store
    flip = bytearray(raw)
    flip[len(raw) // 2] ^= 0x10
    cases["bit_flip"] = bytes(flip)
    for name, data in cases.items():
        f = tmp_path / f"{name}.plan"
        f.write_bytes(data)
        expect_io(f)


def test_consistent_checksum_but_invalid_program(saved, tmp_path):
    """A program whose first op reads past the factor store is refused even
    with a matching checksum."""
    p, path = saved
    raw = bytearray(open(path, "rb").read())
    prog = p.program(("ops",))
    # locate the ops array: it is stored as (u64 count, 64-byte records)
    ops_bytes = prog["ops"].tobytes()
    at = bytes(raw).find(ops_bytes)
    assert at > HEADER and struct.unpack_from("<Q", raw, at - 8)[0] == len(prog["ops"])
    struct.pack_into("<q", raw, at, 1 << 40)  # b_off of op 0
    body = bytes(raw[:-8])
    bad = tmp_path / "forged.plan"
    bad.write_bytes(body + struct.pack("<Q", fnv1a(body)))
    expect_io(bad)
    # the same forgery without the change loads: the checksum routine matches
    good = tmp_path / "resealed.plan"
    orig = open(path, "rb").read()
    good.write_bytes(orig[:-8] + struct.pack("<Q", fnv1a(orig[:-8])))
    assert sht.Plan.load(str(good)).N == p.N


def test_statistics_must_describe_the_program(saved, tmp_path):
    """The statistics stored in the file carry N, which callers use to size
    their buffers: a file whose statistics name another N (or op count) than
    its program is refused even with a matching checksum."""
    import ctypes
    p, path = saved
    raw = open(path, "rb").read()
    info = HEADER + ctypes.sizeof(_lib.sht_opts)  # sht_plan_info follows the options
    assert struct.unpack_from("<i", raw, info)[0] == p.N
    n_ops = info + _lib.sht_plan_info.n_ops.offset
    for field, value, fmt in ((info, p.N - 8, "<i"), (info, p.N + 8, "<i"), (n_ops, 1, "<q")):
        b = bytearray(raw)
        struct.pack_into(fmt, b, field, value)
        body = bytes(b[:-8])
        bad = tmp_path / "stats.plan"
        bad.write_bytes(body + struct.pack("<Q", fnv1a(body)))
        expect_io(bad)


def test_counts_beyond_the_file_are_refused(saved, tmp_path):
    """An element count larger than the rest of the file is refused before
    anything is allocated (here: 2^39 ops, 32 TB)."""
    p, path = saved
    raw = bytearray(open(path, "rb").read())
    at = bytes(raw).find(p.program(("ops",))["ops"].tobytes())
    struct.pack_into("<Q", raw, at - 8, 1 << 39)
    body = bytes(raw[:-8])
    bad = tmp_path / "count.plan"
    bad.write_bytes(body + struct.pack("<Q", fnv1a(body)))
    expect_io(bad)


def check_bounds(q):
    """What the kernels rely on, restated independently of the library's check."""
    P = q.program(("units", "ops", "phases", "factors", "order"))
    N = q.N
    u, o, ph, f = P["units"], P["ops"], P["phases"], P["factors"]
    assert len(u) == 2 * N and sorted(P["order"]) == list(range(2 * N))
    for a in range(2 * N):
        U = u[a]
        assert U["am"] == a and 0 <= U["op_begin"] <= U["op_end"] <= len(o)
        assert U["ph_begin"] >= 0 and U["ph_begin"] + U["nphase"] + 1 <= len(ph)
        for op in o[U["op_begin"]: U["op_end"]]:
            assert op["ld"] >= op["mo"] >= 1 and op["b_off"] >= 0
            assert op["b_off"] + int(op["ld"]) * int(op["ni"]) <= len(f)
            assert op["in_len"].sum() == op["ni"] and op["out_len"].sum() == op["mo"]
            for s in range(2):
                assert op["in_len"][s] >= 0 and 0 <= op["in_off"][s] <= U["nrows"] - op["in_len"][s]
                assert op["out_len"][s] >= 0 and 0 <= op["out_off"][s] <= U["nrows"] - op["out_len"][s]
            assert 0 <= op["phase"] < U["nphase"]


def test_forged_metadata_is_refused_or_safe(tmp_path):
    """Random changes to the header, options, statistics, units, ops, phase
    table and schedule of a file, resealed with a matching checksum: every
    file either is refused or loads a program that passes check_bounds."""
    import random
    p = sht.Plan(12, 1e-10, flags=HOST | _lib.SHT_FLAG_FORCE_FACTOR, n0=6, n_leaf=3)
    path = tmp_path / "small.plan"
    p.save(str(path))
    raw = open(path, "rb").read()
    body0 = raw[:-8]
    prog = p.program(("units", "ops", "phases", "order"))
    regions = [(0, HEADER + 200)]
    for k in ("units", "ops", "phases", "order"):
        b = prog[k].tobytes()
        at = body0.find(b)
        assert at > 0
        regions.append((at - 8, at + len(b)))
    rng = random.Random(2004)
    vals = [0, 1, -1, 2, 7, 8, 9, 63, 64, 65, 1 << 15, 1 << 30, -(1 << 31), (1 << 31) - 1]
    outcomes = {}
    for t in range(150):
        b = bytearray(body0)
        for _ in range(rng.randint(1, 2)):
            lo, hi = rng.choice(regions)
            off = rng.randrange(lo, hi - 4) & ~3
            if rng.random() < 0.5:
                struct.pack_into("<i", b, off, rng.choice(vals))
            else:
                struct.pack_into("<i", b, off, struct.unpack_from("<i", b, off)[0] + rng.choice([-9, -8, -1, 1, 8, 9]))
        body = bytes(b)
        f = tmp_path / "forged.plan"
        f.write_bytes(body + struct.pack("<Q", fnv1a(body)))
        try:
            q = sht.Plan.load(str(f))
        except _lib.ShtError as e:
            assert e.status in (_lib.SHT_ERR_IO, _lib.SHT_ERR_OOM, _lib.SHT_ERR_CUDA), e.status
            outcomes[e.status] = outcomes.get(e.status, 0) + 1
            continue
        check_bounds(q)
        outcomes["loaded"] = outcomes.get("loaded", 0) + 1
        q.close()
    assert outcomes.get(_lib.SHT_ERR_IO, 0) > 50 and outcomes.get("loaded", 0) > 5


def test_intermediate_segments_must_start_on_row_groups(tmp_path):
    """Moving one intermediate output segment off its 8-row boundary makes a
    file with a consistent checksum fail the program check; moving it by a
    whole group (still inside the vector space) does not."""
    p = sht.Plan(40, 1e-10, flags=HOST | _lib.SHT_FLAG_FORCE_FACTOR, n0=12, n_leaf=6)
    path = str(tmp_path / "factored.plan")
    p.save(path)
    raw = bytes(open(path, "rb").read())
    prog = p.program(("units", "ops"))
    units, ops = prog["units"], prog["ops"]
    at = raw.find(ops.tobytes())
    assert at > HEADER
    pick = None
    for u in units:
        for k in range(u["op_begin"], u["op_end"]):
            o = ops[k]
            if o["out_len"][0] > 0 and o["out_off"][0] >= u["yo"] + p.N and \
                    o["out_off"][0] + o["out_len"][0] + 8 <= u["nrows"]:
                pick = k
                break
        if pick is not None:
            break
    assert pick is not None

    def forged(shift, name):
        b = bytearray(raw)
        field = at + 64 * pick + 40  # Op.out_off[0]
        struct.pack_into("<i", b, field, int(ops[pick]["out_off"][0]) + shift)
        body = bytes(b[:-8])
        out = tmp_path / name
        out.write_bytes(body + struct.pack("<Q", fnv1a(body)))
        return out

    expect_io(forged(1, "unaligned.plan"))
    assert sht.Plan.load(str(forged(8, "shifted.plan"))).N == p.N


@pytest.mark.gpu
@pytest.mark.parametrize("prec,F,tol", [(_lib.SHT_FP64, 2, 1e-13), (_lib.SHT_MIXED, 33, 1e-6)])
def test_loaded_plan_on_gpu(tmp_path, prec, F, tol):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N = 96
    p = sht.Plan(N, 1e-12 if prec == _lib.SHT_FP64 else 1e-7, precision=prec)
    path = str(tmp_path / "p.plan")
    p.save(path)
    q = sht.Plan.load(path)
    beta = torch.from_numpy(inputs.coefficients(N, F, seed=8)).cuda()
    ga, gb = p.forward(beta), q.forward(beta)
    ba, bb = p.inverse(ga), q.inverse(gb)
    torch.cuda.synchronize()
    p.sync()
    q.sync()
    assert float((ga - gb).norm() / ga.norm()) <= tol
    assert float((ba - bb).norm() / ba.norm()) <= tol
    ref = oracle.alt_forward(N, beta.cpu().numpy())
    e = np.linalg.norm(gb.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert e <= (1e-10 if prec == _lib.SHT_FP64 else 1e-6)
