"""Host-side checks of libsht.so (no GPU needed).

- the library builds, loads and exports every function include/sht.h declares;
- argument errors are reported before any device work;
- host-only plans: the exported apply program, evaluated in numpy by the
  test-only host_apply module, reproduces the oracle's forward and inverse ALT,
  which pins the precomputation (Legendre matrices, partition, ID, IDBF, rSVD)
  independently of the kernels.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import host_apply
import oracle
import paper_2004_11346_gb300 as sht
from paper_2004_11346_gb300 import _lib, build, inputs

HOST = _lib.SHT_FLAG_HOST_ONLY
FORCE = _lib.SHT_FLAG_FORCE_FACTOR


def declared_functions():
    text = open(os.path.join(build.INCLUDE, "sht.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_functions()
    assert "alt_forward" in names and "sht_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(_lib.EXPORTED) <= set(names)


def test_status_strings():
    lib = _lib.load()
    assert lib.sht_status_str(0) == b"ok"
    assert lib.sht_status_str(3).startswith(b"CUDA")


def test_argument_errors_need_no_device():
    lib = _lib.load()
    h = ctypes.c_void_p()
    assert lib.sht_plan_create(0, 1e-12, None, ctypes.byref(h)) == 1
    assert lib.sht_plan_create(16, 0.0, None, ctypes.byref(h)) == 1
    assert lib.sht_plan_create(16, 1.5, None, ctypes.byref(h)) == 1
    assert lib.alt_forward(None, None, None, 1, None) == 1
    o = sht.opts(16, 1e-12, n_leaf=0)
    assert lib.sht_plan_create(16, 1e-12, ctypes.byref(o), ctypes.byref(h)) == 1
    # host-only plans cannot take the device's Legendre matrices nor be direct
    for fl in (_lib.SHT_FLAG_GPU_LEGENDRE, _lib.SHT_FLAG_DIRECT):
        o = sht.opts(16, 1e-12, flags=HOST | fl)
        assert lib.sht_plan_create(16, 1e-12, ctypes.byref(o), ctypes.byref(h)) == 1


def test_host_only_plan_refuses_device_calls():
    p = sht.Plan(8, 1e-12, flags=HOST)
    with pytest.raises(_lib.ShtError) as e:
        _lib.alt_forward(p.handle, 16, 16, 1, 0)
    assert e.value.status == 7


def test_batch_argument_errors_need_no_device():
    lib = _lib.load()
    h = ctypes.c_void_p()
    assert lib.sht_batch_create(0, None, None, ctypes.byref(h)) == _lib.SHT_ERR_ARG
    p = sht.Plan(8, 1e-7, flags=HOST, precision=_lib.SHT_MIXED)
    with pytest.raises(_lib.ShtError) as e:  # more plans than one launch takes
        _lib.sht_batch_create([p.handle] * 9, [1] * 9)
    assert e.value.status == _lib.SHT_ERR_ARG
    with pytest.raises(_lib.ShtError) as e:
        _lib.sht_batch_create([p.handle], [-1])
    assert e.value.status == _lib.SHT_ERR_ARG
    with pytest.raises(_lib.ShtError) as e:  # host-only plans have no device program
        _lib.sht_batch_create([p.handle], [1])
    assert e.value.status == _lib.SHT_ERR_UNSUPPORTED
    assert lib.alt_forward_batch(None, None, None, None) == _lib.SHT_ERR_ARG


def test_selftest_argument_errors_need_no_device():
    lib = _lib.load()
    assert lib.sht_selftest_timeout(None, None) == _lib.SHT_ERR_ARG
    p = sht.Plan(8, 1e-7, flags=HOST, precision=_lib.SHT_MIXED)
    assert lib.sht_selftest_timeout(p.handle, None) == _lib.SHT_ERR_UNSUPPORTED


def test_plan_nodes_match_oracle():
    for N in [1, 8, 300]:
        p = sht.Plan(N, 1e-12, flags=HOST)
        x, w = p.nodes()
        xo, wo = oracle.gl_rule(2 * N)
        np.testing.assert_allclose(x, xo, atol=3e-16)
        # end weights of either rule carry ~1e-12 relative rounding error
        np.testing.assert_allclose(w, wo, rtol=5e-12)


CASES = [
    (4, {}),
    (64, {}),
    (64, dict(n0=16, n_leaf=8, flags=FORCE)),
    (96, dict(n0=16, n_leaf=8, flags=FORCE, sampling=1)),
    (128, dict(n0=32, n_leaf=16)),
]


@pytest.mark.parametrize("N,kw", CASES)
def test_program_reproduces_oracle(N, kw):
    p = sht.Plan(N, 1e-12, **{**kw, "flags": kw.get("flags", 0) | HOST})
    prog = p.program()
    x, w = p.nodes()
    beta = inputs.coefficients(N, 1, seed=0, real_m0=True)
    g_ref = oracle.alt_forward(N, beta)[0]
    g = host_apply.forward(prog, N, beta[0])
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-12
    b_ref = oracle.alt_inverse(N, g_ref[None])[0]
    b = host_apply.inverse(prog, N, g_ref, w)
    assert np.linalg.norm(b - b_ref) / np.linalg.norm(b_ref) < 1e-12


def test_program_mixed_tolerance():
    # eps = 1e-7: the factorisation error stays at the tolerance's scale
    N = 96
    p = sht.Plan(N, 1e-7, n0=16, n_leaf=8, flags=HOST | FORCE)
    beta = inputs.coefficients(N, 1, seed=4)
    g_ref = oracle.alt_forward(N, beta)[0]
    g = host_apply.forward(p.program(), N, beta[0])
    e = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert 1e-13 < e < 1e-6


def test_program_structure():
    N = 64
    p = sht.Plan(N, 1e-12, n0=16, n_leaf=8, flags=HOST | FORCE)
    prog = p.program()
    st = p.stats()
    units, ops = prog["units"], prog["ops"]
    assert len(units) == 2 * N and st["n_units"] == 2 * N
    assert st["n_blocks_idbf"] > 0 and st["n_ops"] == len(ops)
    assert sorted(prog["order"].tolist()) == list(range(2 * N))
    costs = units["cost"][prog["order"]]
    assert np.all(np.diff(costs) <= 0)
    for u in units:
        seg = ops[u["op_begin"]: u["op_end"]]
        assert np.all(np.diff(seg["phase"]) >= 0)
        assert u["nce"] == (2 * N - u["am"] + 1) // 2 and u["nco"] == (2 * N - u["am"]) // 2
    # every intermediate row is written by at most one op (single writer);
    # intermediate segments start on 8-row groups, so the unwritten rows are
    # the padding at the end of a group
    u = units[0]
    seg = ops[u["op_begin"]: u["op_end"]]
    writes = np.zeros(u["nrows"], dtype=int)
    for op in seg:
        if op["flags"] & 1:
            continue
        for s in range(2):
            writes[op["out_off"][s]: op["out_off"][s] + op["out_len"][s]] += 1
            if op["out_len"][s] > 0 and op["out_off"][s] >= u["yo"] + N:
                assert op["out_off"][s] % 8 == 0
    z0 = (u["yo"] + N + 7) // 8 * 8
    assert np.all(writes[z0:] <= 1)
    grp = np.zeros((u["nrows"] - z0 + 7) // 8 * 8, dtype=int)
    grp[: u["nrows"] - z0] = writes[z0:]
    grp = grp.reshape(-1, 8)
    assert np.all(np.diff(grp, axis=1) <= 0)  # written rows first, padding after
    assert grp[:, 0].all()


def test_kernel_time_needs_timing_plan():
    p = sht.Plan(16, 1e-10, flags=HOST)
    with pytest.raises(_lib.ShtError) as ei:
        p.kernel_time()
    assert ei.value.status == _lib.SHT_ERR_UNSUPPORTED
