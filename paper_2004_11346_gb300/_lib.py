"""ctypes binding of libsht.so (the C ABI declared in include/sht.h).

Argument marshalling only: every step of the transform runs in the library.
The functions keep the C names; pointers are plain integers (device
addresses, e.g. ``tensor.data_ptr()``) and the stream is a ``cudaStream_t``
as an integer (``torch.cuda.current_stream().cuda_stream``).  Loading fails
loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

(SHT_OK, SHT_ERR_ARG, SHT_ERR_OOM, SHT_ERR_CUDA, SHT_ERR_TIMEOUT, SHT_ERR_NUMERIC, SHT_ERR_IO,
 SHT_ERR_UNSUPPORTED) = range(8)
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error or no device",
          4: "device wait timed out", 5: "precomputation did not reach the tolerance",
          6: "plan file error", 7: "unsupported"}
SHT_FP64, SHT_FP32, SHT_MIXED = 0, 1, 2
SHT_FLAG_FORCE_FACTOR = 1
SHT_FLAG_HOST_ONLY = 2
SHT_FLAG_DENSE = 4
SHT_FLAG_TIMING = 8
SHT_FLAG_DIRECT = 16
SHT_FLAG_GPU_LEGENDRE = 32
(SHT_EXPORT_UNITS, SHT_EXPORT_OPS, SHT_EXPORT_PHASES, SHT_EXPORT_FACTORS, SHT_EXPORT_ORDER, SHT_EXPORT_OPTS,
 SHT_EXPORT_UNIT_BLOCKS) = range(7)


class sht_opts(ctypes.Structure):
    _fields_ = [
        ("eps", ctypes.c_double),
        ("n0", ctypes.c_int),
        ("n_leaf", ctypes.c_int),
        ("r_k", ctypes.c_int),
        ("oversample", ctypes.c_double),
        ("rsvd_r", ctypes.c_int),
        ("rsvd_q", ctypes.c_int),
        ("trim_delta", ctypes.c_double),
        ("sampling", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("max_fields", ctypes.c_int),
        ("flags", ctypes.c_int),
        ("seed", ctypes.c_uint64),
    ]


class sht_plan_info(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("n_units", ctypes.c_int64),
        ("n_ops", ctypes.c_int64),
        ("n_blocks_idbf", ctypes.c_int64),
        ("n_blocks_lowrank", ctypes.c_int64),
        ("n_blocks_dense", ctypes.c_int64),
        ("n_blocks_dropped", ctypes.c_int64),
        ("entries_idbf", ctypes.c_int64),
        ("entries_lowrank", ctypes.c_int64),
        ("entries_dense", ctypes.c_int64),
        ("entries_total", ctypes.c_int64),
        ("entries_matrix", ctypes.c_int64),
        ("max_rank", ctypes.c_int64),
        ("max_phases", ctypes.c_int64),
        ("workspace_bytes", ctypes.c_int64),
        ("factor_bytes", ctypes.c_int64),
        ("t_factor_s", ctypes.c_double),
        ("t_upload_s", ctypes.c_double),
        ("threads", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sht_order_info(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int),
        ("am", ctypes.c_int),
        ("cols_even", ctypes.c_int64),
        ("cols_odd", ctypes.c_int64),
        ("n_blocks_idbf", ctypes.c_int64),
        ("n_blocks_lowrank", ctypes.c_int64),
        ("n_blocks_dense", ctypes.c_int64),
        ("n_blocks_dropped", ctypes.c_int64),
        ("entries_idbf", ctypes.c_int64),
        ("entries_lowrank", ctypes.c_int64),
        ("entries_dense", ctypes.c_int64),
        ("entries_total", ctypes.c_int64),
        ("entries_matrix", ctypes.c_int64),
        ("factor_doubles", ctypes.c_int64),
        ("image_elems", ctypes.c_int64),
        ("tc_stages", ctypes.c_int64),
        ("tc_tiles", ctypes.c_int64),
        ("tc_image_fwd_bytes", ctypes.c_int64),
        ("tc_act_bytes", ctypes.c_int64),
        ("max_rank", ctypes.c_int64),
        ("n_ops", ctypes.c_int64),
        ("n_phases", ctypes.c_int64),
        ("rows", ctypes.c_int64),
        ("flops_per_rhs", ctypes.c_double),
        ("t_mat_s", ctypes.c_double),
        ("t_fac_s", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ShtError(RuntimeError):
    def __init__(self, what: str, status: int):
        super().__init__(f"{what}: {STATUS.get(status, status)} (status {status})")
        self.status = status


_lib = None
EXPORTED = [
    "sht_opts_default", "sht_plan_create", "sht_plan_destroy", "sht_plan_stats", "sht_plan_nodes",
    "sht_plan_export", "alt_forward", "alt_inverse", "alt_forward_m", "alt_inverse_m", "sht_sync",
    "sht_status_str", "alt_forward_m_noalloc", "sht_phi_synthesis", "sht_phi_analysis", "sht_forward",
    "sht_inverse", "sht_plan_save", "sht_plan_load", "sht_plan_kernel_time", "sht_batch_create",
    "sht_batch_destroy", "alt_forward_batch", "alt_inverse_batch", "sht_forward_batch", "sht_inverse_batch",
    "sht_batch_sync", "sht_selftest_timeout", "sht_plan_op_image", "sht_order_stats", "sht_plan_set_timing",
    "sht_selftest_convert", "sht_plan_set_order", "sht_legendre",
]


def load(build: bool = True):
    """Load (building first if stale) libsht.so and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise OSError(f"libsht.so not found at {path}")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    plan_p = ctypes.POINTER(ctypes.c_void_p)
    lib.sht_opts_default.argtypes = [i, d, ctypes.POINTER(sht_opts)]
    lib.sht_opts_default.restype = None
    lib.sht_plan_create.argtypes = [i, d, ctypes.POINTER(sht_opts), plan_p]
    lib.sht_plan_destroy.argtypes = [vp]
    lib.sht_plan_stats.argtypes = [vp, ctypes.POINTER(sht_plan_info)]
    lib.sht_plan_nodes.argtypes = [vp, vp, vp]
    lib.sht_plan_export.argtypes = [vp, i, vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.sht_plan_save.argtypes = [vp, ctypes.c_char_p]
    lib.sht_plan_kernel_time.argtypes = [vp, i, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(ctypes.c_int64)]
    lib.sht_plan_load.argtypes = [ctypes.c_char_p, plan_p]
    lib.sht_plan_set_timing.argtypes = [vp, i]
    for name in ("alt_forward", "alt_inverse", "sht_phi_synthesis", "sht_phi_analysis", "sht_forward",
                 "sht_inverse"):
        getattr(lib, name).argtypes = [vp, vp, vp, i, vp]
    for name in ("alt_forward_m", "alt_inverse_m", "alt_forward_m_noalloc"):
        getattr(lib, name).argtypes = [vp, i, vp, vp, i, vp]
    lib.sht_sync.argtypes = [vp, vp]
    lib.sht_batch_create.argtypes = [i, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int), plan_p]
    lib.sht_batch_destroy.argtypes = [vp]
    lib.sht_batch_sync.argtypes = [vp, vp]
    lib.sht_selftest_timeout.argtypes = [vp, vp]
    lib.sht_selftest_convert.argtypes = [vp, vp, vp, ctypes.c_int64, vp]
    lib.sht_plan_set_order.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), i]
    lib.sht_legendre.argtypes = [vp, i, vp, vp]
    lib.sht_plan_op_image.argtypes = [vp, ctypes.c_int64, i, vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.sht_order_stats.argtypes = [i, d, ctypes.POINTER(sht_opts), i, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(sht_order_info)]
    for name in ("alt_forward_batch", "alt_inverse_batch", "sht_forward_batch", "sht_inverse_batch"):
        getattr(lib, name).argtypes = [vp, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), vp]
    lib.sht_status_str.argtypes = [i]
    lib.sht_status_str.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("sht_opts_default", "sht_status_str"):
            getattr(lib, name).restype = i
    _lib = lib
    return lib


def check(status: int, what: str):
    if status != SHT_OK:
        raise ShtError(what, status)


def sht_opts_default(N: int, eps: float) -> sht_opts:
    o = sht_opts()
    load().sht_opts_default(N, eps, ctypes.byref(o))
    return o


def sht_plan_create(N: int, eps: float, opts: sht_opts | None = None) -> int:
    h = ctypes.c_void_p()
    check(load().sht_plan_create(N, eps, ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)),
          "sht_plan_create")
    return h.value


def sht_plan_destroy(plan: int):
    check(load().sht_plan_destroy(plan), "sht_plan_destroy")


def sht_plan_stats(plan: int) -> dict:
    info = sht_plan_info()
    check(load().sht_plan_stats(plan, ctypes.byref(info)), "sht_plan_stats")
    return info.as_dict()


def sht_plan_nodes(plan: int, x_host: int, w_host: int):
    check(load().sht_plan_nodes(plan, x_host, w_host), "sht_plan_nodes")


def sht_plan_export(plan: int, what: int):
    """The exported array's bytes, copied once into a new numpy uint8 array."""
    import numpy as np
    n = ctypes.c_size_t(0)
    check(load().sht_plan_export(plan, what, None, ctypes.byref(n)), "sht_plan_export")
    buf = np.empty(max(1, n.value), dtype=np.uint8)
    check(load().sht_plan_export(plan, what, buf.ctypes.data, ctypes.byref(n)), "sht_plan_export")
    return buf[: n.value]


def sht_plan_save(plan: int, path: str):
    check(load().sht_plan_save(plan, os.fsencode(path)), "sht_plan_save")


def sht_plan_load(path: str) -> int:
    h = ctypes.c_void_p()
    check(load().sht_plan_load(os.fsencode(path), ctypes.byref(h)), "sht_plan_load")
    return h.value


def sht_plan_kernel_time(plan: int, reset: bool = True) -> dict:
    a, o, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    check(load().sht_plan_kernel_time(plan, 1 if reset else 0, ctypes.byref(a), ctypes.byref(o), ctypes.byref(n)),
          "sht_plan_kernel_time")
    return {"apply_ms": a.value, "output_ms": o.value, "launches": n.value}


def sht_plan_set_timing(plan: int, enable: bool):
    check(load().sht_plan_set_timing(plan, 1 if enable else 0), "sht_plan_set_timing")


def sht_plan_opts(plan: int) -> sht_opts:
    raw = sht_plan_export(plan, SHT_EXPORT_OPTS)
    if len(raw) != ctypes.sizeof(sht_opts):
        raise ShtError("sht_plan_export", SHT_ERR_ARG)
    return sht_opts.from_buffer_copy(raw)


def alt_forward(plan: int, beta: int, g: int, F: int, stream: int = 0):
    check(load().alt_forward(plan, beta, g, F, stream), "alt_forward")


def alt_inverse(plan: int, g: int, beta: int, F: int, stream: int = 0):
    check(load().alt_inverse(plan, g, beta, F, stream), "alt_inverse")


def alt_forward_m(plan: int, m: int, beta_m: int, g_m: int, F: int, stream: int = 0):
    check(load().alt_forward_m(plan, m, beta_m, g_m, F, stream), "alt_forward_m")


def alt_inverse_m(plan: int, m: int, g_m: int, beta_m: int, F: int, stream: int = 0):
    check(load().alt_inverse_m(plan, m, g_m, beta_m, F, stream), "alt_inverse_m")


def alt_forward_m_noalloc(plan: int, m: int, beta_m: int, g_m: int, F: int, stream: int = 0):
    check(load().alt_forward_m_noalloc(plan, m, beta_m, g_m, F, stream), "alt_forward_m_noalloc")


def sht_phi_synthesis(plan: int, g: int, f: int, F: int, stream: int = 0):
    check(load().sht_phi_synthesis(plan, g, f, F, stream), "sht_phi_synthesis")


def sht_phi_analysis(plan: int, f: int, g: int, F: int, stream: int = 0):
    check(load().sht_phi_analysis(plan, f, g, F, stream), "sht_phi_analysis")


def sht_forward(plan: int, beta: int, f: int, F: int, stream: int = 0):
    check(load().sht_forward(plan, beta, f, F, stream), "sht_forward")


def sht_inverse(plan: int, f: int, beta: int, F: int, stream: int = 0):
    check(load().sht_inverse(plan, f, beta, F, stream), "sht_inverse")


def sht_sync(plan: int, stream: int = 0):
    check(load().sht_sync(plan, stream), "sht_sync")


def sht_batch_create(plans, fields) -> int:
    """A batch of plans with fields[q] fields for plans[q] (sht_batch_create)."""
    P = len(plans)
    parr = (ctypes.c_void_p * max(1, P))(*plans)
    farr = (ctypes.c_int * max(1, P))(*fields)
    h = ctypes.c_void_p()
    check(load().sht_batch_create(P, parr, farr, ctypes.byref(h)), "sht_batch_create")
    return h.value


def sht_batch_destroy(batch: int):
    check(load().sht_batch_destroy(batch), "sht_batch_destroy")


def _ptrs(ptrs):
    return (ctypes.c_void_p * max(1, len(ptrs)))(*[p or None for p in ptrs])


def alt_forward_batch(batch: int, beta_ptrs, g_ptrs, stream: int = 0):
    check(load().alt_forward_batch(batch, _ptrs(beta_ptrs), _ptrs(g_ptrs), stream), "alt_forward_batch")


def alt_inverse_batch(batch: int, g_ptrs, beta_ptrs, stream: int = 0):
    check(load().alt_inverse_batch(batch, _ptrs(g_ptrs), _ptrs(beta_ptrs), stream), "alt_inverse_batch")


def sht_forward_batch(batch: int, beta_ptrs, f_ptrs, stream: int = 0):
    check(load().sht_forward_batch(batch, _ptrs(beta_ptrs), _ptrs(f_ptrs), stream), "sht_forward_batch")


def sht_inverse_batch(batch: int, f_ptrs, beta_ptrs, stream: int = 0):
    check(load().sht_inverse_batch(batch, _ptrs(f_ptrs), _ptrs(beta_ptrs), stream), "sht_inverse_batch")


def sht_batch_sync(batch: int, stream: int = 0):
    check(load().sht_batch_sync(batch, stream), "sht_batch_sync")


def sht_selftest_timeout(plan: int, stream: int = 0):
    check(load().sht_selftest_timeout(plan, stream), "sht_selftest_timeout")


def sht_legendre(plan: int, am: int, out: int, stream: int = 0):
    check(load().sht_legendre(plan, am, out, stream), "sht_legendre")


def sht_plan_set_order(plan: int, order):
    """Set the plan's unit queue order (a permutation of 0 .. 2N-1)."""
    import numpy as np
    a = np.ascontiguousarray(order, dtype=np.int32)
    check(load().sht_plan_set_order(plan, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(a.size)),
          "sht_plan_set_order")


def sht_selftest_convert(f64: int, f32: int, back: int, n: int, stream: int = 0):
    check(load().sht_selftest_convert(f64, f32, back, n, stream), "sht_selftest_convert")


def sht_plan_op_image(plan: int, op: int, transposed: bool):
    """The BF16 bits (uint16 numpy array) of one op's tensor-core operand image."""
    import numpy as np
    n = ctypes.c_size_t(0)
    check(load().sht_plan_op_image(plan, op, 1 if transposed else 0, None, ctypes.byref(n)), "sht_plan_op_image")
    out = np.zeros(max(1, n.value), dtype=np.uint16)
    check(load().sht_plan_op_image(plan, op, 1 if transposed else 0, out.ctypes.data, ctypes.byref(n)),
          "sht_plan_op_image")
    return out[: n.value]


def sht_order_stats(N: int, eps: float, orders, opts: sht_opts | None = None) -> list:
    """One dict per order (sht_order_info) of the plan sht_plan_create(N, eps, opts) would build."""
    orders = [int(v) for v in orders]
    n = len(orders)
    marr = (ctypes.c_int * max(1, n))(*orders)
    out = (sht_order_info * max(1, n))()
    check(load().sht_order_stats(N, eps, ctypes.byref(opts) if opts is not None else None, n, marr, out),
          "sht_order_stats")
    return [out[k].as_dict() for k in range(n)]
