"""GB300-native IDBF associated Legendre / spherical harmonic transform.

Bremer, Chen & Yang, arXiv:2004.11346.  The transform runs in libsht.so
(CUDA kernels for sm_103a behind the C ABI of include/sht.h); this package
holds the ctypes binding (``_lib``), torch-tensor convenience wrappers
(``Plan``, ``Batch``), the in-tree build (``build``), the seeded input
generators (``inputs``), the plan-parameter autotuner (``autotune``) and the
per-order statistics and plan sizing (``orders``).
"""
from __future__ import annotations

import numpy as np

from . import _lib

__all__ = ["Plan", "Batch", "OP_DTYPE", "UNIT_DTYPE", "opts"]

OP_DTYPE = np.dtype([
    ("b_off", "<i8"), ("mo", "<i4"), ("ni", "<i4"), ("ld", "<i4"), ("flags", "<i4"),
    ("in_off", "<i4", 2), ("in_len", "<i4", 2), ("out_off", "<i4", 2), ("out_len", "<i4", 2),
    ("phase", "<i4"), ("pad", "<i4"),
])
UNIT_DTYPE = np.dtype([
    ("am", "<i4"), ("op_begin", "<i4"), ("op_end", "<i4"), ("ph_begin", "<i4"), ("nphase", "<i4"),
    ("nrows", "<i4"), ("xe", "<i4"), ("xo", "<i4"), ("ye", "<i4"), ("yo", "<i4"), ("nce", "<i4"),
    ("nco", "<i4"), ("pad", "<i4"), ("cost", "<f4"),
])
assert OP_DTYPE.itemsize == 64 and UNIT_DTYPE.itemsize == 56


def opts(N: int, eps: float, **kw) -> _lib.sht_opts:
    """Default plan options for (N, eps) with fields overridden by keyword."""
    o = _lib.sht_opts_default(N, eps)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Plan:
    """A plan for order N at tolerance eps (see sht_plan_create in include/sht.h).

    forward/inverse take CUDA float64 tensors shaped like the oracle's arrays:
    beta (F, 4N^2, 2) and g (F, 4N-1, 2N, 2).  Work is queued on torch's
    current CUDA stream.
    """

    def __init__(self, N: int, eps: float, **kw):
        self.N = N
        self.eps = eps
        self.opts = opts(N, eps, **kw)
        self.handle = _lib.sht_plan_create(N, eps, self.opts)

    @classmethod
    def load(cls, path: str) -> "Plan":
        """A plan read back from a file written by save() (sht_plan_load)."""
        self = cls.__new__(cls)
        self.handle = None
        self.handle = _lib.sht_plan_load(path)
        self.opts = _lib.sht_plan_opts(self.handle)
        self.N = int(self.stats()["N"])
        self.eps = float(self.opts.eps)
        return self

    def save(self, path: str):
        """Write the plan's precomputation to `path` (sht_plan_save)."""
        _lib.sht_plan_save(self.handle, path)

    def close(self):
        if self.handle:
            _lib.sht_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def host_only(self) -> bool:
        return bool(self.opts.flags & _lib.SHT_FLAG_HOST_ONLY)

    def stats(self) -> dict:
        return _lib.sht_plan_stats(self.handle)

    def order(self) -> np.ndarray:
        """The unit queue order of the apply (|m| of each unit in the order taken)."""
        return self.program(("order",))["order"].copy()

    def legendre(self, am: int):
        """Pbar_{am+t}^{am} at the N positive nodes from the device recurrence
        (sht_legendre): a CUDA float64 tensor (2N - am, N)."""
        import torch
        out = torch.empty((2 * self.N - am, self.N), dtype=torch.float64, device="cuda")
        _lib.sht_legendre(self.handle, am, out.data_ptr(), self._stream())
        return out

    def set_order(self, order):
        """Set the unit queue order (sht_plan_set_order): any permutation of 0 .. 2N-1."""
        _lib.sht_plan_set_order(self.handle, order)

    def nodes(self):
        x = np.empty(2 * self.N)
        w = np.empty(2 * self.N)
        _lib.sht_plan_nodes(self.handle, x.ctypes.data, w.ctypes.data)
        return x, w

    def program(self, parts=("units", "ops", "phases", "factors", "order")) -> dict:
        """Host copies of the apply program (for inspection and tests)."""
        kinds = {"units": (_lib.SHT_EXPORT_UNITS, UNIT_DTYPE), "ops": (_lib.SHT_EXPORT_OPS, OP_DTYPE),
                 "phases": (_lib.SHT_EXPORT_PHASES, np.int32), "factors": (_lib.SHT_EXPORT_FACTORS, np.float64),
                 "order": (_lib.SHT_EXPORT_ORDER, np.int32),
                 "unit_blocks": (_lib.SHT_EXPORT_UNIT_BLOCKS, np.int32)}
        return {k: _lib.sht_plan_export(self.handle, kinds[k][0]).view(kinds[k][1]) for k in parts}

    # ---- device entry points (torch tensors)
    @staticmethod
    def _stream():
        import torch
        return torch.cuda.current_stream().cuda_stream

    @staticmethod
    def _dev(t, shape):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError("expected a contiguous CUDA float64 tensor")
        if tuple(t.shape[1:]) != tuple(shape):
            raise ValueError(f"expected shape (F, {', '.join(map(str, shape))}), got {tuple(t.shape)}")
        return t

    def forward(self, beta, out=None):
        import torch
        N = self.N
        beta = self._dev(beta, (4 * N * N, 2))
        F = beta.shape[0]
        g = out if out is not None else torch.empty((F, 4 * N - 1, 2 * N, 2), dtype=torch.float64,
                                                    device=beta.device)
        self._dev(g, (4 * N - 1, 2 * N, 2))
        _lib.alt_forward(self.handle, beta.data_ptr(), g.data_ptr(), F, self._stream())
        return g

    def inverse(self, g, out=None):
        import torch
        N = self.N
        g = self._dev(g, (4 * N - 1, 2 * N, 2))
        F = g.shape[0]
        beta = out if out is not None else torch.empty((F, 4 * N * N, 2), dtype=torch.float64, device=g.device)
        self._dev(beta, (4 * N * N, 2))
        _lib.alt_inverse(self.handle, g.data_ptr(), beta.data_ptr(), F, self._stream())
        return beta

    def forward_m(self, m: int, beta_m, out=None):
        import torch
        N = self.N
        beta_m = self._dev(beta_m, (2 * N - abs(m), 2))
        F = beta_m.shape[0]
        g = out if out is not None else torch.empty((F, 2 * N, 2), dtype=torch.float64, device=beta_m.device)
        self._dev(g, (2 * N, 2))
        _lib.alt_forward_m(self.handle, m, beta_m.data_ptr(), g.data_ptr(), F, self._stream())
        return g

    def inverse_m(self, m: int, g_m, out=None):
        import torch
        N = self.N
        g_m = self._dev(g_m, (2 * N, 2))
        F = g_m.shape[0]
        b = out if out is not None else torch.empty((F, 2 * N - abs(m), 2), dtype=torch.float64,
                                                    device=g_m.device)
        self._dev(b, (2 * N - abs(m), 2))
        _lib.alt_inverse_m(self.handle, m, g_m.data_ptr(), b.data_ptr(), F, self._stream())
        return b

    def phi_synthesis(self, g, out=None):
        """f(theta_l, phi_j) from g(m, theta_l): (F, 4N-1, 2N, 2) -> (F, 2N, 4N-1, 2)."""
        import torch
        N = self.N
        g = self._dev(g, (4 * N - 1, 2 * N, 2))
        F = g.shape[0]
        f = out if out is not None else torch.empty((F, 2 * N, 4 * N - 1, 2), dtype=torch.float64, device=g.device)
        self._dev(f, (2 * N, 4 * N - 1, 2))
        _lib.sht_phi_synthesis(self.handle, g.data_ptr(), f.data_ptr(), F, self._stream())
        return f

    def phi_analysis(self, f, out=None):
        """g(m, theta_l) from f(theta_l, phi_j): (F, 2N, 4N-1, 2) -> (F, 4N-1, 2N, 2)."""
        import torch
        N = self.N
        f = self._dev(f, (2 * N, 4 * N - 1, 2))
        F = f.shape[0]
        g = out if out is not None else torch.empty((F, 4 * N - 1, 2 * N, 2), dtype=torch.float64, device=f.device)
        self._dev(g, (4 * N - 1, 2 * N, 2))
        _lib.sht_phi_analysis(self.handle, f.data_ptr(), g.data_ptr(), F, self._stream())
        return g

    def sht_forward(self, beta, out=None):
        """Full SHT: coefficients (F, 4N^2, 2) -> grid values (F, 2N, 4N-1, 2)."""
        import torch
        N = self.N
        beta = self._dev(beta, (4 * N * N, 2))
        F = beta.shape[0]
        f = out if out is not None else torch.empty((F, 2 * N, 4 * N - 1, 2), dtype=torch.float64,
                                                    device=beta.device)
        self._dev(f, (2 * N, 4 * N - 1, 2))
        _lib.sht_forward(self.handle, beta.data_ptr(), f.data_ptr(), F, self._stream())
        return f

    def sht_inverse(self, f, out=None):
        """Inverse SHT: grid values (F, 2N, 4N-1, 2) -> coefficients (F, 4N^2, 2)."""
        import torch
        N = self.N
        f = self._dev(f, (2 * N, 4 * N - 1, 2))
        F = f.shape[0]
        beta = out if out is not None else torch.empty((F, 4 * N * N, 2), dtype=torch.float64, device=f.device)
        self._dev(beta, (4 * N * N, 2))
        _lib.sht_inverse(self.handle, f.data_ptr(), beta.data_ptr(), F, self._stream())
        return beta

    def kernel_time(self, reset: bool = True) -> dict:
        """Summed device time of the apply kernels since the last reset (plans
        created with flags including SHT_FLAG_TIMING; sht_plan_kernel_time)."""
        return _lib.sht_plan_kernel_time(self.handle, reset)

    def set_timing(self, enable: bool):
        """Pause or resume the kernel-time events of a SHT_FLAG_TIMING plan."""
        _lib.sht_plan_set_timing(self.handle, enable)

    def sync(self):
        _lib.sht_sync(self.handle, self._stream())


class Batch:
    """Several SHT_MIXED plans applied to their own fields in one launch
    (sht_batch_create in include/sht.h).  fields[q] fields go with plans[q];
    the tensors passed to the methods are per plan, shaped as for Plan."""

    def __init__(self, plans, fields):
        self.plans = list(plans)
        self.fields = [int(f) for f in fields]
        self.handle = _lib.sht_batch_create([p.handle for p in self.plans], self.fields)

    def close(self):
        if self.handle:
            _lib.sht_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _args(self, xs, shape_in, shape_out):
        import torch
        outs = []
        for p, F, x in zip(self.plans, self.fields, xs):
            if F == 0:
                outs.append(None)
                continue
            Plan._dev(x, shape_in(p.N))
            if x.shape[0] != F:
                raise ValueError(f"expected {F} fields, got {x.shape[0]}")
            outs.append(torch.empty((F, *shape_out(p.N)), dtype=torch.float64, device=x.device))
        ins = [x.data_ptr() if F else 0 for F, x in zip(self.fields, xs)]
        return ins, outs, [o.data_ptr() if o is not None else 0 for o in outs]

    def forward(self, betas):
        """Forward ALT of every plan's fields: list of (F_q, 4N^2, 2) -> list of (F_q, 4N-1, 2N, 2)."""
        ins, outs, optr = self._args(betas, lambda N: (4 * N * N, 2), lambda N: (4 * N - 1, 2 * N, 2))
        _lib.alt_forward_batch(self.handle, ins, optr, Plan._stream())
        return outs

    def inverse(self, gs):
        """Inverse ALT of every plan's fields: list of (F_q, 4N-1, 2N, 2) -> list of (F_q, 4N^2, 2)."""
        ins, outs, optr = self._args(gs, lambda N: (4 * N - 1, 2 * N, 2), lambda N: (4 * N * N, 2))
        _lib.alt_inverse_batch(self.handle, ins, optr, Plan._stream())
        return outs

    def sht_forward(self, betas):
        """Full SHT of every plan's fields: list of (F_q, 4N^2, 2) -> list of (F_q, 2N, 4N-1, 2)."""
        ins, outs, optr = self._args(betas, lambda N: (4 * N * N, 2), lambda N: (2 * N, 4 * N - 1, 2))
        _lib.sht_forward_batch(self.handle, ins, optr, Plan._stream())
        return outs

    def sht_inverse(self, fs):
        """Inverse SHT of every plan's fields: list of (F_q, 2N, 4N-1, 2) -> list of (F_q, 4N^2, 2)."""
        ins, outs, optr = self._args(fs, lambda N: (2 * N, 4 * N - 1, 2), lambda N: (4 * N * N, 2))
        _lib.sht_inverse_batch(self.handle, ins, optr, Plan._stream())
        return outs

    def sync(self):
        _lib.sht_batch_sync(self.handle, Plan._stream())
