"""Python binding of libsip.so (include/sip.h): argument marshalling only.

Every step of the solver runs in the library's sm_103a kernels; this module
passes device pointers of torch CUDA tensors and host scalars through ctypes.
There is no fallback: if the library cannot be loaded, or no CUDA device is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsip.so")

SIP_OK = 0
SIP_NOT_CONVERGED = 1
SIP_ERR_INVALID_ARG = -1
SIP_NOALLOC_MAX_CELLS = 67108864  # include/sip.h
SIP_ERR_NO_DEVICE = -2
SIP_ERR_CUDA = -3
SIP_ERR_OOM = -4
SIP_ERR_BREAKDOWN = -5
SIP_ERR_DEVICE_TIMEOUT = -6
SIP_ERR_BUSY = -7
SIP_ERR_NOT_FOUND = -8

SIP_MODE_F64 = 0
SIP_MODE_F32_REFINED = 1
SIP_MODE_F32 = 2

ERROR_NAMES = {
    SIP_ERR_INVALID_ARG: "SIP_ERR_INVALID_ARG", SIP_ERR_NO_DEVICE: "SIP_ERR_NO_DEVICE",
    SIP_ERR_CUDA: "SIP_ERR_CUDA", SIP_ERR_OOM: "SIP_ERR_OOM", SIP_ERR_BREAKDOWN: "SIP_ERR_BREAKDOWN",
    SIP_ERR_DEVICE_TIMEOUT: "SIP_ERR_DEVICE_TIMEOUT", SIP_ERR_BUSY: "SIP_ERR_BUSY",
    SIP_ERR_NOT_FOUND: "SIP_ERR_NOT_FOUND",
}

# every symbol include/sip.h declares
EXPORTED = (
    "sip_default_options", "sip_create", "sip_destroy", "sip_trim", "sip_last_error", "sip_factor",
    "sip_iterate", "sip_solve", "sip_get_history", "sip_export_factors", "sip_plan_bytes", "sip_plan_shape",
    "sip_plan_destroy", "sip_plane_layout", "sip_profile_enable", "sip_profile_read",
    "sip_launch_count", "sip_kernel_name", "sip_residual_norm",
    "sip_residual_norm_noalloc", "sip_server_start", "sip_server_submit", "sip_server_poll", "sip_server_stop",
    "sip_server_get_stats", "sip_assemble_pcorr", "sip_tile_model",
)


class sip_block_desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("coef_dtype", ctypes.c_int32),
        ("ap", ctypes.c_void_p), ("aw", ctypes.c_void_p), ("ae", ctypes.c_void_p),
        ("as_", ctypes.c_void_p), ("an", ctypes.c_void_p), ("ab", ctypes.c_void_p),
        ("at", ctypes.c_void_p),
        ("b", ctypes.c_void_p), ("x", ctypes.c_void_p),
        ("symmetric", ctypes.c_int32),
    ]


class sip_server_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
        ("queued", ctypes.c_uint32), ("running", ctypes.c_uint32), ("slots", ctypes.c_uint32),
        ("budget_bytes", ctypes.c_size_t), ("in_use_bytes", ctypes.c_size_t), ("peak_in_use_bytes", ctypes.c_size_t),
        ("oldest_running_ms", ctypes.c_double), ("busy_ms", ctypes.c_double),
    ]


class sip_interface(ctypes.Structure):
    _fields_ = [("blk_lo", ctypes.c_int32), ("blk_hi", ctypes.c_int32),
                ("nj", ctypes.c_int32), ("nk", ctypes.c_int32)]


class sip_options(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double), ("mode", ctypes.c_int32), ("inner_iters", ctypes.c_int32),
        ("max_spin", ctypes.c_int64), ("tile_j", ctypes.c_int32), ("tile_k", ctypes.c_int32),
        ("stages", ctypes.c_int32), ("debug_stall", ctypes.c_int32), ("graphs", ctypes.c_int32),
        ("rows_per_thread", ctypes.c_int32), ("autotune", ctypes.c_int32),
    ]


class sip_pcorr_desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("dirichlet_bottom", ctypes.c_int32),
        ("dx", ctypes.c_void_p), ("dy", ctypes.c_void_p), ("dz", ctypes.c_void_p),
        ("rho", ctypes.c_void_p), ("g", ctypes.c_void_p),
        ("ux", ctypes.c_void_p), ("uy", ctypes.c_void_p), ("uz", ctypes.c_void_p),
    ]


class SipError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libsip.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not built; run paper_1303_4538_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        L.sip_default_options.argtypes = [ctypes.POINTER(sip_options)]
        L.sip_default_options.restype = None
        L.sip_create.argtypes = [ctypes.POINTER(P), I, P]
        L.sip_destroy.argtypes = [P]
        L.sip_trim.argtypes = [P]
        L.sip_last_error.argtypes = [P]
        L.sip_last_error.restype = ctypes.c_char_p
        L.sip_factor.argtypes = [P, ctypes.POINTER(sip_block_desc), I, ctypes.POINTER(sip_interface), I,
                                 ctypes.POINTER(sip_options), ctypes.POINTER(P)]
        L.sip_iterate.argtypes = [P, I, ctypes.POINTER(D)]
        L.sip_solve.argtypes = [P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]
        L.sip_get_history.argtypes = [P, ctypes.POINTER(D), I, ctypes.POINTER(I)]
        L.sip_export_factors.argtypes = [P, I, ctypes.POINTER(P)]
        L.sip_plan_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.sip_plan_shape.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]
        L.sip_plan_destroy.argtypes = [P]
        L.sip_plane_layout.argtypes = [I, I, I, P]
        L.sip_profile_enable.argtypes = [P, I]
        L.sip_profile_read.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_int64), I]
        L.sip_launch_count.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
        L.sip_kernel_name.argtypes = [I]
        L.sip_residual_norm.argtypes = [P, ctypes.POINTER(sip_block_desc), ctypes.POINTER(D), ctypes.POINTER(D)]
        L.sip_residual_norm_noalloc.argtypes = [P, ctypes.POINTER(sip_block_desc), P]
        L.sip_server_start.argtypes = [P, ctypes.c_size_t, I, ctypes.POINTER(P)]
        L.sip_server_submit.argtypes = [P, ctypes.POINTER(sip_block_desc), ctypes.POINTER(sip_options), D, I,
                                        ctypes.POINTER(ctypes.c_uint64)]
        L.sip_server_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                      ctypes.POINTER(D)]
        L.sip_server_stop.argtypes = [P]
        L.sip_server_get_stats.argtypes = [P, ctypes.c_void_p]
        L.sip_assemble_pcorr.argtypes = [P, ctypes.POINTER(sip_pcorr_desc)] + [P] * 8
        L.sip_kernel_name.restype = ctypes.c_char_p
        for name in EXPORTED:
            if name not in ("sip_default_options", "sip_last_error", "sip_kernel_name"):
                getattr(L, name).restype = I
        _lib = L
    return _lib


def default_options(**kw) -> sip_options:
    o = sip_options()
    lib().sip_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return int(t.data_ptr())


class Context:
    """sip_create / sip_destroy around a device and a CUDA stream handle."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        self.h = ctypes.c_void_p()
        self.device = int(device)
        rc = lib().sip_create(ctypes.byref(self.h), int(device), ctypes.c_void_p(stream or 0))
        if rc != SIP_OK:
            raise SipError(rc, "sip_create failed: " + lib().sip_last_error(None).decode())

    def check(self, rc: int, allow_not_converged: bool = False) -> int:
        if rc == SIP_OK or (allow_not_converged and rc == SIP_NOT_CONVERGED):
            return rc
        raise SipError(rc, lib().sip_last_error(self.h).decode())

    def residual_norm(self, desc: "sip_block_desc"):
        """sip_residual_norm: (||b - A x||_2, ||b||_2) of one block descriptor."""
        r = ctypes.c_double(0.0)
        b = ctypes.c_double(0.0)
        self.check(lib().sip_residual_norm(self.h, ctypes.byref(desc), ctypes.byref(r), ctypes.byref(b)))
        return r.value, b.value

    def residual_norm_noalloc(self, desc: "sip_block_desc", out) -> None:
        """sip_residual_norm_noalloc: writes (||b - A x||_2, ||b||_2) into the
        device array `out` (2 doubles) in stream order; no allocation, no sync."""
        if not isinstance(out, int):
            import torch
            if not (out.is_cuda and out.dtype == torch.float64 and out.numel() >= 2
                    and out.device.index == self.device):
                raise ValueError("out must be a float64 tensor of >= 2 elements on the context's device")
        self.check(lib().sip_residual_norm_noalloc(self.h, ctypes.byref(desc), ctypes.c_void_p(_ptr(out))))

    def assemble_pcorr(self, nx: int, ny: int, nz: int, dx, dy, dz, rho, g, ux, uy, uz, outs,
                       dirichlet_bottom: bool = True) -> None:
        """sip_assemble_pcorr: pressure-correction coefficients and rhs of one
        block into `outs` = (ap, aw, ae, as, an, ab, at, b) (device float64
        tensors of nx*ny*nz; aw / as / ab may be None), in stream order."""
        import torch
        n = nx * ny * nz
        sizes = (nx, ny, nz, n, n, (nx + 1) * ny * nz, nx * (ny + 1) * nz, nx * ny * (nz + 1))
        for t, m in zip((dx, dy, dz, rho, g, ux, uy, uz), sizes):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == m
                    and t.device.index == self.device):
                raise ValueError("inputs must be contiguous float64 tensors of the documented sizes on the "
                                 "context's device")
        if len(outs) != 8:
            raise ValueError("outs: (ap, aw, ae, as, an, ab, at, b)")
        for q, t in enumerate(outs):
            if t is None and q in (1, 3, 5):
                continue
            if t is None or not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == n
                                 and t.device.index == self.device):
                raise ValueError("outputs must be contiguous float64 tensors of nx*ny*nz on the context's device")
        d = sip_pcorr_desc(nx, ny, nz, 1 if dirichlet_bottom else 0,
                           *[_ptr(t) for t in (dx, dy, dz, rho, g, ux, uy, uz)])
        self.check(lib().sip_assemble_pcorr(self.h, ctypes.byref(d), *[ctypes.c_void_p(_ptr(t)) for t in outs]))

    def trim(self) -> None:
        """sip_trim: return the pool's cached device memory (not held by a
        live plan) to the device."""
        self.check(lib().sip_trim(self.h))

    def close(self):
        if self.h:
            lib().sip_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_desc(nx, ny, nz, coefs: Sequence, b, x, symmetric: bool = False,
              coef_dtype: int = 0) -> sip_block_desc:
    """coefs: (ap, aw, ae, as, an, ab, at) device tensors or pointers (aw/as/ab
    may be None when symmetric); b, x: FP64 device tensors (natural layout)."""
    d = sip_block_desc()
    d.nx, d.ny, d.nz = int(nx), int(ny), int(nz)
    d.coef_dtype = int(coef_dtype)
    d.ap, d.aw, d.ae, d.as_, d.an, d.ab, d.at = [_ptr(c) for c in coefs]
    d.b = _ptr(b)
    d.x = _ptr(x)
    d.symmetric = 1 if symmetric else 0
    return d


class Plan:
    """sip_factor / sip_iterate / sip_solve / sip_plan_destroy."""

    def __init__(self, ctx: Context, descs: List[sip_block_desc], opts: Optional[sip_options] = None,
                 ifaces: Optional[List[sip_interface]] = None, keep=None):
        self.ctx = ctx
        self.h = ctypes.c_void_p()
        self._keep = keep  # tensors that must outlive the plan (b, x, ...)
        arr = (sip_block_desc * len(descs))(*descs)
        nif = len(ifaces) if ifaces else 0
        iarr = (sip_interface * nif)(*ifaces) if nif else None
        rc = lib().sip_factor(ctx.h, arr, len(descs), iarr, nif,
                              ctypes.byref(opts) if opts is not None else None, ctypes.byref(self.h))
        ctx.check(rc)

    def iterate(self, niters: int) -> float:
        rel = ctypes.c_double(0.0)
        self.ctx.check(lib().sip_iterate(self.h, int(niters), ctypes.byref(rel)))
        return rel.value

    def solve(self, rtol: float, max_iters: int):
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        rc = lib().sip_solve(self.h, float(rtol), int(max_iters), ctypes.byref(it), ctypes.byref(rel))
        self.ctx.check(rc, allow_not_converged=True)
        return it.value, rel.value, rc == SIP_OK

    def history(self) -> List[float]:
        n = ctypes.c_int(0)
        self.ctx.check(lib().sip_get_history(self.h, None, 0, ctypes.byref(n)))
        buf = (ctypes.c_double * max(n.value, 1))()
        self.ctx.check(lib().sip_get_history(self.h, buf, n.value, ctypes.byref(n)))
        return list(buf[: n.value])

    def export_factors(self, blk: int, outs) -> None:
        arr = (ctypes.c_void_p * 7)(*[_ptr(o) for o in outs])
        self.ctx.check(lib().sip_export_factors(self.h, int(blk), arr))

    def profile(self, enable: bool = True) -> None:
        self.ctx.check(lib().sip_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self, reset: bool = True):
        """{kernel name: (total ms, launches)} since the last reset."""
        names = kernel_names()
        ms = (ctypes.c_double * len(names))()
        n = (ctypes.c_int64 * len(names))()
        self.ctx.check(lib().sip_profile_read(self.h, len(names), ms, n, 1 if reset else 0))
        return {names[k]: (ms[k], n[k]) for k in range(len(names)) if n[k]}

    def launches(self) -> int:
        c = ctypes.c_int64(0)
        self.ctx.check(lib().sip_launch_count(self.h, ctypes.byref(c)))
        return c.value

    def nbytes(self) -> int:
        b = ctypes.c_size_t(0)
        self.ctx.check(lib().sip_plan_bytes(self.h, ctypes.byref(b)))
        return b.value

    def shape(self) -> Tuple[int, int, int]:
        """(rows_per_thread, tile_k, stages) of the plan's sweeps."""
        q, tk, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self.ctx.check(lib().sip_plan_shape(self.h, ctypes.byref(q), ctypes.byref(tk), ctypes.byref(r)))
        return q.value, tk.value, r.value

    def close(self):
        if self.h:
            lib().sip_plan_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plane_layout(nx: int, ny: int, nz: int):
    """Host-side plane layout table (no GPU needed): int32 array of shape
    (nz, nx+ny+nz-2); cell (i, j, k) sits at table[k, i+j+k] + j."""
    import numpy as np
    npl = nx + ny + nz - 2
    out = np.zeros((nz, npl), dtype=np.int32)
    rc = lib().sip_plane_layout(int(nx), int(ny), int(nz), out.ctypes.data_as(ctypes.c_void_p))
    if rc != SIP_OK:
        raise SipError(rc, "sip_plane_layout failed")
    return out


def tile_model(dims, rows_per_thread: int, warps: int, ctas: int, nsm: int = 152, fp64: bool = False) -> float:
    """Modelled SM cycles of one sweep launch (host only, no GPU needed):
    dims = [(nx, ny, nz), ...], tiles of 32 x (rows_per_thread * warps)."""
    import numpy as np
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1, 3))
    out = ctypes.c_double()
    rc = lib().sip_tile_model(d.ctypes.data_as(ctypes.c_void_p), int(d.shape[0]), int(rows_per_thread), int(warps),
                              int(ctas), int(nsm), int(bool(fp64)), ctypes.byref(out))
    if rc != SIP_OK:
        raise SipError(rc, "sip_tile_model failed")
    return out.value


class Server:
    """sip_server_start / submit / poll / stop (continuous batching)."""

    def __init__(self, ctx: "Context", hbm_budget_bytes: int, max_slots: int):
        self.ctx = ctx
        self.h = ctypes.c_void_p()
        rc = lib().sip_server_start(ctx.h, ctypes.c_size_t(int(hbm_budget_bytes)), int(max_slots),
                                    ctypes.byref(self.h))
        if rc != SIP_OK:
            raise SipError(rc, "sip_server_start failed")
        self._keep = {}

    def submit(self, desc: sip_block_desc, opts: Optional[sip_options], rtol: float, max_iters: int,
               keep=None) -> int:
        t = ctypes.c_uint64(0)
        rc = lib().sip_server_submit(self.h, ctypes.byref(desc), ctypes.byref(opts) if opts is not None else None,
                                     float(rtol), int(max_iters), ctypes.byref(t))
        if rc != SIP_OK:
            raise SipError(rc, "sip_server_submit failed")
        self._keep[t.value] = keep  # tensors that must outlive the request
        return t.value

    def poll(self, ticket: int):
        """None while running, else (status, iters, relres)."""
        d, st, it = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        rc = lib().sip_server_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(d), ctypes.byref(st),
                                   ctypes.byref(it), ctypes.byref(rel))
        if rc != SIP_OK:
            raise SipError(rc, "sip_server_poll failed")
        if not d.value:
            return None
        self._keep.pop(ticket, None)
        return st.value, it.value, rel.value

    def stats(self) -> dict:
        """sip_server_get_stats as a dict."""
        st = sip_server_stats()
        rc = lib().sip_server_get_stats(self.h, ctypes.byref(st))
        if rc != SIP_OK:
            raise SipError(rc, "sip_server_get_stats failed")
        return {name: getattr(st, name) for name, _ in st._fields_}

    def stop(self):
        if self.h:
            lib().sip_server_stop(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def kernel_names() -> List[str]:
    out = []
    k = 0
    while True:
        nm = lib().sip_kernel_name(k)
        if nm is None:
            return out
        out.append(nm.decode())
        k += 1
