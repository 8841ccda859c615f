"""Python binding of libdwt's C ABI (include/dwt.h) -- argument marshalling only.

The functions keep the C names and return/raise on the status code; every
step of the transform runs in the CUDA kernels of ``lib/libdwt.so``.  There
is no fallback: if the library is missing or fails to load, :func:`lib`
raises.  :class:`Plan` is a convenience wrapper taking PyTorch CUDA tensors
(it only reads their data pointers and strides).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

__all__ = [
    "DwtError", "lib", "LIB_PATH",
    "DWT_OK", "DWT_EINVAL", "DWT_ENOMEM", "DWT_EUNSUPPORTED", "DWT_ECUDA", "DWT_ETIMEOUT", "DWT_EBUSY",
    "DWT_CDF53", "DWT_CDF97", "DWT_DD137", "DWT_F32", "DWT_F16S", "DWT_I32",
    "SCHEMES", "DWT_NORM_JPEG2000", "DWT_NORM_ZETA",
    "dwt_plan_create", "dwt_plan_set_scheme", "dwt_plan_set_tile", "dwt_plan_set_fusion", "dwt_plan_get_fusion", "dwt_plan_get_tile", "dwt_plan_get_scheme", "dwt_plan_set_normalization",
    "dwt2_forward", "dwt2_inverse", "dwt2_forward_noalloc", "dwt2_forward_host", "dwt2_inverse_host", "dwt_batch_submit",
    "dwt_plan_device_status", "dwt_noalloc_device_status", "dwt_set_wait_limits", "dwt_debug_inject",
    "DWT_INJECT_NONE", "DWT_INJECT_ENOMEM", "DWT_INJECT_HOLD", "DWT_INJECT_BATCH_DEP", "dwt_plan_set_profiling", "dwt_plan_read_profile", "dwt_plan_autotune",
    "dwt_plan_destroy", "dwt_scheme_counts", "dwt_status_string", "dwt_version", "Plan", "DwtRequest",
]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libdwt.so")

DWT_OK, DWT_EINVAL, DWT_ENOMEM, DWT_EUNSUPPORTED, DWT_ECUDA, DWT_ETIMEOUT, DWT_EBUSY = range(7)
DWT_CDF53, DWT_CDF97, DWT_DD137 = 0, 1, 2
DWT_F32, DWT_F16S, DWT_I32 = 0, 1, 2
DWT_NORM_JPEG2000, DWT_NORM_ZETA = 0, 1
DWT_INJECT_NONE, DWT_INJECT_ENOMEM, DWT_INJECT_HOLD, DWT_INJECT_BATCH_DEP = range(4)
SCHEMES = {
    "auto": 0, "rowcol": 1, "sweldens": 2, "iwahashi": 3, "iwahashi*": 4, "explosive": 5,
    "explosive*": 6, "monolithic": 7, "monolithic*": 8, "polyphase": 9, "polyphase*": 10,
    "convolution": 11,
}
SCHEME_NAMES = {v: k for k, v in SCHEMES.items()}


class DwtError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {dwt_status_string(status)} (status {status})" if what else
                         f"{dwt_status_string(status)} (status {status})")


class DwtRequest(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("in_pitch", ctypes.c_size_t),
                ("out", ctypes.c_void_p), ("out_pitch", ctypes.c_size_t), ("inverse", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int), ("total_ms", ctypes.c_double),
                ("algorithmic_bytes", ctypes.c_double)]


EXPORTS = {
    "dwt_plan_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                         ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "dwt_plan_set_scheme": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "dwt_plan_get_scheme": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "dwt_plan_set_tile": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "dwt_plan_get_tile": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                          ctypes.c_int),
    "dwt_plan_set_normalization": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "dwt_plan_set_fusion": ([ctypes.c_void_p, ctypes.c_longlong], ctypes.c_int),
    "dwt_plan_get_fusion": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "dwt2_forward": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t,
                      ctypes.c_void_p], ctypes.c_int),
    "dwt2_inverse": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t,
                      ctypes.c_void_p], ctypes.c_int),
    "dwt2_forward_noalloc": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t,
                              ctypes.c_void_p], ctypes.c_int),
    "dwt2_forward_host": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                           ctypes.c_size_t, ctypes.c_void_p], ctypes.c_int),
    "dwt2_inverse_host": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                           ctypes.c_size_t, ctypes.c_void_p], ctypes.c_int),
    "dwt_batch_submit": ([ctypes.POINTER(DwtRequest), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
                         ctypes.c_int),
    "dwt_plan_device_status": ([ctypes.c_void_p], ctypes.c_int),
    "dwt_noalloc_device_status": ([ctypes.c_void_p], ctypes.c_int),
    "dwt_set_wait_limits": ([ctypes.c_uint, ctypes.c_uint], ctypes.c_int),
    "dwt_debug_inject": ([ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "dwt_plan_set_profiling": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "dwt_plan_read_profile": ([ctypes.c_void_p, ctypes.POINTER(KernelStat), ctypes.c_int,
                               ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "dwt_plan_autotune": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "dwt_plan_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "dwt_scheme_counts": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "dwt_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "dwt_version": ([], ctypes.c_char_p),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libdwt.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libdwt is not built ({LIB_PATH} missing); run __graft_entry__.build()")
        l = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in EXPORTS.items():
            fn = getattr(l, name)
            fn.argtypes = args
            fn.restype = res
        _lib = l
    return _lib


def _check(st: int, what: str) -> None:
    if st != DWT_OK:
        raise DwtError(st, what)


def dwt_status_string(status: int) -> str:
    return lib().dwt_status_string(status).decode()


def dwt_version() -> str:
    return lib().dwt_version().decode()


def dwt_plan_create(w: int, h: int, wavelet: int, levels: int, dtype: int) -> int:
    out = ctypes.c_void_p()
    _check(lib().dwt_plan_create(w, h, wavelet, levels, dtype, ctypes.byref(out)), "dwt_plan_create")
    return out.value


def dwt_plan_set_scheme(plan: int, scheme: int) -> None:
    _check(lib().dwt_plan_set_scheme(plan, scheme), "dwt_plan_set_scheme")


def dwt_plan_set_tile(plan: int, strip_rows: int = 0, stages: int = 0) -> None:
    _check(lib().dwt_plan_set_tile(plan, strip_rows, stages), "dwt_plan_set_tile")


def dwt_plan_get_tile(plan: int):
    """(strip_rows, stages) the plan's calls use."""
    r, st = ctypes.c_int(), ctypes.c_int()
    _check(lib().dwt_plan_get_tile(plan, ctypes.byref(r), ctypes.byref(st)), "dwt_plan_get_tile")
    return r.value, st.value


def dwt_plan_set_fusion(plan: int, max_pixels: int = -1) -> None:
    """Levels whose input has at most max_pixels samples run in one fused
    launch (-1: default, 0: off)."""
    _check(lib().dwt_plan_set_fusion(plan, max_pixels), "dwt_plan_set_fusion")


def dwt_plan_get_fusion(plan: int) -> int:
    v = ctypes.c_longlong()
    _check(lib().dwt_plan_get_fusion(plan, ctypes.byref(v)), "dwt_plan_get_fusion")
    return v.value


def dwt_plan_get_scheme(plan: int) -> int:
    s = ctypes.c_int()
    _check(lib().dwt_plan_get_scheme(plan, ctypes.byref(s)), "dwt_plan_get_scheme")
    return s.value


def dwt_plan_set_normalization(plan: int, norm: int) -> None:
    _check(lib().dwt_plan_set_normalization(plan, norm), "dwt_plan_set_normalization")


def dwt2_forward(plan: int, d_in: int, in_pitch: int, d_out: int, out_pitch: int, stream: int = 0) -> None:
    _check(lib().dwt2_forward(plan, d_in, in_pitch, d_out, out_pitch, stream), "dwt2_forward")


def dwt2_inverse(plan: int, d_coef: int, coef_pitch: int, d_out: int, out_pitch: int, stream: int = 0) -> None:
    _check(lib().dwt2_inverse(plan, d_coef, coef_pitch, d_out, out_pitch, stream), "dwt2_inverse")


def dwt2_forward_noalloc(w: int, h: int, wavelet: int, levels: int, dtype: int, d_in: int, in_pitch: int,
                         d_out: int, out_pitch: int, stream: int = 0) -> None:
    """Forward transform without a plan and without any device allocation
    (scratch in a fixed 32 MiB device array of the library; see dwt.h).
    Device-side timeouts are read with :func:`dwt_noalloc_device_status`."""
    _check(lib().dwt2_forward_noalloc(w, h, wavelet, levels, dtype, d_in, in_pitch, d_out, out_pitch, stream),
           "dwt2_forward_noalloc")


def dwt2_forward_host(plan: int, h_in: int, in_pitch: int, h_out: int, out_pitch: int, stream: int = 0) -> None:
    _check(lib().dwt2_forward_host(plan, h_in, in_pitch, h_out, out_pitch, stream), "dwt2_forward_host")


def dwt2_inverse_host(plan: int, h_coef: int, coef_pitch: int, h_out: int, out_pitch: int,
                      stream: int = 0) -> None:
    _check(lib().dwt2_inverse_host(plan, h_coef, coef_pitch, h_out, out_pitch, stream), "dwt2_inverse_host")


def dwt_batch_submit(reqs: Sequence[DwtRequest], stream: int = 0, d_status: int = 0) -> None:
    arr = (DwtRequest * len(reqs))(*reqs)
    _check(lib().dwt_batch_submit(arr, len(reqs), stream, d_status), "dwt_batch_submit")


def dwt_plan_device_status(plan: int) -> int:
    return lib().dwt_plan_device_status(plan)


def dwt_noalloc_device_status(stream: int = 0) -> int:
    return lib().dwt_noalloc_device_status(stream)


def dwt_set_wait_limits(ring_probes: int = 0, dep_spins: int = 0) -> None:
    _check(lib().dwt_set_wait_limits(ring_probes, dep_spins), "dwt_set_wait_limits")


def dwt_debug_inject(what: int, skip: int = 0, count: int = 0) -> None:
    _check(lib().dwt_debug_inject(what, skip, count), "dwt_debug_inject")


def dwt_plan_set_profiling(plan: int, enable: bool) -> None:
    _check(lib().dwt_plan_set_profiling(plan, int(enable)), "dwt_plan_set_profiling")


def dwt_plan_read_profile(plan: int, capacity: int = 64):
    arr = (KernelStat * capacity)()
    n = ctypes.c_int()
    _check(lib().dwt_plan_read_profile(plan, arr, capacity, ctypes.byref(n)), "dwt_plan_read_profile")
    return [dict(name=arr[i].name.decode(), launches=arr[i].launches, total_ms=arr[i].total_ms,
                 algorithmic_bytes=arr[i].algorithmic_bytes) for i in range(min(n.value, capacity))]


def dwt_plan_autotune(plan: int, stream: int = 0) -> None:
    _check(lib().dwt_plan_autotune(plan, stream), "dwt_plan_autotune")


def dwt_scheme_counts(wavelet: int, scheme: int):
    """(multiply-accumulates per quadruple, barriers, tile shared-memory words
    per quadruple) of a scheme's forward program."""
    m, b, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().dwt_scheme_counts(wavelet, scheme, ctypes.byref(m), ctypes.byref(b), ctypes.byref(w)),
           "dwt_scheme_counts")
    return m.value, b.value, w.value


def dwt_plan_destroy(plan: int) -> None:
    _check(lib().dwt_plan_destroy(plan), "dwt_plan_destroy")


# ---------------------------------------------------------------------------
# Tensor convenience wrapper
# ---------------------------------------------------------------------------
_DTYPES = {"f32": DWT_F32, "f16s": DWT_F16S, "i32": DWT_I32}
_WAVELETS = {"cdf53": DWT_CDF53, "cdf97": DWT_CDF97, "dd137": DWT_DD137}


def _pitch(t) -> int:
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a 2-D tensor with unit column stride")
    return t.stride(0) * t.element_size()


class Plan:
    """A dwt_plan for one image size.  ``wavelet``: "cdf53" | "cdf97";
    ``dtype``: "f32" | "f16s" | "i32"; ``scheme``: a key of :data:`SCHEMES`."""

    def __init__(self, w: int, h: int, wavelet: str = "cdf97", levels: int = 1, dtype: str = "f32",
                 scheme: Optional[str] = None):
        self.w, self.h, self.levels = w, h, levels
        self.wavelet, self.dtype = wavelet, dtype
        self.handle = dwt_plan_create(w, h, _WAVELETS[wavelet], levels, _DTYPES[dtype])
        if scheme is not None:
            dwt_plan_set_scheme(self.handle, SCHEMES[scheme])

    @property
    def scheme(self) -> str:
        return SCHEME_NAMES[dwt_plan_get_scheme(self.handle)]

    def forward(self, x, out, stream: int = 0):
        dwt2_forward(self.handle, x.data_ptr(), _pitch(x), out.data_ptr(), _pitch(out), stream)
        return out

    def inverse(self, c, out, stream: int = 0):
        dwt2_inverse(self.handle, c.data_ptr(), _pitch(c), out.data_ptr(), _pitch(out), stream)
        return out

    def forward_host(self, x, out, stream: int = 0):
        dwt2_forward_host(self.handle, x.data_ptr(), _pitch(x), out.data_ptr(), _pitch(out), stream)
        return out

    def inverse_host(self, c, out, stream: int = 0):
        dwt2_inverse_host(self.handle, c.data_ptr(), _pitch(c), out.data_ptr(), _pitch(out), stream)
        return out

    def request(self, src, dst, inverse: bool = False) -> DwtRequest:
        """One entry of a batch (see :func:`submit`)."""
        return DwtRequest(self.handle, src.data_ptr(), _pitch(src), dst.data_ptr(), _pitch(dst), int(inverse))

    def close(self):
        if self.handle:
            dwt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def submit(requests: Sequence[DwtRequest], status=None, stream: int = 0) -> None:
    """Run many transforms in one launch (dwt_batch_submit).  ``requests``
    come from :meth:`Plan.request`; ``status``, if given, is a device int32
    tensor with one slot per request."""
    if status is not None and (status.numel() < len(requests) or status.dtype.itemsize != 4):
        raise ValueError("status needs one int32 slot per request")
    dwt_batch_submit(list(requests), stream, status.data_ptr() if status is not None else 0)
