"""ctypes binding of ``include/wave2d.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``libwave2d.so``; this
module converts arguments and raises on error codes.  There is no fallback:
if the library is missing or cannot load, importing the binding fails.

PyTorch is used for device memory (its caching allocator is installed as the
library's allocation hook by ``use_torch_allocator``) and for streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libwave2d.so")

OK = 0
ERR_ARG, ERR_UNSTABLE, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE = -1, -2, -3, -4, -5, -6, -7
BC_ZERO, BC_PERIODIC, BC_ODD = 0, 1, 2
F64, F32, F32X2 = 0, 1, 2
ALLOW_UNSTABLE, CONVENTIONAL, DIFF_SUMS, DIFF_FORM, CANARY = 1, 2, 4, 8, 16
EXACT_NONE, EXACT_STANDING, EXACT_PLANE = 0, 1, 2
KERNEL_AUTO, KERNEL_SIMPLE, KERNEL_TMA, KERNEL_TEMPORAL, KERNEL_STREAM, KERNEL_PERSISTENT = 0, 1, 2, 3, 4, 5

_NAMES = {ERR_ARG: "ERR_ARG", ERR_UNSTABLE: "ERR_UNSTABLE", ERR_OOM: "ERR_OOM", ERR_CUDA: "ERR_CUDA",
          ERR_NONFINITE: "ERR_NONFINITE", ERR_TIMEOUT: "ERR_TIMEOUT", ERR_STATE: "ERR_STATE"}


class Wave2DError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class wave2d_exact(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("amp", ctypes.c_double),
                ("m", ctypes.c_double), ("k1", ctypes.c_double), ("k2", ctypes.c_double),
                ("x_off", ctypes.c_double)]


class wave2d_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("bc", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class wave2d_tune(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("temporal_t", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


class wave2d_info_t(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("h", ctypes.c_double), ("tau", ctypes.c_double),
                ("c", ctypes.c_double), ("a", ctypes.c_double * 3), ("b", ctypes.c_double * 3),
                ("lambda_max", ctypes.c_double), ("k", ctypes.c_int64), ("scheme", ctypes.c_int32),
                ("radius", ctypes.c_int32), ("dtype", ctypes.c_int32), ("bc", ctypes.c_int32),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("ghost", ctypes.c_int32), ("device_bytes", ctypes.c_int64), ("kernel", ctypes.c_int32),
                ("temporal_t", ctypes.c_int32), ("n_classes", ctypes.c_int32), ("n_points", ctypes.c_int32),
                ("class_a", ctypes.c_double * 8), ("class_b", ctypes.c_double * 8)]


# Classes of the derived schemes, in chain order (include/wave2d.h).
CLASS_CHAIN = ((1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (2, 2), (3, 1), (4, 0))


class wave2d_scheme(ctypes.Structure):
    _fields_ = [("segment", ctypes.c_int32), ("n_classes", ctypes.c_int32), ("radius", ctypes.c_int32),
                ("n_points", ctypes.c_int32), ("a", (ctypes.c_double * 9) * 8), ("b", (ctypes.c_double * 9) * 8)]

    def a_poly(self, c):
        """Coefficients of a_c(lambda) by power 0..8."""
        return [self.a[c][p] for p in range(9)]

    def b_poly(self, c):
        return [self.b[c][p] for p in range(9)]


class wave2d_request(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("h", ctypes.c_double), ("tau", ctypes.c_double),
                ("c", ctypes.c_double), ("steps", ctypes.c_int64), ("u0", ctypes.c_void_p),
                ("v0", ctypes.c_void_p), ("pulse_amp", ctypes.c_double), ("pulse_cx", ctypes.c_double),
                ("pulse_cy", ctypes.c_double), ("pulse_sigma", ctypes.c_double),
                ("out_field", ctypes.c_void_p), ("tag", ctypes.c_uint64)]


class wave2d_completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("l2", ctypes.c_double), ("linf", ctypes.c_double), ("k", ctypes.c_int64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class wave2d_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("node_updates", ctypes.c_int64), ("rounds", ctypes.c_int64), ("used_bytes", ctypes.c_int64),
                ("max_resident_seen", ctypes.c_int32), ("reserved", ctypes.c_int32), ("gpu_busy_s", ctypes.c_double)]


class wave2d_alu_peaks_t(ctypes.Structure):
    _fields_ = [("fp32_fma", ctypes.c_double), ("fp32_fma2", ctypes.c_double), ("fp32_add", ctypes.c_double),
                ("fp64_fma", ctypes.c_double), ("sms", ctypes.c_int32), ("clock_khz", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

# Every exported symbol of include/wave2d.h with (restype, argtypes).
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I64P = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "wave2d_set_allocator": (ctypes.c_int, [ALLOC_FN, FREE_FN, _P]),
    "wave2d_create": (ctypes.c_int, [ctypes.POINTER(wave2d_grid), ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, ctypes.POINTER(_P)]),
    "wave2d_derive_scheme": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(wave2d_scheme)]),
    "wave2d_scheme_lambda_max": (ctypes.c_int, [ctypes.POINTER(wave2d_scheme), _D]),
    "wave2d_create_scheme": (ctypes.c_int, [ctypes.POINTER(wave2d_grid), ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.POINTER(wave2d_scheme), ctypes.POINTER(_P)]),
    "wave2d_first_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "wave2d_step_n": (ctypes.c_int, [_P, ctypes.c_int64]),
    "wave2d_error_vs_exact": (ctypes.c_int, [_P, ctypes.POINTER(wave2d_exact), _D, _D, _D]),
    "wave2d_track_error": (ctypes.c_int, [_P, ctypes.POINTER(wave2d_exact)]),
    "wave2d_get_state": (ctypes.c_int, [_P, _P, _P, _I64P]),
    "wave2d_set_state": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int]),
    "wave2d_raw_bytes": (ctypes.c_int64, [_P]),
    "wave2d_get_raw": (ctypes.c_int, [_P, _P, ctypes.c_int64, _I64P]),
    "wave2d_set_raw": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int64]),
    "wave2d_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(wave2d_tune)]),
    "wave2d_autotune": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(wave2d_tune)]),
    "wave2d_get_info": (ctypes.c_int, [_P, ctypes.POINTER(wave2d_info_t)]),
    "wave2d_sync": (ctypes.c_int, [_P]),
    "wave2d_selftest_timeout": (ctypes.c_int, [_P, ctypes.c_int64]),
    "wave2d_canary_check": (ctypes.c_int, [_P, _I64P]),
    "wave2d_destroy": (None, [_P]),
    "wave2d_last_error": (ctypes.c_char_p, []),
    "wave2d_launch_count": (ctypes.c_int64, []),
    "wave2d_lambda_max": (ctypes.c_double, [ctypes.c_int, ctypes.c_int]),
    "wave2d_alu_peaks": (ctypes.c_int, [ctypes.POINTER(wave2d_alu_peaks_t), _P]),
    "wave2d_diff_norms": (ctypes.c_int, [_P, _P, _D, _D]),
    "wave2d_get_rows": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int]),
    "wave2d_set_rows": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int]),
    "wave2d_error_sums": (ctypes.c_int, [_P, ctypes.POINTER(wave2d_exact), ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int64, _D]),
    "wave2d_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(wave2d_tune),
                                           ctypes.POINTER(_P)]),
    "wave2d_batch_first_step": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int]),
    "wave2d_batch_run": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "wave2d_batch_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                                             ctypes.POINTER(wave2d_tune)]),
    "wave2d_batch_norms": (ctypes.c_int, [_P, _D]),
    "wave2d_batch_destroy": (None, [_P]),
    "wave2d_required_bytes": (ctypes.c_int64, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "wave2d_server_create": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(wave2d_tune),
                                            _P, ctypes.POINTER(_P)]),
    "wave2d_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(wave2d_request)]),
    "wave2d_server_poll": (ctypes.c_int, [_P, ctypes.POINTER(wave2d_completion), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]),
    "wave2d_server_drain": (ctypes.c_int, [_P, ctypes.c_double]),
    "wave2d_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(wave2d_server_stats_t)]),
    "wave2d_server_destroy": (None, [_P]),
    "wave2d_error_norms_noalloc": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                                  ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                  ctypes.POINTER(wave2d_exact), _D, _D, _P]),
}

_lib = None


def lib():
    """Load libwave2d.so (raises if it is missing: there is no CPU path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"wave2d CUDA library not built: {LIB_PATH} is missing "
                              "(run paper_1904_04048_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().wave2d_last_error().decode()


def check(rc: int) -> int:
    if rc < 0:
        raise Wave2DError(rc, last_error())
    return rc


def launch_count() -> int:
    return lib().wave2d_launch_count()


def lambda_max(scheme: int, conventional: bool = False) -> float:
    return lib().wave2d_lambda_max(scheme, int(conventional))


def alu_peaks(stream=None) -> wave2d_alu_peaks_t:
    """wave2d_alu_peaks: measured FP32 / FP64 lane operations per second of
    the current device (``stream``: a cudaStream_t as int, or None)."""
    out = wave2d_alu_peaks_t()
    check(lib().wave2d_alu_peaks(ctypes.byref(out), stream))
    return out


def derive_scheme(m: int) -> wave2d_scheme:
    """Scheme of the monomial segment M*_{<=m} (host-side derivation)."""
    s = wave2d_scheme()
    check(lib().wave2d_derive_scheme(int(m), ctypes.byref(s)))
    return s


def scheme_lambda_max(s: wave2d_scheme) -> float:
    out = ctypes.c_double()
    check(lib().wave2d_scheme_lambda_max(ctypes.byref(s), ctypes.byref(out)))
    return out.value


def error_norms_noalloc(field_ptr: int, dtype: int, nx: int, ny: int, ld: int, h: float, c: float,
                        t: float, ex: wave2d_exact | None = None, stream: int = 0):
    """(rel_l2, rel_linf) of a caller-owned device field through the
    allocation-free entry point (see include/wave2d.h)."""
    l2, linf = ctypes.c_double(), ctypes.c_double()
    check(lib().wave2d_error_norms_noalloc(ctypes.c_void_p(int(field_ptr)), int(dtype), int(nx), int(ny),
                                           int(ld), float(h), float(c), float(t),
                                           ctypes.byref(ex) if ex is not None else None,
                                           ctypes.byref(l2), ctypes.byref(linf),
                                           ctypes.c_void_p(int(stream) if stream else 0)))
    return l2.value, linf.value


# ----------------------------------------------------------------- allocator
_alloc_refs = None


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _alloc_refs
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0))
        except Exception:  # out of memory: the library reports WAVE2D_ERR_OOM
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    refs = (ALLOC_FN(_alloc), FREE_FN(_free))
    check(lib().wave2d_set_allocator(refs[0], refs[1], None))
    _alloc_refs = refs


def use_default_allocator():
    global _alloc_refs
    check(lib().wave2d_set_allocator(ALLOC_FN(), FREE_FN(), None))
    _alloc_refs = None


# ----------------------------------------------------------------- helpers
def exact(kind=EXACT_NONE, amp=1.0, m=1.0, k1=0.0, k2=0.0, x_off=0.0) -> wave2d_exact:
    return wave2d_exact(kind, 0, amp, m, k1, k2, x_off)


def _host_f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _ptr(a):
    """(pointer, on_device) of a numpy array or CUDA torch tensor of float64."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p), 0
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("device inputs must be contiguous float64 tensors")
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda)
    raise TypeError(type(a))


def _buf_ptr(a):
    """(pointer, on_device) of a contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("row buffers must be contiguous")
        return a.ctypes.data_as(ctypes.c_void_p), 0
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("row buffers must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda)
    raise TypeError(type(a))


class Wave2D:
    """One simulation handle (``wave2d_t``)."""

    def __init__(self, nx, ny, h, tau, c=1.0, scheme=13, bc=BC_ZERO, dtype=F32, flags=0, stream=None):
        """``scheme``: 5, 9 or 13 (Section 6), or a ``wave2d_scheme`` (derived)."""
        g = wave2d_grid(int(nx), int(ny), int(bc), int(dtype), int(flags), 0,
                        ctypes.c_void_p(int(stream) if stream else 0))
        out = ctypes.c_void_p()
        if isinstance(scheme, wave2d_scheme):
            check(lib().wave2d_create_scheme(ctypes.byref(g), float(h), float(tau), float(c),
                                             ctypes.byref(scheme), ctypes.byref(out)))
        else:
            check(lib().wave2d_create(ctypes.byref(g), float(h), float(tau), float(c), int(scheme),
                                      ctypes.byref(out)))
        self._h = out
        self.nx, self.ny = int(nx), int(ny)

    def close(self):
        if getattr(self, "_h", None):
            lib().wave2d_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def first_step(self, u0, v0):
        n = self.nx * self.ny
        if isinstance(u0, np.ndarray) or not hasattr(u0, "data_ptr"):
            u0 = _host_f64(u0, n)
            v0 = _host_f64(v0, n)
        pu, du = _ptr(u0)
        pv, dv = _ptr(v0)
        if du != dv:
            raise ValueError("u0 and v0 must both be on the host or both on the device")
        check(lib().wave2d_first_step(self._h, pu, pv, du))

    def step_n(self, n):
        check(lib().wave2d_step_n(self._h, int(n)))

    def error_vs_exact(self, ex: wave2d_exact | None = None):
        l2, linf, E = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        rc = lib().wave2d_error_vs_exact(self._h, ctypes.byref(ex) if ex is not None else None,
                                         ctypes.byref(l2), ctypes.byref(linf), ctypes.byref(E))
        check(rc)
        return l2.value, linf.value, E.value

    def track_error(self, ex: wave2d_exact | None):
        check(lib().wave2d_track_error(self._h, ctypes.byref(ex) if ex is not None else None))

    def get_state(self):
        up = np.empty((self.ny, self.nx))
        uc = np.empty((self.ny, self.nx))
        k = ctypes.c_int64()
        check(lib().wave2d_get_state(self._h, up.ctypes.data_as(ctypes.c_void_p),
                                     uc.ctypes.data_as(ctypes.c_void_p), ctypes.byref(k)))
        return up, uc, k.value

    def set_state(self, u_prev, u_cur, k):
        n = self.nx * self.ny
        up, uc = _host_f64(u_prev, n), _host_f64(u_cur, n)
        check(lib().wave2d_set_state(self._h, up.ctypes.data_as(ctypes.c_void_p),
                                     uc.ctypes.data_as(ctypes.c_void_p), int(k), 0))

    def diff_norms(self, ref: "Wave2D"):
        """wave2d_diff_norms: (relative L2, relative L-infinity) of this
        handle's current level against ``ref``'s (same grid, same k)."""
        l2, linf = ctypes.c_double(), ctypes.c_double()
        check(lib().wave2d_diff_norms(self._h, ref.handle, ctypes.byref(l2), ctypes.byref(linf)))
        return l2.value, linf.value

    def row_block_shape(self, nrows):
        """Shape and numpy dtype of one plane's packed row block of
        wave2d_get_rows / wave2d_set_rows for this handle's storage type."""
        dt = self.info().dtype
        if dt == F64:
            return (nrows, self.nx), np.float64
        if dt == F32X2:
            return (2, nrows, self.nx), np.float32
        return (nrows, self.nx), np.float32

    def get_rows(self, j0, nrows, prev, cur):
        """wave2d_get_rows into caller buffers of ``row_block_shape(nrows)``:
        numpy arrays (host) or contiguous CUDA tensors (device, queued on the
        handle's stream)."""
        pp, dp = _buf_ptr(prev)
        pc, dc = _buf_ptr(cur)
        if dp != dc:
            raise ValueError("prev and cur must both be on the host or both on the device")
        check(lib().wave2d_get_rows(self._h, int(j0), int(nrows), pp, pc, dp))

    def set_rows(self, j0, nrows, prev, cur):
        """wave2d_set_rows from buffers of ``row_block_shape(nrows)``."""
        pp, dp = _buf_ptr(prev)
        pc, dc = _buf_ptr(cur)
        if dp != dc:
            raise ValueError("prev and cur must both be on the host or both on the device")
        check(lib().wave2d_set_rows(self._h, int(j0), int(nrows), pp, pc, dp))

    def error_sums(self, ex, j0, nrows, row_shift=0):
        """wave2d_error_sums: [sum (u-u_e)^2, sum u_e^2, max |u-u_e|, max |u_e|]
        over rows j0 .. j0 + nrows - 1, u_e placed at rows + row_shift."""
        out = (ctypes.c_double * 4)()
        check(lib().wave2d_error_sums(self._h, ctypes.byref(ex) if ex is not None else None, int(j0), int(nrows),
                                      int(row_shift), out))
        return [out[0], out[1], out[2], out[3]]

    def get_raw(self):
        nb = check(lib().wave2d_raw_bytes(self._h))
        buf = np.empty(nb, dtype=np.uint8)
        k = ctypes.c_int64()
        check(lib().wave2d_get_raw(self._h, buf.ctypes.data_as(ctypes.c_void_p), nb, ctypes.byref(k)))
        return buf, k.value

    def set_raw(self, buf, k):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        check(lib().wave2d_set_raw(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.size, int(k)))

    def set_tuning(self, kernel=KERNEL_AUTO, tile_h=0, temporal_t=0, use_graph=-1, ctas_per_sm=0):
        """wave2d_set_tuning: ``kernel`` one of KERNEL_AUTO / SIMPLE / TMA /
        TEMPORAL / STREAM; ``tile_h`` rows per tile (TEMPORAL: 16, 24, 32, 64)
        or per strip (STREAM: 8 .. 4096), 0 = default; ``temporal_t`` levels
        per launch of the two multi-level kernels (TEMPORAL: 2, 3, 4; STREAM:
        2, 3, 4, 6, in the difference form 2, 3, 4; 0 = the default depth)."""
        t = wave2d_tune(int(kernel), int(tile_h), int(temporal_t), int(use_graph), int(ctas_per_sm))
        check(lib().wave2d_set_tuning(self._h, ctypes.byref(t)))

    def autotune(self, steps=16) -> wave2d_tune:
        best = wave2d_tune()
        check(lib().wave2d_autotune(self._h, int(steps), ctypes.byref(best)))
        return best

    def info(self) -> wave2d_info_t:
        inf = wave2d_info_t()
        check(lib().wave2d_get_info(self._h, ctypes.byref(inf)))
        return inf

    def canary_check(self) -> int:
        """Number of guard-band cells that changed (handles with CANARY)."""
        out = ctypes.c_int64()
        check(lib().wave2d_canary_check(self._h, ctypes.byref(out)))
        return out.value

    def sync(self):
        check(lib().wave2d_sync(self._h))

    def selftest_timeout(self, limit_cycles=1 << 20):
        check(lib().wave2d_selftest_timeout(self._h, int(limit_cycles)))


class Batch:
    """A batch of handles stepped together (``wave2d_batch_t``)."""

    def __init__(self, sims, temporal_t=0, tile_h=0, kernel=KERNEL_TEMPORAL):
        """kernel: KERNEL_TEMPORAL (shared-memory regions, any boundary) or
        KERNEL_STREAM (register streaming, zero boundary); tile_h: rows per
        region (32, 64) or per strip (8..1024); temporal_t: levels per launch."""
        self.sims = list(sims)
        arr = (ctypes.c_void_p * len(self.sims))(*[s.handle.value for s in self.sims])
        opt = wave2d_tune(int(kernel), int(tile_h), int(temporal_t), -1, 0)
        out = ctypes.c_void_p()
        check(lib().wave2d_batch_create(arr, len(self.sims), ctypes.byref(opt), ctypes.byref(out)))
        self._b = out
        self._keep = arr

    def close(self):
        if getattr(self, "_b", None):
            lib().wave2d_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def first_step(self, u0s, v0s):
        """Host (numpy) or device (torch float64) initial data, one pair per instance."""
        n = len(self.sims)
        keep = []
        on_dev = None
        pu, pv = (ctypes.c_void_p * n)(), (ctypes.c_void_p * n)()
        for i, (s, a, b) in enumerate(zip(self.sims, u0s, v0s)):
            if isinstance(a, np.ndarray) or not hasattr(a, "data_ptr"):
                a = _host_f64(a, s.nx * s.ny)
                b = _host_f64(b, s.nx * s.ny)
            keep += [a, b]
            (p1, d1), (p2, d2) = _ptr(a), _ptr(b)
            if on_dev is None:
                on_dev = d1
            if d1 != on_dev or d2 != on_dev:
                raise ValueError("all initial data must be on the host or all on the device")
            pu[i], pv[i] = p1, p2
        check(lib().wave2d_batch_first_step(self._b, pu, pv, int(on_dev or 0)))

    def run(self, steps):
        arr = (ctypes.c_int64 * len(self.sims))(*[int(x) for x in steps])
        check(lib().wave2d_batch_run(self._b, arr))

    def autotune(self, steps, probe_steps=32) -> wave2d_tune:
        arr = (ctypes.c_int64 * len(self.sims))(*[int(x) for x in steps])
        best = wave2d_tune()
        check(lib().wave2d_batch_autotune(self._b, arr, int(probe_steps), ctypes.byref(best)))
        return best

    def norms(self):
        out = np.zeros(2 * len(self.sims))
        check(lib().wave2d_batch_norms(self._b, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out.reshape(-1, 2)


class Server:
    """Continuous-batching server (``wave2d_server_t``)."""

    def __init__(self, budget_bytes=16 << 30, max_resident=512, quantum=64, temporal_t=0, tile_h=0, stream=None,
                 kernel=KERNEL_STREAM):
        opt = wave2d_tune(int(kernel), int(tile_h), int(temporal_t), 0, 0)
        out = ctypes.c_void_p()
        check(lib().wave2d_server_create(int(budget_bytes), int(max_resident), int(quantum), ctypes.byref(opt),
                                         ctypes.c_void_p(int(stream) if stream else 0), ctypes.byref(out)))
        self._s = out
        self._keep = {}

    def submit(self, nx, ny, h, tau, steps, scheme=13, c=1.0, u0=None, v0=None, pulse=None, tag=0,
               out_field=None, flags=0):
        """Queue a request; pulse = (amp, cx, cy, sigma) when u0/v0 are not given;
        out_field: numpy (ny, nx) float64 array receiving the final level."""
        r = wave2d_request()
        r.nx, r.ny, r.scheme, r.flags = int(nx), int(ny), int(scheme), int(flags)
        r.h, r.tau, r.c, r.steps, r.tag = float(h), float(tau), float(c), int(steps), int(tag)
        if u0 is not None:
            a = _host_f64(u0, nx * ny)
            b = _host_f64(v0, nx * ny)
            r.u0 = a.ctypes.data_as(ctypes.c_void_p)
            r.v0 = b.ctypes.data_as(ctypes.c_void_p)
        elif pulse is not None:
            r.pulse_amp, r.pulse_cx, r.pulse_cy, r.pulse_sigma = (float(x) for x in pulse)
        if out_field is not None:
            assert out_field.dtype == np.float64 and out_field.flags.c_contiguous and out_field.size == nx * ny
            r.out_field = out_field.ctypes.data_as(ctypes.c_void_p)
            self._keep[int(tag)] = out_field
        check(lib().wave2d_server_submit(self._s, ctypes.byref(r)))

    def poll(self, max_n=1024):
        buf = (wave2d_completion * max_n)()
        n = ctypes.c_int()
        check(lib().wave2d_server_poll(self._s, buf, max_n, ctypes.byref(n)))
        out = [buf[i] for i in range(n.value)]
        for c in out:
            self._keep.pop(int(c.tag), None)
        return out

    def drain(self, timeout_s=600.0):
        check(lib().wave2d_server_drain(self._s, float(timeout_s)))

    def stats(self) -> wave2d_server_stats_t:
        st = wave2d_server_stats_t()
        check(lib().wave2d_server_stats(self._s, ctypes.byref(st)))
        return st

    def close(self):
        if getattr(self, "_s", None):
            lib().wave2d_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
