"""ctypes binding of the lutc C ABI (``include/lutc.h``).

Argument marshalling only: every step of the correction runs in the CUDA
library.  Tensors are torch CUDA tensors; the stream defaults to torch's
current stream of the tensor's device.  If the compiled library is missing
(and cannot be built) importing raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

LUTC_OK = 0
LUTC_EINVAL = -1
LUTC_EUNSUPPORTED = -2
LUTC_ENOMEM = -3
LUTC_ECUDA = -4
LUTC_ETIMEOUT = -5
LUTC_EBUSY = -6
LUTC_ESHUTDOWN = -7
LUTC_ECANCELED = -8
LUTC_STRETCH = 1
LUTC_MAX_BANDS = 64
LUTC_TRACE_PHASES = 3
LUTC_PATH_AUTO = 0
LUTC_PATH_TMA = 1
LUTC_PATH_STRIP = 2
LUTC_REQ_HOST = 2
LUTC_STATIC_SCRATCH_BYTES = 1 << 20
LUTC_TASK_LUTGEN, LUTC_TASK_HIST, LUTC_TASK_STRETCH, LUTC_TASK_COMPOSE = 1, 2, 3, 4
LUTC_TASK_APPLY, LUTC_TASK_CORRECT_IMAGE, LUTC_TASK_DEVICE_INFO, LUTC_TASK_DEMOSAIC, LUTC_TASK_FIT = 5, 6, 7, 8, 9
LUTC_BAYER = {"rggb": 0, "bggr": 1, "grbg": 2, "gbrg": 3}


class LutcError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (where, _strerror(status), status))


class Coeffs(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("G", ctypes.c_void_p), ("O", ctypes.c_void_p), ("ncols", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("column_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int32), ("max_wait_us", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("max_queue", ctypes.c_int32), ("fake_device", ctypes.c_int32),
                ("fake_latency_us", ctypes.c_int32), ("fail_every", ctypes.c_int32), ("hold_when_idle", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batch_size", ctypes.c_int32), ("submit_s", ctypes.c_double),
                ("start_s", ctypes.c_double), ("launched_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("cache_miss", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class ReplayRequest(ctypes.Structure):
    _fields_ = [("at_s", ctypes.c_double), ("raster", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("pitch_bytes", ctypes.c_int64), ("out_pitch_bytes", ctypes.c_int64), ("sensor_id", ctypes.c_int32),
                ("height", ctypes.c_int32), ("flags", ctypes.c_int32), ("pad", ctypes.c_int32)]


class Raster(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("pitch_bytes", ctypes.c_int64), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("bands", ctypes.c_int32), ("bits", ctypes.c_int32)]


class Job(ctypes.Structure):
    _fields_ = [("in_", Raster), ("per_band", ctypes.POINTER(Coeffs)), ("out", ctypes.c_void_p),
                ("out_pitch_bytes", ctypes.c_int64), ("flags", ctypes.c_int32)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("column_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("use_graph", ctypes.c_int32)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_RP = ctypes.POINTER(Raster)
_CP = ctypes.POINTER(Coeffs)

#: name -> (restype, argtypes) for every entry point declared in include/lutc.h
SIGNATURES = {
    "lutc_version": (_I, []),
    "lutc_strerror": (ctypes.c_char_p, [_I]),
    "lutc_lutgen": (_I, [_CP, _I, _P, _P]),
    "lutc_apply_u16": (_I, [_RP, _P, _P, _I64, _P]),
    "lutc_hist": (_I, [_RP, _CP, _P, _P]),
    "lutc_stretch": (_I, [_P, _I, _I, _P, _P, _P]),
    "lutc_compose": (_I, [_P, _P, _I, _I, _P, _P]),
    "lutc_apply_u8": (_I, [_RP, _P, _P, _I64, _P]),
    "lutc_correct_image_workspace": (_SZ, [_RP]),
    "lutc_correct_image_tables": (_I, [_RP, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "lutc_correct_image": (_I, [_RP, _CP, _I, _P, _I64, _P, _SZ, _P]),
    "lutc_apply_stretch": (_I, [_RP, _CP, _P, _P, _I64, _P]),
    "lutc_correct_image_static": (_I, [_RP, _CP, _I, _P, _I64, _P]),
    "lutc_trace_enable": (_I, [_I]),
    "lutc_device_status": (_I, [ctypes.POINTER(_I), _P]),
    "lutc_set_tuning": (_I, [_I, ctypes.POINTER(Tuning)]),
    "lutc_submit": (_I, [_I, ctypes.c_char_p, ctypes.POINTER(_P), _I, ctypes.POINTER(_P), _I, _P, _SZ, _P]),
    "lutc_device_info": (_I, [ctypes.c_char_p, _SZ, ctypes.POINTER(_SZ)]),
    "lutc_fit": (_I, [_P, _I64, _P, _I64, _I, _I, _I, _P, _P, _P, _P]),
    "lutc_correct_image_host_workspace": (_SZ, [ctypes.POINTER(Raster), _I]),
    "lutc_correct_image_host": (_I, [ctypes.POINTER(Raster), ctypes.POINTER(Coeffs), _I, _P, _I64, _P, _SZ, _P]),
    "lutc_net_server_create": (_I, [ctypes.c_char_p, _I, _I, ctypes.POINTER(_P)]),
    "lutc_net_server_port": (_I, [_P]),
    "lutc_net_server_stats": (_I, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "lutc_net_server_destroy": (_I, [_P]),
    "lutc_selftest_wait_timeout": (_I, [ctypes.c_longlong, _P]),
    "lutc_correct_frames_host_workspace": (_SZ, [ctypes.POINTER(Raster), _I, _I]),
    "lutc_correct_frames_host": (_I, [ctypes.POINTER(Raster), ctypes.POINTER(_P), _I, ctypes.POINTER(Coeffs), _I,
                                      ctypes.POINTER(_P), _I64, _P, _SZ, _P]),
    "lutc_demosaic": (_I, [ctypes.POINTER(Raster), ctypes.POINTER(Coeffs), _I, _P, _I64, _P]),
    "lutc_batch_workspace": (_SZ, [ctypes.POINTER(Job), _I]),
    "lutc_server_create": (_I, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)]),
    "lutc_server_register_sensor": (_I, [_P, _I, _I, _I, _I, _P, _P, _P]),
    "lutc_server_submit": (_I, [_P, _I, _P, _I, _I64, _P, _I64, _I, ctypes.POINTER(ctypes.c_uint64)]),
    "lutc_server_wait": (_I, [_P, ctypes.c_uint64, _I64, ctypes.POINTER(RequestInfo)]),
    "lutc_server_stats": (_I, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                               ctypes.POINTER(_SZ), ctypes.POINTER(ctypes.c_int32)]),
    "lutc_server_destroy": (_I, [_P]),
    "lutc_server_cancel": (_I, [_P, ctypes.c_uint64]),
    "lutc_server_replay": (_I, [_P, ctypes.POINTER(ReplayRequest), _I, ctypes.POINTER(RequestInfo),
                                ctypes.POINTER(ctypes.c_double)]),
    "lutc_batch_create": (_I, [ctypes.POINTER(Job), _I, ctypes.POINTER(BatchConfig), _P, _SZ, _P,
                               ctypes.POINTER(_P)]),
    "lutc_batch_run": (_I, [_P, _P]),
    "lutc_batch_tables": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "lutc_batch_destroy": (_I, [_P]),
    "lutc_batch_correct": (_I, [ctypes.POINTER(Job), _I, ctypes.POINTER(BatchConfig), _P, _SZ, _P]),
    "lutc_batch_autotune": (_I, [ctypes.POINTER(Job), _I, _P, _SZ, _P, _I, ctypes.POINTER(BatchConfig),
                                 ctypes.POINTER(ctypes.c_float)]),
    "lutc_get_tuning": (_I, [_I, ctypes.POINTER(Tuning)]),
    "lutc_last_path": (_I, [ctypes.POINTER(_I)]),
    "lutc_probe_fp64_fma": (_I, [_I, ctypes.c_longlong, _P, ctypes.POINTER(ctypes.c_longlong), _P]),
    "lutc_trace_read": (_I, [ctypes.POINTER(ctypes.c_float), _I]),
}

_lib = None


def checked() -> bool:
    """True when ``LUTC_CHECKED=1`` selects the bounds-checking build of the library."""
    return os.environ.get("LUTC_CHECKED") == "1"


def lib(build_if_stale: bool = True) -> ctypes.CDLL:
    """The loaded ``liblutc.so`` (built first if it is missing or older than its sources), or its
    bounds-checking variant under ``LUTC_CHECKED=1``."""
    global _lib
    if _lib is None:
        if checked():
            path = _build.build(checked=True) if build_if_stale else _build.CHECKED_LIB
        else:
            path = _build.build() if build_if_stale else _build.LIB
        if not os.path.exists(path):
            raise ImportError("lutc CUDA library not built: %s" % path)
        handle = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _strerror(status: int) -> str:
    try:
        return lib().lutc_strerror(status).decode()
    except Exception:  # pragma: no cover - only while the library is unusable
        return "status %d" % status


def check(status: int, where: str) -> None:
    if status != LUTC_OK:
        raise LutcError(status, where)
