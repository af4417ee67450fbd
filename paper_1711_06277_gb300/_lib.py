"""ctypes declarations of the C ABI in ``include/art.h`` (argument marshalling only).

The library is loaded from the in-tree build folder. There is no fallback: if the library
is missing or fails to load, importing the binding raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

ART_OK = 0
ART_EINVAL = -1
ART_ENOMEM = -2
ART_EQUEUE_OVERFLOW = -3
ART_ETIMEOUT = -4
ART_EACCOUNTING = -5
ART_ECUDA = -6
ART_ESTATE = -7
ART_EINTERNAL = -8
ART_MAX_LEVEL = 13
ART_NLEVELS = 20
ART_SCHED_PERSISTENT = 0
ART_SCHED_PLAIN = 1
ART_F_ROTATE = 1

EXPORTED = [
    "art_params_default", "art_create_grid", "art_update_fields", "art_add_sources",
    "art_set_nonionizing", "art_clear_sources", "art_num_sources", "art_trace", "art_get_stats", "art_trace_backward",
    "art_xn_update", "art_dt_substep", "art_dt_scratch_bytes", "art_dt_substep_static",
    "art_estimate_work", "art_partition_sources", "art_destroy_grid", "art_strerror",
]
ART_DT_STATIC_MAX_CELLS = 1 << 24


class ArtParams(ctypes.Structure):
    _fields_ = [
        ("level0", ctypes.c_int),
        ("level_max", ctypes.c_int),
        ("m_ray", ctypes.c_double),
        ("tau_max", ctypes.c_double),
        ("sigma_H", ctypes.c_double),
        ("sigma_d", ctypes.c_double),
        ("rot", ctypes.c_double * 9),
        ("flags", ctypes.c_uint),
        ("schedule", ctypes.c_int),
        ("block_threads", ctypes.c_int),
        ("chunk", ctypes.c_int),
        ("queue_capacity", ctypes.c_longlong),
        ("wait_limit_s", ctypes.c_double),
        ("blocks_per_sm", ctypes.c_int),
        ("d_max", ctypes.c_double),
    ]


class ArtStats(ctypes.Structure):
    _fields_ = [
        ("crossings", ctypes.c_ulonglong),
        ("rays_total", ctypes.c_ulonglong),
        ("rays_per_level", ctypes.c_ulonglong * ART_NLEVELS),
        ("destroy", ctypes.c_ulonglong),
        ("destroy_expected", ctypes.c_ulonglong),
        ("L_in", ctypes.c_double),
        ("L_absorbed", ctypes.c_double),
        ("L_escaped", ctypes.c_double),
        ("L_dropped", ctypes.c_double),
        ("level_reached", ctypes.c_int),
        ("level_max", ctypes.c_int),
        ("status", ctypes.c_int),
        ("pad", ctypes.c_int),
        ("Ln_in", ctypes.c_double),
        ("Ln_absorbed", ctypes.c_double),
        ("Ln_escaped", ctypes.c_double),
        ("Ln_dropped", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("rays_per_level", "pad")}
        d["rays_per_level"] = list(self.rays_per_level)
        return d


class ArtError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})" if what else strerror(status))


_lib = None


def lib():
    """The loaded library (built first if needed)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            path = _build.build()
        L = ctypes.CDLL(path)
        vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        P = ctypes.POINTER
        L.art_params_default.argtypes = [P(ArtParams)]
        L.art_params_default.restype = None
        L.art_create_grid.argtypes = [P(vp), i, i, i, P(d), d, vp, vp, vp]
        L.art_create_grid.restype = i
        L.art_update_fields.argtypes = [vp, vp, vp]
        L.art_update_fields.restype = i
        L.art_add_sources.argtypes = [vp, i, P(d), P(d)]
        L.art_add_sources.restype = i
        L.art_set_nonionizing.argtypes = [vp, P(d)]
        L.art_set_nonionizing.restype = i
        L.art_clear_sources.argtypes = [vp]
        L.art_clear_sources.restype = i
        L.art_num_sources.argtypes = [vp]
        L.art_num_sources.restype = i
        L.art_trace.argtypes = [vp, P(ArtParams), vp, vp, vp, P(ArtStats)]
        L.art_trace.restype = i
        L.art_get_stats.argtypes = [vp, P(ArtStats)]
        L.art_get_stats.restype = i
        L.art_trace_backward.argtypes = [vp, P(ArtParams), vp, vp, vp, vp, P(ArtStats)]
        L.art_trace_backward.restype = i
        L.art_xn_update.argtypes = [vp, ll, vp, vp, vp, vp, d, d, i]
        L.art_xn_update.restype = i
        L.art_dt_substep.argtypes = [vp, ll, vp, vp, vp, d, d, vp, vp]
        L.art_dt_substep.restype = i
        L.art_dt_scratch_bytes.argtypes = [ll]
        L.art_dt_scratch_bytes.restype = ll
        L.art_dt_substep_static.argtypes = [vp, ll, vp, vp, vp, d, d, vp]
        L.art_dt_substep_static.restype = i
        L.art_estimate_work.argtypes = [vp, P(ArtParams), P(d)]
        L.art_estimate_work.restype = i
        L.art_partition_sources.argtypes = [i, P(d), i, P(i), P(d)]
        L.art_partition_sources.restype = i
        L.art_destroy_grid.argtypes = [vp]
        L.art_destroy_grid.restype = None
        L.art_strerror.argtypes = [i]
        L.art_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().art_strerror(status).decode()


def check(status: int, what: str = "") -> int:
    if status != ART_OK:
        raise ArtError(status, what)
    return status
