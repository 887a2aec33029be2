"""ctypes declarations of the C ABI in ``include/geraf.h``.

Loads the in-tree ``libgeraf.so`` and fails loudly when it is missing: there
is no CPU fallback for any call.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgeraf.so")

c_float_p = ctypes.POINTER(ctypes.c_float)
vp = ctypes.c_void_p
i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
f32, sz = ctypes.c_float, ctypes.c_size_t
szp = ctypes.POINTER(ctypes.c_size_t)


class GerafGrid(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("pitch", ctypes.c_float * 3), ("n", ctypes.c_int32 * 3),
                ("aperture_z", ctypes.c_float)]


class GerafBand(ctypes.Structure):
    _fields_ = [("f0", ctypes.c_double), ("df", ctypes.c_double), ("n_f", ctypes.c_int32), ("method", ctypes.c_int32)]


class GerafFieldDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("prims", vp), ("n_prims", ctypes.c_int32), ("params", vp),
                ("n_levels", ctypes.c_int32), ("width", ctypes.c_int32), ("n_hidden", ctypes.c_int32),
                ("beta", ctypes.c_float), ("center", ctypes.c_float * 3), ("half", ctypes.c_float),
                ("precision", ctypes.c_int32), ("refl_hidden", ctypes.c_int32), ("refl_width", ctypes.c_int32)]


class GerafProposal(ctypes.Structure):
    _fields_ = [("features", vp), ("params", vp), ("g", ctypes.c_int32 * 3), ("feat", ctypes.c_int32),
                ("width", ctypes.c_int32), ("n_hidden", ctypes.c_int32), ("beta", ctypes.c_float),
                ("eps", ctypes.c_float), ("depth", ctypes.c_int32)]


# name -> argtypes (all return geraf_status as int)
SIGNATURES = {
    "geraf_poll_device_error": [vp],
    "geraf_check_bounded_wait": [u64, vp],
    "geraf_sample": [ctypes.POINTER(GerafGrid), i32, u64, u64, vp, vp, vp],
    "geraf_fields_saved_bytes": [ctypes.POINTER(GerafFieldDesc), i64, szp],
    "geraf_fields": [ctypes.POINTER(GerafFieldDesc), vp, i64, vp, vp, vp, vp, sz, vp],
    "geraf_fields_backward": [ctypes.POINTER(GerafFieldDesc), vp, i64, vp, vp, vp, vp, vp, vp, szp, vp],
    "geraf_blend": [vp, vp, i32, i32, vp, vp, i32, f32, f32, vp, vp, vp, vp, vp, vp, vp],
    "geraf_blend_backward": [vp, vp, vp, vp, i32, i32, f32, f32, vp, vp, vp, vp, vp, vp, vp, szp, vp],
    "geraf_render": [vp, vp, vp, vp, i64, vp, vp, i32, ctypes.POINTER(GerafBand), i32, vp, szp, vp, vp],
    "geraf_render_noalloc": [vp, vp, vp, vp, i64, vp, vp, i32, ctypes.POINTER(GerafBand), i32, vp, vp],
    "geraf_render_backward": [vp, vp, vp, vp, i64, vp, vp, i32, ctypes.POINTER(GerafBand), i32, vp, vp, szp,
                              vp, vp, vp, vp],
    "geraf_filter": [vp, vp, i32, ctypes.POINTER(GerafBand), vp, i64, vp, vp, vp, szp, vp, vp, vp, vp, vp],
    "geraf_filter_backward": [vp, i32, ctypes.POINTER(GerafBand), vp, i64, vp, vp, vp, szp, vp, vp],
    "geraf_chebyshev_order": [vp, i64, vp, i32, ctypes.POINTER(GerafBand), vp, szp, ctypes.POINTER(i32), vp],
    "geraf_chebyshev_work": [vp, i64, vp, i32, ctypes.POINTER(GerafBand), i32, vp, szp, ctypes.POINTER(i32),
                             ctypes.POINTER(ctypes.c_double), vp],
    "geraf_masked_loss": [vp, vp, vp, i64, f32, f32, vp, szp, vp, vp, vp, vp],
    "geraf_proposal_saved_bytes": [ctypes.POINTER(GerafProposal), szp],
    "geraf_proposal_density": [ctypes.POINTER(GerafProposal), vp, vp, vp, sz, vp],
    "geraf_sample_proposal": [ctypes.POINTER(GerafGrid), ctypes.POINTER(GerafProposal), vp, u64, u64, vp, vp, vp, vp],
    "geraf_sample_cells": [ctypes.POINTER(GerafGrid), ctypes.POINTER(GerafProposal), vp, i32, i32, i32, u64, u64, vp,
                           vp, vp, vp, vp, szp, vp],
    "geraf_sample_backward": [ctypes.POINTER(GerafProposal), ctypes.POINTER(GerafGrid), i32, vp, vp, vp, vp, vp, vp,
                              vp, vp, vp, szp, vp],
}

STATUS = {0: "GERAF_OK", 1: "GERAF_ERR_INVALID_ARG", 2: "GERAF_ERR_ALIGNMENT", 3: "GERAF_ERR_CUDA",
          4: "GERAF_ERR_WORKSPACE", 5: "GERAF_ERR_TIMEOUT", 6: "GERAF_ERR_UNSUPPORTED"}


class GerafError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """The loaded C library (raises if the extension was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA extension {LIB_PATH} is missing; run __graft_entry__.build() first "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.geraf_last_error_string.restype = ctypes.c_char_p
        L.geraf_last_error_string.argtypes = []
        L.geraf_version.restype = ctypes.c_int32
        L.geraf_version.argtypes = []
        _lib = L
    return _lib


def check(status):
    if status != 0:
        raise GerafError(status, lib().geraf_last_error_string().decode())
