"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/geraf.h declares; argument errors come back as status
codes without touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libgeraf():
    from paper_2605_29097_gb300 import _build, _lib
    _build.build()
    return _lib.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "geraf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(geraf_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(libgeraf):
    names = _declared()
    assert len(names) >= 13
    for nm in names:
        assert hasattr(libgeraf, nm), nm


def test_argument_errors_return_status_without_device(libgeraf):
    from paper_2605_29097_gb300 import _lib
    n = ctypes.c_size_t(0)
    band = _lib.GerafBand(77e9, 1e8, 32)
    # n_pts = 0 is rejected before anything is launched
    st = libgeraf.geraf_render(None, None, None, None, 0, None, None, 4, ctypes.byref(band), 1, None,
                               ctypes.byref(n), None, None)
    assert st == 1 and b"n_pts" in libgeraf.geraf_last_error_string()
    # misaligned workspace
    st = libgeraf.geraf_filter_backward(None, 4, ctypes.byref(band), None, 10, None, None,
                                        ctypes.c_void_p(8), ctypes.byref(n), None, None)
    assert st == 2
    # workspace size query needs no device memory
    st = libgeraf.geraf_render(None, None, None, None, 1000, None, None, 64, ctypes.byref(band), 1, None,
                               ctypes.byref(n), None, None)
    assert st == 0 and n.value > 0
    bad = _lib.GerafBand(77e9, 1e8, 0)
    st = libgeraf.geraf_render(None, None, None, None, 1000, None, None, 64, ctypes.byref(bad), 1, None,
                               ctypes.byref(n), None, None)
    assert st == 1
    # unknown phasor method
    bad = _lib.GerafBand(77e9, 1e8, 32, 7)
    st = libgeraf.geraf_render(None, None, None, None, 1000, None, None, 64, ctypes.byref(bad), 1, None,
                               ctypes.byref(n), None, None)
    assert st == 1 and b"method" in libgeraf.geraf_last_error_string()
    # the Chebyshev form's workspace (moment partials, coefficient table) is part of the size query
    cheb = _lib.GerafBand(77e9, 1e8, 128, 2)
    rec = _lib.GerafBand(77e9, 1e8, 128, 1)
    n_rec = ctypes.c_size_t(0)
    assert libgeraf.geraf_render(None, None, None, None, 1000, None, None, 64, ctypes.byref(cheb), 1, None,
                                 ctypes.byref(n), None, None) == 0
    assert libgeraf.geraf_render(None, None, None, None, 1000, None, None, 64, ctypes.byref(rec), 1, None,
                                 ctypes.byref(n_rec), None, None) == 0
    assert n.value > n_rec.value
    order = ctypes.c_int32(-1)
    assert libgeraf.geraf_chebyshev_order(None, 100, None, 4, ctypes.byref(cheb), None, ctypes.byref(n),
                                          ctypes.byref(order), None) == 0 and n.value > 0
    # the orders query: size query in both directions, bad direction rejected
    orders = (ctypes.c_int32 * 3)()
    mean = ctypes.c_double(0.0)
    for to_points in (0, 1):
        n.value = 0
        assert libgeraf.geraf_chebyshev_work(None, 5000, None, 300, ctypes.byref(cheb), to_points, None,
                                             ctypes.byref(n), orders, ctypes.byref(mean), None) == 0
        assert n.value > 0
    assert libgeraf.geraf_chebyshev_work(None, 5000, None, 300, ctypes.byref(cheb), 2, None, ctypes.byref(n),
                                         orders, ctypes.byref(mean), None) == 1
    assert b"to_points" in libgeraf.geraf_last_error_string()
    assert libgeraf.geraf_version() >= 1
