"""Host-side checks of the serving engine's C ABI: argument validation
answers before any device work (no request is run here)."""
import ctypes

import numpy as np

from paper_1511_01353_gb300 import fmt as F


def test_server_rejects_bad_arguments():
    L = F.load()
    h = ctypes.c_void_p()
    assert L.fmt_server_create(0, 1e9, 1000, ctypes.byref(h)) == F.FMT_EINVAL
    assert L.fmt_server_create(2, 0.0, 1000, ctypes.byref(h)) == F.FMT_EINVAL
    assert L.fmt_server_create(2, 1e9, 0, ctypes.byref(h)) == F.FMT_EINVAL
    assert L.fmt_server_create(2, 1e9, 1000, ctypes.byref(h)) == F.FMT_OK
    x = np.zeros(4)
    r = F.fmt_request()
    r.params = F.make_params(4, 3, 1, 1e-4)
    t = ctypes.c_int64()
    r.n = 0
    r.x = r.y = r.z = r.f = x.ctypes.data
    assert L.fmt_server_submit(h, ctypes.byref(r), ctypes.byref(t)) == F.FMT_EINVAL
    r.n, r.m = 4, 3  # targets without arrays
    assert L.fmt_server_submit(h, ctypes.byref(r), ctypes.byref(t)) == F.FMT_EINVAL
    r.m = 0
    r.params.degree = 15
    assert L.fmt_server_submit(h, ctypes.byref(r), ctypes.byref(t)) == F.FMT_EINVAL
    res = F.fmt_request_result()
    assert L.fmt_server_wait(h, 12345, 0.0, ctypes.byref(res)) == F.FMT_EINVAL
    assert F.fmt_last_error()
    assert L.fmt_server_destroy(h) == F.FMT_OK


def test_server_clock_is_monotone():
    a = F.Server.clock()
    b = F.Server.clock()
    assert b >= a


def test_resident_calls_reject_unknown_ids():
    L = F.load()
    h = ctypes.c_void_p()
    assert L.fmt_server_create(1, 1e9, 1000, ctypes.byref(h)) == F.FMT_OK
    t = ctypes.c_int64()
    x = np.zeros(3)
    assert L.fmt_server_submit_eval(h, 7, 3, x.ctypes.data, x.ctypes.data, x.ctypes.data, x.ctypes.data,
                                    ctypes.byref(t)) == F.FMT_EINVAL
    assert L.fmt_server_submit_eval(h, 7, -1, None, None, None, None, ctypes.byref(t)) == F.FMT_EINVAL
    assert L.fmt_server_release(h, 7) == F.FMT_EINVAL
    a, p, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    assert L.fmt_server_memory(h, ctypes.byref(a), ctypes.byref(p), ctypes.byref(n)) == F.FMT_OK
    assert a.value == 0.0 and n.value == 0
    r = F.fmt_request()
    r.params = F.make_params(4, 3, 1, 1e-4)
    r.n = 3
    r.x = r.y = r.z = r.f = x.ctypes.data
    r.keep = 2
    assert L.fmt_server_submit(h, ctypes.byref(r), ctypes.byref(t)) == F.FMT_EINVAL
    assert L.fmt_server_destroy(h) == F.FMT_OK
