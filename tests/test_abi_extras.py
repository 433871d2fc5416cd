"""CPU checks of the host-side logic of dd_post.h, dd_subband.h and
dd_binned.h: argument errors are reported before any device work (so they
need no GPU), and the boxcar workspace size follows its layout."""
import ctypes

import numpy as np
import pytest

import paper_1401_8258_gb300 as dd
from paper_1401_8258_gb300 import _native

DD_ERR_ARG, DD_ERR_SIZE, DD_ERR_DTYPE, DD_ERR_RANGE = -1, -2, -3, -8


@pytest.fixture(scope="module")
def lib():
    dd.build()
    return _native.load()


FAKE = ctypes.c_void_p(0x1000)  # never dereferenced: every call below fails validation first


def test_median_filter_argument_errors(lib):
    f = lib.dd_median_filter
    assert f(FAKE, 100, 7, 2, 100, 5, ctypes.c_void_p(0x100000), 100, None) == DD_ERR_DTYPE
    assert f(None, 100, 0, 2, 100, 5, FAKE, 100, None) == DD_ERR_ARG
    for width in (0, 2, 16, 17):
        assert f(FAKE, 100, 0, 2, 100, width, ctypes.c_void_p(0x100000), 100, None) == DD_ERR_ARG
    assert f(FAKE, 100, 0, 0, 100, 5, ctypes.c_void_p(0x100000), 100, None) == DD_ERR_SIZE
    assert f(FAKE, 99, 0, 2, 100, 5, ctypes.c_void_p(0x100000), 100, None) == DD_ERR_ARG
    # overlapping input and output
    assert f(FAKE, 100, 0, 2, 100, 5, ctypes.c_void_p(0x1000 + 40), 100, None) == DD_ERR_ARG


def test_detrend_argument_errors(lib):
    f = lib.dd_detrend
    out = ctypes.c_void_p(0x100000)
    assert f(FAKE, 100, 5, 2, 100, out, 100, None, None) == DD_ERR_DTYPE
    assert f(FAKE, 100, 0, 2, (1 << 24) + 1, out, 100, None, None) == DD_ERR_SIZE
    assert f(FAKE, 100, 0, 2, 0, out, 100, None, None) == DD_ERR_SIZE
    assert f(FAKE, 100, 0, 2, 100, FAKE, 100, None, None) == DD_ERR_ARG  # int rows in place
    assert f(ctypes.c_void_p(0x1002), 100, 1, 2, 100, out, 100, None, None) == DD_ERR_ARG


def test_boxcar_workspace_and_argument_errors(lib):
    b = ctypes.c_int64(0)
    assert lib.dd_boxcar_workspace_bytes(3, 10000, ctypes.addressof(b)) == 0
    tiles = (10000 + 4095) // 4096
    assert b.value == 8 * (3 * 12 + 2 * 3 * tiles + 2)
    assert lib.dd_boxcar_workspace_bytes(0, 10, ctypes.addressof(b)) == DD_ERR_SIZE
    need = _native.dd_boxcar_workspace_bytes(2, 100)
    cnt = ctypes.c_int64(0)
    f = lib.dd_boxcar_detect
    ws = ctypes.c_void_p(0x200000)
    args = lambda **k: [k.get("rows", FAKE), 100, k.get("rt", 1), 2, 100, None, None,
                        k.get("nw", 4), k.get("ns", 3.0), k.get("ws", ws),
                        k.get("wsb", need), ctypes.c_void_p(0x300000), 4,
                        ctypes.addressof(cnt), None]
    assert f(*args(rt=9)) == DD_ERR_DTYPE
    assert f(*args(nw=0)) == DD_ERR_ARG and f(*args(nw=13)) == DD_ERR_ARG
    assert f(*args(ns=float("inf"))) == DD_ERR_ARG
    assert f(*args(wsb=need - 8)) == DD_ERR_ARG
    assert f(*args(ws=ctypes.c_void_p(0x200008))) == DD_ERR_ARG  # workspace not 16-byte aligned


def test_subband_and_binned_creation_errors(lib):
    dms = np.arange(16, dtype=np.float64)
    h = ctypes.c_void_p()
    sc = lib.dd_subband_create
    assert sc(ctypes.addressof(h), 64, 416.0, 0.25, 1e-4, dms.ctypes.data, 16, 0, 0, 4, 0) == DD_ERR_ARG
    assert sc(ctypes.addressof(h), 64, 416.0, 0.25, 1e-4, dms.ctypes.data, 16, 0, 8, 0, 0) == DD_ERR_ARG
    assert sc(ctypes.addressof(h), 64, 416.0, 0.25, 1e-4, dms.ctypes.data, 16, 9, 8, 4, 0) == DD_ERR_DTYPE
    assert sc(ctypes.addressof(h), 70000, 1500.0, 0.001, 64e-6, dms.ctypes.data, 16, 0, 64, 4,
              0) == DD_ERR_RANGE
    bc = lib.dd_binned_create
    rev = dms[::-1].copy()
    assert bc(ctypes.addressof(h), 64, 416.0, 0.25, 1e-4, rev.ctypes.data, 16, 0, 4, 0,
              0) == DD_ERR_ARG
    for mf in (0, 3, 6, 128):
        assert bc(ctypes.addressof(h), 64, 416.0, 0.25, 1e-4, dms.ctypes.data, 16, 0, mf, 0,
                  0) == DD_ERR_ARG
    assert bc(ctypes.addressof(h), 4096, 1500.0, 0.07, 64e-6, dms.ctypes.data, 16, 0, 64, 0,
              0) == DD_ERR_RANGE
    for mode in (-1, 2):  # no such binning mode
        assert bc(ctypes.addressof(h), 64, 416.0, 0.25, 1e-4, dms.ctypes.data, 16, 0, 4, mode,
                  0) == DD_ERR_ARG
    for dtype in (1, 2):  # 8-bit means need u8 input
        assert bc(ctypes.addressof(h), 64, 416.0, 0.25, 1e-4, dms.ctypes.data, 16, dtype, 4, 1,
                  0) == DD_ERR_DTYPE
    assert h.value is None  # nothing was created


def test_plan_from_delays_rejects_bad_tables(lib):
    h = ctypes.c_void_p()
    bad = np.array([[0, 1], [-1, 2]], dtype=np.int32)
    assert lib.dd_plan_create_from_delays(ctypes.addressof(h), 2, 2, bad.ctypes.data, 0, 0) == DD_ERR_ARG
    big = np.array([[0, 1 << 30], [1, (1 << 30) + 1]], dtype=np.int32)
    assert lib.dd_plan_create_from_delays(ctypes.addressof(h), 2, 2, big.ctypes.data, 0, 0) == DD_ERR_ARG
    assert lib.dd_plan_create_from_delays(ctypes.addressof(h), 2, 2, None, 0, 0) == DD_ERR_ARG
    assert lib.dd_plan_create_from_delays(ctypes.addressof(h), 2, 2, bad.ctypes.data, 7, 0) == DD_ERR_DTYPE


def test_host_pipe_argument_errors(lib):
    """dd_host_pipe_*: null handles and outputs are refused before any device
    work; destroying a null pipe is a no-op."""
    h = ctypes.c_void_p()
    cnt, has = ctypes.c_int64(0), ctypes.c_int32(0)
    assert lib.dd_host_pipe_create(None, FAKE, 100, 100, ctypes.c_float(5.0), 10) == DD_ERR_ARG
    assert lib.dd_host_pipe_create(ctypes.addressof(h), None, 100, 100, ctypes.c_float(5.0),
                                   10) == DD_ERR_ARG
    assert h.value is None
    assert lib.dd_host_pipe_push(None, FAKE, FAKE, ctypes.addressof(cnt), ctypes.addressof(has),
                                 None) == DD_ERR_ARG
    assert lib.dd_host_pipe_flush(None, FAKE, ctypes.addressof(cnt), ctypes.addressof(has),
                                  None) == DD_ERR_ARG
    assert lib.dd_host_pipe_destroy(None) == 0


def test_subband_and_binned_sync_reject_null(lib):
    assert lib.dd_subband_sync(None, None) == DD_ERR_ARG
    assert lib.dd_binned_sync(None, None) == DD_ERR_ARG


def fused_sums_fit(nchan, nsamp_out) -> bool:
    """The library's decision (ddi_fused_sums_fit, a host-only test hook) of
    whether dd_run's fused path may total a row's sum of squares in 64 bits."""
    f = _native.load().ddi_fused_sums_fit
    f.argtypes = [ctypes.c_int32, ctypes.c_int64]
    return bool(f(nchan, nsamp_out))


@pytest.mark.parametrize("nchan", [1, 64, 1024, 4096, 16384, 1 << 20])
def test_fused_sum_limit_is_exact(lib, nchan):
    """The fused path is taken exactly while (255 nchan)^2 nsamp_out < 2^64,
    the range of its 64-bit sum of squares; the largest such nsamp_out is
    (2^64 - 1) // (255 nchan)^2, computed here in Python's exact integers."""
    m2 = (255 * nchan) ** 2
    last = (2 ** 64 - 1) // m2
    for n in (1, 1000, last - 1, last):
        if 1 <= n <= min(last, 2 ** 62):
            assert fused_sums_fit(nchan, n), (nchan, n)
    if last + 1 <= 2 ** 62:
        assert not fused_sums_fit(nchan, last + 1)
    assert not fused_sums_fit(nchan, 0)
    # 16384 channels: the limit lies near 1.06 M outputs, within a block that
    # fits GB300 memory
    if nchan == 16384:
        assert last == 1056816
