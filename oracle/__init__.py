"""CPU oracle for brute-force dedispersion and n-sigma detection.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The CUDA library in
``paper_1401_8258_gb300`` neither imports nor links it, and this package takes
nothing from the library: the arithmetic lives in ``dd_oracle.c`` (plain C,
compiled with ``-ffp-contract=off``), written from the thesis:

* ``delay_table``   -- Sec. 2.1.1, the discretised-delay (deltaT) equation,
                       with the dispersion constant of Sec. 1.2.1;
* ``dedisperse``    -- Sec. 2.1.1, the brute-force dedispersion equation,
                       valid length nsamp - maxshift per Sec. 3.4;
* ``stats``         -- Sec. 3.5, per-DM normalisation (mean, population rms);
* ``detect``        -- Sec. 3.6, n-sigma thresholding into (DM, time,
                       intensity) triplets.

Each function is pinned by ``tests/test_oracle_pins.py`` to facts that do not
come from the oracle itself (exact rational delays, library sums, impulse
responses, injected pulses, closed forms printed in the thesis).

``oracle.post`` (numpy) holds the post-processing of the dedispersed series
(Sec. 3.5 median filtering, detrending and normalisation; Sec. 1.5.1 boxcar
smoothing and single-pulse thresholding), pinned by
``tests/test_oracle_post_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

U8, F16, F32 = 0, 1, 2
_DTYPE_CODE = {np.dtype(np.uint8): U8, np.dtype(np.float16): F16, np.dtype(np.float32): F32}

CANDIDATE_DTYPE = np.dtype(
    [("dm_idx", np.int32), ("t", np.int32), ("value", np.float32), ("snr", np.float32)]
)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``dd_oracle.c`` into ``_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _bind(lib):
    """Declare argument and return types on a loaded oracle library."""
    i32, i64, f32, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
    vp = ctypes.c_void_p
    lib.oracle_delay_table.argtypes = [i32, f64, f64, f64, vp, i32, vp, vp]
    lib.oracle_dedisperse.argtypes = [i32, vp, i32, i64, i64, vp, i32, i64, vp, i32]
    lib.oracle_stats_i32.argtypes = [vp, i32, i64, vp, vp]
    lib.oracle_stats_f64.argtypes = [vp, i32, i64, vp, vp]
    lib.oracle_detect_i32.argtypes = [vp, i32, i64, vp, vp, f32, vp, i64, vp]
    lib.oracle_detect_f64.argtypes = [vp, i32, i64, vp, vp, f32, vp, i64, vp]
    for fn in ("oracle_delay_table", "oracle_dedisperse", "oracle_stats_i32",
               "oracle_stats_f64", "oracle_detect_i32", "oracle_detect_f64",
               "oracle_max_threads"):
        getattr(lib, fn).restype = i32
    return lib


def _use_library(path: str | None):
    """Point this module at another build of ``dd_oracle.c`` (``None``
    restores the default).  Used by the tests that plant mistakes in a copy
    of the oracle to show that the pins catch them."""
    global _lib
    with _lock:
        _lib = None if path is None else _bind(ctypes.CDLL(path))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _check(status: int, what: str) -> None:
    if status != 0:
        raise RuntimeError(f"oracle {what} failed with status {status}")


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def delay_table(nchan: int, f_top_mhz: float, chan_width_mhz: float, t_samp_s: float,
                dms) -> tuple[np.ndarray, int]:
    """Integer delays ``[nchan][ndm]`` (int32) and their maximum (Sec. 2.1.1)."""
    dms = np.ascontiguousarray(dms, dtype=np.float64)
    out = np.empty((nchan, dms.size), dtype=np.int32)
    mx = np.zeros(1, dtype=np.int32)
    st = _load().oracle_delay_table(int(nchan), float(f_top_mhz), float(chan_width_mhz),
                                    float(t_samp_s), _ptr(dms), int(dms.size), _ptr(out), _ptr(mx))
    _check(st, "delay_table")
    return out, int(mx[0])


def dedisperse(block: np.ndarray, delays: np.ndarray, nsamp_out: int | None = None,
               nsamp_in: int | None = None, nthreads: int = 0) -> np.ndarray:
    """Brute-force dedispersion of ``block[nchan][pitch]`` (Sec. 2.1.1).

    Returns int32 ``[ndm][nsamp_out]`` for uint8 input, float64 otherwise.
    ``nsamp_in`` defaults to the row length; ``nsamp_out`` to
    ``nsamp_in - max(delays)``.
    """
    if block.ndim != 2 or block.strides[1] != block.itemsize:
        raise ValueError("block must be 2-D with unit time stride")
    code = _DTYPE_CODE[block.dtype]
    nchan = block.shape[0]
    pitch = block.strides[0] // block.itemsize
    if nsamp_in is None:
        nsamp_in = block.shape[1]
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    if delays.shape[0] != nchan:
        raise ValueError("delays must be [nchan][ndm]")
    ndm = delays.shape[1]
    if nsamp_out is None:
        nsamp_out = nsamp_in - int(delays.max())
    out = np.empty((ndm, nsamp_out), dtype=np.int32 if code == U8 else np.float64)
    view = block.view(np.uint16) if code == F16 else block
    st = _load().oracle_dedisperse(code, _ptr(view), nchan, int(nsamp_in), int(pitch),
                                   _ptr(delays), ndm, int(nsamp_out), _ptr(out), int(nthreads))
    _check(st, "dedisperse")
    return out


def stats(D: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Per-row mean and population standard deviation (Sec. 3.5).

    int32 rows use exact integer sums and the written double finaliser;
    float64 rows use a two-pass double computation.
    """
    ndm, n = D.shape
    mean = np.empty(ndm, dtype=np.float64)
    sigma = np.empty(ndm, dtype=np.float64)
    if D.dtype == np.int32:
        D = np.ascontiguousarray(D)
        st = _load().oracle_stats_i32(_ptr(D), ndm, n, _ptr(mean), _ptr(sigma))
    else:
        D = np.ascontiguousarray(D, dtype=np.float64)
        st = _load().oracle_stats_f64(_ptr(D), ndm, n, _ptr(mean), _ptr(sigma))
    _check(st, "stats")
    return mean, sigma


def detect(D: np.ndarray, mean: np.ndarray, sigma: np.ndarray, nsigma: float,
           capacity: int | None = None) -> tuple[np.ndarray, int]:
    """n-sigma candidates of ``D`` in (dm_idx, t) order (Sec. 3.6).

    Returns ``(candidates[:min(total, capacity)], total)``.
    """
    ndm, n = D.shape
    mean = np.ascontiguousarray(mean, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    lib = _load()
    total = np.zeros(1, dtype=np.int64)
    is_int = D.dtype == np.int32
    if is_int:
        D = np.ascontiguousarray(D)
        fn = lib.oracle_detect_i32
    else:
        D = np.ascontiguousarray(D, dtype=np.float64)
        fn = lib.oracle_detect_f64
    if capacity is None:
        st = fn(_ptr(D), ndm, n, _ptr(mean), _ptr(sigma), float(nsigma), None, 0, _ptr(total))
        _check(st, "detect")
        capacity = int(total[0])
    cands = np.zeros(max(capacity, 1), dtype=CANDIDATE_DTYPE)
    st = fn(_ptr(D), ndm, n, _ptr(mean), _ptr(sigma), float(nsigma), _ptr(cands),
            int(capacity), _ptr(total))
    _check(st, "detect")
    tot = int(total[0])
    return cands[:min(tot, capacity)].copy(), tot
