"""ctypes binding of ``libdd.so`` (declared in ``include/dd.h``).

One Python function per C entry point, with the same name; each only
marshals arguments (pointers, sizes, stream handles) and turns a negative
status into :class:`DDError`.  No arithmetic of the method happens here: every
step runs in the library's CUDA kernels, and loading fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

DD_U8, DD_F16, DD_F32 = 0, 1, 2
DTYPE_CODES = {"u8": DD_U8, "f16": DD_F16, "f32": DD_F32}

DD_OK = 0
DD_ERR_ARG = -1
DD_ERR_SIZE = -2
DD_ERR_DTYPE = -3
DD_ERR_CUDA = -4
DD_ERR_OOM = -5
DD_ERR_OVERFLOW = -6
DD_ERR_DEVICE_TIMEOUT = -7
DD_ERR_RANGE = -8

CANDIDATE_DTYPE = np.dtype(
    [("dm_idx", np.int32), ("t", np.int32), ("value", np.float32), ("snr", np.float32)]
)

DD_ROWS_I32, DD_ROWS_F32 = 0, 1
PULSE_DTYPE = np.dtype([("dm_idx", np.int32), ("t", np.int32), ("width", np.int32),
                        ("snr", np.float32), ("value", np.float64)])


class DDError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {dd_status_string(status)} ({status})")


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) for every entry point in dd.h
_i32, _i64, _f32, _f64, _vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double,
                               ctypes.c_void_p)
SIGNATURES = [
    ("dd_compute_delays", ctypes.c_int, [_i32, _f64, _f64, _f64, _vp, _i32, _vp, _vp]),
    ("dd_plan_create", ctypes.c_int, [_vp, _i32, _f64, _f64, _f64, _vp, _i32, _i32, _i32]),
    ("dd_plan_destroy", ctypes.c_int, [_vp]),
    ("dd_plan_create_like", ctypes.c_int, [_vp, _vp]),
    ("dd_plan_max_delay", ctypes.c_int, [_vp, _vp]),
    ("dd_plan_nsamp_out", ctypes.c_int, [_vp, _i64, _vp]),
    ("dd_plan_delays", ctypes.c_int, [_vp, _vp]),
    ("dd_execute", ctypes.c_int, [_vp, _vp, _i64, _i64, _vp, _vp]),
    ("dd_detect", ctypes.c_int, [_vp, _vp, _i64, _f32, _vp, _i64, _vp, _vp]),
    ("dd_get_stats", ctypes.c_int, [_vp, _vp, _vp]),
    ("dd_sync", ctypes.c_int, [_vp, _vp]),
    ("dd_process_host", ctypes.c_int, [_vp, _vp, _i64, _i64, _f32, _vp, _i64, _vp, _vp]),
    ("dd_host_pipe_create", ctypes.c_int, [_vp, _vp, _i64, _i64, _f32, _i64]),
    ("dd_host_pipe_destroy", ctypes.c_int, [_vp]),
    ("dd_host_pipe_push", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("dd_host_pipe_flush", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    ("dd_plan_launch_count", ctypes.c_int, [_vp, _vp]),
    ("dd_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("dd_measure_add_peak", ctypes.c_int, [_i32, _i32, _vp, _vp]),
    ("dd_plan_set_path", ctypes.c_int, [_vp, _i32]),
    ("dd_plan_set_staging_depth", ctypes.c_int, [_vp, _i32]),
    ("dd_plan_set_wait_timeout", ctypes.c_int, [_vp, _i64]),
    ("dd_plan_inject_fault", ctypes.c_int, [_vp, _i32]),
    ("dd_plan_kernel_info", ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    ("dd_detect_noalloc", ctypes.c_int, [_vp, _i32, _i32, _i64, _f32, _vp, _i64, _vp, _vp]),
    ("dd_run", ctypes.c_int, [_vp, _vp, _i64, _i64, _vp, _f32, _vp, _i64, _vp, _vp, _vp]),
    ("dd_plan_autotune", ctypes.c_int, [_vp, _i64, _vp, _vp]),
    ("dd_stream_bytes", ctypes.c_int, [_vp, _i64, _vp]),
    ("dd_stream_create", ctypes.c_int, [_vp, _vp, _i64]),
    ("dd_stream_destroy", ctypes.c_int, [_vp]),
    ("dd_streams_push", ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _f32, _vp, _vp, _vp, _vp]),
    ("dd_batch_create", ctypes.c_int, [_vp, _vp, _i32]),
    ("dd_batch_destroy", ctypes.c_int, [_vp]),
    ("dd_batch_run", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _f32, _vp, _vp, _vp, _vp]),
    ("dd_batch_graph_replays", ctypes.c_int, [_vp, _vp]),
    ("dd_plan_create_from_delays", ctypes.c_int, [_vp, _i32, _i32, _vp, _i32, _i32]),
    ("dd_execute_pitched", ctypes.c_int, [_vp, _vp, _i64, _i64, _vp, _i64, _vp]),
    # dd_subband.h
    ("dd_subband_create", ctypes.c_int, [_vp, _i32, _f64, _f64, _f64, _vp, _i32, _i32, _i32, _i32,
                                         _i32]),
    ("dd_subband_destroy", ctypes.c_int, [_vp]),
    ("dd_subband_max_delay", ctypes.c_int, [_vp, _vp]),
    ("dd_subband_nominal", ctypes.c_int, [_vp, _vp, _vp]),
    ("dd_subband_execute", ctypes.c_int, [_vp, _vp, _i64, _i64, _vp, _vp]),
    ("dd_subband_launch_count", ctypes.c_int, [_vp, _vp]),
    ("dd_subband_sync", ctypes.c_int, [_vp, _vp]),
    # dd_binned.h
    ("dd_binned_create", ctypes.c_int,
     [_vp, _i32, _f64, _f64, _f64, _vp, _i32, _i32, _i32, _i32, _i32]),
    ("dd_binned_destroy", ctypes.c_int, [_vp]),
    ("dd_binned_diagonal_dm", ctypes.c_int, [_vp, _vp]),
    ("dd_binned_rows", ctypes.c_int, [_vp, _i64, _vp, _vp]),
    ("dd_binned_execute", ctypes.c_int, [_vp, _vp, _i64, _i64, _vp, _i64, _vp]),
    ("dd_binned_launch_count", ctypes.c_int, [_vp, _vp]),
    ("dd_binned_sync", ctypes.c_int, [_vp, _vp]),
    # dd_post.h
    ("dd_median_filter", ctypes.c_int, [_vp, _i64, _i32, _i32, _i64, _i32, _vp, _i64, _vp]),
    ("dd_detrend", ctypes.c_int, [_vp, _i64, _i32, _i32, _i64, _vp, _i64, _vp, _vp]),
    ("dd_boxcar_workspace_bytes", ctypes.c_int, [_i32, _i64, _vp]),
    ("dd_boxcar_detect", ctypes.c_int, [_vp, _i64, _i32, _i32, _i64, _vp, _vp, _i32, _f32, _vp,
                                        _i64, _vp, _i64, _vp, _vp]),
]

PEAK_KINDS = {"fadd": 0, "fadd2": 1, "iadd": 2, "iadd3": 3, "imad": 4, "lop3": 5, "prmt": 6,
              "hadd2": 7, "fadd_f16": 8, "prmt_iadd": 9, "lop3_iadd": 10}


def library_path() -> str:
    return _build.LIB


def load():
    """Load ``libdd.so``; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libdd.so is not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, what: str, allow=()) -> int:
    if status < 0 and status not in allow:
        raise DDError(status, what)
    return status


def _addr(x) -> int | None:
    """Device or host address of a torch tensor / numpy array / int."""
    try:
        return x.data_ptr()  # torch tensors, the common case first
    except AttributeError:
        pass
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def dd_status_string(status: int) -> str:
    return load().dd_status_string(int(status)).decode()


def dd_compute_delays(nchan, f_top_mhz, chan_width_mhz, t_samp_s, dms):
    dms = np.ascontiguousarray(dms, dtype=np.float64)
    out = np.empty((nchan, dms.size), dtype=np.int32)
    mx = ctypes.c_int32(0)
    _check(load().dd_compute_delays(int(nchan), float(f_top_mhz), float(chan_width_mhz),
                                    float(t_samp_s), dms.ctypes.data, int(dms.size),
                                    out.ctypes.data, ctypes.addressof(mx)), "dd_compute_delays")
    return out, int(mx.value)


def dd_plan_create(nchan, f_top_mhz, chan_width_mhz, t_samp_s, dms, dtype, device=0):
    dms = np.ascontiguousarray(dms, dtype=np.float64)
    code = DTYPE_CODES[dtype] if isinstance(dtype, str) else int(dtype)
    handle = ctypes.c_void_p()
    _check(load().dd_plan_create(ctypes.addressof(handle), int(nchan), float(f_top_mhz),
                                 float(chan_width_mhz), float(t_samp_s), dms.ctypes.data,
                                 int(dms.size), code, int(device)), "dd_plan_create")
    return handle.value


def dd_plan_create_like(src):
    """A plan of src's geometry sharing its tables; returns the handle."""
    handle = ctypes.c_void_p()
    _check(load().dd_plan_create_like(ctypes.addressof(handle), src), "dd_plan_create_like")
    return handle.value


def dd_plan_destroy(plan) -> None:
    _check(load().dd_plan_destroy(plan), "dd_plan_destroy")


def dd_plan_max_delay(plan) -> int:
    v = ctypes.c_int32(0)
    _check(load().dd_plan_max_delay(plan, ctypes.addressof(v)), "dd_plan_max_delay")
    return int(v.value)


def dd_plan_nsamp_out(plan, nsamp_in) -> int:
    v = ctypes.c_int64(0)
    _check(load().dd_plan_nsamp_out(plan, int(nsamp_in), ctypes.addressof(v)), "dd_plan_nsamp_out")
    return int(v.value)


def dd_plan_delays(plan, nchan, ndm) -> np.ndarray:
    out = np.empty((nchan, ndm), dtype=np.int32)
    _check(load().dd_plan_delays(plan, out.ctypes.data), "dd_plan_delays")
    return out


def dd_plan_launch_count(plan) -> int:
    v = ctypes.c_int64(0)
    _check(load().dd_plan_launch_count(plan, ctypes.addressof(v)), "dd_plan_launch_count")
    return int(v.value)


def dd_execute(plan, block, nsamp_in, pitch_elems, out, stream=None) -> None:
    _check(load().dd_execute(plan, _addr(block), int(nsamp_in), int(pitch_elems), _addr(out),
                             _stream(stream)), "dd_execute")


def dd_detect(plan, out, nsamp_out, nsigma, cands, capacity, stream=None) -> tuple[int, int]:
    """Returns ``(status, count)``; status is DD_OK or DD_ERR_OVERFLOW."""
    cnt = ctypes.c_int64(0)
    st = load().dd_detect(plan, _addr(out), int(nsamp_out), float(nsigma), _addr(cands),
                          int(capacity), ctypes.addressof(cnt), _stream(stream))
    _check(st, "dd_detect", allow=(DD_ERR_OVERFLOW,))
    return st, int(cnt.value)


def dd_run(plan, block, nsamp_in, pitch_elems, out, nsigma, cands, capacity, stream=None,
           event=None) -> tuple[int, int]:
    """Dedispersion + detection in one call; returns ``(status, count)``
    (DD_OK or DD_ERR_OVERFLOW).  ``event``: optional CUDA event (torch Event
    or raw handle) recorded after the dedispersion kernel."""
    cnt = ctypes.c_int64(0)
    ev = None if event is None else int(getattr(event, "cuda_event", event))
    st = (_lib or load()).dd_run(plan, _addr(block), int(nsamp_in), int(pitch_elems), _addr(out),
                                 float(nsigma), _addr(cands), int(capacity),
                                 ctypes.addressof(cnt), _stream(stream), ev)
    _check(st, "dd_run", allow=(DD_ERR_OVERFLOW,))
    return st, int(cnt.value)


def dd_plan_autotune(plan, nsamp_in) -> tuple[int, float]:
    """(DM trials per CTA chosen, its median ms per launch)."""
    nd, ms = ctypes.c_int32(0), ctypes.c_float(0)
    _check(load().dd_plan_autotune(plan, int(nsamp_in), ctypes.addressof(nd), ctypes.addressof(ms)),
           "dd_plan_autotune")
    return nd.value, ms.value


def dd_stream_bytes(plan, block_samples) -> int:
    v = ctypes.c_int64(0)
    _check(load().dd_stream_bytes(plan, int(block_samples), ctypes.addressof(v)), "dd_stream_bytes")
    return int(v.value)


def dd_stream_create(plan, block_samples) -> int:
    h = ctypes.c_void_p()
    _check(load().dd_stream_create(ctypes.addressof(h), plan, int(block_samples)),
           "dd_stream_create")
    return h.value


def dd_stream_destroy(stream_handle) -> None:
    _check(load().dd_stream_destroy(stream_handle), "dd_stream_destroy")


def dd_streams_push(streams, blocks, pitch_elems, outs, nsigma, cands, capacity,
                    stream=None) -> tuple[int, list[int]]:
    """One wave: a block per stream handle; returns ``(status, counts)``."""
    n = len(streams)
    vp_arr, i64_arr = ctypes.c_void_p * n, ctypes.c_int64 * n
    st_ = vp_arr(*[int(x) for x in streams])
    b_ = vp_arr(*[_addr(x) for x in blocks])
    o_ = vp_arr(*[_addr(x) for x in outs])
    c_ = vp_arr(*[_addr(x) if x is not None else None for x in cands])
    pe = i64_arr(*[int(x) for x in pitch_elems])
    cap = i64_arr(*[int(x) for x in capacity])
    cnt = i64_arr()
    st = load().dd_streams_push(st_, n, b_, pe, o_, float(nsigma), c_, cap, cnt, _stream(stream))
    _check(st, "dd_streams_push", allow=(DD_ERR_OVERFLOW,))
    return st, [int(x) for x in cnt]


def dd_batch_create(plans) -> int:
    """Handle of a batch over the given plan handles."""
    arr = (ctypes.c_void_p * len(plans))(*[int(p) for p in plans])
    h = ctypes.c_void_p()
    _check(load().dd_batch_create(ctypes.addressof(h), arr, len(plans)), "dd_batch_create")
    return h.value


def dd_batch_destroy(batch) -> None:
    _check(load().dd_batch_destroy(batch), "dd_batch_destroy")


def dd_batch_run(batch, blocks, nsamp_in, pitch_elems, outs, nsigma, cands, capacity,
                 stream=None) -> tuple[int, list[int]]:
    """Per-beam lists; returns ``(status, counts)`` (DD_OK or DD_ERR_OVERFLOW)."""
    n = len(blocks)
    vp_arr = ctypes.c_void_p * n
    i64_arr = ctypes.c_int64 * n
    b_ = vp_arr(*[_addr(x) for x in blocks])
    o_ = vp_arr(*[_addr(x) for x in outs])
    c_ = vp_arr(*[_addr(x) if x is not None else None for x in cands])
    ns = i64_arr(*[int(x) for x in nsamp_in])
    pe = i64_arr(*[int(x) for x in pitch_elems])
    cap = i64_arr(*[int(x) for x in capacity])
    cnt = i64_arr()
    st = load().dd_batch_run(batch, b_, ns, pe, o_, float(nsigma), c_, cap, cnt, _stream(stream))
    _check(st, "dd_batch_run", allow=(DD_ERR_OVERFLOW,))
    return st, [int(x) for x in cnt]


def dd_get_stats(plan, ndm) -> tuple[np.ndarray, np.ndarray]:
    mean = np.empty(ndm, dtype=np.float64)
    sigma = np.empty(ndm, dtype=np.float64)
    _check(load().dd_get_stats(plan, mean.ctypes.data, sigma.ctypes.data), "dd_get_stats")
    return mean, sigma


def dd_sync(plan, stream=None) -> None:
    _check(load().dd_sync(plan, _stream(stream)), "dd_sync")


def dd_process_host(plan, host_block, nsamp_in, pitch_elems, nsigma, host_cands, capacity,
                    stream=None) -> tuple[int, int]:
    cnt = ctypes.c_int64(0)
    st = load().dd_process_host(plan, _addr(host_block), int(nsamp_in), int(pitch_elems),
                                float(nsigma), _addr(host_cands), int(capacity),
                                ctypes.addressof(cnt), _stream(stream))
    _check(st, "dd_process_host", allow=(DD_ERR_OVERFLOW,))
    return st, int(cnt.value)


def dd_host_pipe_create(plan, nsamp_in, pitch_elems, nsigma, capacity) -> int:
    h = ctypes.c_void_p()
    _check(load().dd_host_pipe_create(ctypes.addressof(h), plan, int(nsamp_in), int(pitch_elems),
                                      float(nsigma), int(capacity)), "dd_host_pipe_create")
    return h.value


def dd_host_pipe_destroy(pipe) -> None:
    _check(load().dd_host_pipe_destroy(pipe), "dd_host_pipe_destroy")


def dd_host_pipe_push(pipe, host_block, host_cands, stream=None) -> tuple[int, int, bool]:
    """(status, count, has_result) of the block pushed before this one."""
    cnt, has = ctypes.c_int64(0), ctypes.c_int32(0)
    st = load().dd_host_pipe_push(pipe, _addr(host_block), _addr(host_cands),
                                  ctypes.addressof(cnt), ctypes.addressof(has), _stream(stream))
    _check(st, "dd_host_pipe_push", allow=(DD_ERR_OVERFLOW,))
    return st, int(cnt.value), bool(has.value)


def dd_host_pipe_flush(pipe, host_cands, stream=None) -> tuple[int, int, bool]:
    """(status, count, has_result) of the last pushed block."""
    cnt, has = ctypes.c_int64(0), ctypes.c_int32(0)
    st = load().dd_host_pipe_flush(pipe, _addr(host_cands), ctypes.addressof(cnt),
                                   ctypes.addressof(has), _stream(stream))
    _check(st, "dd_host_pipe_flush", allow=(DD_ERR_OVERFLOW,))
    return st, int(cnt.value), bool(has.value)


def dd_measure_add_peak(kind, device=0) -> tuple[float, float]:
    """(ops/s, ops per clock per SM) of one add-pipe instruction form."""
    code = PEAK_KINDS[kind] if isinstance(kind, str) else int(kind)
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    _check(load().dd_measure_add_peak(code, int(device), ctypes.addressof(a), ctypes.addressof(b)),
           "dd_measure_add_peak")
    return a.value, b.value


def dd_plan_set_path(plan, path) -> None:
    _check(load().dd_plan_set_path(plan, int(path)), "dd_plan_set_path")


def dd_plan_set_wait_timeout(plan, timeout_ns) -> None:
    _check(load().dd_plan_set_wait_timeout(plan, int(timeout_ns)), "dd_plan_set_wait_timeout")


def dd_plan_inject_fault(plan, skip_copies) -> None:
    _check(load().dd_plan_inject_fault(plan, int(skip_copies)), "dd_plan_inject_fault")


def dd_plan_set_staging_depth(plan, copy_ahead) -> None:
    _check(load().dd_plan_set_staging_depth(plan, int(copy_ahead)), "dd_plan_set_staging_depth")


def dd_plan_kernel_info(plan, block, pitch_elems) -> dict:
    st, nd, sm, ca = (ctypes.c_int32(0) for _ in range(4))
    _check(load().dd_plan_kernel_info(plan, _addr(block), int(pitch_elems), ctypes.addressof(st),
                                      ctypes.addressof(nd), ctypes.addressof(sm),
                                      ctypes.addressof(ca)),
           "dd_plan_kernel_info")
    return {"staged": bool(st.value), "dms_per_cta": nd.value, "smem_bytes": sm.value,
            "copy_ahead": ca.value}


def dd_detect_noalloc(out, dtype, ndm, nsamp_out, nsigma, cands, capacity, stream=None):
    """Returns ``(status, count)``; status is DD_OK or DD_ERR_OVERFLOW."""
    code = DTYPE_CODES[dtype] if isinstance(dtype, str) else int(dtype)
    cnt = ctypes.c_int64(0)
    st = load().dd_detect_noalloc(_addr(out), code, int(ndm), int(nsamp_out), float(nsigma),
                                  _addr(cands), int(capacity), ctypes.addressof(cnt),
                                  _stream(stream))
    _check(st, "dd_detect_noalloc", allow=(DD_ERR_OVERFLOW,))
    return st, int(cnt.value)


def dd_median_filter(rows, in_pitch, rows_type, nrows, ncols, width, out, out_pitch, stream=None):
    _check(load().dd_median_filter(_addr(rows), int(in_pitch), int(rows_type), int(nrows),
                                   int(ncols), int(width), _addr(out), int(out_pitch),
                                   _stream(stream)), "dd_median_filter")


def dd_detrend(rows, in_pitch, rows_type, nrows, ncols, out, out_pitch, coef=None, stream=None):
    _check(load().dd_detrend(_addr(rows), int(in_pitch), int(rows_type), int(nrows), int(ncols),
                             _addr(out), int(out_pitch), _addr(coef), _stream(stream)),
           "dd_detrend")


def dd_boxcar_workspace_bytes(nrows, ncols) -> int:
    b = ctypes.c_int64(0)
    _check(load().dd_boxcar_workspace_bytes(int(nrows), int(ncols), ctypes.addressof(b)),
           "dd_boxcar_workspace_bytes")
    return int(b.value)


def dd_boxcar_detect(rows, pitch, rows_type, nrows, ncols, mean, sigma, nwidths, nsigma,
                     workspace, workspace_bytes, pulses, capacity, stream=None):
    """Returns ``(status, count)``; status is DD_OK or DD_ERR_OVERFLOW."""
    cnt = ctypes.c_int64(0)
    st = load().dd_boxcar_detect(_addr(rows), int(pitch), int(rows_type), int(nrows), int(ncols),
                                 _addr(mean), _addr(sigma), int(nwidths), float(nsigma),
                                 _addr(workspace), int(workspace_bytes), _addr(pulses),
                                 int(capacity), ctypes.addressof(cnt), _stream(stream))
    _check(st, "dd_boxcar_detect", allow=(DD_ERR_OVERFLOW,))
    return st, int(cnt.value)


def dd_plan_create_from_delays(delays, dtype, device=0) -> int:
    code = DTYPE_CODES[dtype] if isinstance(dtype, str) else int(dtype)
    d = np.ascontiguousarray(delays, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(load().dd_plan_create_from_delays(ctypes.addressof(h), int(d.shape[0]),
                                             int(d.shape[1]), d.ctypes.data, code, int(device)),
           "dd_plan_create_from_delays")
    return h.value


def dd_execute_pitched(plan, block, nsamp_in, pitch_elems, out, out_pitch, stream=None) -> None:
    _check(load().dd_execute_pitched(plan, _addr(block), int(nsamp_in), int(pitch_elems),
                                     _addr(out), int(out_pitch), _stream(stream)),
           "dd_execute_pitched")


def dd_subband_create(nchan, f_top_mhz, chan_width_mhz, t_samp_s, dms, dtype, chans_per_subband,
                      dms_per_group, device=0) -> int:
    code = DTYPE_CODES[dtype] if isinstance(dtype, str) else int(dtype)
    dms = np.ascontiguousarray(dms, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(load().dd_subband_create(ctypes.addressof(h), int(nchan), float(f_top_mhz),
                                    float(chan_width_mhz), float(t_samp_s), dms.ctypes.data,
                                    int(dms.size), code, int(chans_per_subband),
                                    int(dms_per_group), int(device)), "dd_subband_create")
    return h.value


def dd_subband_destroy(sub) -> None:
    _check(load().dd_subband_destroy(sub), "dd_subband_destroy")


def dd_subband_max_delay(sub) -> int:
    m = ctypes.c_int32(0)
    _check(load().dd_subband_max_delay(sub, ctypes.addressof(m)), "dd_subband_max_delay")
    return int(m.value)


def dd_subband_nominal(sub) -> np.ndarray:
    n = ctypes.c_int32(0)
    _check(load().dd_subband_nominal(sub, None, ctypes.addressof(n)), "dd_subband_nominal")
    nom = np.zeros(n.value, dtype=np.int32)
    _check(load().dd_subband_nominal(sub, nom.ctypes.data, None), "dd_subband_nominal")
    return nom


def dd_subband_execute(sub, block, nsamp_in, pitch_elems, out, stream=None) -> None:
    _check(load().dd_subband_execute(sub, _addr(block), int(nsamp_in), int(pitch_elems),
                                     _addr(out), _stream(stream)), "dd_subband_execute")


def dd_subband_sync(sub, stream=None) -> None:
    _check(load().dd_subband_sync(sub, _stream(stream)), "dd_subband_sync")


def dd_binned_sync(b, stream=None) -> None:
    _check(load().dd_binned_sync(b, _stream(stream)), "dd_binned_sync")


def dd_subband_launch_count(sub) -> int:
    n = ctypes.c_int64(0)
    _check(load().dd_subband_launch_count(sub, ctypes.addressof(n)), "dd_subband_launch_count")
    return int(n.value)


BIN_MODES = {"sum": 0, "mean8": 1}  # dd_bin_mode


def dd_binned_create(nchan, f_top_mhz, chan_width_mhz, t_samp_s, dms, dtype, max_factor,
                     mode="sum", device=0) -> int:
    code = DTYPE_CODES[dtype] if isinstance(dtype, str) else int(dtype)
    mcode = BIN_MODES[mode] if isinstance(mode, str) else int(mode)
    dms = np.ascontiguousarray(dms, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(load().dd_binned_create(ctypes.addressof(h), int(nchan), float(f_top_mhz),
                                   float(chan_width_mhz), float(t_samp_s), dms.ctypes.data,
                                   int(dms.size), code, int(max_factor), mcode, int(device)),
           "dd_binned_create")
    return h.value


def dd_binned_destroy(b) -> None:
    _check(load().dd_binned_destroy(b), "dd_binned_destroy")


def dd_binned_diagonal_dm(b) -> float:
    v = ctypes.c_double(0)
    _check(load().dd_binned_diagonal_dm(b, ctypes.addressof(v)), "dd_binned_diagonal_dm")
    return float(v.value)


def dd_binned_rows(b, ndm, nsamp_in) -> tuple[np.ndarray, np.ndarray]:
    fac = np.zeros(ndm, dtype=np.int32)
    n = np.zeros(ndm, dtype=np.int64)
    _check(load().dd_binned_rows(b, int(nsamp_in), fac.ctypes.data, n.ctypes.data),
           "dd_binned_rows")
    return fac, n


def dd_binned_execute(b, block, nsamp_in, pitch_elems, out, out_pitch, stream=None) -> None:
    _check(load().dd_binned_execute(b, _addr(block), int(nsamp_in), int(pitch_elems), _addr(out),
                                    int(out_pitch), _stream(stream)), "dd_binned_execute")


def dd_binned_launch_count(b) -> int:
    n = ctypes.c_int64(0)
    _check(load().dd_binned_launch_count(b, ctypes.addressof(n)), "dd_binned_launch_count")
    return int(n.value)


def dd_batch_graph_replays(batch) -> int:
    n = ctypes.c_int64(0)
    _check(load().dd_batch_graph_replays(batch, ctypes.addressof(n)), "dd_batch_graph_replays")
    return int(n.value)
