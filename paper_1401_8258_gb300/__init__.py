"""GB300-native brute-force incoherent dedispersion and n-sigma detection.

The compute path lives in ``libdd.so`` (hand-written CUDA for sm_103a behind
the C ABI of ``include/dd.h``).  This package is the thin Python side:

* :mod:`._native` -- one ctypes function per C entry point (same names);
* :class:`Plan`   -- a small owner of a plan handle that passes torch device
  tensors and streams to those functions (PyTorch supplies memory and
  streams only);
* :func:`median_filter`, :func:`detrend`, :func:`boxcar_detect` -- the
  post-processing of ``include/dd_post.h`` on torch device rows.
"""
from __future__ import annotations

import numpy as np

from . import _native
from ._native import (CANDIDATE_DTYPE, DD_ERR_OVERFLOW, DD_F16, DD_F32, DD_OK, DD_U8, DTYPE_CODES,
                      DDError, dd_compute_delays, dd_detect, dd_execute, dd_get_stats,
                      dd_plan_create, dd_plan_delays, dd_plan_destroy, dd_plan_launch_count,
                      dd_plan_max_delay, dd_plan_nsamp_out, dd_process_host, dd_run,
                      dd_batch_create, dd_batch_destroy, dd_batch_run, dd_status_string, dd_sync)
from ._native import DD_ROWS_F32, DD_ROWS_I32, PULSE_DTYPE
from .build import build

__all__ = [
    "Plan", "build", "DDError", "CANDIDATE_DTYPE", "DD_U8", "DD_F16", "DD_F32", "DD_OK",
    "DD_ERR_OVERFLOW", "DTYPE_CODES", "dd_compute_delays", "dd_plan_create", "dd_plan_destroy",
    "dd_plan_max_delay", "dd_plan_nsamp_out", "dd_plan_delays", "dd_execute", "dd_detect",
    "dd_get_stats", "dd_sync", "dd_process_host", "dd_plan_launch_count", "dd_status_string",
    "dd_run", "Batch", "dd_batch_create", "dd_batch_destroy", "dd_batch_run", "Stream",
    "push_streams", "median_filter", "detrend", "boxcar_detect", "PULSE_DTYPE", "Subband",
    "Binned", "HostPipe",
]

_TORCH_IN = {"u8": "uint8", "f16": "float16", "f32": "float32"}


class Plan:
    """A dedispersion plan on one CUDA device (wraps ``dd_plan``)."""

    def __init__(self, nchan, f_top_mhz, chan_width_mhz, t_samp_s, dms, dtype="u8", device=0):
        self.nchan = int(nchan)
        self.dms = np.ascontiguousarray(dms, dtype=np.float64)
        self.ndm = int(self.dms.size)
        self.dtype = dtype
        self.device = int(device)
        self.handle = dd_plan_create(nchan, f_top_mhz, chan_width_mhz, t_samp_s, self.dms, dtype,
                                     device)
        self.maxshift = dd_plan_max_delay(self.handle)

    @classmethod
    def like(cls, other: "Plan") -> "Plan":
        """A plan of ``other``'s geometry that shares its tables
        (dd_plan_create_like): its own workspaces, no table build."""
        p = cls.__new__(cls)
        p.nchan, p.dms, p.ndm, p.dtype, p.device = (other.nchan, other.dms, other.ndm,
                                                     other.dtype, other.device)
        p.handle = _native.dd_plan_create_like(other.handle)
        p.maxshift = dd_plan_max_delay(p.handle)
        return p

    def close(self) -> None:
        if getattr(self, "handle", None):
            dd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def delays(self) -> np.ndarray:
        return dd_plan_delays(self.handle, self.nchan, self.ndm)

    def nsamp_out(self, nsamp_in: int) -> int:
        return dd_plan_nsamp_out(self.handle, nsamp_in)

    @property
    def out_torch_dtype(self):
        import torch
        return torch.int32 if self.dtype == "u8" else torch.float32

    def execute(self, block, out=None, nsamp_in=None, stream=None):
        """Dedisperse a device tensor ``block[nchan][pitch]`` into ``out``.

        f16 blocks may be passed as ``torch.float16`` tensors.  Returns ``out``
        (allocated on the block's device when not given).
        """
        import torch
        if block.dim() != 2 or block.stride(1) != 1 or block.shape[0] != self.nchan:
            raise ValueError("block must be [nchan][pitch] with unit time stride")
        if str(block.dtype).split(".")[-1] != _TORCH_IN[self.dtype]:
            raise TypeError(f"block dtype {block.dtype} does not match plan dtype {self.dtype}")
        nsamp_in = block.shape[1] if nsamp_in is None else int(nsamp_in)
        n_out = self.nsamp_out(nsamp_in)
        if out is None:
            out = torch.empty((self.ndm, n_out), dtype=self.out_torch_dtype, device=block.device)
        dd_execute(self.handle, block, nsamp_in, block.stride(0), out, stream)
        return out

    def detect(self, out, nsigma, cands=None, capacity=None, stream=None):
        """Threshold ``out``; returns ``(candidates numpy array, total)``."""
        import torch
        n_out = out.shape[1]
        if cands is None:
            capacity = 1 << 16 if capacity is None else int(capacity)
            cands = torch.empty((max(capacity, 1), 16), dtype=torch.uint8, device=out.device)
        else:
            capacity = cands.numel() * cands.element_size() // 16 if capacity is None else capacity
        st, total = dd_detect(self.handle, out, n_out, nsigma, cands if capacity else None,
                              capacity, stream)
        k = min(total, capacity)
        host = cands[:k].cpu().numpy().view(CANDIDATE_DTYPE).reshape(-1) if k else \
            np.zeros(0, dtype=CANDIDATE_DTYPE)
        return host, total

    def run(self, block, nsigma, out=None, nsamp_in=None, capacity=1 << 16, stream=None):
        """Dedisperse and detect in one call (dd_run); returns
        ``(out, candidates numpy array, total)``."""
        import torch
        if block.dim() != 2 or block.stride(1) != 1 or block.shape[0] != self.nchan:
            raise ValueError("block must be [nchan][pitch] with unit time stride")
        if str(block.dtype).split(".")[-1] != _TORCH_IN[self.dtype]:
            raise TypeError(f"block dtype {block.dtype} does not match plan dtype {self.dtype}")
        nsamp_in = block.shape[1] if nsamp_in is None else int(nsamp_in)
        n_out = self.nsamp_out(nsamp_in)
        if out is None:
            out = torch.empty((self.ndm, n_out), dtype=self.out_torch_dtype, device=block.device)
        capacity = int(capacity)
        cands = torch.empty((max(capacity, 1), 16), dtype=torch.uint8, device=block.device)
        st, total = dd_run(self.handle, block, nsamp_in, block.stride(0), out, nsigma,
                           cands if capacity else None, capacity, stream)
        k = min(total, capacity)
        host = cands[:k].cpu().numpy().view(CANDIDATE_DTYPE).reshape(-1) if k else \
            np.zeros(0, dtype=CANDIDATE_DTYPE)
        return out, host, total

    def autotune(self, nsamp_in):
        """Time every staged tile width (and, for u8, staging depth) that fits
        and keep the fastest; returns (DM trials per CTA, ms per launch)."""
        return _native.dd_plan_autotune(self.handle, nsamp_in)

    def stats(self):
        return dd_get_stats(self.handle, self.ndm)

    def launch_count(self) -> int:
        return dd_plan_launch_count(self.handle)


class Batch:
    """Several plans run together (dd_batch_*); keeps the plans alive."""

    def __init__(self, plans):
        self.plans = list(plans)
        self.handle = dd_batch_create([p.handle for p in self.plans])

    def run(self, blocks, nsigma, outs=None, nsamp_in=None, capacity=1 << 16, stream=None):
        """Dedisperse and detect every beam; returns ``(outs, candidate arrays,
        totals)``, one entry per plan."""
        import torch
        n = len(self.plans)
        nsamp_in = [b.shape[1] for b in blocks] if nsamp_in is None else list(nsamp_in)
        if outs is None:
            outs = [torch.empty((p.ndm, p.nsamp_out(ns)), dtype=p.out_torch_dtype,
                                device=b.device) for p, b, ns in zip(self.plans, blocks, nsamp_in)]
        caps = [int(capacity)] * n if np.isscalar(capacity) else [int(c) for c in capacity]
        # candidate buffers persist between runs, so that runs with the same
        # blocks and outs replay the batch's captured graph
        ckey = (tuple(caps), tuple(str(b.device) for b in blocks))
        if getattr(self, "_ckey", None) != ckey:
            self._cands = [torch.empty((max(c, 1), 16), dtype=torch.uint8, device=b.device)
                           for c, b in zip(caps, blocks)]
            self._ckey = ckey
        cands = self._cands
        st, totals = dd_batch_run(self.handle, blocks, nsamp_in, [b.stride(0) for b in blocks],
                                  outs, nsigma, [c if k else None for c, k in zip(cands, caps)],
                                  caps, stream)
        hosts = []
        for c, k, t in zip(cands, caps, totals):
            m = min(t, k)
            hosts.append(c[:m].cpu().numpy().view(CANDIDATE_DTYPE).reshape(-1) if m else
                         np.zeros(0, dtype=CANDIDATE_DTYPE))
        return outs, hosts, totals

    def graph_replays(self):
        """Runs served by the batch's captured CUDA graph."""
        return _native.dd_batch_graph_replays(self.handle)

    def close(self):
        if self.handle:
            dd_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stream:
    """Block-by-block dedispersion of one beam with its overlap tail kept on
    the device (dd_stream_*); keeps its plan alive."""

    def __init__(self, plan, block_samples):
        self.plan = plan
        self.block_samples = int(block_samples)
        self.handle = _native.dd_stream_create(plan.handle, self.block_samples)

    @staticmethod
    def bytes_needed(plan, block_samples) -> int:
        return _native.dd_stream_bytes(plan.handle, block_samples)

    def push(self, block, nsigma, capacity=1 << 16, out=None, stream=None):
        """One block [nchan][>= block_samples]; returns (out, candidates, total)."""
        outs, cands, totals = push_streams([self], [block], nsigma, capacity,
                                           None if out is None else [out], stream)
        return outs[0], cands[0], totals[0]

    def close(self):
        if self.handle:
            _native.dd_stream_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def push_streams(streams, blocks, nsigma, capacity=1 << 16, outs=None, stream=None):
    """One wave: a block for each stream (distinct plans); returns
    ``(outs, candidate arrays, totals)``."""
    import torch
    n = len(streams)
    if outs is None:
        outs = [torch.empty((s.plan.ndm, s.block_samples), dtype=s.plan.out_torch_dtype,
                            device=b.device) for s, b in zip(streams, blocks)]
    caps = [int(capacity)] * n if np.isscalar(capacity) else [int(c) for c in capacity]
    cands = [torch.empty((max(c, 1), 16), dtype=torch.uint8, device=b.device)
             for c, b in zip(caps, blocks)]
    st, totals = _native.dd_streams_push([s.handle for s in streams], blocks,
                                         [b.stride(0) for b in blocks], outs, nsigma,
                                         [c if k else None for c, k in zip(cands, caps)], caps,
                                         stream)
    hosts = []
    for c, k, t in zip(cands, caps, totals):
        m = min(t, k)
        hosts.append(c[:m].cpu().numpy().view(CANDIDATE_DTYPE).reshape(-1) if m else
                     np.zeros(0, dtype=CANDIDATE_DTYPE))
    return outs, hosts, totals


def _rows_type(rows) -> int:
    import torch
    if rows.dim() != 2 or rows.stride(1) != 1:
        raise ValueError("rows must be a 2-D tensor with contiguous rows")
    if rows.dtype == torch.int32:
        return DD_ROWS_I32
    if rows.dtype == torch.float32:
        return DD_ROWS_F32
    raise ValueError("rows must be int32 or float32")


def median_filter(rows, width, out=None, stream=None):
    """Windowed median of each row (dd_median_filter); returns ``out``."""
    import torch
    rt = _rows_type(rows)
    if out is None:
        out = torch.empty(rows.shape, dtype=rows.dtype, device=rows.device)
    _native.dd_median_filter(rows, rows.stride(0), rt, rows.shape[0], rows.shape[1], width, out,
                             out.stride(0), stream)
    return out


def detrend(rows, out=None, coef=False, stream=None):
    """Detrended, normalised float rows (dd_detrend); with ``coef`` also the
    per-row (a, b, s) as a float64 device tensor."""
    import torch
    rt = _rows_type(rows)
    if out is None:
        out = torch.empty(rows.shape, dtype=torch.float32, device=rows.device)
    c = torch.empty((rows.shape[0], 3), dtype=torch.float64, device=rows.device) if coef else None
    _native.dd_detrend(rows, rows.stride(0), rt, rows.shape[0], rows.shape[1], out, out.stride(0),
                       c, stream)
    return (out, c) if coef else out


def boxcar_detect(rows, nwidths, nsigma, mean=None, sigma=None, capacity=1 << 16,
                  workspace=None, stream=None):
    """Boxcar single-pulse search (dd_boxcar_detect).  ``mean`` / ``sigma``:
    float64 device tensors per row or None (0 and 1).  Returns (pulses as a
    PULSE_DTYPE numpy array, total found)."""
    import torch
    rt = _rows_type(rows)
    nrows, ncols = rows.shape
    need = _native.dd_boxcar_workspace_bytes(nrows, ncols)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=rows.device)
    pulses = torch.empty((max(capacity, 1), PULSE_DTYPE.itemsize), dtype=torch.uint8,
                         device=rows.device)
    _, total = _native.dd_boxcar_detect(rows, rows.stride(0), rt, nrows, ncols, mean, sigma,
                                        nwidths, nsigma, workspace, workspace.numel(), pulses,
                                        capacity, stream)
    got = pulses[:min(total, capacity)].cpu().numpy().view(PULSE_DTYPE).reshape(-1)
    return got, total


class Subband:
    """Owner of a dd_subband handle (two-step subband dedispersion,
    include/dd_subband.h) working on torch device tensors."""

    def __init__(self, nchan, f_top_mhz, chan_width_mhz, t_samp_s, dms, dtype,
                 chans_per_subband, dms_per_group, device=0):
        self.nchan, self.ndm, self.dtype = int(nchan), len(dms), dtype
        self.device = device
        self.handle = _native.dd_subband_create(nchan, f_top_mhz, chan_width_mhz, t_samp_s, dms,
                                                dtype, chans_per_subband, dms_per_group, device)
        self.maxshift = _native.dd_subband_max_delay(self.handle)
        self.nominal = _native.dd_subband_nominal(self.handle)

    def nsamp_out(self, nsamp_in):
        return int(nsamp_in) - self.maxshift

    def execute(self, block, nsamp_in=None, out=None, stream=None):
        import torch
        nsamp_in = block.shape[1] if nsamp_in is None else nsamp_in
        n = self.nsamp_out(nsamp_in)
        if out is None:
            dt = torch.int32 if self.dtype == "u8" else torch.float32
            out = torch.empty((self.ndm, n), dtype=dt, device=block.device)
        _native.dd_subband_execute(self.handle, block, nsamp_in, block.stride(0), out, stream)
        return out

    def launch_count(self):
        return _native.dd_subband_launch_count(self.handle)

    def sync(self, stream=None):
        """Wait for this object's work on `stream`; raises DDError if a
        bounded device wait of one of its launches ran out."""
        _native.dd_subband_sync(self.handle, stream)

    def close(self):
        if self.handle:
            _native.dd_subband_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostPipe:
    """Owner of a dd_host_pipe handle: host blocks of one shape through a
    plan, each block's copy overlapped with the previous block's work
    (include/dd.h).  ``push`` returns the previous block's candidates,
    ``flush`` the last block's; both return None when no result is due."""

    def __init__(self, plan, nsamp_in, pitch_elems, nsigma, capacity=1 << 16):
        self.plan, self.capacity = plan, int(capacity)
        self.handle = _native.dd_host_pipe_create(plan.handle, nsamp_in, pitch_elems, nsigma,
                                                  capacity)
        self._cands = np.zeros(max(1, self.capacity), dtype=CANDIDATE_DTYPE)

    def _result(self, st, total, has):
        if not has:
            return None
        return self._cands[:min(total, self.capacity)].copy(), total

    def push(self, host_block, stream=None):
        """host_block: host numpy array or (pinned) torch tensor [nchan][pitch],
        unchanged until the next push or flush returns."""
        return self._result(*_native.dd_host_pipe_push(self.handle, host_block, self._cands,
                                                       stream))

    def flush(self, stream=None):
        return self._result(*_native.dd_host_pipe_flush(self.handle, self._cands, stream))

    def close(self):
        if self.handle:
            _native.dd_host_pipe_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Binned:
    """Owner of a dd_binned handle (time-binned dedispersion past the
    diagonal DM, include/dd_binned.h) working on torch device tensors.
    mode "sum" bins by pair sums (the thesis's downfactoring), "mean8" (u8
    input) by 8-bit pair means rounded half up."""

    def __init__(self, nchan, f_top_mhz, chan_width_mhz, t_samp_s, dms, dtype, max_factor,
                 mode="sum", device=0):
        self.ndm, self.dtype, self.mode = len(dms), dtype, mode
        self.handle = _native.dd_binned_create(nchan, f_top_mhz, chan_width_mhz, t_samp_s, dms,
                                               dtype, max_factor, mode, device)
        self.dm_diag = _native.dd_binned_diagonal_dm(self.handle)

    def rows(self, nsamp_in):
        """(downfactor, output length) per trial for nsamp_in input samples."""
        return _native.dd_binned_rows(self.handle, self.ndm, nsamp_in)

    def execute(self, block, nsamp_in=None, out=None, stream=None):
        import torch
        nsamp_in = block.shape[1] if nsamp_in is None else nsamp_in
        _, lens = self.rows(nsamp_in)
        if out is None:
            dt = torch.int32 if self.dtype == "u8" else torch.float32
            out = torch.zeros((self.ndm, int(lens.max())), dtype=dt, device=block.device)
        _native.dd_binned_execute(self.handle, block, nsamp_in, block.stride(0), out,
                                  out.stride(0), stream)
        return out

    def launch_count(self):
        return _native.dd_binned_launch_count(self.handle)

    def sync(self, stream=None):
        """Wait for this object's work on `stream`; raises DDError if a
        bounded device wait of one of its launches ran out."""
        _native.dd_binned_sync(self.handle, stream)

    def close(self):
        if self.handle:
            _native.dd_binned_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
