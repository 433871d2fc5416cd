"""Continuous-batching server for streams of filterbank blocks.

The thesis's back-end processes several beams per GPU in real time: each
beam's samples arrive block by block, each block is dedispersed together with
the previous block's last maxshift samples (Sec. 3.4), input buffers are
double-buffered so that the next block's transfer overlaps the current
block's processing (Sec. 4.2), and the detection output of every beam goes
on to the post-processing stages (Sec. 3.8).  ``Server`` runs that loop on
one GPU over the library's C ABI:

* **Admission by memory.**  A beam is opened with its plan and block length
  and waits in arrival order until its device memory -- the stream's own
  buffers and workspace (``dd_stream_bytes``), two input staging slots and a
  candidate buffer -- fits the server's budget (a fraction of the device's
  free memory at start-up).  A beam that ends (``close_beam``) releases its
  memory once its last block is processed, which admits the beams waiting.
* **Host arrivals, copies on a copy stream.**  ``submit`` (from any host
  thread) queues a block; as soon as one of the beam's two staging slots is
  free its host-to-device copy is queued on the copy stream, so blocks that
  arrive while a wave runs are copied during it.
* **Continuous batching.**  The server thread repeatedly takes every admitted
  beam whose next block has been copied and runs them as one wave
  (``dd_streams_push``: the 8-bit beams of the wave share persistent
  launches), on the compute stream after the wave's copies; beams that arrive
  or are admitted while a wave runs join the next one.  ``per_beam=True``
  runs the same beams one push per beam instead (the plain per-beam form).
* **Latency.**  Each block's result records its arrival time (given by the
  caller, or the time of ``submit``) and the wall-clock time its candidates
  were on the host.

Every step of the method runs in the library's kernels; this module only
schedules, copies and keeps the books.
"""
from __future__ import annotations

import collections
import threading
import time

import numpy as np

from . import _native
from ._native import CANDIDATE_DTYPE

_ELEM = {"u8": 1, "f16": 2, "f32": 4}

BlockResult = collections.namedtuple(
    "BlockResult", "seq candidates total arrival done latency wave_size out")


class _Beam:
    def __init__(self, key, plan, block_samples, capacity, nbytes):
        self.key = key
        self.plan = plan
        self.block = int(block_samples)
        self.capacity = int(capacity)
        self.nbytes = int(nbytes)
        self.queue = collections.deque()   # (seq, arrival, host block), oldest first
        self.submitted = 0                 # blocks queued so far
        self.copied = 0                    # blocks whose copy has been queued
        self.done = 0                      # blocks processed
        self.closing = False
        self.admitted = False
        self.released = False
        self.stream = None
        self.slots = None                  # two device staging blocks [nchan][block]
        self.events = [None, None]         # copy-done event of each slot
        self.out = None
        self.cands = None
        self.opened = time.perf_counter()
        self.admit_time = None


class Server:
    """See the module docstring.  Beams are identified by any hashable key;
    one plan per beam (plans of one geometry may share tables: ``Plan.like``)."""

    def __init__(self, nsigma, capacity=1 << 16, device=0, mem_budget=None, mem_fraction=0.8,
                 per_beam=False, keep_outputs=False):
        import torch
        self._torch = torch
        self.nsigma = float(nsigma)
        self.capacity = int(capacity)
        self.device = torch.device("cuda", int(device))
        self.per_beam = bool(per_beam)
        self.keep_outputs = bool(keep_outputs)
        self.compute = torch.cuda.Stream(self.device)
        self.copy = torch.cuda.Stream(self.device)
        free, _ = torch.cuda.mem_get_info(self.device)
        self.budget = int(mem_budget) if mem_budget is not None else int(mem_fraction * free)
        self.used = 0
        self.peak_used = 0
        self._cv = threading.Condition()
        self._beams = {}                          # key -> _Beam, until released
        self._pending = collections.deque()       # opened, awaiting admission
        self._active = []                         # admitted, in admission order
        self.results = collections.defaultdict(list)
        self.waves = []                           # (beams, start, end) wall-clock
        self.admissions = []                      # (key, opened, admitted)
        self._stop = False
        self._abort = False
        self._error = None
        self._thread = threading.Thread(target=self._run, name="dd-server", daemon=True)
        self._thread.start()

    # ------------------------------------------------------------ client side

    def beam_bytes(self, plan, block_samples) -> int:
        """Device bytes a beam of this plan and block length holds while
        admitted: its stream, two staging slots, a candidate buffer."""
        return (_native.dd_stream_bytes(plan.handle, int(block_samples)) +
                2 * plan.nchan * int(block_samples) * _ELEM[plan.dtype] + 16 * self.capacity)

    def open(self, key, plan, block_samples):
        """Register a beam; it is admitted when its memory fits the budget."""
        nbytes = self.beam_bytes(plan, block_samples)
        if nbytes > self.budget:
            raise ValueError(f"beam {key!r} needs {nbytes} bytes, over the budget {self.budget}")
        with self._cv:
            self._raise_error()
            if key in self._beams:
                raise KeyError(f"beam {key!r} is open")
            b = _Beam(key, plan, block_samples, self.capacity, nbytes)
            self._beams[key] = b
            self._pending.append(b)
            self._cv.notify_all()

    def submit(self, key, host_block, arrival=None):
        """Queue one block of beam ``key``: a host tensor or array [nchan][>=
        block] (pinned memory gives asynchronous copies).  ``arrival``: its
        arrival time on the ``time.perf_counter`` clock (default: now)."""
        torch = self._torch
        blk = host_block if isinstance(host_block, torch.Tensor) else torch.from_numpy(
            np.ascontiguousarray(host_block))
        with self._cv:
            self._raise_error()
            b = self._beams[key]
            if b.closing:
                raise ValueError(f"beam {key!r} is closed")
            if blk.shape[0] != b.plan.nchan or blk.shape[1] < b.block or blk.stride(1) != 1:
                raise ValueError("block must be [nchan][>= block_samples] with unit time stride")
            b.queue.append((b.submitted, time.perf_counter() if arrival is None else arrival, blk))
            b.submitted += 1
            if b.admitted:
                self._issue_copies(b)
            self._cv.notify_all()

    def close_beam(self, key):
        """No more blocks for ``key``: it is released after its last block."""
        with self._cv:
            self._beams[key].closing = True
            self._cv.notify_all()

    def drain(self, timeout=None):
        """Wait until every beam opened so far is closed, processed and
        released; raises what the server thread raised."""
        end = None if timeout is None else time.perf_counter() + timeout
        with self._cv:
            while self._beams and self._error is None:
                if not all(b.closing for b in self._beams.values()):
                    raise RuntimeError("drain() needs every beam closed (close_beam)")
                left = None if end is None else end - time.perf_counter()
                if left is not None and left <= 0:
                    raise TimeoutError("server did not drain")
                self._cv.wait(left)
            self._raise_error()

    def shutdown(self):
        """Stop once nothing copied is left to run; release the streams."""
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        self._thread.join()
        self._raise_error()

    def abort(self):
        """Stop after the push in flight, dropping queued blocks (an
        overloaded run); release the streams."""
        with self._cv:
            self._stop = self._abort = True
            self._cv.notify_all()
        self._thread.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.shutdown()

    def _raise_error(self):
        if self._error is not None:
            raise RuntimeError("server thread failed") from self._error

    # ------------------------------------------------------------ server side

    def _issue_copies(self, b):
        """Queue host-to-device copies of b's next blocks into its free
        slots (block n uses slot n % 2, free once block n - 2 is done).
        Called with the lock held."""
        torch = self._torch
        while b.copied < b.submitted and b.copied - b.done < 2:
            seq = b.copied
            _, _, blk = b.queue[seq - b.done]
            slot = b.slots[seq % 2]
            with torch.cuda.stream(self.copy):
                slot.copy_(blk[:, :b.block], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.copy)
            b.events[seq % 2] = ev
            b.copied += 1

    def _admit(self):
        """Admit waiting beams in arrival order while they fit.  Lock held."""
        torch = self._torch
        while self._pending and self.used + self._pending[0].nbytes <= self.budget:
            b = self._pending.popleft()
            p = b.plan
            b.stream = _native.dd_stream_create(p.handle, b.block)
            in_dtype = {"u8": torch.uint8, "f16": torch.float16, "f32": torch.float32}[p.dtype]
            b.slots = [torch.empty((p.nchan, b.block), dtype=in_dtype, device=self.device)
                       for _ in range(2)]
            b.out = torch.empty((p.ndm, b.block), dtype=p.out_torch_dtype, device=self.device)
            b.cands = torch.empty((max(self.capacity, 1), 16), dtype=torch.uint8,
                                  device=self.device)
            b.admitted = True
            b.admit_time = time.perf_counter()
            self.admissions.append((b.key, b.opened, b.admit_time))
            self.used += b.nbytes
            self.peak_used = max(self.peak_used, self.used)
            self._active.append(b)
            self._issue_copies(b)

    def _release(self):
        """Release closed beams with nothing left to do.  Lock held."""
        keep = []
        freed = False
        for b in self._active:
            if b.closing and b.done == b.submitted:
                _native.dd_stream_destroy(b.stream)
                b.stream = b.slots = b.out = b.cands = None
                b.events = [None, None]
                b.released = True
                self.used -= b.nbytes
                del self._beams[b.key]
                freed = True
            else:
                keep.append(b)
        self._active = keep
        # a beam closed before it was admitted
        for b in list(self._pending):
            if b.closing and b.submitted == 0:
                self._pending.remove(b)
                del self._beams[b.key]
        if freed:
            self._torch.cuda.empty_cache()

    def _run(self):
        torch = self._torch
        torch.cuda.set_device(self.device)
        try:
            while True:
                with self._cv:
                    while True:
                        self._release()
                        self._admit()
                        # every admitted beam whose next block has been copied
                        wave = [] if self._abort else [b for b in self._active
                                                        if b.copied > b.done]
                        if wave or self._stop:
                            break
                        self._cv.notify_all()
                        self._cv.wait(0.05)
                    if not wave:  # stopping, nothing copied left to run
                        for b in self._active:
                            _native.dd_stream_destroy(b.stream)
                            b.stream = None
                        self._active = []
                        self._cv.notify_all()
                        return
                    items = [(b, b.done % 2, b.events[b.done % 2]) + b.queue[0][:2]
                             for b in wave]
                self._push(items)
        except BaseException as e:  # reported to the client threads
            with self._cv:
                self._error = e
                self._cv.notify_all()

    def _push(self, items):
        """One wave (or, per_beam, one push per beam) on the compute stream,
        then the candidates to the host; books the results of each push."""
        for _, _, ev, _, _ in items:
            self.compute.wait_event(ev)
        groups = [[it] for it in items] if self.per_beam else [items]
        for g in groups:
            t0 = time.perf_counter()
            _, totals = _native.dd_streams_push(
                [b.stream for b, *_ in g], [b.slots[s] for b, s, *_ in g],
                [b.block for b, *_ in g], [b.out for b, *_ in g], self.nsigma,
                [b.cands if self.capacity else None for b, *_ in g],
                [self.capacity] * len(g), self.compute)
            hosts = []
            for (b, *_), t in zip(g, totals):
                k = min(t, self.capacity)
                hosts.append(b.cands[:k].cpu().numpy().view(CANDIDATE_DTYPE).reshape(-1).copy()
                             if k else np.zeros(0, dtype=CANDIDATE_DTYPE))
            outs = [b.out.cpu() if self.keep_outputs else None for b, *_ in g]
            t1 = time.perf_counter()
            with self._cv:
                self.waves.append((len(g), t0, t1))
                for (b, _, _, seq, arrival), c, t, o in zip(g, hosts, totals, outs):
                    self.results[b.key].append(
                        BlockResult(seq, c, t, arrival, t1, t1 - arrival, len(g), o))
                    b.queue.popleft()
                    b.done += 1
                    self._issue_copies(b)
                self._cv.notify_all()

    # ------------------------------------------------------------ reports

    def latencies(self, keys=None):
        """Per-block latencies (seconds) of the given beams (default all)."""
        with self._cv:
            ks = self.results.keys() if keys is None else keys
            return np.array([r.latency for k in ks for r in self.results.get(k, [])])
