"""Seeded synthetic filterbank generators shared by the tests, the smoke check
and the benchmark.

This module holds no dedispersion arithmetic.  Where a dispersed pulse is
injected, the caller passes the integer delay of every channel for the pulse's
DM trial (taken from whichever delay table it is testing), and the generator
only adds the pulse amplitude at those samples.

Workloads follow the shapes of the thesis's observations (Ch. 4: BEST-II at
400-416 MHz with 1024 channels and 51.2 us sampling; Sec. 2.4 functional test
with a boxcar pulse in N(0,1) noise; Sec. 3.3.4 narrowband RFI with a 6.5 ms
period) and an L-band survey shape (1200-1500 MHz, 4096 channels).  All draws
come from ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DTYPES = {"u8": np.uint8, "f16": np.float16, "f32": np.float32}


@dataclass
class Workload:
    """Geometry of one filterbank block and its DM-trial list."""

    name: str
    nchan: int
    nsamp: int
    f_top_mhz: float
    chan_width_mhz: float
    t_samp_s: float
    dms: np.ndarray
    dtype: str
    n_pulses: int = 0
    pulse_amp: float = 0.0
    pulse_width: tuple = (1, 1)
    pulse_dm_idx: int | None = None
    rfi_frac: float = 0.0
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def ndm(self) -> int:
        return int(self.dms.size)


def dm_grid(lo: float, step: float, n: int) -> np.ndarray:
    """DM trials lo + d*step (not accumulated), float64."""
    return lo + step * np.arange(n, dtype=np.float64)


def workload(name: str) -> Workload:
    """Named workloads.

    * ``single_beam_f32`` -- 64 ch x 8192 f32, 416 MHz top, 0.25 MHz channels,
      100 us, DM 0..63 step 1, one boxcar pulse of amplitude 5 per channel,
      width 4, at DM trial 30.
    * ``full_block_u8``  -- 1024 ch x 65536 u8 (round(N(128,16)) clipped),
      400-416 MHz, 51.2 us, DM 0..204.7 step 0.1, 8 pulses (amplitude 16 per
      channel, widths 1..32) at random DM trials and times.
    * ``single_beam_f16`` -- ``single_beam_f32`` stored as f16.
    * ``lband_f32`` / ``lband_f16`` -- 4096 ch x 131072, 1200-1500 MHz, 64 us,
      DM 0..409.5 step 0.1, N(0,1) noise, 1% of channels with a 6.5 ms
      narrowband sinusoid of amplitude 3, one pulse.
    """
    if name in ("single_beam_f32", "single_beam_f16"):
        return Workload(name, 64, 8192, 416.0, 0.25, 100e-6, dm_grid(0.0, 1.0, 64),
                        "f32" if name.endswith("f32") else "f16",
                        n_pulses=1, pulse_amp=5.0, pulse_width=(4, 4), pulse_dm_idx=30)
    if name == "full_block_u8":
        return Workload(name, 1024, 65536, 416.0, 16.0 / 1024, 51.2e-6,
                        dm_grid(0.0, 0.1, 2048), "u8",
                        n_pulses=8, pulse_amp=16.0, pulse_width=(1, 32))
    if name in ("lband_f32", "lband_f16"):
        return Workload(name, 4096, 131072, 1500.0, 300.0 / 4096, 64e-6,
                        dm_grid(0.0, 0.1, 4096), name[-3:],
                        n_pulses=1, pulse_amp=1.0, pulse_width=(1, 32), rfi_frac=0.01)
    raise KeyError(name)


def batch_workloads(seed: int, maxshift_of, n: int = 32, nchan_choices=(256, 512, 1024, 4096),
                    nsamp_range=(16384, 131072), ndm_range=(128, 4096)) -> list[Workload]:
    """A batch of 32 uneven u8 beams of varied geometry (multi-beam batching).

    Per beam, drawn with ``default_rng(seed)``: nchan from ``nchan_choices``;
    nsamp uniform over multiples of 1024 in ``nsamp_range``; ndm uniform over
    multiples of 128 in ``ndm_range``; band A (416 MHz top, 16 MHz wide,
    51.2 us) or band B (1500 MHz top, 300 MHz wide, 64 us), channel width =
    bandwidth / nchan; DM trials 0, 0.1, ...; data and pulses as
    ``full_block_u8``.  A beam whose largest delay (``maxshift_of(beam)``,
    supplied by the caller) reaches nsamp / 2 is drawn again.
    """
    rng = np.random.default_rng(seed)
    beams = []
    while len(beams) < n:
        nchan = int(rng.choice(nchan_choices))
        nsamp = 1024 * int(rng.integers(nsamp_range[0] // 1024, nsamp_range[1] // 1024 + 1))
        ndm = 128 * int(rng.integers(ndm_range[0] // 128, ndm_range[1] // 128 + 1))
        if rng.integers(0, 2) == 0:
            f_top, bw, ts = 416.0, 16.0, 51.2e-6
        else:
            f_top, bw, ts = 1500.0, 300.0, 64e-6
        wl = Workload(f"beam{len(beams)}", nchan, nsamp, f_top, bw / nchan, ts,
                      dm_grid(0.0, 0.1, ndm), "u8", n_pulses=8, pulse_amp=16.0,
                      pulse_width=(1, 32))
        if maxshift_of(wl) < nsamp // 2:
            beams.append(wl)
    return beams


def serving_workloads(seed: int, maxshift_of, n: int = 64) -> list[Workload]:
    """64 streaming beams with 1 s blocks (real-time serving).

    Per beam, drawn with ``default_rng(seed)``: sampling time 51.2, 64, 128
    or 256 us (n/4 beams each); nchan from {512, 1024, 2048, 4096}; ndm
    uniform over multiples of 128 in [512, 4096]; band A (416 MHz top,
    16 MHz wide) or band B (1500 MHz top, 300 MHz wide), channel width =
    bandwidth / nchan; DM trials 0, 0.1, ...  ``nsamp`` is the block length,
    1 s of samples rounded half away from zero (19531, 15625, 7813, 3906).
    A beam whose largest delay (``maxshift_of(beam)``, supplied by the
    caller) reaches half a block is drawn again.
    """
    rng = np.random.default_rng(seed)
    tsamps = (51.2e-6, 64e-6, 128e-6, 256e-6)
    blocks = {51.2e-6: 19531, 64e-6: 15625, 128e-6: 7813, 256e-6: 3906}
    beams = []
    while len(beams) < n:
        ts = tsamps[len(beams) * len(tsamps) // n]
        nchan = int(rng.choice((512, 1024, 2048, 4096)))
        ndm = 128 * int(rng.integers(4, 33))
        f_top, bw = (416.0, 16.0) if rng.integers(0, 2) == 0 else (1500.0, 300.0)
        wl = Workload(f"serve{len(beams)}", nchan, blocks[ts], f_top, bw / nchan, ts,
                      dm_grid(0.0, 0.1, ndm), "u8")
        if maxshift_of(wl) < wl.nsamp // 2:
            beams.append(wl)
    return beams


def scaled(wl: Workload, nchan: int | None = None, nsamp: int | None = None,
           ndm: int | None = None) -> Workload:
    """Same band and DM step, smaller sizes (for tests)."""
    out = Workload(**{k: getattr(wl, k) for k in wl.__dataclass_fields__})
    if nchan is not None:
        bw = wl.chan_width_mhz * wl.nchan
        out.nchan = nchan
        out.chan_width_mhz = bw / nchan
    if nsamp is not None:
        out.nsamp = nsamp
    if ndm is not None:
        step = float(wl.dms[1] - wl.dms[0]) if wl.ndm > 1 else 1.0
        out.dms = dm_grid(float(wl.dms[0]), step, ndm)
        if out.pulse_dm_idx is not None and out.pulse_dm_idx >= ndm:
            out.pulse_dm_idx = ndm // 2
    return out


@dataclass
class Pulse:
    dm_idx: int
    t0: int
    width: int
    amp: float


def draw_pulses(rng: np.random.Generator, wl: Workload, nsamp_out: int) -> list[Pulse]:
    """Pulse parameters: DM trial, arrival sample t0 at the band top, width."""
    pulses = []
    for _ in range(wl.n_pulses):
        lo, hi = wl.pulse_width
        w = int(rng.integers(lo, hi + 1))
        d = wl.pulse_dm_idx if wl.pulse_dm_idx is not None else int(rng.integers(0, wl.ndm))
        t0 = int(rng.integers(0, max(nsamp_out - w, 1)))
        pulses.append(Pulse(d, t0, w, float(wl.pulse_amp)))
    return pulses


def add_pulse(block: np.ndarray, delay_row: np.ndarray, p: Pulse) -> None:
    """Add ``p.amp`` to ``block[c, t0 + delay_row[c] : +width]`` for every c.

    ``delay_row[c]`` is the integer delay of channel c at the pulse's DM
    trial, supplied by the caller.
    """
    for c in range(block.shape[0]):
        s = p.t0 + int(delay_row[c])
        block[c, s:s + p.width] += p.amp


def add_narrowband_rfi(rng: np.random.Generator, block: np.ndarray, t_samp_s: float,
                       frac: float, amp: float = 3.0, period_s: float = 6.5e-3) -> np.ndarray:
    """Add ``amp*sin(2 pi t t_samp / period + phi)`` to a seeded 1% of channels."""
    nchan, nsamp = block.shape
    k = max(1, int(round(frac * nchan)))
    chans = np.sort(rng.choice(nchan, size=k, replace=False))
    t = np.arange(nsamp, dtype=np.float64) * t_samp_s
    for c in chans:
        phi = rng.uniform(0.0, 2 * np.pi)
        block[c] += (amp * np.sin(2 * np.pi * t / period_s + phi)).astype(block.dtype)
    return chans


def make_block(wl: Workload, seed: int, delays: np.ndarray, pitch: int | None = None):
    """Seeded filterbank ``[nchan][pitch]`` for workload ``wl``.

    ``delays`` is the ``[nchan][ndm]`` integer delay table used to place the
    pulses (and whose maximum sets the valid output length).  Returns
    ``(block, pulses)``; for pitch > nsamp the padding holds zeros.
    """
    rng = np.random.default_rng(seed)
    nchan, nsamp = wl.nchan, wl.nsamp
    z = rng.standard_normal((nchan, nsamp), dtype=np.float32)
    nsamp_out = nsamp - int(delays.max())
    pulses = draw_pulses(rng, wl, nsamp_out)
    if wl.dtype == "u8":
        z *= 16.0
        z += 128.0
    for p in pulses:
        add_pulse(z, delays[:, p.dm_idx], p)
    if wl.rfi_frac > 0:
        add_narrowband_rfi(rng, z, wl.t_samp_s, wl.rfi_frac)
    if wl.dtype == "u8":
        data = np.clip(np.rint(z), 0, 255).astype(np.uint8)
    else:
        data = z.astype(DTYPES[wl.dtype])
    if pitch is None or pitch == nsamp:
        return data, pulses
    out = np.zeros((nchan, pitch), dtype=data.dtype)
    out[:, :nsamp] = data
    return out, pulses


def random_block(rng: np.random.Generator, nchan: int, nsamp: int, dtype: str,
                 pitch: int | None = None) -> np.ndarray:
    """Plain random block: u8 uniform 0..255, floats N(0,1)."""
    pitch = nsamp if pitch is None else pitch
    if dtype == "u8":
        b = rng.integers(0, 256, size=(nchan, pitch), dtype=np.uint8)
    else:
        b = rng.standard_normal((nchan, pitch), dtype=np.float32).astype(DTYPES[dtype])
    if pitch > nsamp:
        b[:, nsamp:] = 0
    return b


def series_rows(rng: np.random.Generator, nrows: int, ncols: int, dtype: str,
                level: float = 0.0, noise: float = 1.0, slope: float = 0.0,
                pulses: int = 0, pulse_amp: float = 0.0, pulse_width=(1, 64),
                pitch: int | None = None) -> np.ndarray:
    """Rows shaped like dedispersed series, for the post-processing tests.

    Per row: ``level`` + a linear drift of ``slope`` per sample with a
    random sign + N(0, noise^2) noise + ``pulses`` top-hat pulses of height
    ``pulse_amp`` x noise, widths uniform in ``pulse_width``, at uniform
    start samples.  ``dtype`` "i32" rounds half away from zero to int32,
    "f32" keeps float32.  Columns past ncols (pitch > ncols) hold a large
    sentinel that no result may read."""
    pitch = ncols if pitch is None else pitch
    t = np.arange(ncols, dtype=np.float64)
    y = level + np.outer(rng.choice((-1.0, 1.0), nrows) * slope, t)
    y = y + noise * rng.standard_normal((nrows, ncols))
    for r in range(nrows):
        for _ in range(pulses):
            w = int(rng.integers(pulse_width[0], pulse_width[1] + 1))
            t0 = int(rng.integers(0, max(1, ncols - w)))
            y[r, t0:t0 + w] += pulse_amp * noise
    out_dtype = np.int32 if dtype == "i32" else np.float32
    rows = np.full((nrows, pitch), 1 << 30, dtype=out_dtype)
    if dtype == "i32":
        rows[:, :ncols] = (np.sign(y) * np.floor(np.abs(y) + 0.5)).astype(np.int32)
    else:
        rows[:, :ncols] = y.astype(np.float32)
    return rows
