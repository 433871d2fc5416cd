"""GPU: the path at the edges of its size limits, against the oracle on
sampled output ranges (each range computed by the oracle from the slice of
the block it reads).

* The staged float kernel is persistent, so its time tiles have no grid
  limit: 65535 x 256 outputs and one more (the old grid-row limit) both run
  on it and must give the oracle's sums.
* The staged u8 kernel's work queue has no tile-count limit: a 20-million-
  sample block runs through it.
* 16384 channels: 64 drains of the u8 kernel's 16-bit partial sums into its
  32-bit sums, and exact int32 sums up to 16384 x 255.
* Past the 64-bit limit of dd_run's fused row sums of squares, dd_run keeps
  the statistics exact through the 128-bit passes.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1401_8258_gb300 as dd
import synth
from tests.test_abi_extras import fused_sums_fit

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FLOAT_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    dd.build()
    oracle.build()


def sampled_ranges(n_out, width=2048, seed=0):
    rng = np.random.default_rng(seed)
    mids = rng.integers(width, n_out - 2 * width, 2).tolist()
    return [(0, width), (n_out - width, n_out)] + [(m, m + width) for m in mids]


def check_ranges(block, delays, got, n_out, dtype):
    mx = int(delays.max())
    for a, b in sampled_ranges(n_out):
        part = block[:, a:b + mx]
        ref = oracle.dedisperse(part, delays, nsamp_out=b - a)
        if dtype == "u8":
            assert np.array_equal(got[:, a:b], ref), (a, b)
        else:
            scale = oracle.dedisperse(np.abs(part.astype(np.float32)), delays, nsamp_out=b - a)
            err = np.abs(got[:, a:b].astype(np.float64) - ref) / np.maximum(scale, 1e-30)
            assert err.max() <= FLOAT_RTOL, (a, b, err.max())


@pytest.mark.parametrize("extra", [0, 1])
def test_float_kernel_time_tile_limit(extra):
    """nsamp_out = 65535 x 256 (+1): both sizes on the staged kernel."""
    # L-band channel spacing, trials far enough apart for non-zero delays and
    # close enough for the staged kernel's tables
    nchan, f_top, df, ts = 8, 1500.0, 300.0 / 4096, 64e-6
    dms = synth.dm_grid(0.0, 50.0, 4)
    delays, mx = oracle.delay_table(nchan, f_top, df, ts, dms)
    assert mx > 0
    n_out = 65535 * 256 + extra
    nsamp = n_out + mx
    pitch = (nsamp + 3) // 4 * 4
    block = synth.random_block(np.random.default_rng(21), nchan, nsamp, "f32", pitch=pitch)
    with dd.Plan(nchan, f_top, df, ts, dms, "f32") as plan:
        assert plan.maxshift == mx and plan.nsamp_out(nsamp) == n_out
        dblock = torch.from_numpy(block).to(DEV)
        # the staged tables exist, so the time-tile count alone picks the kernel
        assert dd._native.dd_plan_kernel_info(plan.handle, dblock, pitch)["staged"]
        out = plan.execute(dblock, nsamp_in=nsamp)
        got = out.cpu().numpy()
    assert got.shape == (4, n_out)
    check_ranges(block, delays, got, n_out, "f32")


def test_u8_kernel_twenty_million_samples():
    nchan, f_top, df, ts = 16, 416.0, 1.0, 51.2e-6
    dms = synth.dm_grid(0.0, 0.5, 8)
    delays, mx = oracle.delay_table(nchan, f_top, df, ts, dms)
    nsamp = 20_000_000
    block = synth.random_block(np.random.default_rng(22), nchan, nsamp, "u8")
    with dd.Plan(nchan, f_top, df, ts, dms, "u8") as plan:
        out = plan.execute(torch.from_numpy(block).to(DEV))
        got = out.cpu().numpy()
    assert got.shape == (8, nsamp - mx)
    check_ranges(block, delays, got, nsamp - mx, "u8")


def test_u8_kernel_sixteen_thousand_channels():
    nchan, f_top, df, ts = 16384, 1500.0, 300.0 / 16384, 64e-6
    dms = synth.dm_grid(0.0, 0.1, 64)
    delays, mx = oracle.delay_table(nchan, f_top, df, ts, dms)
    nsamp = mx + 5000
    block = np.full((nchan, nsamp), 255, dtype=np.uint8)  # the largest sums
    block[:, ::7] = np.random.default_rng(23).integers(0, 256, (nchan, (nsamp + 6) // 7))
    with dd.Plan(nchan, f_top, df, ts, dms, "u8") as plan:
        out, cands, total = plan.run(torch.from_numpy(block).to(DEV), 3.0)
        got = out.cpu().numpy()
        mean, sigma = plan.stats()
    ref = oracle.dedisperse(block, delays)
    assert np.array_equal(got, ref)
    assert ref.max() > 255 * nchan * 0.8
    m, s = oracle.stats(ref)
    assert np.array_equal(mean, m) and np.array_equal(sigma, s)
    c_ref, tot = oracle.detect(ref, m, s, 3.0)
    assert total == tot and np.array_equal(cands, c_ref)


def test_u8_run_past_the_fused_sum_limit_keeps_exact_statistics():
    """dd_run totals each row's sum of squares in 64 bits only while
    (255 nchan)^2 nsamp_out < 2^64; 16384 saturated channels x 1.1 M outputs
    are past that, so dd_run must take the passes that keep it in 128 bits and
    still give the oracle's statistics and candidates exactly.  Both trials
    are DM 0, so each row is the plain channel sum (a pinned identity of the
    oracle) and the block can be checked at this size in seconds."""
    nchan, nsamp = 16384, 1_100_000
    assert not fused_sums_fit(nchan, nsamp)
    dms = np.zeros(2)
    block = np.full((nchan, nsamp), 255, dtype=np.uint8)
    rng = np.random.default_rng(24)
    block[rng.integers(0, nchan, 40000), rng.integers(0, nsamp, 40000)] = 0
    with dd.Plan(nchan, 1500.0, 300.0 / nchan, 64e-6, dms, "u8") as plan:
        assert plan.maxshift == 0
        # the full columns sit about 0.19 sigma above the mean
        out, cands, total = plan.run(torch.from_numpy(block).to(DEV), 0.1, capacity=0)
        got = out.cpu().numpy()
        mean, sigma = plan.stats()
    row = (255 * nchan - 255 * np.count_nonzero(block == 0, axis=0)).astype(np.int32)
    ref = np.stack([row, row])
    assert np.array_equal(got, ref)
    m, s = oracle.stats(ref)
    assert np.array_equal(mean, m) and np.array_equal(sigma, s) and s[0] > 0
    _, tot = oracle.detect(ref, m, s, 0.1, capacity=0)
    assert total == tot > 0
