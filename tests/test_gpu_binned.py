"""GPU: time-binned dedispersion (include/dd_binned.h) against the binning
oracle (oracle/approx.py).

u8 input: binned series are integer sums (exact in float below 2^24) and the
rows are compared exactly, with the downfactors, lengths and diagonal DM.
Float input: pair sums are float adds in the same order on both sides; the
dedispersion adds nchan binned samples of up to max_factor inputs each, so
each output agrees within 1e-5 x nchan x factor x max|I| (the brute-force
float bound with the binned samples' magnitude).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import approx
import paper_1401_8258_gb300 as dd
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    dd.build()
    oracle.build()


def geometry(nchan, ndm, step):
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=nchan, ndm=ndm)
    wl.dms = synth.dm_grid(0.0, step, ndm)
    return wl


@pytest.mark.parametrize("nchan,ndm,step,max_factor,extra,pitch_pad", [
    (128, 160, 1.0, 8, 3000, 0),
    (256, 100, 1.5, 4, 2001, 0),     # odd length: binned levels drop a sample
    (200, 90, 2.0, 16, 1500, 3),     # unaligned pitch: plain-load full-rate kernel
    (64, 40, 0.5, 1, 1000, 0),       # max_factor 1: the brute-force sum
])
def test_binned_u8_matches_oracle_exactly(nchan, ndm, step, max_factor, extra, pitch_pad):
    wl = geometry(nchan, ndm, step)
    _, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    nsamp = mx + extra
    pitch = (nsamp + 15) // 16 * 16 + pitch_pad
    block = synth.random_block(np.random.default_rng(nchan), nchan, nsamp, "u8", pitch=pitch)
    rows, fac, lens = approx.binned_dedisperse(block, wl.nchan, wl.f_top_mhz, wl.chan_width_mhz,
                                               wl.t_samp_s, wl.dms, max_factor, nsamp_in=nsamp)
    with dd.Binned(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8",
                   max_factor) as b:
        assert b.dm_diag == approx.diagonal_dm(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz,
                                               wl.t_samp_s)
        gf, gl = b.rows(nsamp)
        assert np.array_equal(gf, fac) and np.array_equal(gl, lens)
        out = b.execute(torch.from_numpy(block).to(DEV), nsamp_in=nsamp).cpu().numpy()
        assert b.launch_count() > 0
    if max_factor > 1:
        assert fac.max() > 1  # the geometry reaches past twice the diagonal DM
    for d in range(wl.ndm):
        assert np.array_equal(out[d, :lens[d]], rows[d]), d


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_binned_float_matches_oracle_within_bound(dtype):
    wl = geometry(128, 120, 1.0)
    _, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    nsamp = mx + 2500
    block = synth.random_block(np.random.default_rng(2), wl.nchan, nsamp, dtype, pitch=nsamp + 8)
    rows, fac, lens = approx.binned_dedisperse(block, wl.nchan, wl.f_top_mhz, wl.chan_width_mhz,
                                               wl.t_samp_s, wl.dms, 8, nsamp_in=nsamp)
    dblock = torch.from_numpy(block.view(np.uint16) if dtype == "f16" else block).to(DEV)
    with dd.Binned(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, dtype,
                   8) as b:
        out = b.execute(dblock, nsamp_in=nsamp).cpu().numpy().astype(np.float64)
    amax = np.abs(block[:, :nsamp].astype(np.float64)).max()
    for d in range(wl.ndm):
        bound = 1e-5 * wl.nchan * fac[d] * amax
        assert np.abs(out[d, :lens[d]] - rows[d]).max() <= bound, d


def test_binned_argument_errors():
    wl = geometry(64, 16, 1.0)
    with pytest.raises(dd.DDError):  # DM list must not decrease
        dd._native.dd_binned_create(64, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s,
                                    wl.dms[::-1].copy(), "u8", 4)
    with pytest.raises(dd.DDError):  # max_factor a power of two
        dd._native.dd_binned_create(64, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms,
                                    "u8", 6)
    with dd.Binned(64, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8", 4) as b:
        x = torch.zeros((64, 64), dtype=torch.uint8, device=DEV)
        o = torch.zeros((16, 64), dtype=torch.int32, device=DEV)
        with pytest.raises(dd.DDError):  # too short for the trials' delays
            dd._native.dd_binned_execute(b.handle, x, 64, 64, o, 64)
