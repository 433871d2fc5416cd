"""GPU: time-binned dedispersion (include/dd_binned.h) against the binning
oracle (oracle/approx.py).

u8 input: binned series are integer sums (exact in float below 2^24), or in
the 8-bit mode integer rounded means, and the rows are compared exactly, with
the downfactors, lengths and diagonal DM.
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


@pytest.mark.parametrize("mode", ["sum", "mean8"])
@pytest.mark.parametrize("nchan,ndm,step,max_factor,extra,pitch_pad", [
    (128, 160, 1.0, 8, 3000, 0),
    (256, 100, 1.5, 4, 2001, 0),     # odd length: binned levels drop a sample
    (200, 90, 2.0, 16, 1500, 3),     # unaligned pitch: plain-load full-rate kernel
    (64, 40, 0.5, 1, 1000, 0),       # max_factor 1: the brute-force sum
    (96, 200, 1.0, 64, 9000, 0),     # six binning levels
])
def test_binned_u8_matches_oracle_exactly(nchan, ndm, step, max_factor, extra, pitch_pad, mode):
    wl = geometry(nchan, ndm, step)
    _, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    nsamp = mx + extra
    pitch = (nsamp + 15) // 16 * 16 + pitch_pad
    block = synth.random_block(np.random.default_rng(nchan), nchan, nsamp, "u8", pitch=pitch)
    rows, fac, lens = approx.binned_dedisperse(block, wl.nchan, wl.f_top_mhz, wl.chan_width_mhz,
                                               wl.t_samp_s, wl.dms, max_factor, nsamp_in=nsamp,
                                               mode=mode)
    with dd.Binned(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8",
                   max_factor, mode=mode) as b:
        assert b.dm_diag == approx.diagonal_dm(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz,
                                               wl.t_samp_s)
        gf, gl = b.rows(nsamp)
        assert np.array_equal(gf, fac) and np.array_equal(gl, lens)
        out = b.execute(torch.from_numpy(block).to(DEV), nsamp_in=nsamp).cpu().numpy()
        assert b.launch_count() > 0
        b.sync()  # no bounded wait ran out
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
    with pytest.raises(dd.DDError) as e:  # 8-bit means of float input
        dd._native.dd_binned_create(64, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms,
                                    "f32", 4, "mean8")
    assert e.value.status == -3
    with pytest.raises(dd.DDError) as e:  # no such mode
        dd._native.dd_binned_create(64, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms,
                                    "u8", 4, 2)
    assert e.value.status == -1
    with dd.Binned(64, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8", 4) as b:
        x = torch.zeros((64, 64), dtype=torch.uint8, device=DEV)
        o = torch.zeros((16, 64), dtype=torch.int32, device=DEV)
        with pytest.raises(dd.DDError):  # too short for the trials' delays
            dd._native.dd_binned_execute(b.handle, x, 64, 64, o, 64)


@pytest.mark.parametrize("mode", ["sum", "mean8"])
def test_binned_full_block_u8_full_size_sampled_rows(mode):
    """1024 ch x 65536 u8, 2048 trials DM 0..204.7, downfactors up to 8 (the
    timed binned workload): rows sampled in every downfactor range against
    the oracle's binned series, dedispersed one by one with that range's
    delays and length, bit-exact."""
    wl = synth.workload("full_block_u8")
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, _ = synth.make_block(wl, seed=1, delays=delays)
    with dd.Binned(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8", 8,
                   mode=mode) as b:
        out = b.execute(torch.from_numpy(block).to(DEV)).cpu().numpy()
        fac, lens = b.rows(wl.nsamp)
    assert np.array_equal(fac, approx.binning_factors(
        wl.dms, approx.diagonal_dm(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s), 8))
    rng = np.random.default_rng(5)
    for f in sorted(set(fac.tolist())):
        idx = np.nonzero(fac == f)[0]
        ftab, fmx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz,
                                       wl.t_samp_s * f, wl.dms[idx])
        if f == 1:
            src = block
        elif mode == "sum":
            src = approx.decimate(block, wl.nsamp, f).astype(np.float32)
        else:
            src = approx.decimate_mean8(block, wl.nsamp, f)
        n_out = src.shape[1] - fmx
        assert np.all(lens[idx] == n_out)
        pick = sorted(set([0, len(idx) - 1] + rng.integers(0, len(idx), 4).tolist()))
        ref = oracle.dedisperse(np.ascontiguousarray(src), ftab[:, pick], nsamp_out=n_out)
        if ref.dtype != np.int32:
            ref = np.rint(ref).astype(np.int32)
        for j, i in enumerate(pick):
            assert np.array_equal(out[idx[i], :n_out], ref[j]), (mode, f, idx[i])
