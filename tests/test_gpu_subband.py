"""GPU: subband dedispersion (include/dd_subband.h) against the subband oracle
(oracle/approx.py), and at the nominal trials against the brute-force sum.

u8 input: integer sums throughout (step-1 series as 16-bit integers, or
carried as float below 2^24 for subbands wider than 257 channels), so the
comparison is exact.  Float input: step 1 and step 2 each
accumulate in float on the device and in double in the oracle; with the
step-1 series rounded to float on both sides, each output agrees within
1e-5 of the sum of |I| over the channels it adds (the bound of the
brute-force float tests, applied to the whole two-step sum).
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


def geometry(nchan, ndm, step=0.5, bw=16.0):
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=nchan, ndm=ndm)
    wl.chan_width_mhz = bw / nchan
    wl.dms = synth.dm_grid(0.0, step, ndm)
    return wl


def make(wl, dtype, cps, dpg):
    return dd.Subband(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, dtype,
                      cps, dpg)


@pytest.mark.parametrize("nchan,ndm,cps,dpg,pitch_pad", [
    (256, 96, 32, 16, 0),
    (256, 96, 48, 7, 0),     # ragged last subband and last group
    (300, 70, 32, 16, 5),    # unaligned pitch: plain-load kernels in both steps
    (512, 128, 64, 32, 0),
    (256, 64, 1, 8, 0),      # one channel per subband: the brute-force sum
    (600, 64, 300, 16, 0),   # subbands too wide for 16-bit sums: float step-1 series
])
def test_subband_u8_matches_oracle_exactly(nchan, ndm, cps, dpg, pitch_pad):
    wl = geometry(nchan, ndm)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s,
                                    wl.dms)
    nsamp = mx + 5000
    pitch = (nsamp + 15) // 16 * 16 + pitch_pad
    block = synth.random_block(np.random.default_rng(nchan + ndm), nchan, nsamp, "u8", pitch=pitch)
    ref = approx.subband_dedisperse(block, delays, cps, dpg, nsamp_in=nsamp)
    tb = approx.SubbandTables(delays, cps, dpg)
    with make(wl, "u8", cps, dpg) as sub:
        assert sub.maxshift == tb.maxshift
        assert list(sub.nominal) == tb.nominal
        got = sub.execute(torch.from_numpy(block).to(DEV), nsamp_in=nsamp).cpu().numpy()
        sub.sync()  # no bounded wait ran out
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)
    if cps == 1:
        brute = oracle.dedisperse(block, delays, nsamp_in=nsamp)
        assert np.array_equal(got, brute[:, :got.shape[1]])


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_subband_float_matches_oracle_within_bound(dtype):
    wl = geometry(256, 80)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s,
                                    wl.dms)
    nsamp = mx + 3000
    block = synth.random_block(np.random.default_rng(9), wl.nchan, nsamp, dtype, pitch=nsamp + 8)
    with make(wl, dtype, 32, 16) as sub:
        dblock = torch.from_numpy(block.view(np.uint16) if dtype == "f16" else block).to(DEV)
        got = sub.execute(dblock, nsamp_in=nsamp).cpu().numpy().astype(np.float64)
    ref = approx.subband_dedisperse(block, delays, 32, 16, nsamp_in=nsamp)
    # every output adds nchan samples; bound by nchan x the block's largest |I|
    bound = 1e-5 * wl.nchan * np.abs(block[:, :nsamp].astype(np.float64)).max()
    assert np.abs(got - ref).max() <= bound


def test_subband_nominal_trials_equal_brute_force_on_gpu():
    wl = geometry(512, 128)
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8") as plan:
        delays = plan.delays()
        block, _ = synth.make_block(synth.scaled(wl, nsamp=plan.maxshift + 8000), 5, delays)
        dblock = torch.from_numpy(block).to(DEV)
        brute = plan.run(dblock, 6.0)[0].cpu().numpy()
    with make(wl, "u8", 32, 16) as sub:
        got = sub.execute(dblock).cpu().numpy()
        n = min(got.shape[1], brute.shape[1])
        assert np.array_equal(got[sub.nominal, :n], brute[sub.nominal, :n])
        assert sub.launch_count() > 0


def test_subband_argument_errors():
    wl = geometry(64, 16)
    with pytest.raises(dd.DDError):
        dd._native.dd_subband_create(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s,
                                     wl.dms, "u8", 0, 4)
    with pytest.raises(dd.DDError):  # u8 sums must stay below 2^24
        dd._native.dd_subband_create(70000, 1500.0, 0.001, 64e-6, np.zeros(4), "u8", 64, 2)
    with make(wl, "u8", 16, 4) as sub:
        x = torch.zeros((64, sub.maxshift), dtype=torch.uint8, device=DEV)
        out = torch.zeros((16, 1), dtype=torch.int32, device=DEV)
        with pytest.raises(dd.DDError):  # nsamp_in <= maxshift
            dd._native.dd_subband_execute(sub.handle, x, sub.maxshift, sub.maxshift, out)
