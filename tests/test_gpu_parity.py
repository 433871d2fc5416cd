"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer (u8) input must match bit for bit, including the per-DM statistics
and the candidate list.  Float input (f16, f32) must satisfy, per output,
  |D_gpu - D_oracle| <= 1e-5 * sum_c |I[c][t + delay(c,d)]|
i.e. a relative error of 1e-5 against the conditioning of each sum (the
oracle sums in double); candidates must agree except for samples whose oracle
snr lies within 1e-4*max(1,|nsigma|) of the threshold.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1401_8258_gb300 as dd
import synth

pytestmark = pytest.mark.gpu

FLOAT_RTOL = 1e-5
BAND = 1e-4

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    dd.build()
    oracle.build()


def _to_dev(block: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(block)).to(DEV)


def run_plan(wl, block, nsamp_in=None, offset=0, nsigma=None, capacity=1 << 16):
    """Dedisperse (and optionally detect) ``block`` on the GPU.

    ``offset`` shifts the block's start by that many elements inside a larger
    device buffer, so that misaligned pointers are exercised.
    """
    nchan, pitch = block.shape
    nsamp_in = pitch if nsamp_in is None else nsamp_in
    with dd.Plan(nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, wl.dtype) as plan:
        flat = np.zeros(nchan * pitch + offset + 64, dtype=block.dtype)
        flat[offset:offset + nchan * pitch] = block.reshape(-1)
        dbuf = _to_dev(flat)
        dblock = dbuf[offset:offset + nchan * pitch].view(nchan, pitch)
        out = plan.execute(dblock, nsamp_in=nsamp_in)
        res = {"D": None, "cands": None, "total": None, "mean": None, "sigma": None}
        if nsigma is not None:
            cands, total = plan.detect(out, nsigma, capacity=capacity)
            mean, sigma = plan.stats()
            res.update(cands=cands, total=total, mean=mean, sigma=sigma)
        torch.cuda.synchronize()
        res["D"] = out.cpu().numpy()
        res["delays"] = plan.delays()
        res["launches"] = plan.launch_count()
    return res


def float_rel_errs(block, delays, got, ref, nsamp_in=None, rows=None):
    """|got - ref| / sum_c |I[c][t + delay]| for every output."""
    absblock = np.abs(block.astype(np.float32))
    d = delays if rows is None else delays[:, rows]
    scale = oracle.dedisperse(absblock, d, nsamp_out=ref.shape[1], nsamp_in=nsamp_in)
    return np.abs(got.astype(np.float64) - ref) / np.maximum(scale, 1e-30)


def float_rel_err(block, delays, got, ref, nsamp_in=None, rows=None):
    """max |got - ref| / sum_c |I[c][t + delay]| over all outputs."""
    return float(np.max(float_rel_errs(block, delays, got, ref, nsamp_in, rows)))


def report_errs(label, errs):
    """Print the max and 99th percentile of the per-output relative error."""
    print(f"\n{label}: relative error max {errs.max():.3e} p99 {np.percentile(errs, 99):.3e}")


def assert_parity(wl, block, res, nsamp_in=None):
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    assert np.array_equal(res["delays"], delays)
    ref = oracle.dedisperse(block, delays, nsamp_in=nsamp_in)
    got = res["D"]
    assert got.shape == ref.shape
    if wl.dtype == "u8":
        assert got.dtype == np.int32
        bad = np.argwhere(got != ref)
        assert bad.size == 0, f"{bad.shape[0]} mismatches, first {bad[:5].tolist()}"
    else:
        err = float_rel_err(block, delays, got, ref, nsamp_in)
        assert err <= FLOAT_RTOL, err
    return ref


def assert_float_candidates(got, D, ref, scale, mean, sigma, ref_mean, ref_sigma):
    """Every float candidate (Sec. 3.6 triplet: DM index, time, intensity,
    plus its S/N) against the FP64 oracle.

    value: the GPU output at (d, t) itself, hence within the stated bound
      1e-5 * sum_c |I| of the oracle's D.
    snr: computed from the GPU's D, mean and rms; against the oracle's
      (D - mean) / rms its error is at most
        (|dD| + |dmean|) / rms_gpu + |snr_oracle| * |d rms| / rms_gpu
      with |dD| <= 1e-5 * sum_c |I| and the measured differences of the row
      statistics, plus the rounding of snr to float (2^-24 relative)."""
    d, t = got["dm_idx"].astype(np.int64), got["t"].astype(np.int64)
    assert np.array_equal(got["value"], D[d, t].astype(np.float32))
    dv = np.abs(got["value"].astype(np.float64) - ref[d, t])
    assert np.all(dv <= FLOAT_RTOL * scale[d, t]), float(np.max(dv / scale[d, t]))
    snr_ref = (ref[d, t] - ref_mean[d]) / ref_sigma[d]
    bound = ((FLOAT_RTOL * scale[d, t] + np.abs(mean[d] - ref_mean[d])) / sigma[d] +
             np.abs(snr_ref) * np.abs(sigma[d] - ref_sigma[d]) / sigma[d] +
             2.0 ** -23 * np.abs(snr_ref) + 1e-9)
    err = np.abs(got["snr"].astype(np.float64) - snr_ref)
    assert np.all(err <= bound), float(np.max(err - bound))


def assert_detection(wl, ref, res, nsigma, block=None, delays=None, nsamp_in=None):
    if wl.dtype == "u8":
        mean, sigma = oracle.stats(ref)
        assert np.array_equal(res["mean"], mean)
        assert np.array_equal(res["sigma"], sigma)
        cands, total = oracle.detect(ref, mean, sigma, nsigma)
        assert res["total"] == total
        assert np.array_equal(res["cands"], cands)
    else:
        mean, sigma = oracle.stats(ref)
        np.testing.assert_allclose(res["mean"], mean, rtol=1e-5, atol=1e-4 * np.sqrt(wl.nchan))
        np.testing.assert_allclose(res["sigma"], sigma, rtol=1e-5)
        ok = sigma > 0
        snr = np.full(ref.shape, -np.inf)
        snr[ok] = (ref[ok] - mean[ok, None]) / sigma[ok, None]
        band = BAND * max(1.0, abs(nsigma))
        sure = set(map(tuple, np.argwhere(snr > nsigma + band)))
        maybe = set(map(tuple, np.argwhere(snr > nsigma - band)))
        got = set(zip(res["cands"]["dm_idx"].tolist(), res["cands"]["t"].tolist()))
        assert sure <= got <= maybe
        order = list(zip(res["cands"]["dm_idx"].tolist(), res["cands"]["t"].tolist()))
        assert order == sorted(order)
        assert res["total"] == res["cands"].size
        if res["cands"].size:
            assert block is not None, "float candidates need the block for their bounds"
            scale = oracle.dedisperse(np.abs(block.astype(np.float32)), delays,
                                      nsamp_out=ref.shape[1], nsamp_in=nsamp_in)
            assert_float_candidates(res["cands"], res["D"], ref, scale, res["mean"],
                                    res["sigma"], mean, sigma)


# ------------------------------------------------------------------ tiny

@pytest.mark.parametrize("dtype", ["u8", "f16", "f32"])
@pytest.mark.parametrize("seed", range(6))
def test_tiny_random_shapes(dtype, seed):
    rng = np.random.default_rng(1000 + seed)
    nchan = int(rng.integers(1, 38))
    ndm = int(rng.integers(1, 20))
    f_top = float(rng.uniform(300, 1500))
    df = float(rng.uniform(0.001, 0.05)) * f_top / max(nchan, 1)
    ts = float(rng.uniform(20e-6, 200e-6))
    dms = np.sort(rng.uniform(0, 40, ndm))
    wl = synth.Workload("tiny", nchan, 0, f_top, df, ts, dms, dtype)
    _, mx = oracle.delay_table(nchan, f_top, df, ts, dms)
    nsamp = mx + int(rng.integers(1, 300))
    pitch = nsamp + int(rng.integers(0, 19))
    block = synth.random_block(rng, nchan, nsamp, dtype, pitch)
    offset = int(rng.integers(0, 5))
    res = run_plan(wl, block, nsamp_in=nsamp, offset=offset, nsigma=1.5)
    ref = assert_parity(wl, block, res, nsamp_in=nsamp)
    assert_detection(wl, ref, res, 1.5, block, res["delays"], nsamp)


@pytest.mark.parametrize("dtype", ["u8", "f16", "f32"])
def test_single_output_sample_and_single_trial(dtype):
    rng = np.random.default_rng(5)
    wl = synth.Workload("edge", 8, 0, 416.0, 0.25, 100e-6, np.array([17.0]), dtype)
    _, mx = oracle.delay_table(8, 416.0, 0.25, 100e-6, wl.dms)
    block = synth.random_block(rng, 8, mx + 1, dtype)
    res = run_plan(wl, block)
    assert res["D"].shape == (1, 1)
    assert_parity(wl, block, res)


def test_all_zero_dm_and_one_channel():
    rng = np.random.default_rng(6)
    wl = synth.Workload("zero", 1, 0, 416.0, 0.25, 100e-6, np.zeros(5), "u8")
    block = synth.random_block(rng, 1, 777, "u8")
    res = run_plan(wl, block, nsigma=2.0)
    ref = assert_parity(wl, block, res)
    assert np.array_equal(res["D"][0], block[0].astype(np.int32))
    assert_detection(wl, ref, res, 2.0)


def test_constant_input_gives_zero_sigma_and_no_candidates():
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=32, ndm=40)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block = np.full((32, mx + 5000), 200, dtype=np.uint8)
    res = run_plan(wl, block, nsigma=0.0)
    assert np.all(res["sigma"] == 0) and res["total"] == 0
    assert np.all(res["D"] == 200 * 32)


# ---------------------------------------------------------------- configs

@pytest.mark.parametrize("dtype", ["f32", "f16", "u8"])
def test_single_beam_full_config(dtype):
    """64 ch x 8192, DM 0..63: every output against the oracle."""
    wl = synth.workload("single_beam_f32")
    wl.dtype = dtype
    if dtype == "u8":
        wl.pulse_amp = 80.0
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, pulses = synth.make_block(wl, seed=1, delays=delays)
    res = run_plan(wl, block, nsigma=6.0)
    ref = assert_parity(wl, block, res)
    assert_detection(wl, ref, res, 6.0, block, delays)
    if dtype != "u8":
        report_errs(f"single_beam {dtype}", float_rel_errs(block, delays, res["D"], ref))
    p = pulses[0]
    hit = (res["cands"]["dm_idx"] == p.dm_idx) & (res["cands"]["t"] >= p.t0) & \
        (res["cands"]["t"] < p.t0 + p.width)
    assert hit.any()


@pytest.mark.parametrize("pitch_pad, offset", [(0, 0), (13, 0), (0, 3), (16, 16)])
def test_full_block_geometry_reduced_size(pitch_pad, offset):
    """400-416 MHz, 51.2 us geometry at 256 channels, 128 trials: covers
    many time tiles, a ragged tail, odd pitches and misaligned pointers."""
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=256, nsamp=12000, ndm=128)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, _ = synth.make_block(wl, seed=2, delays=delays, pitch=wl.nsamp + pitch_pad)
    res = run_plan(wl, block, nsamp_in=wl.nsamp, offset=offset, nsigma=4.0)
    ref = assert_parity(wl, block, res, nsamp_in=wl.nsamp)
    assert_detection(wl, ref, res, 4.0, block, delays, wl.nsamp)


def test_full_block_u8_full_size_sampled_rows():
    """1024 ch x 65536 u8, 2048 trials DM 0..204.7: rows sampled across the
    DM range (first, last and spread) against the oracle, bit-exact, with
    their statistics and candidates; pulses recovered at their true trial."""
    wl = synth.workload("full_block_u8")
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, pulses = synth.make_block(wl, seed=1, delays=delays)
    res = run_plan(wl, block, nsigma=6.0)
    D = res["D"]
    rows = sorted(set([0, 1, 2, 1023, 2046, 2047] + [p.dm_idx for p in pulses] +
                      np.random.default_rng(3).integers(0, wl.ndm, 10).tolist()))
    ref = oracle.dedisperse(block, delays[:, rows], nsamp_out=D.shape[1])
    assert np.array_equal(D[rows], ref)
    mean, sigma = oracle.stats(ref)
    assert np.array_equal(res["mean"][rows], mean)
    assert np.array_equal(res["sigma"][rows], sigma)
    for p in pulses:
        hit = (res["cands"]["dm_idx"] == p.dm_idx) & (res["cands"]["t"] >= p.t0) & \
            (res["cands"]["t"] < p.t0 + p.width)
        assert hit.any(), p
    for i, r in enumerate(rows):
        c_ref, tot = oracle.detect(ref[i:i + 1], mean[i:i + 1], sigma[i:i + 1], 6.0)
        mine = res["cands"][res["cands"]["dm_idx"] == r]
        assert mine.size == tot
        assert np.array_equal(mine["t"], c_ref["t"])
        assert np.array_equal(mine["value"], c_ref["value"])
        assert np.array_equal(mine["snr"], c_ref["snr"])


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_lband_full_size_sampled_rows(dtype):
    """4096 ch x 131072, 4096 trials DM 0..409.5 with narrowband RFI, detected
    at 6 sigma in the launch configuration the bench times: sampled rows
    within 1e-5 of the FP64 oracle (relative to the sum of |I|), their
    statistics within 1e-5, and their candidates (set, order, value, snr)
    against the oracle's; the pulse is found at its trial and time."""
    wl = synth.workload("lband_" + dtype)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, pulses = synth.make_block(wl, seed=1, delays=delays)
    nsigma = 6.0
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, wl.dtype) as plan:
        out, cands, total = plan.run(_to_dev(block), nsigma)
        mean_g, sigma_g = plan.stats()
        D = out.cpu().numpy()
    del out
    assert total == cands.size
    p = pulses[0]
    rows = [0, 1, 2048, 4094, 4095, p.dm_idx]
    ref = oracle.dedisperse(block, delays[:, rows], nsamp_out=D.shape[1])
    errs = float_rel_errs(block, delays, D[rows], ref, rows=rows)
    report_errs(f"lband {dtype} (rows {rows})", errs)
    assert errs.max() <= FLOAT_RTOL
    mean, sigma = oracle.stats(ref)
    np.testing.assert_allclose(mean_g[rows], mean, rtol=1e-5, atol=1e-4 * np.sqrt(wl.nchan))
    np.testing.assert_allclose(sigma_g[rows], sigma, rtol=1e-5)
    scale = oracle.dedisperse(np.abs(block.astype(np.float32)), delays[:, rows],
                              nsamp_out=D.shape[1])
    band = BAND * max(1.0, abs(nsigma))
    for i, r in enumerate(rows):
        snr = (ref[i] - mean[i]) / sigma[i]
        mine = cands[cands["dm_idx"] == r]
        got = set(mine["t"].tolist())
        assert set(np.flatnonzero(snr > nsigma + band).tolist()) <= got
        assert got <= set(np.flatnonzero(snr > nsigma - band).tolist())
        assert np.all(np.diff(mine["t"]) > 0)
        sub = mine.copy()
        sub["dm_idx"] = i
        assert_float_candidates(sub, D[rows], ref, scale, mean_g[rows], sigma_g[rows],
                                mean, sigma)
    hit = (cands["dm_idx"] == p.dm_idx) & (cands["t"] >= p.t0) & (cands["t"] < p.t0 + p.width)
    assert hit.any()


# ------------------------------------------------------------ error paths

def test_argument_errors():
    wl = synth.workload("single_beam_f32")
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "f32") as plan:
        h = plan.handle
        blk = torch.zeros((wl.nchan, 2000), device=DEV)
        out = torch.zeros((wl.ndm, 2000), device=DEV)
        with pytest.raises(dd.DDError) as e:
            dd.dd_execute(h, blk, plan.maxshift, 2000, out)          # nsamp_in <= maxshift
        assert e.value.status == -2
        with pytest.raises(dd.DDError) as e:
            dd.dd_execute(h, blk, 2000, 1999, out)                    # pitch < nsamp_in
        assert e.value.status == -2
        with pytest.raises(dd.DDError) as e:
            dd.dd_execute(h, None, 2000, 2000, out)
        assert e.value.status == -1
        with pytest.raises(dd.DDError) as e:
            dd.dd_detect(h, out, 100, 5.0, None, 10)                  # capacity without buffer
        assert e.value.status == -1
        with pytest.raises(dd.DDError) as e:
            dd.dd_get_stats(h, wl.ndm)                                # no detect yet
        assert e.value.status == -1
    with pytest.raises(dd.DDError) as e:
        dd.dd_plan_create(64, 416.0, 0.25, 1e-4, [1.0], 7)
    assert e.value.status == -3
    with pytest.raises(dd.DDError) as e:
        dd.dd_plan_create(64, 416.0, 0.25, 1e-4, np.zeros(70000), "u8")
    assert e.value.status == -2


def test_capacity_overflow_keeps_first_candidates_in_order():
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=64, nsamp=8000, ndm=32)
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, _ = synth.make_block(wl, seed=4, delays=delays)
    full = run_plan(wl, block, nsigma=1.0)
    part = run_plan(wl, block, nsigma=1.0, capacity=100)
    assert full["total"] == part["total"] > 100
    assert np.array_equal(part["cands"], full["cands"][:100])
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8") as plan:
        out = plan.execute(_to_dev(block))
        cands = torch.empty((10, 16), dtype=torch.uint8, device=DEV)
        st, total = dd.dd_detect(plan.handle, out, out.shape[1], 1.0, cands, 10)
        assert st == dd.DD_ERR_OVERFLOW and total == full["total"]
        st, total = dd.dd_detect(plan.handle, out, out.shape[1], 1.0, None, 0)
        assert total == full["total"]


def test_process_host_matches_device_path():
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=128, nsamp=9000, ndm=64)
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, _ = synth.make_block(wl, seed=5, delays=delays)
    dev = run_plan(wl, block, nsigma=3.0)
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8") as plan:
        host = torch.from_numpy(block).pin_memory()
        cands = np.zeros(1 << 16, dtype=dd.CANDIDATE_DTYPE)
        for _ in range(2):  # second call reuses the plan's buffers
            st, total = dd.dd_process_host(plan.handle, host, wl.nsamp, wl.nsamp, 3.0, cands,
                                           cands.size)
            assert st == 0 and total == dev["total"]
            assert np.array_equal(cands[:total], dev["cands"])


def test_add_pipe_probe_reports_positive_rates():
    ops, per_clk = dd._native.dd_measure_add_peak("fadd")
    assert ops > 1e12 and 16 <= per_clk <= 512


# ------------------------------------------------------- staged u8 kernel

STAGED_CASES = [
    # (workload, nchan, ndm, extra samples past maxshift, pitch pad)
    ("full_block_u8", 1024, 128, 1100, 0),
    ("full_block_u8", 1021, 100, 700, 16),
    ("full_block_u8", 1024, 2048, 3000, 0),
    ("lband_f32", 4096, 96, 1500, 32),
    ("full_block_u8", 1036, 64, 900, 0),   # last chunk holds 3 quads
    ("full_block_u8", 68, 64, 300, 0),     # last chunk holds 1 quad
]

# Geometries whose first DM tile builds rows from before sample 0 (window of
# the band-top channel starting at -16): (f_top MHz, channel width MHz,
# t_samp s, first DM, DM step, nchan, ndm)
SLACK_GEOMETRIES = [
    (559.74, 0.7752, 51.2e-6, 0.8816, 0.02105, 64, 100),
    (728.89, 5.5687, 64e-6, 0.917, 0.00745, 16, 40),
]


@pytest.mark.parametrize("name,nchan,ndm,extra,pad", STAGED_CASES)
def test_staged_kernel_matches_oracle_and_plain_kernel(name, nchan, ndm, extra, pad):
    base = synth.workload(name)
    wl = synth.scaled(base, nchan=nchan, ndm=ndm)
    wl.chan_width_mhz = base.chan_width_mhz
    wl.dtype = "u8"
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    nsamp = mx + extra
    pitch = (nsamp + 15) // 16 * 16 + pad
    rng = np.random.default_rng(77)
    block = synth.random_block(rng, wl.nchan, nsamp, "u8", pitch)
    block[:, nsamp:] = 0xEE
    dblock = _to_dev(block)
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8") as plan:
        info = dd._native.dd_plan_kernel_info(plan.handle, dblock, pitch)
        assert info["staged"], info
        staged = plan.execute(dblock, nsamp_in=nsamp)
        dd._native.dd_plan_set_path(plan.handle, 1)
        assert not dd._native.dd_plan_kernel_info(plan.handle, dblock, pitch)["staged"]
        plain = plan.execute(dblock, nsamp_in=nsamp)
        dd.dd_sync(plan.handle)
        s, p = staged.cpu().numpy(), plain.cpu().numpy()
    assert np.array_equal(s, p)
    rows = sorted(set([0, ndm - 1] + np.random.default_rng(1).integers(0, ndm, 12).tolist()))
    ref = oracle.dedisperse(block, delays[:, rows], nsamp_out=s.shape[1], nsamp_in=nsamp)
    assert np.array_equal(s[rows], ref)


@pytest.mark.parametrize("geo", SLACK_GEOMETRIES)
def test_staged_kernel_row_origin_before_first_sample(geo):
    f_top, df, ts, dm0, step, nchan, ndm = geo
    dms = dm0 + step * np.arange(ndm)
    delays, mx = oracle.delay_table(nchan, f_top, df, ts, dms)
    nsamp = mx + 1300
    pitch = (nsamp + 15) // 16 * 16
    block = synth.random_block(np.random.default_rng(4), nchan, nsamp, "u8", pitch)
    dblock = _to_dev(block)
    with dd.Plan(nchan, f_top, df, ts, dms, "u8") as plan:
        assert dd._native.dd_plan_kernel_info(plan.handle, dblock, pitch)["staged"]
        out = plan.execute(dblock, nsamp_in=nsamp)
        dd.dd_sync(plan.handle)
        got = out.cpu().numpy()
    assert np.array_equal(got, oracle.dedisperse(block, delays, nsamp_in=nsamp))


def test_staged_kernel_16_trial_tiles_on_wide_channels():
    """256 channels of 62.5 kHz in the 400-416 MHz band: relative delays vary
    too much for 64- or 32-trial tiles, so the plan takes 16-trial tiles."""
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=256, ndm=300)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    nsamp = mx + 1500
    pitch = (nsamp + 15) // 16 * 16
    block = synth.random_block(np.random.default_rng(8), wl.nchan, nsamp, "u8", pitch)
    dblock = _to_dev(block)
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8") as plan:
        info = dd._native.dd_plan_kernel_info(plan.handle, dblock, pitch)
        assert info["staged"] and info["dms_per_cta"] == 16, info
        out, cands, total = plan.run(dblock, 3.0, nsamp_in=nsamp)
        mean, sigma = plan.stats()
        got = out.cpu().numpy()
    ref = oracle.dedisperse(block, delays, nsamp_in=nsamp)
    assert np.array_equal(got, ref)
    m, s = oracle.stats(ref)
    assert np.array_equal(mean, m) and np.array_equal(sigma, s)
    c, t = oracle.detect(ref, m, s, 3.0)
    assert total == t and np.array_equal(cands, c)


def test_staged_kernel_bounded_wait_reports_timeout_and_recovers():
    """Fault injection: the staged kernel queues no copies, so its first
    bounded wait (50 ms) runs out; the launch reports DD_ERR_DEVICE_TIMEOUT
    through dd_sync, the context stays usable, and the next launch is exact."""
    base = synth.workload("full_block_u8")
    wl = synth.scaled(base, nchan=256, ndm=64)
    wl.chan_width_mhz = base.chan_width_mhz
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    nsamp = mx + 2000
    pitch = (nsamp + 15) // 16 * 16
    block = synth.random_block(np.random.default_rng(3), wl.nchan, nsamp, "u8", pitch)
    dblock = _to_dev(block)
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8") as plan:
        assert dd._native.dd_plan_kernel_info(plan.handle, dblock, pitch)["staged"]
        dd._native.dd_plan_set_wait_timeout(plan.handle, 50_000_000)
        dd._native.dd_plan_inject_fault(plan.handle, 1)
        plan.execute(dblock, nsamp_in=nsamp)
        with pytest.raises(dd.DDError) as e:
            dd.dd_sync(plan.handle)
        assert e.value.status == -7
        dd._native.dd_plan_inject_fault(plan.handle, 0)
        out = plan.execute(dblock, nsamp_in=nsamp)
        dd.dd_sync(plan.handle)
        got = out.cpu().numpy()
    assert np.array_equal(got, oracle.dedisperse(block, delays, nsamp_in=nsamp))


# ----------------------------------------------------- staged f16/f32 kernel

FLOAT_STAGED_CASES = [
    # (workload, nchan, ndm, samples past maxshift, pitch pad, dtype)
    ("lband_f32", 1024, 96, 1500, 0, "f32"),
    ("lband_f32", 1021, 70, 700, 8, "f16"),     # padding channels, pitch padding
    ("lband_f32", 4096, 128, 900, 0, "f16"),
    ("full_block_u8", 512, 64, 1000, 16, "f32"),
]


@pytest.mark.parametrize("name,nchan,ndm,extra,pad,dtype", FLOAT_STAGED_CASES)
def test_staged_float_kernel_matches_oracle_and_plain_kernel(name, nchan, ndm, extra, pad, dtype):
    base = synth.workload(name)
    wl = synth.scaled(base, nchan=nchan, ndm=ndm)
    wl.chan_width_mhz = base.chan_width_mhz
    wl.dtype = dtype
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    nsamp = mx + extra
    pitch = (nsamp + 7) // 8 * 8 + pad
    block = synth.random_block(np.random.default_rng(21), wl.nchan, nsamp, dtype, pitch)
    block[:, nsamp:] = 1e4  # row padding must never reach a stored output
    dblock = _to_dev(block)
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, dtype) as plan:
        assert dd._native.dd_plan_kernel_info(plan.handle, dblock, pitch)["staged"]
        staged = plan.execute(dblock, nsamp_in=nsamp)
        dd._native.dd_plan_set_path(plan.handle, 1)
        plain = plan.execute(dblock, nsamp_in=nsamp)
        dd.dd_sync(plan.handle)
        s, p = staged.cpu().numpy(), plain.cpu().numpy()
    ref = oracle.dedisperse(block[:, :nsamp], delays)
    err_s = float_rel_err(block[:, :nsamp], delays, s, ref)
    err_p = float_rel_err(block[:, :nsamp], delays, p, ref)
    print(f"{name} {dtype} {nchan}x{ndm}: staged {err_s:.2e}, plain {err_p:.2e}")
    assert err_s <= FLOAT_RTOL and err_p <= FLOAT_RTOL


def test_staged_float_kernel_bounded_wait_reports_timeout_and_recovers():
    base = synth.workload("lband_f32")
    wl = synth.scaled(base, nchan=256, ndm=64)
    wl.chan_width_mhz = base.chan_width_mhz
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    nsamp = mx + 2000
    pitch = (nsamp + 7) // 8 * 8
    block = synth.random_block(np.random.default_rng(3), wl.nchan, nsamp, "f32", pitch)
    dblock = _to_dev(block)
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "f32") as plan:
        assert dd._native.dd_plan_kernel_info(plan.handle, dblock, pitch)["staged"]
        dd._native.dd_plan_set_wait_timeout(plan.handle, 50_000_000)
        dd._native.dd_plan_inject_fault(plan.handle, 1)
        plan.execute(dblock, nsamp_in=nsamp)
        with pytest.raises(dd.DDError) as e:
            dd.dd_sync(plan.handle)
        assert e.value.status == -7
        dd._native.dd_plan_inject_fault(plan.handle, 0)
        out = plan.execute(dblock, nsamp_in=nsamp)
        dd.dd_sync(plan.handle)
        got = out.cpu().numpy()
    ref = oracle.dedisperse(block[:, :nsamp], delays)
    assert float_rel_err(block[:, :nsamp], delays, got, ref) <= FLOAT_RTOL
