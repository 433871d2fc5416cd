"""GPU: dd_run (dedispersion + detection in one call) against the separate
dd_execute + dd_detect calls, which the parity tests pin to the oracle, and
directly against the oracle on reduced shapes.

With the staged u8 kernel, dd_run takes each row's sums and tile maxima from
the dedispersion kernel and reads the output only in tiles that can hold a
candidate; everything it returns must still be bit-identical.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1401_8258_gb300 as dd
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    dd.build()
    oracle.build()


def both_paths(wl, block, nsigma, capacity=1 << 16, nsamp_in=None, expect_staged=True):
    """(separate calls, dd_run) results for the same device block."""
    nchan, pitch = block.shape
    nsamp_in = pitch if nsamp_in is None else nsamp_in
    dblock = torch.from_numpy(np.ascontiguousarray(block)).to(DEV)
    res = []
    with dd.Plan(nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, wl.dtype) as plan:
        info = dd._native.dd_plan_kernel_info(plan.handle, dblock, pitch)
        assert bool(info["staged"]) == expect_staged, info
        n_out = plan.nsamp_out(nsamp_in)
        cap = max(capacity, 1)
        for fused in (False, True):
            out = torch.full((wl.ndm, n_out), -7, dtype=plan.out_torch_dtype, device=DEV)
            cands = torch.zeros((cap, 16), dtype=torch.uint8, device=DEV)
            if fused:
                st, total = dd.dd_run(plan.handle, dblock, nsamp_in, pitch, out, nsigma,
                                      cands if capacity else None, capacity)
            else:
                dd.dd_execute(plan.handle, dblock, nsamp_in, pitch, out)
                st, total = dd.dd_detect(plan.handle, out, n_out, nsigma,
                                         cands if capacity else None, capacity)
            mean, sigma = plan.stats()
            k = min(total, capacity)
            c = cands[:k].cpu().numpy().view(dd.CANDIDATE_DTYPE).reshape(-1)
            res.append({"st": st, "total": total, "out": out, "cands": c, "mean": mean,
                        "sigma": sigma})
    return res


def assert_same(a, b):
    assert a["st"] == b["st"] and a["total"] == b["total"]
    assert torch.equal(a["out"], b["out"])
    assert np.array_equal(a["cands"], b["cands"])
    assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["sigma"], b["sigma"])


def test_run_full_block_u8_full_size_matches_separate_calls():
    wl = synth.workload("full_block_u8")
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, pulses = synth.make_block(wl, seed=1, delays=delays)
    sep, run = both_paths(wl, block, 6.0, capacity=1 << 20)
    assert_same(sep, run)
    assert run["total"] > 0
    for p in pulses:
        hit = (run["cands"]["dm_idx"] == p.dm_idx) & (run["cands"]["t"] >= p.t0) & \
            (run["cands"]["t"] < p.t0 + p.width)
        assert hit.any(), p


CASES = [
    # (nchan, ndm, samples past maxshift, pitch pad, nsigma)
    (1024, 128, 3000, 0, 6.0),
    (1021, 100, 1700, 16, 3.0),     # ragged channels, pitch padding, ragged last tile
    (512, 70, 513, 0, -1.0),        # every tile holds candidates
    (256, 64, 900, 32, 1e9),        # none
    (68, 64, 600, 0, 2.5),          # last chunk holds one quad
]


@pytest.mark.parametrize("nchan,ndm,extra,pad,nsigma", CASES)
def test_run_matches_oracle_and_separate_calls(nchan, ndm, extra, pad, nsigma):
    base = synth.workload("full_block_u8")
    wl = synth.scaled(base, nchan=nchan, ndm=ndm)
    wl.chan_width_mhz = base.chan_width_mhz
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    wl.nsamp = mx + extra
    block, _ = synth.make_block(wl, seed=9, delays=delays)
    pitch = (wl.nsamp + 15) // 16 * 16 + pad
    padded = np.zeros((nchan, pitch), dtype=np.uint8)
    padded[:, :wl.nsamp] = block
    padded[:, wl.nsamp:] = 0xEE  # row padding must never reach a stored output
    sep, run = both_paths(wl, padded, nsigma, capacity=1 << 20, nsamp_in=wl.nsamp)
    assert_same(sep, run)
    ref = oracle.dedisperse(block, delays)
    assert np.array_equal(run["out"].cpu().numpy(), ref)
    mean, sigma = oracle.stats(ref)
    assert np.array_equal(run["mean"], mean) and np.array_equal(run["sigma"], sigma)
    cands, total = oracle.detect(ref, mean, sigma, nsigma)
    assert run["total"] == total
    assert np.array_equal(run["cands"], cands)


def narrow(nchan, nsamp, ndm):
    """The top nchan channels of the 400-416 MHz band (staged-kernel geometry)."""
    base = synth.workload("full_block_u8")
    wl = synth.scaled(base, nchan=nchan, nsamp=nsamp, ndm=ndm)
    wl.chan_width_mhz = base.chan_width_mhz
    return wl


def test_run_capacity_overflow_keeps_first_candidates_in_order():
    wl = narrow(64, 8000, 32)
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, _ = synth.make_block(wl, seed=4, delays=delays)
    sep, run = both_paths(wl, block, 1.0, capacity=100)
    assert_same(sep, run)
    assert run["st"] == dd.DD_ERR_OVERFLOW and run["total"] > 100
    _, full = both_paths(wl, block, 1.0, capacity=1 << 20)
    assert np.array_equal(run["cands"], full["cands"][:100])
    _, none = both_paths(wl, block, 1.0, capacity=0)
    assert none["total"] == full["total"] and none["st"] == dd.DD_ERR_OVERFLOW


def test_run_constant_rows_have_no_candidates():
    wl = narrow(128, 6000, 64)
    block = np.full((wl.nchan, wl.nsamp), 77, dtype=np.uint8)
    sep, run = both_paths(wl, block, 0.0)
    assert_same(sep, run)
    assert run["total"] == 0 and np.all(run["sigma"] == 0.0)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_run_float_plan_on_the_plain_kernel_fuses_detection(dtype):
    """The single-beam geometry (64 wide channels, DM step 1) takes the
    plain-load kernel, which also keeps per-tile partial statistics for
    dd_run: output identical to dd_execute, statistics within 1e-6 of the
    separate pass, statistics and candidates against the FP64 oracle."""
    from tests.test_gpu_parity import assert_detection
    wl = synth.workload("single_beam_f32")
    wl.dtype = dtype
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, pulses = synth.make_block(wl, seed=2, delays=delays)
    sep, run = both_paths(wl, block, 5.0, expect_staged=False)
    assert torch.equal(sep["out"], run["out"]) and sep["st"] == run["st"]
    np.testing.assert_allclose(run["mean"], sep["mean"], rtol=1e-6, atol=1e-6 * np.sqrt(wl.nchan))
    np.testing.assert_allclose(run["sigma"], sep["sigma"], rtol=1e-6)
    ref = oracle.dedisperse(block, delays)
    res = {"D": run["out"].cpu().numpy(), "cands": run["cands"], "total": run["total"],
           "mean": run["mean"], "sigma": run["sigma"]}
    assert_detection(wl, ref, res, 5.0, block, delays)
    p = pulses[0]
    hit = (run["cands"]["dm_idx"] == p.dm_idx) & (run["cands"]["t"] >= p.t0) & \
        (run["cands"]["t"] < p.t0 + p.width)
    assert hit.any()


def test_run_records_the_phase_event():
    wl = narrow(256, 9000, 128)
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, _ = synth.make_block(wl, seed=3, delays=delays)
    dblock = torch.from_numpy(block).to(DEV)
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8") as plan:
        out = torch.empty((wl.ndm, plan.nsamp_out(wl.nsamp)), dtype=torch.int32, device=DEV)
        cands = torch.empty((1 << 12, 16), dtype=torch.uint8, device=DEV)
        start, mid = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        mid.record()  # creates the event
        start.record()
        dd.dd_run(plan.handle, dblock, wl.nsamp, wl.nsamp, out, 6.0, cands, 1 << 12,
                  torch.cuda.current_stream(), mid)
        end = torch.cuda.Event(enable_timing=True)
        end.record()
        torch.cuda.synchronize()
        assert 0.0 < start.elapsed_time(mid) <= start.elapsed_time(end)


@pytest.mark.parametrize("name,nchan,ndm,dtype", [
    ("full_block_u8", 1024, 256, "u8"),
    ("lband_f32", 1024, 256, "f32"),
    ("lband_f32", 512, 192, "f16"),
])
def test_autotune_keeps_results_identical(name, nchan, ndm, dtype):
    """The plan's tile width is chosen by timing; no width changes a result
    (integer sums are exact, and the float kernel's summation order per output
    does not depend on the tiling)."""
    base = synth.workload(name)
    wl = synth.scaled(base, nchan=nchan, ndm=ndm)
    wl.chan_width_mhz = base.chan_width_mhz
    wl.dtype = dtype
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    wl.nsamp = mx + 3000
    pitch = (wl.nsamp + 15) // 16 * 16
    block, _ = synth.make_block(wl, seed=6, delays=delays, pitch=pitch)
    dblock = torch.from_numpy(block).to(DEV)
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, dtype) as plan:
        assert dd._native.dd_plan_kernel_info(plan.handle, dblock, pitch)["staged"]
        before = plan.run(dblock, 4.0, nsamp_in=wl.nsamp)
        nd, ms = plan.autotune(wl.nsamp)
        assert nd in ((64, 32, 16) if dtype == "u8" else (128, 64)) and ms > 0
        print(f"{name} {dtype}: autotune chose {nd} trials per CTA ({ms:.3f} ms)")
        info = dd._native.dd_plan_kernel_info(plan.handle, dblock, pitch)
        assert info["staged"] and info["dms_per_cta"] == nd
        assert info["copy_ahead"] in ((1, 2, 3) if dtype == "u8" else (0,))
        print(f"  staging depth {info['copy_ahead']}")
        after = plan.run(dblock, 4.0, nsamp_in=wl.nsamp)
    assert torch.equal(before[0], after[0])
    assert before[2] == after[2] and np.array_equal(before[1], after[1])


@pytest.mark.parametrize("dtype,capacity", [("u8", 1 << 14), ("f32", 1 << 14), ("u8", 5)])
def test_host_pipe_results_equal_process_host_per_block(dtype, capacity):
    """dd_host_pipe: push k returns block k-1's candidates, flush the last
    block's; each equals dd_process_host of that block (candidates, total,
    statistics), also after a flush and with a capacity below the total."""
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=256, nsamp=24000, ndm=160)
    wl.dtype = dtype
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    blocks = [torch.from_numpy(synth.make_block(wl, seed=s, delays=delays)[0]).pin_memory()
              for s in (1, 2, 3)]
    nsigma = 4.0
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, dtype) as plan:
        want = []
        host = np.zeros(max(capacity, 1), dtype=dd.CANDIDATE_DTYPE)
        for b in blocks:
            st, total = dd.dd_process_host(plan.handle, b, wl.nsamp, wl.nsamp, nsigma, host,
                                           capacity)
            want.append((host[:min(total, capacity)].copy(), total, plan.stats()))
        assert want[0][1] > capacity or capacity > 5
        with dd.HostPipe(plan, wl.nsamp, wl.nsamp, nsigma, capacity) as pipe:
            got = [pipe.push(blocks[0])]
            got.append((pipe.push(blocks[1]), plan.stats()))
            got.append((pipe.push(blocks[2]), plan.stats()))
            got.append((pipe.flush(), plan.stats()))
            assert got[0] is None and pipe.flush() is None
            assert pipe.push(blocks[0]) is None  # the previous result went out with the flush
            got.append((pipe.flush(), plan.stats()))
    for (res, stats), (c, total, wstats) in zip(got[1:], want + [want[0]]):
        assert res is not None and res[1] == total
        assert np.array_equal(res[0], c)
        assert np.array_equal(stats[0], wstats[0]) and np.array_equal(stats[1], wstats[1])


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_staging_depths_give_identical_results(depth):
    """Each staging depth of the u8 kernel (input windows queued 1, 2 or 3
    chunks ahead) gives the oracle's output, statistics and candidates, alone
    and in a batch that mixes depths (one shared launch per depth)."""
    wl = synth.scaled(synth.workload("full_block_u8"), nchan=512, nsamp=30000, ndm=192)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, _ = synth.make_block(wl, seed=8, delays=delays)
    dblock = torch.from_numpy(block).to(DEV)
    ref = oracle.dedisperse(block, delays)
    m, sd = oracle.stats(ref)
    c_ref, tot = oracle.detect(ref, m, sd, 4.0)
    other = 1 + depth % 3
    with dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8") as p1, \
            dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8") as p2:
        dd._native.dd_plan_set_staging_depth(p1.handle, depth)
        dd._native.dd_plan_set_staging_depth(p2.handle, other)
        assert dd._native.dd_plan_kernel_info(p1.handle, dblock, wl.nsamp)["copy_ahead"] == depth
        out, cands, total = p1.run(dblock, 4.0)
        assert np.array_equal(out.cpu().numpy(), ref)
        assert total == tot and np.array_equal(cands, c_ref)
        mean, sigma = p1.stats()
        assert np.array_equal(mean, m) and np.array_equal(sigma, sd)
        batch = dd.Batch([p1, p2])
        outs, bc, totals = batch.run([dblock, dblock], 4.0)
        batch.close()
        for o, c, t in zip(outs, bc, totals):
            assert np.array_equal(o.cpu().numpy(), ref)
            assert t == tot and np.array_equal(c, c_ref)
        with pytest.raises(dd.DDError):
            dd._native.dd_plan_set_staging_depth(p1.handle, 4)
        # the timeout path at this depth: no copies queued, the wait runs out
        dd._native.dd_plan_set_wait_timeout(p1.handle, 50_000_000)
        dd._native.dd_plan_inject_fault(p1.handle, 1)
        with pytest.raises(dd.DDError) as e:
            p1.run(dblock, 4.0)
        assert e.value.status == -7
        dd._native.dd_plan_inject_fault(p1.handle, 0)
        out, cands, total = p1.run(dblock, 4.0)
        assert np.array_equal(out.cpu().numpy(), ref) and total == tot


FLOAT_CASES = [
    # (nchan, ndm, samples past maxshift, pitch pad, dtype, nsigma)
    (1024, 128, 1500, 0, "f32", 4.0),
    (1021, 70, 700, 8, "f16", 3.0),    # padding channels and trials, pitch padding, ragged tail
    (512, 64, 257, 0, "f32", -1.0),    # nearly every tile holds candidates
    (256, 64, 900, 0, "f32", 1e9),     # none
]


@pytest.mark.parametrize("nchan,ndm,extra,pad,dtype,nsigma", FLOAT_CASES)
def test_run_float_fused_statistics_and_candidates(nchan, ndm, extra, pad, dtype, nsigma):
    """dd_run on the staged float kernel keeps per-tile partial statistics in
    its epilogue and reads the output only in tiles that can hold a
    candidate.  Its output is dd_execute's bit for bit; its statistics agree
    with the separate statistics pass to 1e-6 (both FP64 evaluations of the
    same rows); statistics and candidates (set, order, value, snr) against the
    FP64 oracle as in the parity tests (Sec. 3.5, 3.6)."""
    from tests.test_gpu_parity import assert_detection
    base = synth.workload("lband_f32")
    wl = synth.scaled(base, nchan=nchan, ndm=ndm)
    wl.chan_width_mhz = base.chan_width_mhz
    wl.dtype = dtype
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    nsamp = mx + extra
    pitch = (nsamp + 7) // 8 * 8 + pad
    block = synth.random_block(np.random.default_rng(31), nchan, nsamp, dtype, pitch)
    block[:, nsamp:] = 1e4  # row padding must never reach an output or a statistic
    sep, run = both_paths(wl, block, nsigma, capacity=1 << 20, nsamp_in=nsamp)
    assert torch.equal(sep["out"], run["out"])
    np.testing.assert_allclose(run["mean"], sep["mean"], rtol=1e-6, atol=1e-6 * np.sqrt(nchan))
    np.testing.assert_allclose(run["sigma"], sep["sigma"], rtol=1e-6)
    ref = oracle.dedisperse(block[:, :nsamp], delays)
    res = {"D": run["out"].cpu().numpy(), "cands": run["cands"], "total": run["total"],
           "mean": run["mean"], "sigma": run["sigma"]}
    assert_detection(wl, ref, res, nsigma, block[:, :nsamp], delays)
    if nsigma > 100:
        assert run["total"] == 0
    if nsigma < 0:
        assert run["total"] > ref.size // 2
