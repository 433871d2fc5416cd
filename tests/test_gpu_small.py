"""GPU: dd_run in one launch for small float beams (the single-beam
functional-test shape of Sec. 2.4, and any small float beam that the staged
float kernel does not take).

The one-launch path runs the plain-load kernel's sums, the per-tile partial
statistics, the row statistics (Sec. 3.5) and the candidate extraction
(Sec. 3.6) in one cooperative launch with a grid barrier.  It uses the same
device arithmetic as the multi-launch plain-kernel path (dd_run on a plan
held to the plain-load kernel, itself pinned to the oracle in
test_gpu_run.py), so outputs, statistics and candidates must equal that
path's bit for bit; the single-beam case is also checked against the oracle.
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


def single_beam(dtype="f32", ndm=None, nchan=None):
    wl = synth.workload("single_beam_f32")
    wl.dtype = dtype
    if ndm is not None or nchan is not None:
        wl = synth.scaled(wl, nchan=nchan or wl.nchan, ndm=ndm or wl.ndm)
        wl.chan_width_mhz = 0.25
        wl.dtype = dtype
    return wl


def plan_of(wl, path=0):
    p = dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, wl.dtype)
    if path:
        dd._native.dd_plan_set_path(p.handle, path)
    return p


def run(plan, dblock, nsamp_in, nsigma, capacity):
    n_out = plan.nsamp_out(nsamp_in)
    out = torch.full((plan.ndm, n_out), -7.0, dtype=torch.float32, device=DEV)
    cands = torch.zeros((max(capacity, 1), 16), dtype=torch.uint8, device=DEV)
    before = plan.launch_count()
    st, total = dd.dd_run(plan.handle, dblock, nsamp_in, dblock.stride(0), out, nsigma,
                          cands if capacity else None, capacity)
    launches = plan.launch_count() - before
    mean, sigma = plan.stats()
    k = min(total, capacity)
    c = cands[:k].cpu().numpy().view(dd.CANDIDATE_DTYPE).reshape(-1)
    return {"st": st, "total": total, "out": out, "cands": c, "mean": mean, "sigma": sigma,
            "launches": launches}


def assert_identical(a, b):
    assert a["st"] == b["st"] and a["total"] == b["total"]
    assert torch.equal(a["out"], b["out"])
    assert np.array_equal(a["cands"], b["cands"])
    assert np.array_equal(a["mean"], b["mean"]) and np.array_equal(a["sigma"], b["sigma"])


def both(wl, block, nsamp_in, nsigma, capacity=1 << 16):
    dblock = torch.from_numpy(np.ascontiguousarray(block)).to(DEV)
    with plan_of(wl) as p0, plan_of(wl, path=1) as p1:
        one = run(p0, dblock, nsamp_in, nsigma, capacity)
        multi = run(p1, dblock, nsamp_in, nsigma, capacity)
    assert one["launches"] == 1, one["launches"]
    assert multi["launches"] >= 3, multi["launches"]
    return one, multi


CASES = [
    # (dtype, nchan, ndm, samples past maxshift, pitch pad, nsigma)
    ("f32", 64, 64, None, 0, 5.0),       # the single-beam geometry as given
    ("f16", 64, 64, None, 0, 3.0),
    ("f32", 64, 61, 1001, 1, 2.0),       # ragged trials and tail, unaligned pitch
    ("f32", 200, 1000, 700, 3, 3.0),     # more rows than CTAs: rows per row worker > 1
    ("f32", 64, 64, 300, 0, -1.0),       # every sample a candidate
    ("f32", 64, 64, 300, 0, 1e9),        # none
    ("f16", 129, 37, 5000, 5, 2.5),      # channels past one delay stage of 64
]


@pytest.mark.parametrize("dtype,nchan,ndm,extra,pad,nsigma", CASES)
def test_one_launch_equals_the_multi_launch_path(dtype, nchan, ndm, extra, pad, nsigma):
    wl = single_beam(dtype, ndm=ndm, nchan=nchan)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    nsamp = wl.nsamp if extra is None else mx + extra
    pitch = nsamp + pad
    while pad and (pitch * (2 if dtype == "f16" else 4)) % 16 == 0:
        pitch += 1  # rows off the 16-byte grid: the staged float kernel cannot take them
    block = synth.random_block(np.random.default_rng(7), wl.nchan, nsamp, dtype, pitch)
    if pad:
        block[:, nsamp:] = 1e4  # row padding must never reach an output or a statistic
    one, multi = both(wl, block, nsamp, nsigma, capacity=1 << 20)
    assert_identical(one, multi)
    if nsigma < 0:
        assert one["total"] > one["out"].numel() // 2
    if nsigma > 100:
        assert one["total"] == 0


def test_one_launch_single_beam_against_the_oracle():
    """Statistics and candidates (set, order, value, snr) of the single-beam
    block with its pulse, against the FP64 oracle (Sec. 3.5, 3.6)."""
    from tests.test_gpu_parity import assert_detection
    wl = single_beam("f32")
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, pulses = synth.make_block(wl, seed=2, delays=delays)
    dblock = torch.from_numpy(block).to(DEV)
    with plan_of(wl) as p:
        r = run(p, dblock, wl.nsamp, 5.0, 1 << 16)
    assert r["launches"] == 1
    from tests.test_gpu_parity import FLOAT_RTOL, float_rel_err
    ref = oracle.dedisperse(block, delays)
    assert float_rel_err(block, delays, r["out"].cpu().numpy(), ref) <= FLOAT_RTOL
    res = {"D": r["out"].cpu().numpy(), "cands": r["cands"], "total": r["total"],
           "mean": r["mean"], "sigma": r["sigma"]}
    assert_detection(wl, ref, res, 5.0, block, delays)
    p0 = pulses[0]
    hit = (r["cands"]["dm_idx"] == p0.dm_idx) & (r["cands"]["t"] >= p0.t0) & \
        (r["cands"]["t"] < p0.t0 + p0.width)
    assert hit.any()


def test_one_launch_capacity_overflow_keeps_the_first_candidates():
    wl = single_beam("f32")
    block = synth.random_block(np.random.default_rng(9), wl.nchan, wl.nsamp, "f32")
    full, _ = both(wl, block, wl.nsamp, 1.0, capacity=1 << 20)
    assert full["total"] > 200
    cut, multi = both(wl, block, wl.nsamp, 1.0, capacity=100)
    assert cut["st"] == dd._native.DD_ERR_OVERFLOW and cut["total"] == full["total"]
    assert np.array_equal(cut["cands"], full["cands"][:100])
    assert_identical(cut, multi)
    none, _ = both(wl, block, wl.nsamp, 1.0, capacity=0)
    assert none["total"] == full["total"] and none["cands"].size == 0


def test_one_launch_repeats_and_changing_sizes():
    """The grid barrier's arrivals counter and the launch epochs of the
    published row counts carry over launches of different grid sizes on one
    plan: every run equals a fresh multi-launch run."""
    wl = single_beam("f32")
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    rng = np.random.default_rng(11)
    sizes = [wl.nsamp, mx + 300, wl.nsamp, mx + 2000]
    blocks = {n: torch.from_numpy(synth.random_block(rng, wl.nchan, n, "f32")).to(DEV)
              for n in set(sizes)}
    with plan_of(wl) as p0, plan_of(wl, path=1) as p1:
        want = {n: run(p1, b, n, 3.0, 1 << 16) for n, b in blocks.items()}
        for i in range(30):
            n = sizes[i % len(sizes)]
            got = run(p0, blocks[n], n, 3.0, 1 << 16)
            assert got["launches"] == 1
            assert_identical(got, want[n])


def test_one_launch_wait_that_runs_out_is_reported_and_recovered():
    """With the plan's fault injection on, the grid barrier waits for
    one arrival more than the grid makes: every row worker's wait runs out
    after the plan's bound, records the status and returns, no total is
    stored, and dd_run returns DD_ERR_DEVICE_TIMEOUT (no device fault, no
    hang).  The next run without injection gives the full result again (the
    host resets the barrier counter)."""
    wl = single_beam("f32")
    block = synth.random_block(np.random.default_rng(13), wl.nchan, wl.nsamp, "f32")
    dblock = torch.from_numpy(block).to(DEV)
    with plan_of(wl) as p0, plan_of(wl, path=1) as p1:
        want = run(p1, dblock, wl.nsamp, 3.0, 1 << 16)
        assert_identical(run(p0, dblock, wl.nsamp, 3.0, 1 << 16), want)
        for _ in range(3):
            dd._native.dd_plan_set_wait_timeout(p0.handle, 1_000_000)
            dd._native.dd_plan_inject_fault(p0.handle, 1)
            with pytest.raises(dd.DDError) as e:
                run(p0, dblock, wl.nsamp, 3.0, 1 << 16)
            assert e.value.status == dd._native.DD_ERR_DEVICE_TIMEOUT
            dd._native.dd_plan_inject_fault(p0.handle, 0)
            dd._native.dd_plan_set_wait_timeout(p0.handle, 2_000_000_000)
            assert_identical(run(p0, dblock, wl.nsamp, 3.0, 1 << 16), want)


def test_batch_with_a_small_float_beam_equals_it_alone():
    """dd_batch_run takes the multi-launch plain-kernel path for such a beam;
    its results equal dd_run's one launch bit for bit."""
    wl = single_beam("f32")
    block = synth.random_block(np.random.default_rng(17), wl.nchan, wl.nsamp, "f32")
    dblock = torch.from_numpy(block).to(DEV)
    with plan_of(wl) as p:
        alone = run(p, dblock, wl.nsamp, 3.0, 1 << 16)
        assert alone["launches"] == 1
        b = dd.Batch([p])
        outs, cands, totals = b.run([dblock], 3.0, capacity=1 << 16)
        mean, sigma = p.stats()
        assert totals[0] == alone["total"]
        assert torch.equal(outs[0], alone["out"])
        assert np.array_equal(cands[0], alone["cands"])
        assert np.array_equal(mean, alone["mean"]) and np.array_equal(sigma, alone["sigma"])
        b.close()
