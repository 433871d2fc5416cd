"""GPU: dd_batch_run over uneven beams against dd_run on each beam alone
(which the other GPU tests pin to the oracle), and directly against the
oracle on small beams.

The staged u8 beams of a batch share persistent launches (one per DM-tile
width) whose work queue interleaves the beams; each beam's output, statistics
and candidates must still be bit-identical to a run of that beam alone.
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


def maxshift(wl):
    _, m = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    return m


def small_batch(seed, n):
    return synth.batch_workloads(seed, maxshift, n=n, nchan_choices=(256, 512, 1024),
                                 nsamp_range=(16384, 24576), ndm_range=(128, 384))


def make_beams(workloads, seed):
    blocks, delays = [], []
    for i, wl in enumerate(workloads):
        d, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
        b, _ = synth.make_block(wl, seed + i, d)
        blocks.append(b)
        delays.append(d)
    return blocks, delays


def plan_of(wl):
    return dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, wl.dtype)


def run_alone(plan, dblock, nsigma, capacity):
    out, cands, total = plan.run(dblock, nsigma, capacity=capacity)
    mean, sigma = plan.stats()
    return out, cands, total, mean, sigma


def assert_batch_matches_alone(workloads, blocks, nsigma, capacity=1 << 16):
    dblocks = [torch.from_numpy(np.ascontiguousarray(b)).to(DEV) for b in blocks]
    plans = [plan_of(wl) for wl in workloads]
    alone = [run_alone(p, b, nsigma, capacity) for p, b in zip(plans, dblocks)]
    with dd.Batch(plans) as batch:
        for _ in range(2):  # a second run reuses every buffer
            outs, cands, totals = batch.run(dblocks, nsigma, capacity=capacity)
            for i, p in enumerate(plans):
                out_a, c_a, t_a, m_a, s_a = alone[i]
                assert totals[i] == t_a, i
                assert torch.equal(outs[i], out_a), i
                assert np.array_equal(cands[i], c_a), i
                mean, sigma = p.stats()
                assert np.array_equal(mean, m_a) and np.array_equal(sigma, s_a), i
    staged = [dd._native.dd_plan_kernel_info(p.handle, b, b.stride(0))["staged"]
              for p, b in zip(plans, dblocks)]
    for p in plans:
        p.close()
    return outs, cands, totals, staged


def test_batch_of_uneven_u8_beams_matches_each_beam_alone_and_the_oracle():
    workloads = small_batch(seed=3, n=7)
    blocks, delays = make_beams(workloads, seed=40)
    outs, cands, totals, staged = assert_batch_matches_alone(workloads, blocks, 5.0)
    assert sum(staged) >= 4  # the shared persistent launches carry most beams
    for i in (0, len(workloads) - 1):
        ref = oracle.dedisperse(blocks[i], delays[i])
        assert np.array_equal(outs[i].cpu().numpy(), ref)
        mean, sigma = oracle.stats(ref)
        c, t = oracle.detect(ref, mean, sigma, 5.0)
        assert totals[i] == t and np.array_equal(cands[i], c)


def test_mixed_batch_with_float_and_plain_kernel_beams():
    wls = small_batch(seed=5, n=3)
    f32 = synth.scaled(synth.workload("lband_f32"), nchan=512, nsamp=12000, ndm=96)
    f32.chan_width_mhz = synth.workload("lband_f32").chan_width_mhz
    wide = synth.scaled(synth.workload("single_beam_f32"), nsamp=4096)
    wide.dtype = "u8"  # 64 wide channels: no staged tables, plain-load kernel
    workloads = wls + [f32, wide]
    blocks, _ = make_beams(workloads, seed=70)
    _, _, _, staged = assert_batch_matches_alone(workloads, blocks, 4.0)
    assert staged[-1] == 0 and sum(staged) >= 3


def test_batch_capacity_overflow_keeps_each_beams_first_candidates():
    workloads = small_batch(seed=7, n=4)
    blocks, _ = make_beams(workloads, seed=90)
    dblocks = [torch.from_numpy(b).to(DEV) for b in blocks]
    plans = [plan_of(wl) for wl in workloads]
    full = [p.run(b, 1.5, capacity=1 << 20) for p, b in zip(plans, dblocks)]
    with dd.Batch(plans) as batch:
        outs = [torch.empty_like(f[0]) for f in full]
        cands = [torch.empty((50, 16), dtype=torch.uint8, device=DEV) for _ in plans]
        st, totals = dd.dd_batch_run(batch.handle, dblocks, [b.shape[1] for b in blocks],
                                     [b.shape[1] for b in blocks], outs, 1.5, cands,
                                     [50] * len(plans))
        assert st == dd.DD_ERR_OVERFLOW
        for i, f in enumerate(full):
            assert totals[i] == f[2] > 50
            got = cands[i].cpu().numpy().view(dd.CANDIDATE_DTYPE).reshape(-1)
            assert np.array_equal(got, f[1][:50])
    for p in plans:
        p.close()


def test_batch_bounded_wait_reports_timeout_and_recovers():
    """Fault injection on the host: the shared launch queues no copies, its
    first bounded wait (50 ms) runs out, the batch reports
    DD_ERR_DEVICE_TIMEOUT, and the next run is exact."""
    workloads = small_batch(seed=9, n=3)
    blocks, _ = make_beams(workloads, seed=110)
    dblocks = [torch.from_numpy(b).to(DEV) for b in blocks]
    plans = [plan_of(wl) for wl in workloads]
    alone = [p.run(b, 5.0) for p, b in zip(plans, dblocks)]
    # the shared launch takes its timeout and fault switch from the costliest
    # beam's plan (queued first); set them on every plan
    for p in plans:
        dd._native.dd_plan_set_wait_timeout(p.handle, 50_000_000)
        dd._native.dd_plan_inject_fault(p.handle, 1)
    with dd.Batch(plans) as batch:
        with pytest.raises(dd.DDError) as e:
            batch.run(dblocks, 5.0)
        assert e.value.status == -7
        for p in plans:
            dd._native.dd_plan_inject_fault(p.handle, 0)
        outs, cands, totals = batch.run(dblocks, 5.0)
        for i, a in enumerate(alone):
            assert torch.equal(outs[i], a[0]) and totals[i] == a[2]
            assert np.array_equal(cands[i], a[1])
    for p in plans:
        p.close()


def test_batch_replays_its_captured_graph_and_recaptures_on_change():
    workloads = small_batch(seed=13, n=5)
    blocks, _ = make_beams(workloads, seed=150)
    dblocks = [torch.from_numpy(np.ascontiguousarray(b)).to(DEV) for b in blocks]
    plans = [plan_of(wl) for wl in workloads]
    alone = [run_alone(p, b, 5.0, 1 << 16) for p, b in zip(plans, dblocks)]
    outs = [torch.empty_like(a[0]) for a in alone]
    with dd.Batch(plans) as batch:
        for rep in range(4):  # run, capture, then replays
            for o in outs:
                o.fill_(-1)
            got, cands, totals = batch.run(dblocks, 5.0, outs=outs)
            for i, a in enumerate(alone):
                assert torch.equal(got[i], a[0]) and totals[i] == a[2], (rep, i)
                assert np.array_equal(cands[i], a[1])
                mean, sigma = plans[i].stats()
                assert np.array_equal(mean, a[3]) and np.array_equal(sigma, a[4])
        assert batch.graph_replays() == 3
        # a new output array: run directly and capture again
        outs[0] = torch.empty_like(outs[0])
        got, _, totals = batch.run(dblocks, 5.0, outs=outs)
        assert torch.equal(got[0], alone[0][0]) and batch.graph_replays() == 3
        got, _, totals = batch.run(dblocks, 5.0, outs=outs)
        assert torch.equal(got[0], alone[0][0]) and batch.graph_replays() == 4
        # a plan's workspace reallocated by a longer block elsewhere: no stale replay
        big = torch.from_numpy(np.ascontiguousarray(
            np.tile(blocks[1], (1, 2)))).to(DEV)
        plans[1].run(big, 5.0)
        got, _, totals = batch.run(dblocks, 5.0, outs=outs)
        assert torch.equal(got[1], alone[1][0]) and totals[1] == alone[1][2]
        assert batch.graph_replays() == 4
    for p in plans:
        p.close()


def test_full_size_batch_of_32_beams_sampled_rows():
    """The 32-beam batch the bench times (same generator and seed), every
    beam checked on two sampled DM rows against the oracle: outputs exactly,
    and the candidates of those rows with the rows' own statistics."""
    import bench
    workloads = bench.batch_workloads(1)
    assert len(workloads) == 32
    plans = [plan_of(wl) for wl in workloads]
    rng = np.random.default_rng(77)
    blocks, dblocks, delays = [], [], []
    for i, (wl, p) in enumerate(zip(workloads, plans)):
        d = p.delays()
        b, _ = synth.make_block(wl, 1000 + i, d)
        blocks.append(b)
        dblocks.append(torch.from_numpy(b).to(DEV))
        delays.append(d)
    with dd.Batch(plans) as batch:
        outs, cands, totals = batch.run(dblocks, 6.0, capacity=1 << 20)
        assert max(totals) <= 1 << 20
        for i, wl in enumerate(workloads):
            rows = rng.choice(wl.ndm, 2, replace=False)
            ref = oracle.dedisperse(blocks[i], np.ascontiguousarray(delays[i][:, rows]),
                                    nsamp_out=outs[i].shape[1])
            got = outs[i][torch.as_tensor(rows, device=DEV)].cpu().numpy()
            assert np.array_equal(got, ref), i
            mean, sigma = oracle.stats(ref)
            c_ref, _ = oracle.detect(ref, mean, sigma, 6.0)
            g_mean, g_sigma = plans[i].stats()
            assert np.array_equal(g_mean[rows], mean) and np.array_equal(g_sigma[rows], sigma)
            for k, r in enumerate(rows):
                mine = cands[i][cands[i]["dm_idx"] == r]
                theirs = c_ref[c_ref["dm_idx"] == k]
                assert np.array_equal(mine["t"], theirs["t"]), (i, r)
                assert np.array_equal(mine["value"], theirs["value"]), (i, r)
    del outs, dblocks
    for p in plans:
        p.close()


def test_batch_of_mixed_widths_and_depths_is_one_launch_and_two_detection_launches():
    """Beams whose plans take 64-, 32- and 16-trial tiles and different
    staging depths share one persistent launch (the kernel dispatches on each
    beam's width; the batch runs at its most common depth), and their
    detection runs as two launches for all of them: at most three kernels per
    batch step, each beam's results still those of the beam alone."""
    base = synth.workload("full_block_u8")
    wide = synth.scaled(base, nchan=256, ndm=160)            # 62.5 kHz channels: 16 trials
    mid = synth.scaled(base, nchan=512, ndm=200)             # 31.25 kHz channels
    narrow = synth.scaled(base, nchan=512, ndm=200)
    narrow.chan_width_mhz = base.chan_width_mhz              # 15.6 kHz: 64 trials
    workloads = [wide, mid, narrow, synth.scaled(base, nchan=384, ndm=96)]
    for wl in workloads:
        wl.nsamp = (maxshift(wl) + 6000 + 15) // 16 * 16  # whole 16-byte rows: staged
    blocks, _ = make_beams(workloads, seed=41)
    dblocks = [torch.from_numpy(np.ascontiguousarray(b)).to(DEV) for b in blocks]
    plans = [plan_of(wl) for wl in workloads]
    infos = [dd._native.dd_plan_kernel_info(p.handle, b, b.stride(0))
             for p, b in zip(plans, dblocks)]
    assert all(i["staged"] for i in infos), infos
    widths = {i["dms_per_cta"] for i in infos}
    assert len(widths) >= 2, widths
    dd._native.dd_plan_set_staging_depth(plans[0].handle, 3)
    dd._native.dd_plan_set_staging_depth(plans[1].handle, 1)
    alone = [run_alone(p, b, 4.0, 1 << 16) for p, b in zip(plans, dblocks)]
    with dd.Batch(plans) as batch:
        batch.run(dblocks, 4.0)
        before = sum(p.launch_count() for p in plans)
        outs, cands, totals = batch.run(dblocks, 4.0)
        launches = sum(p.launch_count() for p in plans) - before
        for i in range(len(plans)):
            out_a, c_a, t_a, m_a, s_a = alone[i]
            assert totals[i] == t_a and torch.equal(outs[i], out_a)
            assert np.array_equal(cands[i], c_a)
            mean, sigma = plans[i].stats()
            assert np.array_equal(mean, m_a) and np.array_equal(sigma, s_a)
    assert launches <= 3, launches
    for p in plans:
        p.close()


def test_batch_of_float_beams_shares_float_kernel_launches():
    """Staged float beams of one input dtype and tile width share one
    persistent launch of the float kernel (its queue holds every beam's
    items); the results equal each beam alone bit for bit."""
    base = synth.workload("lband_f32")
    workloads = []
    for nchan, ndm, dtype in [(512, 96, "f32"), (256, 200, "f32"), (384, 64, "f32"),
                              (256, 128, "f16"), (512, 80, "f16")]:
        wl = synth.scaled(base, nchan=nchan, ndm=ndm)
        wl.chan_width_mhz = base.chan_width_mhz
        wl.dtype = dtype
        wl.nsamp = (maxshift(wl) + 5000 + 15) // 16 * 16  # whole 16-byte rows: staged
        workloads.append(wl)
    blocks, _ = make_beams(workloads, seed=77)
    dblocks = [torch.from_numpy(np.ascontiguousarray(b)).to(DEV) for b in blocks]
    plans = [plan_of(wl) for wl in workloads]
    infos = [dd._native.dd_plan_kernel_info(p.handle, b, b.stride(0)) for p, b in zip(plans, dblocks)]
    assert all(i["staged"] for i in infos), infos
    groups = {(wl.dtype, i["dms_per_cta"]) for wl, i in zip(workloads, infos)}
    alone = [run_alone(p, b, 4.0, 1 << 16) for p, b in zip(plans, dblocks)]
    with dd.Batch(plans) as batch:
        before = sum(p.launch_count() for p in plans)
        outs, cands, totals = batch.run(dblocks, 4.0, capacity=1 << 16)
        launches = sum(p.launch_count() for p in plans) - before
    # one dedispersion launch per (dtype, width) group; detection per float
    # beam: row statistics and counts, scan, write
    assert launches == len(groups) + 3 * len(plans), (launches, groups)
    for i, p in enumerate(plans):
        out_a, c_a, t_a, m_a, s_a = alone[i]
        assert totals[i] == t_a and torch.equal(outs[i], out_a), i
        assert np.array_equal(cands[i], c_a), i
        mean, sigma = p.stats()
        assert np.array_equal(mean, m_a) and np.array_equal(sigma, s_a), i
    for p in plans:
        p.close()
