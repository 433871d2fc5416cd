"""GPU: the continuous-batching server (paper_1401_8258_gb300.serve).

Beams of different geometries (8-bit and f32) join and leave while others run;
one waits for admission until a finished beam frees its memory; blocks
arrive from a host thread and are copied on the copy stream.  Every block's
candidates, total and dedispersed output must equal a solo stream run of that
beam over the same blocks, bit for bit -- the same result alone and in the
mix (Sec. 3.4, 3.8).  The stream path itself is pinned to the oracle in
test_gpu_stream.py; one beam is also checked against the oracle here.
"""
import threading
import time

import numpy as np
import pytest
import torch

import oracle
import paper_1401_8258_gb300 as dd
from paper_1401_8258_gb300.serve import Server
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
NSIGMA = 3.0


@pytest.fixture(scope="module", autouse=True)
def built():
    dd.build()
    oracle.build()


def beam(nchan, ndm, dtype, block, band):
    base = synth.workload("full_block_u8" if band == "A" else "lband_f32")
    wl = synth.scaled(base, nchan=nchan, ndm=ndm)
    wl.dtype = dtype
    plan = dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, dtype)
    assert plan.maxshift < block
    return wl, plan, block


def host_blocks(wl, n, block, seed):
    rng = np.random.default_rng(seed)
    return [torch.from_numpy(synth.random_block(rng, wl.nchan, block, wl.dtype)).pin_memory()
            for _ in range(n)]


def solo(plan, block, blocks):
    """The same blocks through a stream of the plan alone."""
    res = []
    with dd.Stream(plan, block) as s:
        for b in blocks:
            out, cands, total = s.push(b.to(DEV), NSIGMA)
            res.append((cands, total, out.cpu()))
    return res


def test_server_beams_join_and_leave_results_equal_solo_runs():
    specs = {
        "A": beam(256, 64, "u8", 4096, "A"),      # leaves after 3 blocks
        "B": beam(512, 128, "u8", 6000, "A"),
        "C": beam(256, 96, "f32", 5000, "B"),
        "D": beam(384, 64, "u8", 4096, "A"),      # joins late; waits for A's memory
        "E": beam(256, 64, "u8", 3000, "B"),      # joins last
    }
    nblocks = {"A": 3, "B": 6, "C": 5, "D": 4, "E": 3}
    blocks = {k: host_blocks(wl, nblocks[k], blk, seed=i)
              for i, (k, (wl, _, blk)) in enumerate(specs.items())}
    probe = Server(NSIGMA, capacity=1 << 14, mem_budget=1 << 40)
    size = {k: probe.beam_bytes(p, blk) for k, (_, p, blk) in specs.items()}
    probe.shutdown()
    # room for A, B and C together, not for D as well: D waits for A
    budget = size["A"] + size["B"] + size["C"] + size["E"] // 2
    assert size["D"] > size["E"] // 2 and budget >= max(size.values())

    with Server(NSIGMA, capacity=1 << 14, mem_budget=budget, keep_outputs=True) as srv:
        def feed():
            for k in "ABC":
                srv.open(k, specs[k][1], specs[k][2])
            for i in range(6):
                for k in "ABC":
                    if i < nblocks[k]:
                        srv.submit(k, blocks[k][i])
                if i == 2:
                    srv.close_beam("A")
                if i == 1:
                    srv.open("D", specs["D"][1], specs["D"][2])  # A still holds its memory
                    for b in blocks["D"]:
                        srv.submit("D", b)
                    srv.close_beam("D")
                if i == 3:
                    srv.open("E", specs["E"][1], specs["E"][2])
                    for b in blocks["E"]:
                        srv.submit("E", b)
                    srv.close_beam("E")
                time.sleep(0.02)
            srv.close_beam("B")
            srv.close_beam("C")

        t = threading.Thread(target=feed)
        t.start()
        t.join()
        srv.drain(timeout=120)
        results = {k: sorted(srv.results[k], key=lambda r: r.seq) for k in specs}
        waves = list(srv.waves)
        admissions = {k: (o, a) for k, o, a in srv.admissions}
        peak = srv.peak_used

    # every block processed once, in order, within the budget
    assert peak <= budget
    for k in specs:
        assert [r.seq for r in results[k]] == list(range(nblocks[k])), k
        assert all(r.latency > 0 for r in results[k])
    # continuous batching: beams shared waves
    assert max(n for n, _, _ in waves) >= 2
    # D was admitted only after A's last block was done (its memory released)
    a_last = max(r.done for r in results["A"])
    assert admissions["D"][1] >= a_last

    # the same result alone and in the mix
    for k, (wl, plan, blk) in specs.items():
        want = solo(plan, blk, blocks[k])
        for r, (cands, total, out) in zip(results[k], want):
            assert r.total == total, (k, r.seq)
            assert np.array_equal(r.candidates, cands), (k, r.seq)
            assert torch.equal(r.out, out), (k, r.seq)
        plan.close()

    # and one beam against the oracle: its stream output is the dedispersion
    # of the concatenated blocks (zeros before the first)
    wl, _, blk = specs["B"]
    sig = np.concatenate([b.numpy() for b in blocks["B"]], axis=1)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    padded = np.concatenate([np.zeros((wl.nchan, mx), dtype=sig.dtype), sig], axis=1)
    ref = oracle.dedisperse(padded, delays)
    got = np.concatenate([r.out.numpy() for r in results["B"]], axis=1)
    assert np.array_equal(got, ref[:, :got.shape[1]])


def test_server_per_beam_form_gives_the_same_results():
    """per_beam=True (one push per beam, the plain form the serving bench
    compares with) returns the same candidates as waves."""
    specs = {"P": beam(256, 64, "u8", 4096, "A"), "Q": beam(256, 96, "f32", 4096, "B")}
    blocks = {k: host_blocks(wl, 3, blk, seed=10 + i)
              for i, (k, (wl, _, blk)) in enumerate(specs.items())}
    got = {}
    for per_beam in (False, True):
        with Server(NSIGMA, capacity=1 << 14, per_beam=per_beam) as srv:
            for k, (_, p, blk) in specs.items():
                srv.open(k, p, blk)
            for i in range(3):
                for k in specs:
                    srv.submit(k, blocks[k][i])
            for k in specs:
                srv.close_beam(k)
            srv.drain(timeout=60)
            got[per_beam] = {k: sorted(srv.results[k], key=lambda r: r.seq) for k in specs}
            if per_beam:
                assert all(n == 1 for n, _, _ in srv.waves)
    for k in specs:
        for a, b in zip(got[False][k], got[True][k]):
            assert a.total == b.total and np.array_equal(a.candidates, b.candidates)
    for _, p, _ in specs.values():
        p.close()


def test_server_rejects_a_beam_over_the_budget_and_reports_bad_blocks():
    _, plan, blk = beam(256, 64, "u8", 4096, "A")
    with Server(NSIGMA, capacity=1 << 10, mem_budget=1 << 20) as srv:
        with pytest.raises(ValueError):
            srv.open("big", plan, blk)
    with Server(NSIGMA, capacity=1 << 10) as srv:
        srv.open("x", plan, blk)
        with pytest.raises(ValueError):
            srv.submit("x", np.zeros((255, blk), dtype=np.uint8))
        srv.close_beam("x")
        srv.drain(timeout=30)
    plan.close()
