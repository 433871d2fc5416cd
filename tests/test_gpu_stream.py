"""GPU: streams (blocks pushed one after another, overlap tail on the device).

Concatenated push outputs must equal one dd_run over the whole signal with
maxshift zero samples in front (bit-exact, also for float input: the
summation order per output does not depend on where a time tile starts), each
push's candidates must equal the oracle's for that push's output and
statistics, and a wave of several streams must give each stream the results
it gets alone.
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


def narrow(name, nchan, ndm, dtype):
    base = synth.workload(name)
    wl = synth.scaled(base, nchan=nchan, ndm=ndm)
    wl.chan_width_mhz = base.chan_width_mhz
    wl.dtype = dtype
    return wl


def plan_of(wl):
    return dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, wl.dtype)


def signal(wl, nsamp, seed):
    return synth.random_block(np.random.default_rng(seed), wl.nchan, nsamp, wl.dtype)


@pytest.mark.parametrize("name,nchan,ndm,dtype,block", [
    ("full_block_u8", 512, 128, "u8", 4096),
    ("full_block_u8", 256, 96, "u8", 1000),      # block shorter than a time tile
    ("lband_f32", 512, 130, "f32", 3000),
    ("lband_f32", 256, 64, "f16", 2048),
])
def test_stream_pushes_concatenate_to_one_run(name, nchan, ndm, dtype, block):
    wl = narrow(name, nchan, ndm, dtype)
    pushes = 5
    with plan_of(wl) as plan:
        mx = plan.maxshift
        sig = signal(wl, pushes * block, seed=12)
        outs = []
        with dd.Stream(plan, block) as st:
            for k in range(pushes):
                piece = np.ascontiguousarray(sig[:, k * block:(k + 1) * block])
                blk = torch.from_numpy(piece).to(DEV)
                out, cands, total = st.push(blk, 4.0)
                d = out.cpu().numpy()
                outs.append(d)
                if dtype == "u8":  # candidates from this push's own statistics
                    mean, sigma = oracle.stats(d)
                    c, t = oracle.detect(d, mean, sigma, 4.0)
                    assert total == t and np.array_equal(cands, c)
        # the whole signal behind maxshift zeros, 16-byte pitch (staged kernel)
        n_all = mx + pushes * block
        per16 = 16 // sig.dtype.itemsize
        full = np.zeros((nchan, (n_all + per16 - 1) // per16 * per16), dtype=sig.dtype)
        full[:, mx:n_all] = sig
        dfull = torch.from_numpy(full).to(DEV)
        assert dd._native.dd_plan_kernel_info(plan.handle, dfull, full.shape[1])["staged"]
        ref = plan.run(dfull, 4.0, nsamp_in=n_all)[0].cpu().numpy()
    got = np.concatenate(outs, axis=1)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)
    if dtype == "u8":
        delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s,
                                       wl.dms)
        rows = [0, ndm // 2, ndm - 1]
        assert np.array_equal(got[rows], oracle.dedisperse(full[:, :n_all], delays[:, rows]))


def test_wave_of_streams_matches_each_stream_alone():
    wls = [narrow("full_block_u8", 512, 128, "u8"), narrow("full_block_u8", 1024, 64, "u8"),
           narrow("lband_f32", 256, 70, "f32")]
    wide = synth.scaled(synth.workload("single_beam_f32"), nsamp=4096)
    wide.dtype = "u8"  # plain-load kernel
    wls.append(wide)
    blocks_n = [3000, 2048, 2500, 1500]
    pushes = 3
    sigs = [signal(w, pushes * b, seed=20 + i) for i, (w, b) in enumerate(zip(wls, blocks_n))]

    def run(together):
        plans = [plan_of(w) for w in wls]
        streams = [dd.Stream(p, b) for p, b in zip(plans, blocks_n)]
        res = [[] for _ in wls]
        for k in range(pushes):
            blks = [torch.from_numpy(np.ascontiguousarray(s[:, k * b:(k + 1) * b])).to(DEV)
                    for s, b in zip(sigs, blocks_n)]
            if together:
                outs, cands, totals = dd.push_streams(streams, blks, 3.0)
            else:
                outs, cands, totals = zip(*[st.push(b, 3.0) for st, b in zip(streams, blks)])
            for i in range(len(wls)):
                res[i].append((outs[i].cpu().numpy(), cands[i], totals[i]))
        for st in streams:
            st.close()
        for p in plans:
            p.close()
        return res

    alone, mixed = run(False), run(True)
    for i in range(len(wls)):
        for (oa, ca, ta), (om, cm, tm) in zip(alone[i], mixed[i]):
            assert np.array_equal(oa, om) and ta == tm and np.array_equal(ca, cm), i


def test_stream_memory_model_covers_its_buffers():
    wl = narrow("full_block_u8", 1024, 256, "u8")
    with plan_of(wl) as plan:
        block = 19531
        need = dd.Stream.bytes_needed(plan, block)
        free0, _ = torch.cuda.mem_get_info()
        with dd.Stream(plan, block):
            free1, _ = torch.cuda.mem_get_info()
        # the stream itself holds its double buffer (the rest is the caller's
        # output and the plan's workspace, also in the model)
        assert 0 < free0 - free1 <= need
        assert need >= 2 * wl.nchan * (plan.maxshift + block)


def test_full_size_serving_mix_sampled_rows():
    """The 64-beam serving mix the bench runs (same generator and seed), two
    consecutive 1 s blocks pushed as one wave each; every beam checked on two
    sampled DM rows against the oracle over its whole signal (maxshift zeros,
    then both blocks)."""
    import bench
    wls = bench.serving_workloads(1)
    assert len(wls) == 64
    plans = [plan_of(w) for w in wls]
    streams = [dd.Stream(p, w.nsamp) for p, w in zip(plans, wls)]
    rng = np.random.default_rng(5)
    sigs = [synth.random_block(rng, w.nchan, 2 * w.nsamp, "u8") for w in wls]
    results = [[] for _ in wls]
    for k in range(2):
        blks = [torch.from_numpy(np.ascontiguousarray(s[:, k * w.nsamp:(k + 1) * w.nsamp]))
                .to(DEV) for s, w in zip(sigs, wls)]
        outs, _, _ = dd.push_streams(streams, blks, 6.0, capacity=1 << 18)
        for i in range(len(wls)):
            results[i].append(outs[i])
    for i, (w, p) in enumerate(zip(wls, plans)):
        mx = p.maxshift
        full = np.zeros((w.nchan, mx + 2 * w.nsamp), dtype=np.uint8)
        full[:, mx:] = sigs[i]
        rows = rng.choice(w.ndm, 2, replace=False)
        ref = oracle.dedisperse(full, np.ascontiguousarray(p.delays()[:, rows]),
                                nsamp_out=2 * w.nsamp)
        got = torch.cat([r[torch.as_tensor(rows, device=DEV)] for r in results[i]],
                        dim=1).cpu().numpy()
        assert got.shape == ref.shape and np.array_equal(got, ref), i
    for st in streams:
        st.close()
    for p in plans:
        p.close()
