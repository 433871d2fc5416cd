"""The N > 1 path of bench.py on the CPU: two gloo ranks, as torchrun starts
them (RANK / WORLD_SIZE / LOCAL_RANK / MASTER_* in the environment).

Replicas: every rank dedisperses its own beam (here with the CPU oracle, the
GPU kernels being covered by the -m gpu tests), nothing crosses ranks on the
data path, the job time is the slowest rank's (all_reduce MAX) and the rate
counts the units of all ranks.  The reference arm runs on rank 0 only.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    import oracle
    import synth

    oracle.build()  # atomic replace: safe when both ranks build
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    wl = synth.scaled(synth.workload("single_beam_f32"), nsamp=2048)
    wl.dtype = "u8"
    wl.pulse_amp = 5 * 16.0
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s,
                                    wl.dms)
    block, _ = synth.make_block(wl, bench.replica_seed(7, r), delays)
    D = oracle.dedisperse(block, delays)  # this rank's replica of the step
    seconds = 0.5 + r  # rank 1 is the slower one
    t_max = bench.max_over_ranks(seconds, w)
    units = D.size
    rate = bench.whole_job_rate(w, units, 3, t_max)
    dist.barrier()
    queue.put((r, w, local, t_max, rate, units, int(D.astype(np.int64).sum()),
               int(block.astype(np.int64).sum())))
    dist.destroy_process_group()


def test_two_gloo_ranks_run_replicas_and_time_the_slowest():
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(queue.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, t0, rate0, u0, s0, b0), (r1, w1, l1, t1, rate1, u1, s1, b1) = res
    assert (r0, r1) == (0, 1) and w0 == w1 == 2 and (l0, l1) == (0, 1)
    assert t0 == t1 == 1.5                      # both see the slowest rank
    assert rate0 == rate1 == 2 * u0 * 3 / 1.5   # all ranks' units over that time
    assert b0 != b1                             # each replica has its own beam
    assert u0 == u1


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.argparse.Namespace(workload="full_block_u8", impl="reference", gpus=2, steps=1,
                                    warmup=0, seed=1, cpu_seconds=1.0, nsamp=None)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""


def test_single_rank_helpers_need_no_process_group():
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.whole_job_rate(1, 10, 4, 2.0) == 20.0
    assert bench.replica_seed(5, 0) != bench.replica_seed(5, 1)


@pytest.mark.parametrize("workload", ["full_block_u8", "binned8_full_block_u8"])
def test_reference_arm_line_carries_the_contract_keys(monkeypatch, capsys, workload):
    """Rank 0 of the reference arm prints one JSON line with the keys the
    bench contract asks for, the oracle's rate as value, cpu_baseline and
    e2e describing that run (a short sample)."""
    import json

    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    args = bench.argparse.Namespace(workload=workload, impl="reference", gpus=1, steps=1,
                                    warmup=0, seed=1, cpu_seconds=0.2, nsamp=None)
    bench.run_reference(args)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 1
    assert line["config"]["workload"] == workload
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"]
    assert cpu["sample"] and cpu["unit"] == line["unit"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0
