"""Benchmark of the dedispersion + detection hot path on GB300.

One step = one pass of the whole path over one synthetic filterbank block
resident in HBM: dd_run -- brute-force dedispersion, then per-DM statistics,
n-sigma threshold, candidate list and the count to the host.  The default
workload is the largest single-GPU configuration, ``lband_f32``: 4096
channels x 131072 f32 samples (1200-1500 MHz, 64 us), 4096 DM trials
0..409.5; ``--workload full_block_u8`` times the 8-bit block (1024 channels x
65536, 2048 trials), whose dedispersion kernel also accumulates each DM row's
exact sums and per-tile maxima.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints one JSON line.  ``value`` is DM-trial*samples/s summed over ranks
(each rank processes its own beam: weak scaling, no collective on the data
path).  ``e2e`` repeats the metric through a host pipe on pinned host buffers
(every step a host->device copy of its block, dedispersion, detection and
its candidates back to the host, each copy overlapped with the previous
block's work); ``e2e.serial`` the same through dd_process_host, one block at
a time.  ``roofline`` reports the dedispersion kernel against the add-pipe
peak.  ``cpu_baseline`` times the CPU oracle on a bounded sample of the same
workload on this machine's host cores.  ``--impl reference`` times only the
oracle (the reference arm).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "DM-trial*samples/s"
UNIT = "DM-trial*samples/s"
NSIGMA = 6.0
L2_FLUSH_BYTES = 256 << 20
LANES_PER_SM = 128  # 32-bit add lanes per SM (4 partitions x 32)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="lband_f32")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the bounded oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-probes", action="store_true", help="skip the add-pipe probes")
    ap.add_argument("--nsamp", type=int, default=None,
                    help="input samples per channel (default: the workload's); a shorter "
                         "block for profiling captures")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# Replicas: with N ranks each dedisperses its own beam (no data-path
# collective); the job's time is the slowest rank's and its rate counts the
# units every rank processed.

def replica_seed(seed, rank):
    """Seed of rank `rank`'s beam (each replica gets its own data)."""
    return seed + rank


def max_over_ranks(value, world, device=None):
    """The largest `value` over all ranks (all_reduce MAX; needs an initialised
    process group when world > 1)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_step, steps, seconds):
    """Units all ranks processed per second of the slowest rank."""
    return world * units_per_step * steps / seconds


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ helpers

def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def kernel_source_sha(workload: str) -> str:
    """Hash of the code of the dedispersion kernel that dominates `workload`
    (the 8-bit kernel for u8 workloads, the float kernel otherwise; comments
    and blank lines dropped), to tell whether a recorded ncu traffic figure
    still applies."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1401_8258_gb300", "csrc")
    kind = "quad" if workload.endswith("u8") else "octet"
    files = {"quad": ["dd_dedisp_quad.cu"], "octet": ["dd_dedisp_octet.cu"]}[kind]
    for f in sorted([os.path.join(csrc, n) for n in files] +
                    glob.glob(os.path.join(csrc, f"dd_{kind}*")) +
                    [os.path.join(csrc, "dd_device.cuh")]):
        with open(f) as fh:
            for line in fh:
                code = line.split("//", 1)[0].strip()
                if code:
                    h.update(code.encode())
    return h.hexdigest()[:12]


def recorded_traffic(workload: str) -> tuple[float | None, str | None]:
    """DRAM bytes per dedispersion launch from the committed ncu summary, if
    it was taken on the current kernel source (``source_sha`` line)."""
    path = os.path.join(ROOT, "profiles", f"dedisperse_{workload}.md")
    if not os.path.exists(path):
        return None, None
    text = open(path).read()
    m_b = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    m_s = re.search(r"source_sha:\s*([0-9a-f]+)", text)
    if not (m_b and m_s) or m_s.group(1) != kernel_source_sha(workload):
        return None, os.path.relpath(path, ROOT)
    return float(m_b.group(1)), os.path.relpath(path, ROOT)


def geometry(wl):
    from paper_1401_8258_gb300 import dd_compute_delays
    delays, mx = dd_compute_delays(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    return delays, mx, wl.nsamp - mx


# ----------------------------------------------------------- CPU baseline

def time_oracle_sample(wl, block, delays, nsamp_out, target_s: float) -> dict:
    """Oracle dedispersion + stats + detection on a DM subset sized for about
    ``target_s`` seconds on all host cores; throughput scaled to the metric."""
    import oracle
    oracle.build()
    ndm_total = wl.ndm
    probe = max(1, min(ndm_total, 8))
    idx = np.linspace(0, ndm_total - 1, probe).astype(int)
    t0 = time.perf_counter()
    D = oracle.dedisperse(block, delays[:, idx], nsamp_out=nsamp_out, nsamp_in=wl.nsamp)
    m, s = oracle.stats(D)
    oracle.detect(D, m, s, NSIGMA, capacity=0)
    dt = time.perf_counter() - t0
    per_dm = dt / probe
    n = int(min(ndm_total, max(probe, target_s / max(per_dm, 1e-9))))
    idx = np.linspace(0, ndm_total - 1, n).astype(int)
    t0 = time.perf_counter()
    D = oracle.dedisperse(block, delays[:, idx], nsamp_out=nsamp_out, nsamp_in=wl.nsamp)
    m, s = oracle.stats(D)
    oracle.detect(D, m, s, NSIGMA, capacity=0)
    dt = time.perf_counter() - t0
    # the same work on one core, on a few trials (about a tenth of the time)
    n1 = max(1, min(n, int(0.1 * target_s / max(per_dm * oracle.max_threads(), 1e-9))))
    idx1 = np.linspace(0, ndm_total - 1, n1).astype(int)
    t0 = time.perf_counter()
    D1 = oracle.dedisperse(block, delays[:, idx1], nsamp_out=nsamp_out, nsamp_in=wl.nsamp,
                           nthreads=1)
    m1, s1 = oracle.stats(D1)
    oracle.detect(D1, m1, s1, NSIGMA, capacity=0)
    dt1 = time.perf_counter() - t0
    return {"value": n * nsamp_out / dt, "unit": UNIT, "cores": oracle.max_threads(),
            "kind": "oracle", "seconds": dt,
            "single_core": {"value": n1 * nsamp_out / dt1, "trials": n1, "seconds": dt1},
            "sample": f"{n} of {ndm_total} DM trials (evenly spaced) x {nsamp_out} samples x "
                      f"{wl.nchan} channels of the same block; dedispersion + stats + detection"}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ------------------------------------------------------------- reference arm

def load_workload(args):
    wl = synth.workload(args.workload)
    if args.nsamp is not None:
        wl = synth.scaled(wl, nsamp=args.nsamp)
    return wl


def reference_steps(args, timed):
    """Runs the oracle sample `timed(seconds)` for the reference arm's warm-up
    and timed steps (each sized so the whole run ends within about a
    minute); returns the median rate, the seconds spent and the last
    sample's record."""
    per_step = max(1.0, 60.0 / max(args.steps + args.warmup, 1))
    for _ in range(args.warmup):
        timed(min(per_step, 2.0))
    vals, secs, last = [], 0.0, None
    for _ in range(args.steps):
        last = timed(per_step)
        vals.append(last["value"])
        secs += last["seconds"]
    return statistics.median(vals), secs, last


def print_reference(args, value, secs, last, dtype, config):
    """The reference arm's JSON line (the oracle's rate on the host cores)."""
    cpu = {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
           "sample": last["sample"]}
    for k in ("single_core", "cpu_model"):
        if k in last:
            cpu[k] = last[k]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": config, "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    if args.workload in (POST, BINNED, BINNED8, SUBBAND):
        import oracle
        wl = synth.workload("full_block_u8")
        delays, _, nsamp_out = geometry_oracle(wl)
        block, _ = synth.make_block(wl, args.seed, delays)
        if args.workload == POST:
            # the chain on evenly spaced rows, dedispersed by the oracle first
            rows = np.linspace(0, wl.ndm - 1, 64).astype(np.int64)
            D = oracle.dedisperse(block, np.ascontiguousarray(delays[:, rows]),
                                  nsamp_out=nsamp_out)
            value, secs, last = reference_steps(args, lambda t: time_oracle_post(D, t))
            last["sample"] = "evenly spaced DM rows of the block: " + last["sample"]
            config = {"workload": POST, "rows": wl.ndm, "samples": nsamp_out,
                      "median_width": POST_MEDIAN_WIDTH, "boxcar_widths": POST_WIDTHS,
                      "nsigma": NSIGMA, "parallelism": "replicas1"}
            print_reference(args, value, secs, last, "f64", config)
        elif args.workload in (BINNED, BINNED8):
            mode = bin_mode(args.workload)
            value, secs, last = reference_steps(
                args, lambda t: time_oracle_binned(wl, block, t, mode))
            config = {"workload": args.workload, "max_factor": BIN_MAX_FACTOR, "binning": mode,
                      "parallelism": "replicas1"}
            print_reference(args, value, secs, last, "int32", config)
        else:
            value, secs, last = reference_steps(
                args, lambda t: time_oracle_subband(wl, block, delays, t))
            config = {"workload": SUBBAND, "chans_per_subband": SUB_CHANS,
                      "dms_per_group": SUB_DMS, "parallelism": "replicas1"}
            print_reference(args, value, secs, last, "int32", config)
        return
    if args.workload in (BATCH, BATCH_SMALL, SERVE):
        # the oracle on the first beam (its rate stands for the set)
        ms = lambda w: geometry_oracle(w)[1]  # noqa: E731
        if args.workload == SERVE:
            wl = synth.serving_workloads(args.seed, ms)[0]
        elif args.workload == BATCH_SMALL:
            wl = synth.batch_workloads(args.seed, ms, nchan_choices=(256, 512),
                                       nsamp_range=(16384, 65536), ndm_range=(128, 512))[0]
        else:
            wl = synth.batch_workloads(args.seed, ms)[0]
    else:
        wl = load_workload(args)
    delays, mx, nsamp_out = geometry_oracle(wl)
    block, _ = synth.make_block(wl, args.seed, delays)
    value, secs, last = reference_steps(
        args, lambda t: time_oracle_sample(wl, block, delays, nsamp_out, t))
    last["cpu_model"] = cpu_model()
    config = workload_config(wl, nsamp_out, args.gpus)
    if args.workload in (BATCH, BATCH_SMALL, SERVE):
        config = {"workload": args.workload, "sampled_beam": config,
                  "note": "the oracle's rate on the set's first beam stands for the set"}
        last["sample"] = "first beam of the set: " + last["sample"]
    print_reference(args, value, secs, last, "int64" if wl.dtype == "u8" else "f64", config)


def geometry_oracle(wl):
    import oracle
    oracle.build()
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    return delays, mx, wl.nsamp - mx


def workload_config(wl, nsamp_out, n_gpus):
    return {
        "workload": wl.name, "nchan": wl.nchan, "nsamp_in": wl.nsamp, "nsamp_out": nsamp_out,
        "ndm": wl.ndm, "dm_range": [float(wl.dms[0]), float(wl.dms[-1])],
        "f_top_mhz": wl.f_top_mhz, "chan_width_mhz": wl.chan_width_mhz,
        "t_samp_s": wl.t_samp_s, "input_dtype": wl.dtype, "nsigma": NSIGMA,
        "beams_per_gpu": 1, "parallelism": f"replicas{n_gpus}",
        "l2": "L2 flushed (256 MiB write) before every timed step",
    }


# ------------------------------------------------------------------- ours

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1401_8258_gb300 as dd

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dd.build()

    wl = load_workload(args)
    plan = dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, wl.dtype, local)
    delays = plan.delays()
    nsamp_out = plan.nsamp_out(wl.nsamp)
    block_np, pulses = synth.make_block(wl, replica_seed(args.seed, rank), delays)
    block = torch.from_numpy(block_np).to(dev)
    out = torch.empty((wl.ndm, nsamp_out), dtype=plan.out_torch_dtype, device=dev)
    cap = 1 << 20
    cands = torch.empty((cap, 16), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        # ev_mid is recorded by the library right after the dedispersion kernel
        st, total = dd.dd_run(plan.handle, block, wl.nsamp, block.stride(0), out, NSIGMA, cands,
                              cap, stream, ev_mid)
        return total

    ev_mid = torch.cuda.Event(enable_timing=True)
    ev_mid.record(stream)  # creates the event before its handle is passed on
    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for e in mids:
        e.record(stream)
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = plan.launch_count()
    totals = []
    for i in range(args.steps):
        flush.fill_(1.0)
        starts[i].record(stream)
        ev_mid = mids[i]
        totals.append(step())
        ends[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = plan.launch_count() - launches0
    clock = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    kern_ms = [s.elapsed_time(m) for s, m in zip(starts, mids)]
    t_total = sum(step_ms) / 1e3
    t_kernel = statistics.median(kern_ms) / 1e3  # median of the timed launches
    t_total = max_over_ranks(t_total, world, dev)
    units_per_step = wl.ndm * nsamp_out
    value = whole_job_rate(world, units_per_step, args.steps, t_total)

    # end to end through the C ABI on pinned host buffers: a host pipe (each
    # block's copy overlapped with the previous block's dd_run; K pushes and
    # one flush give K results), and dd_process_host one block at a time
    e2e = None
    if not args.no_e2e:
        host_block = torch.from_numpy(block_np).pin_memory()
        host_cands = torch.empty((cap, 16), dtype=torch.uint8).pin_memory()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pipe = dd.HostPipe(plan, wl.nsamp, wl.nsamp, NSIGMA, cap)
        for _ in range(max(1, args.warmup)):
            pipe.push(host_block, stream)
        pipe.flush(stream)
        torch.cuda.synchronize()
        counts = []
        ev0.record(stream)
        for _ in range(args.steps):
            r = pipe.push(host_block, stream)
            if r is not None:
                counts.append(r[1])
        counts.append(pipe.flush(stream)[1])
        ev1.record(stream)
        torch.cuda.synchronize()
        pipe.close()
        assert len(counts) == args.steps
        t_e2e = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world, dev)
        e2e = {"value": whole_job_rate(world, units_per_step, args.steps, t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": int(block_np.nbytes),
               "d2h_bytes_per_step": int(8 + 16 * statistics.mean(min(c, cap) for c in counts)),
               "api": "dd_host_pipe_push / dd_host_pipe_flush (copy of block k overlapped "
                      "with dd_run of block k-1)"}
        for _ in range(max(1, args.warmup)):
            dd.dd_process_host(plan.handle, host_block, wl.nsamp, wl.nsamp, NSIGMA, host_cands,
                               cap, stream)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            dd.dd_process_host(plan.handle, host_block, wl.nsamp, wl.nsamp, NSIGMA, host_cands,
                               cap, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_ser = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world, dev)
        e2e["serial"] = {"value": whole_job_rate(world, units_per_step, args.steps, t_ser),
                         "api": "dd_process_host (copy, dd_run, candidates back, in turn)"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        plan.close()
        return

    # roofline of the dedispersion kernel (plain 32-bit add pipes)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = measured_peaks()
    smax = float(peaks.get("sm_max_mhz", 2070.0))
    adds = float(wl.ndm) * nsamp_out * wl.nchan
    achieved = adds / t_kernel / 1e12
    peak = sms * LANES_PER_SM * smax * 1e6 / 1e12
    probes = {}
    for kind in () if args.no_probes else ("fadd", "fadd2", "iadd", "iadd3", "imad", "lop3", "prmt", "prmt_iadd",
                 "lop3_iadd", "fadd_f16", "hadd2"):
        try:
            ops, per_clk = dd._native.dd_measure_add_peak(kind, local)
            probes[kind] = {"Tops_per_s": ops / 1e12, "ops_per_clk_per_sm": per_clk}
        except Exception as e:  # probe failure must not hide the bench line
            probes[kind] = {"error": str(e)}
    traffic, prof = recorded_traffic(wl.name)
    algo_bytes = block_np.nbytes + wl.ndm * nsamp_out * 4
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tadd/s",
            "frac": achieved / peak, "traffic": traffic,
            "kernel": "dd_dedisperse", "kernel_ms": t_kernel * 1e3,
            "peak_basis": f"{sms} SMs x {LANES_PER_SM} add lanes x {smax:.0f} MHz (max clock)",
            "frac_at_observed_clock": (achieved / (sms * LANES_PER_SM * clock["sm_mhz"] * 1e6 / 1e12)
                                       if clock.get("sm_mhz") else None),
            "algorithmic_bytes": algo_bytes,
            "hbm_frac_of_measured": (algo_bytes / t_kernel / 1e9) / float(peaks.get("hbm_gbs", 6784.5)),
            # the ncu DRAM bytes of one launch over this run's kernel time
            "hbm_frac_from_traffic": ((traffic / t_kernel / 1e9) / float(peaks.get("hbm_gbs", 6784.5))
                                      if traffic else None),
            "traffic_source": prof, "add_pipe_probes": probes}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = time_oracle_sample(wl, block_np, delays, nsamp_out, args.cpu_seconds)
        cpu["cpu_model"] = cpu_model()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32" if wl.dtype == "u8" else "f32", "data": "synthetic",
        "config": workload_config(wl, nsamp_out, world),
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clock,
        "gpu_launches": int(launches),
        "candidates_per_step": int(statistics.median(totals)),
        "step_ms_median": statistics.median(step_ms),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    plan.close()


# ------------------------------------------------------------- batch

BATCH = "batch32_u8"  # 32 uneven u8 beams (the batching row's configuration)
# 32 small u8 beams (256 or 512 channels, 128..512 trials): the mix where one
# shared launch fills the SMs that each beam alone leaves idle
BATCH_SMALL = "batch32_small_u8"


def batch_workloads(seed, small=False):
    from paper_1401_8258_gb300 import dd_compute_delays

    def maxshift(wl):
        return dd_compute_delays(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)[1]
    if small:
        return synth.batch_workloads(seed, maxshift, n=32, nchan_choices=(256, 512),
                                     nsamp_range=(16384, 65536), ndm_range=(128, 512))
    return synth.batch_workloads(seed, maxshift, n=32)


def run_batch(args):
    """One step = dd_batch_run over 32 uneven beams resident in HBM."""
    import torch

    import paper_1401_8258_gb300 as dd

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dd.build()
    wls = batch_workloads(args.seed, small=args.workload == BATCH_SMALL)
    plans = [dd.Plan(w.nchan, w.f_top_mhz, w.chan_width_mhz, w.t_samp_s, w.dms, "u8", local)
             for w in wls]
    # plan time, outside the timed region: the autotuner times every staged
    # tile width and staging depth on each beam's geometry and keeps the
    # fastest (a shorter scratch block suffices: the choice depends on the
    # geometry)
    tuned = [p.autotune(min(w.nsamp, p.maxshift + 32768)) for p, w in zip(plans, wls)]
    depths = [dd._native.dd_plan_kernel_info(p.handle, None, 0)["copy_ahead"] for p in plans]
    host_blocks, blocks, outs, nouts = [], [], [], []
    for i, (w, p) in enumerate(zip(wls, plans)):
        b, _ = synth.make_block(w, args.seed + 1000 * (rank + 1) + i, p.delays())
        host_blocks.append(b)
        blocks.append(torch.from_numpy(b).to(dev))
        nouts.append(p.nsamp_out(w.nsamp))
        outs.append(torch.empty((w.ndm, nouts[-1]), dtype=torch.int32, device=dev))
    cap = 1 << 16
    cands = [torch.empty((cap, 16), dtype=torch.uint8, device=dev) for _ in wls]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    nsamp = [w.nsamp for w in wls]
    batch = dd.Batch(plans)

    def step():
        st, totals = dd.dd_batch_run(batch.handle, blocks, nsamp, nsamp, outs, NSIGMA, cands,
                                     [cap] * len(wls), stream)
        return sum(totals)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = sum(p.launch_count() for p in plans)
    totals = []
    for i in range(args.steps):
        flush.fill_(1.0)
        starts[i].record(stream)
        totals.append(step())
        ends[i].record(stream)
    torch.cuda.synchronize()
    launches = sum(p.launch_count() for p in plans) - launches0
    clock = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_total = sum(step_ms) / 1e3
    units = sum(w.ndm * n for w, n in zip(wls, nouts))
    value = units * args.steps / t_total

    # the same beams one dd_run after another (the per-beam launch baseline)
    cands1 = torch.empty((cap, 16), dtype=torch.uint8, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rep in range(2):
        flush.fill_(1.0)
        ev0.record(stream)
        for p, b, o, n in zip(plans, blocks, outs, nsamp):
            dd.dd_run(p.handle, b, n, n, o, NSIGMA, cands1, cap, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    per_beam_ms = ev0.elapsed_time(ev1)

    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(b).pin_memory() for b in host_blocks]
        host_cands = [torch.empty((cap, 16), dtype=torch.uint8).pin_memory() for _ in wls]
        counts = []

        def e2e_step():
            for hb, db in zip(pinned, blocks):
                db.copy_(hb, non_blocking=True)
            st, tot = dd.dd_batch_run(batch.handle, blocks, nsamp, nsamp, outs, NSIGMA, cands,
                                      [cap] * len(wls), stream)
            for hc, c, t in zip(host_cands, cands, tot):
                if t:
                    hc[:min(t, cap)].copy_(c[:min(t, cap)], non_blocking=True)
            torch.cuda.synchronize()
            counts.append(sum(min(t, cap) for t in tot))
        e2e_step()
        ev0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        ev1.record(stream)
        torch.cuda.synchronize()
        t_e2e = ev0.elapsed_time(ev1) / 1e3
        e2e = {"value": units * args.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(sum(b.nbytes for b in host_blocks)),
               "d2h_bytes_per_step": int(8 * len(wls) + 16 * statistics.mean(counts[1:]))}

    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = measured_peaks()
    smax = float(peaks.get("sm_max_mhz", 2070.0))
    adds = float(sum(w.ndm * n * w.nchan for w, n in zip(wls, nouts)))
    t_step = t_total / args.steps
    achieved = adds / t_step / 1e12
    peak = sms * LANES_PER_SM * smax * 1e6 / 1e12
    staged = sum(dd._native.dd_plan_kernel_info(p.handle, b, n)["staged"]
                 for p, b, n in zip(plans, blocks, nsamp))
    algo_bytes = sum(b.nbytes for b in host_blocks) + sum(4 * w.ndm * n for w, n in zip(wls, nouts))
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tadd/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": "whole batch step (shared persistent launches, other beams' kernels, "
                      "detection)", "kernel_ms": t_step * 1e3,
            "peak_basis": f"{sms} SMs x {LANES_PER_SM} add lanes x {smax:.0f} MHz (max clock)",
            "algorithmic_bytes": algo_bytes,
            "hbm_frac_of_measured": (algo_bytes / t_step / 1e9) / float(peaks.get("hbm_gbs", 6784.5))}
    cpu = None
    if not args.no_cpu_baseline:
        w0 = wls[0]
        cpu = time_oracle_sample(w0, host_blocks[0], plans[0].delays(), nouts[0], args.cpu_seconds)
        cpu["sample"] = "beam 0 of the batch: " + cpu["sample"]
        cpu["cpu_model"] = cpu_model()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "beams": len(wls), "staged_beams": int(staged),
                   "autotuned_dms_per_cta": [int(t[0]) for t in tuned],
                   "autotuned_staging_depth": depths,
                   "nchan": [w.nchan for w in wls], "ndm": [w.ndm for w in wls],
                   "nsamp_in": nsamp, "input_dtype": "u8", "nsigma": NSIGMA,
                   "parallelism": "replicas1",
                   "l2": "L2 flushed (256 MiB write) before every timed step"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clock,
        "gpu_launches": int(launches),
        "per_beam_dd_run_ms": per_beam_ms,
        "candidates_per_step": int(statistics.median(totals)),
    }
    print(json.dumps(line), flush=True)
    batch.close()
    for p in plans:
        p.close()


# ----------------------------------------------------------- serving

SERVE = "serve64_u8"  # 64 beams streaming 1 s blocks (the serving row's configuration)


def serving_workloads(seed):
    from paper_1401_8258_gb300 import dd_compute_delays

    def maxshift(wl):
        return dd_compute_delays(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)[1]
    return synth.serving_workloads(seed, maxshift, n=64)


def serve_load(dd, Server, wls, plans, host, nbeams, per_beam, seconds, seed, cap,
               drain_s=20.0):
    """One load point through the server: `nbeams` beams of the serving mix
    (beam i has the geometry of base beam i % 64, its own stream, plan and
    memory; replicas share their base plan's tables), each sending
    `seconds` one-second blocks that arrive in real time at phase_i + k
    seconds (phases uniform in [0, 1)), copied from pinned host memory.
    Returns latency percentiles over the blocks after the first two of each
    beam, the GPU's busy share, and whether the load is sustained: every
    block done, p99 latency below the block duration, the last block
    finished within one block duration of its arrival."""
    import threading
    rng = np.random.default_rng(seed)
    phases = rng.uniform(0.0, 1.0, nbeams)
    beam_plans = []
    for i in range(nbeams):
        base = plans[i % len(plans)]
        beam_plans.append(base if i < len(plans) else dd.Plan.like(base))
    srv = Server(NSIGMA, capacity=cap, per_beam=per_beam)
    try:
        for i in range(nbeams):
            srv.open(i, beam_plans[i], wls[i % len(wls)].nsamp)
        t0 = time.perf_counter() + 0.5
        arrivals = sorted((t0 + phases[i] + k, i, k) for i in range(nbeams)
                          for k in range(seconds))

        def feed():
            for t, i, k in arrivals:
                dt = t - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                srv.submit(i, host[i % len(host)][k % 2], arrival=t)
            for i in range(nbeams):
                srv.close_beam(i)

        th = threading.Thread(target=feed, daemon=True)
        th.start()
        th.join()
        drained = True
        try:
            srv.drain(timeout=drain_s)
        except TimeoutError:
            drained = False
        lat = np.array([r.latency for i in range(nbeams) for r in srv.results[i]
                        if r.seq >= 2])
        done = sum(len(srv.results[i]) for i in range(nbeams))
        last = max((r.latency for i in range(nbeams) for r in srv.results[i]
                    if r.seq == seconds - 1), default=float("inf"))
        waves = list(srv.waves)
        busy = sum(b - a for _, a, b in waves)
        span = arrivals[-1][0] - arrivals[0][0] + 1.0
        admitted_at_once = srv.peak_used
    finally:
        srv.abort()
        for i in range(len(plans), nbeams):
            beam_plans[i].close()
    p99 = float(np.percentile(lat, 99)) if lat.size else float("inf")
    ok = bool(drained and done == nbeams * seconds and p99 < 1.0 and last < 1.0)
    return {"beams": nbeams, "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency_s": p99, "max_latency_s": float(lat.max()) if lat.size else None,
            "busy_share": busy / span, "waves": len(waves),
            "beams_per_wave": float(np.mean([n for n, _, _ in waves])) if waves else 0.0,
            "blocks_done": done, "peak_admitted_bytes": int(admitted_at_once),
            "sustained": ok}


def run_serve(args):
    """Real-time serving of the 64-beam mix through the continuous-batching
    server (paper_1401_8258_gb300.serve.Server): beams opened and admitted by
    device memory, 1 s blocks arriving in real time from a host thread,
    copied from pinned memory on the copy stream, waves of every beam with a
    copied block (or one push per beam, the plain form), wall-clock latency
    from arrival to candidates on the host.  For each form the largest load
    (beams of this mix, in steps of 32) sustained with p99 latency below the
    block duration is searched, three times; ``value`` is the real-time
    throughput (DM-trial*samples per second of data) of the largest load the
    waves sustained in every repeat."""
    import torch

    import paper_1401_8258_gb300 as dd
    from paper_1401_8258_gb300.serve import Server

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dd.build()
    wls = serving_workloads(args.seed)
    plans = [dd.Plan(w.nchan, w.f_top_mhz, w.chan_width_mhz, w.t_samp_s, w.dms, "u8", local)
             for w in wls]
    cap = 1 << 14
    rng = np.random.default_rng(args.seed)
    host = [[torch.from_numpy(synth.random_block(rng, w.nchan, w.nsamp, "u8")).pin_memory()
             for _ in range(2)] for w in wls]
    seconds = max(20, args.steps)
    repeats = 3

    # warm-up: every geometry's kernels and the allocator
    serve_load(dd, Server, wls, plans, host, len(wls), False, 3, args.seed, cap)

    step = 32

    def search(per_beam, rep):
        """Largest sustained load in steps of 32 beams: a run at 768 beams
        estimates the capacity from its busy share, then loads around the
        estimate are run until a sustained load and the next one up, not
        sustained, are found."""
        tried, seen = [], {}

        def run(nb):
            if nb not in seen:
                seen[nb] = serve_load(dd, Server, wls, plans, host, nb, per_beam, seconds,
                                      args.seed + 1000 * rep + nb, cap)
                tried.append(seen[nb])
            return seen[nb]

        first = run(768)
        est = 768 / max(first["busy_share"], 1e-3)
        nb = max(step, int(0.97 * est) // step * step)
        for _ in range(8):
            ok = run(nb)["sustained"]
            if ok and (nb + step) in seen and not seen[nb + step]["sustained"]:
                break
            if not ok and (nb - step) in seen and seen[nb - step]["sustained"]:
                break
            nb = nb + step if ok else nb - step
            if nb < step:
                break
        best = max((b for b, r in seen.items() if r["sustained"] and all(
            seen[c]["sustained"] for c in seen if c < b)), default=0)
        return best, tried

    clocks = ClockSampler(local)
    clocks.start()
    results = {"waves": [], "per_beam_launches": []}
    for rep in range(repeats):
        for form, per_beam in (("waves", False), ("per_beam_launches", True)):
            best, tried = search(per_beam, rep)
            results[form].append({"max_realtime_beams": best, "sweep": tried})
    clock = clocks.stop()

    def summary(form):
        bests = [r["max_realtime_beams"] for r in results[form]]
        at = [t for r in results[form] for t in r["sweep"]
              if t["beams"] == r["max_realtime_beams"]]
        return {"max_realtime_beams_each_repeat": bests, "min": min(bests), "max": max(bests),
                "p50_latency_s_at_max": [t["p50_latency_s"] for t in at],
                "p99_latency_s_at_max": [t["p99_latency_s"] for t in at],
                "repeats": results[form]}

    sw, sp = summary("waves"), summary("per_beam_launches")
    beams = sw["min"]
    units = sum(wls[i % len(wls)].ndm * wls[i % len(wls)].nsamp for i in range(beams))
    adds = float(sum(wls[i % len(wls)].ndm * wls[i % len(wls)].nsamp * wls[i % len(wls)].nchan
                     for i in range(beams)))
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    peak = props.multi_processor_count * LANES_PER_SM * float(peaks.get("sm_max_mhz", 2070.0)) / 1e6
    line = {
        "metric": METRIC, "value": float(units), "unit": UNIT + " (real time, 1 s blocks)",
        "n_gpus": 1, "steps": seconds, "warmup": 3, "ms_per_step": 1000.0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": SERVE, "beam_mix": 64, "block_s": 1.0,
                   "seconds_of_arrivals_per_load": seconds, "repeats": repeats,
                   "nchan": [w.nchan for w in wls], "ndm": [w.ndm for w in wls],
                   "t_samp_s": [w.t_samp_s for w in wls], "input_dtype": "u8",
                   "nsigma": NSIGMA, "parallelism": "replicas1",
                   "arrivals": "real time from a host thread, staggered phases, pinned host "
                               "blocks copied on a copy stream"},
        "roofline": {"bound": "alu", "achieved": adds / 1e12, "peak": peak, "unit": "Tadd/s",
                     "frac": adds / 1e12 / peak, "traffic": None,
                     "kernel": "the beams' sample-adds per second of data at the sustained load"},
        "serving": {"waves": sw, "per_beam_launches": sp,
                    "margin_beams": sw["min"] - sp["max"]},
        "cpu_baseline": None, "e2e": None, "clocks": clock, "gpu_launches": None,
    }
    print(json.dumps(line), flush=True)
    for p in plans:
        p.close()


# ------------------------------------------------------ post-processing

POST = "post_full_block_u8"  # median(5) -> detrend -> boxcar on the full_block_u8 output
POST_MEDIAN_WIDTH = 5
POST_WIDTHS = 8  # boxcar widths 1 .. 128 samples


def time_oracle_post(D, seconds):
    """The oracle's post-processing chain on a bounded sample of rows."""
    from oracle import post

    rows = 1
    t0 = time.perf_counter()
    post.boxcar_detect(post.detrend(post.median_filter(D[:1], POST_MEDIAN_WIDTH))[0]
                       .astype(np.float32), None, None, POST_WIDTHS, NSIGMA)
    one = time.perf_counter() - t0
    rows = int(max(1, min(D.shape[0], seconds / max(one, 1e-6))))
    t0 = time.perf_counter()
    z, _ = post.detrend(post.median_filter(D[:rows], POST_MEDIAN_WIDTH))
    post.boxcar_detect(z.astype(np.float32), None, None, POST_WIDTHS, NSIGMA)
    dt = time.perf_counter() - t0
    return {"value": rows * D.shape[1] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "seconds": dt,
            "sample": f"{rows} of {D.shape[0]} rows x {D.shape[1]} samples: median "
                      f"({POST_MEDIAN_WIDTH}), detrend, boxcar ({POST_WIDTHS} widths)"}


def run_post(args):
    """One step = dd_median_filter -> dd_detrend -> dd_boxcar_detect over the
    2048 x 57723 int32 dedispersed rows of full_block_u8 (resident in HBM;
    produced once by dd_run before the timed region)."""
    import torch

    import paper_1401_8258_gb300 as dd

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dd.build()
    wl = synth.workload("full_block_u8")
    plan = dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, wl.dtype, local)
    block, _ = synth.make_block(wl, args.seed + 1000 * (rank + 1), plan.delays())
    D = plan.run(torch.from_numpy(block).to(dev), NSIGMA)[0]
    ndm, n = D.shape
    med = torch.empty_like(D)
    z = torch.empty((ndm, n), dtype=torch.float32, device=dev)
    need = dd._native.dd_boxcar_workspace_bytes(ndm, n)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    cap = 1 << 20
    pulses = torch.empty((cap, dd.PULSE_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]

    def step(e=None):
        if e: e[0].record(stream)
        dd._native.dd_median_filter(D, n, dd.DD_ROWS_I32, ndm, n, POST_MEDIAN_WIDTH, med, n, stream)
        if e: e[1].record(stream)
        dd._native.dd_detrend(med, n, dd.DD_ROWS_I32, ndm, n, z, n, None, stream)
        if e: e[2].record(stream)
        _, total = dd._native.dd_boxcar_detect(z, n, dd.DD_ROWS_F32, ndm, n, None, None,
                                               POST_WIDTHS, NSIGMA, ws, need, pulses, cap, stream)
        if e: e[3].record(stream)
        return total

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    totals = []
    for i in range(args.steps):
        flush.fill_(1.0)
        totals.append(step(ev[i]))
    torch.cuda.synchronize()
    clock = clocks.stop()
    parts = np.array([[e[k].elapsed_time(e[k + 1]) for k in range(3)] for e in ev]) / 1e3
    t_step = float(parts.sum(axis=1).mean())
    units = ndm * n
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6784.5))
    elems = float(ndm * n)
    algo = {"dd_median": 8 * elems, "dd_detrend_rows": 8 * elems, "dd_boxcar": 4 * elems}
    kernels = {}
    for k, name in enumerate(algo):
        t = float(parts[:, k].mean())
        gbs = algo[name] / t / 1e9
        kernels[name] = {"ms": 1e3 * t, "algorithmic_bytes": int(algo[name]), "GB_per_s": gbs,
                         "frac_of_measured_hbm": gbs / hbm}
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    roof = {"bound": "hbm", "achieved": kernels[dom]["GB_per_s"], "peak": hbm, "unit": "GB/s",
            "frac": kernels[dom]["frac_of_measured_hbm"], "traffic": None, "kernel": dom,
            "kernel_ms": kernels[dom]["ms"], "peak_basis": "measured HBM copy bandwidth",
            "post_kernels": kernels,
            "note": "dd_boxcar time is the whole call: thresholds, count sweep, scan, write "
                    "sweep, the count's copy to the host and its synchronisation"}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = time_oracle_post(D.cpu().numpy(), args.cpu_seconds)
        cpu["cpu_model"] = cpu_model()
    line = {
        "metric": METRIC, "value": units / t_step, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": POST, "rows": ndm, "samples": n,
                   "median_width": POST_MEDIAN_WIDTH, "boxcar_widths": POST_WIDTHS,
                   "nsigma": NSIGMA, "parallelism": "replicas1",
                   "l2": "L2 flushed (256 MiB write) before every timed step"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": None, "clocks": clock,
        "gpu_launches": 7 * args.steps,
        "pulses_per_step": int(statistics.median(totals)),
    }
    print(json.dumps(line), flush=True)
    plan.close()


# ------------------------------------------------------------ subband

SUBBAND = "subband_full_block_u8"  # full_block_u8 by subband dedispersion
SUB_CHANS, SUB_DMS = 32, 64        # channels per subband, trials per DM group


def time_oracle_subband(wl, block, delays, seconds):
    """The subband oracle on whole DM groups of the block (a bounded sample)."""
    from oracle import approx

    ngroups_all = (wl.ndm + SUB_DMS - 1) // SUB_DMS
    t0 = time.perf_counter()
    approx.subband_dedisperse(block, np.ascontiguousarray(delays[:, :SUB_DMS]), SUB_CHANS,
                              SUB_DMS)
    one = time.perf_counter() - t0
    groups = int(max(1, min(ngroups_all, seconds / max(one, 1e-6))))
    sub = np.ascontiguousarray(delays[:, :groups * SUB_DMS])
    t0 = time.perf_counter()
    out = approx.subband_dedisperse(block, sub, SUB_CHANS, SUB_DMS)
    dt = time.perf_counter() - t0
    import oracle
    return {"value": out.size / dt, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "seconds": dt,
            "sample": f"{groups} of {ngroups_all} DM groups ({out.shape[0]} trials) x "
                      f"{out.shape[1]} samples, {wl.nchan} channels in subbands of {SUB_CHANS}"}


def run_subband(args):
    """One step = dd_subband_execute over full_block_u8 (resident in HBM);
    the brute-force kernel on the same block is timed beside it."""
    import torch

    import paper_1401_8258_gb300 as dd

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dd.build()
    wl = load_workload(argparse.Namespace(workload="full_block_u8", nsamp=args.nsamp))
    sub = dd.Subband(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8",
                     SUB_CHANS, SUB_DMS, local)
    plan = dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8", local)
    delays = plan.delays()
    block, _ = synth.make_block(wl, args.seed + 1000 * (rank + 1), delays)
    dblock = torch.from_numpy(block).to(dev)
    n_out = sub.nsamp_out(wl.nsamp)
    out = torch.empty((wl.ndm, n_out), dtype=torch.int32, device=dev)
    n_bf = plan.nsamp_out(wl.nsamp)
    out_bf = torch.empty((wl.ndm, n_bf), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        ms = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    run_sub = lambda: sub.execute(dblock, out=out, stream=stream)  # noqa: E731
    run_bf = lambda: dd.dd_execute(plan.handle, dblock, wl.nsamp, wl.nsamp, out_bf,  # noqa: E731
                                   stream)
    timed(run_sub, args.warmup)
    timed(run_bf, args.warmup)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = sub.launch_count()
    sub_ms = timed(run_sub, args.steps)
    launches = sub.launch_count() - l0
    clock = clocks.stop()
    bf_ms = timed(run_bf, max(3, args.steps // 2))
    t_step = statistics.mean(sub_ms) / 1e3
    units = wl.ndm * n_out
    nnom = len(sub.nominal)
    nsub = (wl.nchan + SUB_CHANS - 1) // SUB_CHANS
    # step-1 series run nsamp_in - D1 samples, D1 = the largest delay inside a
    # subband at a nominal trial (from the plan's delay table)
    tn = delays[:, sub.nominal].astype(np.int64)
    d1 = max(int((tn[c0:c0 + SUB_CHANS] - tn[c0]).max()) for c0 in range(0, wl.nchan, SUB_CHANS))
    adds = float(wl.nchan) * nnom * (wl.nsamp - d1) + float(nsub) * wl.ndm * n_out
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    smax = float(peaks.get("sm_max_mhz", 2070.0))
    peak = props.multi_processor_count * LANES_PER_SM * smax * 1e6 / 1e12
    achieved = adds / t_step / 1e12
    dm_step = float(wl.dms[1] - wl.dms[0])
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tadd/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": "whole subband step (step-1 plans, conversions, step-2 plans)",
            "kernel_ms": 1e3 * t_step,
            "peak_basis": f"{props.multi_processor_count} SMs x {LANES_PER_SM} add lanes x "
                          f"{smax:.0f} MHz (max clock)",
            "algorithmic_adds_per_step": adds,
            "brute_force_adds_per_step": float(wl.nchan) * wl.ndm * n_bf}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = time_oracle_subband(wl, block, delays, args.cpu_seconds)
        cpu["cpu_model"] = cpu_model()
    line = {
        "metric": METRIC, "value": units / t_step, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": SUBBAND, "nchan": wl.nchan, "nsamp_in": wl.nsamp,
                   "nsamp_out": n_out, "ndm": wl.ndm, "chans_per_subband": SUB_CHANS,
                   "dms_per_group": SUB_DMS, "nominal_trials": nnom,
                   "max_dm_error": dm_step * (SUB_DMS // 2), "input_dtype": "u8",
                   "parallelism": "replicas1",
                   "l2": "L2 flushed (256 MiB write) before every timed step"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": None, "clocks": clock,
        "gpu_launches": int(launches / max(args.steps, 1)) * args.steps,
        "brute_force": {"ms": statistics.mean(bf_ms),
                        "value": wl.ndm * n_bf / (statistics.mean(bf_ms) / 1e3)},
        "speedup_vs_brute_force": statistics.mean(bf_ms) / (1e3 * t_step),
    }
    print(json.dumps(line), flush=True)
    sub.close()
    plan.close()


# --------------------------------------------------------- time binning

BINNED = "binned_full_block_u8"  # full_block_u8 with downfactors past the diagonal DM
BINNED8 = "binned8_full_block_u8"  # the same, binned series kept as 8-bit rounded means
BIN_MAX_FACTOR = 8


def bin_mode(workload):
    return "mean8" if workload == BINNED8 else "sum"


def time_oracle_binned(wl, block, seconds, mode="sum"):
    """The binning oracle on evenly spaced trials (each at its own rate)."""
    from oracle import approx
    import oracle

    n = 8
    while True:
        idx = np.linspace(0, wl.ndm - 1, n).astype(np.int64)
        t0 = time.perf_counter()
        rows, fac, lens = approx.binned_dedisperse(block, wl.nchan, wl.f_top_mhz,
                                                   wl.chan_width_mhz, wl.t_samp_s, wl.dms[idx],
                                                   BIN_MAX_FACTOR, mode=mode)
        dt = time.perf_counter() - t0
        if dt * 2 > seconds or n >= wl.ndm:
            break
        n = min(wl.ndm, n * 2)
    covered = float(np.sum(lens * fac))
    return {"value": covered / dt, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "seconds": dt,
            "sample": f"{n} of {wl.ndm} evenly spaced trials (downfactors "
                      f"{sorted(set(fac.tolist()))}), full block"}


def run_binned(args):
    """One step = dd_binned_execute over full_block_u8 (resident), binned by
    pair sums or (binned8_full_block_u8) by 8-bit pair means; the brute-force
    kernel on the same block is timed beside it.  value counts each trial's
    output samples times its downfactor (input samples covered)."""
    import torch

    import paper_1401_8258_gb300 as dd

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dd.build()
    wl = load_workload(argparse.Namespace(workload="full_block_u8", nsamp=args.nsamp))
    mode = bin_mode(args.workload)
    b = dd.Binned(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8",
                  BIN_MAX_FACTOR, mode=mode, device=local)
    plan = dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, "u8", local)
    block, _ = synth.make_block(wl, args.seed + 1000 * (rank + 1), plan.delays())
    dblock = torch.from_numpy(block).to(dev)
    fac, lens = b.rows(wl.nsamp)
    out = torch.empty((wl.ndm, int(lens.max())), dtype=torch.int32, device=dev)
    n_bf = plan.nsamp_out(wl.nsamp)
    out_bf = torch.empty((wl.ndm, n_bf), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        ms = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    run_b = lambda: b.execute(dblock, out=out, stream=stream)  # noqa: E731
    run_bf = lambda: dd.dd_execute(plan.handle, dblock, wl.nsamp, wl.nsamp, out_bf,  # noqa: E731
                                   stream)
    timed(run_b, args.warmup)
    timed(run_bf, args.warmup)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = b.launch_count()
    b_ms = timed(run_b, args.steps)
    launches = b.launch_count() - l0
    clock = clocks.stop()
    bf_ms = timed(run_bf, max(3, args.steps // 2))
    t_step = statistics.mean(b_ms) / 1e3
    covered = float(np.sum(lens * fac))
    adds = float(np.sum(lens)) * wl.nchan
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    smax = float(peaks.get("sm_max_mhz", 2070.0))
    peak = props.multi_processor_count * LANES_PER_SM * smax * 1e6 / 1e12
    achieved = adds / t_step / 1e12
    counts = {int(k): int((fac == k).sum()) for k in sorted(set(fac.tolist()))}
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tadd/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": "whole binned step (binning passes, one plan per downfactor)",
            "kernel_ms": 1e3 * t_step,
            "peak_basis": f"{props.multi_processor_count} SMs x {LANES_PER_SM} add lanes x "
                          f"{smax:.0f} MHz (max clock)",
            "algorithmic_adds_per_step": adds,
            "brute_force_adds_per_step": float(wl.nchan) * wl.ndm * n_bf}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = time_oracle_binned(wl, block, args.cpu_seconds, mode)
        cpu["cpu_model"] = cpu_model()
    line = {
        "metric": METRIC, "value": covered / t_step, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "nchan": wl.nchan, "nsamp_in": wl.nsamp,
                   "ndm": wl.ndm, "max_factor": BIN_MAX_FACTOR, "binning": mode,
                   "diagonal_dm": b.dm_diag,
                   "trials_per_downfactor": counts, "input_dtype": "u8",
                   "value_counts": "output samples x downfactor (input samples covered)",
                   "parallelism": "replicas1",
                   "l2": "L2 flushed (256 MiB write) before every timed step"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": None, "clocks": clock,
        "gpu_launches": int(launches),
        "brute_force": {"ms": statistics.mean(bf_ms),
                        "value": wl.ndm * n_bf / (statistics.mean(bf_ms) / 1e3)},
        "speedup_vs_brute_force": statistics.mean(bf_ms) / (1e3 * t_step),
    }
    print(json.dumps(line), flush=True)
    b.close()
    plan.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in (BATCH, BATCH_SMALL):
        run_batch(args)
    elif args.workload == SERVE:
        run_serve(args)
    elif args.workload == POST:
        run_post(args)
    elif args.workload == SUBBAND:
        run_subband(args)
    elif args.workload in (BINNED, BINNED8):
        run_binned(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
