"""CPU checks of the staged f16/f32 kernel's plan-time tables.

The tables (dd_octet_plan.cpp) tell the kernel which input windows to
bulk-copy, how to sum eight channels into pattern rows and where each DM
trial reads.  A numpy model of the kernel's three phases (copy, build,
accumulate) runs on them here, asserting every shared-memory and global index
against the buffer it addresses.  The input holds small integers, so every
summation order is exact and the model must equal the oracle exactly.
Uncopied / unbuilt words hold a sentinel that would show in any output.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1401_8258_gb300 as dd
import synth

GROUP = 8
T_TILE = 256
REC_HEADER = 4
UNIT_WORDS = 16
CODES_WORD = 8  # shift codes within a unit, two patterns per word
BOUNDS_WORD = 6
REF_CHAN = 3
MAX_OCTETS_PER_CHUNK = 2
MAX_UNITS = 64
ZERO_ELEMS = 64
NWARPS = 12  # building warps
ND_THR = 8  # DM trials per thread of the 128-trial tile (16 warps x 8); 4 for 64
SENTINEL = 1e30


@pytest.fixture(scope="module", autouse=True)
def built():
    dd.build()
    oracle.build()


def octet_tables(delays, nchan, ndm, nd_thr, esize):
    lib = ctypes.CDLL(dd._native.library_path())
    fn = lib.ddi_octet_tables
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    info = np.zeros(11, dtype=np.int32)
    fn(delays.ctypes.data, nchan, ndm, nd_thr, esize, info.ctypes.data, None, None)
    if not info[0]:
        return None
    (ok, nd_cta, ntiles, nchunks, nchan_pad, rec_words, raw_stride, prow_words, smem, opc,
     es) = info.tolist()
    recs = np.zeros(ntiles * nchunks * rec_words, dtype=np.int32)
    meta = np.zeros(ntiles * nchan_pad * 2, dtype=np.int32)
    fn(delays.ctypes.data, nchan, ndm, nd_thr, esize, info.ctypes.data, recs.ctypes.data,
       meta.ctypes.data)
    return dict(nd_cta=nd_cta, ntiles=ntiles, nchunks=nchunks, nchan_pad=nchan_pad,
                rec_words=rec_words, raw_stride=raw_stride, prow_words=prow_words, smem=smem,
                opc=opc, esize=es, recs=recs.reshape(ntiles, nchunks, rec_words),
                meta=meta.reshape(ntiles, nchan_pad, 2))


def emulate(block, tb, ndm, nsamp_out):
    """Model of dd_dedisperse_octet on the tables; asserts all indexes."""
    nchan, pitch = block.shape
    nd, rs, pw, opc, es = tb["nd_cta"], tb["raw_stride"], tb["prow_words"], tb["opc"], tb["esize"]
    align = 16 // es
    out = np.zeros((ndm, nsamp_out))
    units_off = REC_HEADER + MAX_OCTETS_PER_CHUNK * nd
    for tile in range(tb["ntiles"]):
        for tt in range((nsamp_out + T_TILE - 1) // T_TILE):
            t_cta = tt * T_TILE
            acc = np.zeros((nd, T_TILE))
            for ch in range(tb["nchunks"]):
                rec = tb["recs"][tile, ch]
                stage = np.full(ZERO_ELEMS + GROUP * opc * rs, SENTINEL)
                stage[:ZERO_ELEMS] = 0.0
                for s in range(GROUP * opc):
                    c = ch * GROUP * opc + s
                    if c >= tb["nchan_pad"]:
                        continue
                    start, need = tb["meta"][tile, c]
                    if need <= 0:
                        assert c >= nchan
                        continue
                    # the window, clipped to the row: a channel below the
                    # reference may start before the first sample
                    off = t_cta + start
                    hi = min(off + (need * es + 15) // 16 * 16 // es, pitch)
                    lo = max(off, 0)
                    assert off % align == 0 and hi % align == 0 and 0 < hi - off <= rs
                    assert off >= -rs
                    base = ZERO_ELEMS + s * rs
                    stage[base + lo - off:base + hi - off] = block[c, lo:hi]
                no, nunits = rec[2], rec[3]
                # the kernel reads each unit's header (words 0..7) as two
                # 16-byte vectors; the record sits 16-byte aligned in shared
                # memory
                assert (units_off * 4) % 16 == 0 and (UNIT_WORDS * 4) % 16 == 0
                assert CODES_WORD + 8 <= UNIT_WORDS
                assert (REC_HEADER * 4) % 16 == 0 and (tb["rec_words"] * 4) % 16 == 0
                units = rec[units_off:units_off + UNIT_WORDS * nunits].reshape(-1, UNIT_WORDS)
                starts = rec[units_off + UNIT_WORDS * MAX_UNITS:].view(np.uint16)[:NWARPS + 1]
                assert starts[0] == 0 and starts[NWARPS] == nunits
                assert np.all(np.diff(starts.astype(int)) >= 0)
                assert starts[1] == 0  # building warp 0 queues the copies and builds nothing
                prow = np.full(pw, SENTINEL)
                written = np.zeros(pw, dtype=np.int64)
                for u in units.astype(np.int64) & 0xFFFFFFFF:
                    dest0, items = u[0] & 0xFFFFF, (u[0] >> 20) & 63
                    npat, L, bound = u[1] & 0xFF, (u[1] >> 8) & 0x1FFFFF, (u[1] >> 29) & 3
                    assert 1 <= items <= 32 and 1 <= npat <= 16 and L % 4 == 0
                    offs = [(u[2 + k // 2] >> (16 * (k & 1))) & 0xFFFF for k in range(GROUP)]
                    chan_bound = [(u[BOUNDS_WORD] >> (2 * k)) & 3 for k in range(GROUP)]
                    lanes = np.arange(items)
                    for p in range(npat):
                        words = dest0 + p * L + lanes
                        assert words.max() < pw
                        written[words] += 1
                        v = np.zeros(items)
                        code = (u[CODES_WORD + p // 2] >> (16 * (p & 1))) & 0xFFFF
                        for k in range(GROUP):
                            sh = (code >> (2 * k)) & 3
                            if k == REF_CHAN:  # the patterns' delay origin
                                assert sh == 0
                            if bound:  # the kernel then only loads shifts 0 .. bound
                                assert sh <= bound
                            assert sh <= chan_bound[k]  # and per channel 0 .. its bound
                            idx = offs[k] + lanes + sh
                            if offs[k] < ZERO_ELEMS:  # padding channel: inside the zero area
                                assert idx.max() < ZERO_ELEMS
                            else:
                                slot = (offs[k] - ZERO_ELEMS) // rs
                                assert (idx.max() - ZERO_ELEMS) // rs == slot
                            v += stage[idx]
                        prow[words] = v
                assert written.max() <= 1
                A = rec[REC_HEADER:REC_HEADER + MAX_OCTETS_PER_CHUNK * nd].reshape(
                    MAX_OCTETS_PER_CHUNK, nd)
                for o in range(no):
                    for i in range(nd):
                        w = A[o, i] + np.arange(T_TILE)
                        assert w[0] >= 0 and w[-1] < pw
                        acc[i] += prow[w]
            d0 = tile * nd
            dn = min(nd, ndm - d0)
            tn = min(T_TILE, nsamp_out - t_cta)
            out[d0:d0 + dn, t_cta:t_cta + tn] = acc[:dn, :tn]
    return out


CASES = [
    # (workload, nchan, ndm, samples past maxshift, pitch pad in elements, esize)
    ("lband_f32", 512, 70, 600, 8, 4),
    ("lband_f32", 509, 64, 900, 0, 2),    # padding channels in the last octet, f16 layout
    ("lband_f32", 515, 66, 800, 4, 4),    # last octet of 3 channels: its reference is channel 2
    ("lband_f32", 1024, 130, 700, 0, 2),
    ("full_block_u8", 256, 64, 800, 4, 4),
]


@pytest.mark.parametrize("name,nchan,ndm,extra,pad,esize", CASES)
def test_octet_kernel_model_matches_oracle(name, nchan, ndm, extra, pad, esize):
    base = synth.workload(name)
    wl = synth.scaled(base, nchan=nchan, ndm=ndm)
    wl.chan_width_mhz = base.chan_width_mhz  # full-band channel width: realistic patterns
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    tb = octet_tables(delays, nchan, ndm, ND_THR, esize) or \
        octet_tables(delays, nchan, ndm, ND_THR // 2, esize)
    assert tb is not None
    nsamp = mx + extra
    align = 16 // esize
    pitch = (nsamp + align - 1) // align * align + pad
    rng = np.random.default_rng(5)
    block = rng.integers(-8, 9, size=(nchan, pitch)).astype(np.float64)
    block[:, nsamp:] = 1e6  # row padding must never reach a stored output
    # the first DM tile starts at DM 0, where the reference channel's delay is
    # 0 while channels below it have negative relative delays at the tile's
    # larger DMs: their windows start before the first sample (clipped)
    assert (tb["meta"][0, :nchan, 0] < 0).any()
    got = emulate(block, tb, ndm, nsamp - mx)
    ref = oracle.dedisperse(block[:, :nsamp].astype(np.float32), delays, nsamp_in=nsamp)
    assert np.array_equal(got, ref)


def test_octet_tables_fit_shared_memory_for_lband():
    wl = synth.workload("lband_f32")
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    for esize in (4, 2):
        tb = octet_tables(delays, wl.nchan, wl.ndm, ND_THR, esize)
        assert tb is not None and tb["nd_cta"] == 128, esize
        stage = ZERO_ELEMS * esize + GROUP * tb["opc"] * tb["raw_stride"] * esize
        smem = 64 + 4 * tb["rec_words"] * 4 + 3 * stage + 2 * tb["prow_words"] * 4
        assert smem == tb["smem"] <= 227 * 1024


def test_octet_tables_refuse_geometries_with_too_many_patterns():
    wl = synth.workload("single_beam_f32")
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    assert octet_tables(delays, wl.nchan, wl.ndm, ND_THR, 4) is None
    assert octet_tables(delays, wl.nchan, wl.ndm, ND_THR // 2, 4) is None


def test_lband_units_select_between_two_candidates_and_stay_balanced():
    """The plan's unit choices on the L-band geometry (Sec. 2.1.1 delays):
    every build unit counts its shifts from its own smallest one, so that
    each channel selects between two candidates (bound 1), and the busiest
    building warp of a chunk carries little more than an even share."""
    wl = synth.workload("lband_f32")
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    tb = octet_tables(delays, wl.nchan, wl.ndm, ND_THR, 4)
    nd = tb["nd_cta"]
    units_off = REC_HEADER + MAX_OCTETS_PER_CHUNK * nd
    starts_off = units_off + UNIT_WORDS * MAX_UNITS
    total = busiest = 0
    for t in range(tb["ntiles"]):
        for c in range(tb["nchunks"]):
            rec = tb["recs"][t, c]
            n = int(rec[3])
            units = (rec[units_off:units_off + UNIT_WORDS * n].astype(np.int64) & 0xFFFFFFFF)
            units = units.reshape(-1, UNIT_WORDS)
            assert np.all((units[:, 1] >> 29) & 3 == 1)
            npat = units[:, 1] & 0xFF
            starts = rec[starts_off:].view(np.uint16)[:NWARPS + 1].astype(int)
            loads = [int(npat[starts[w]:starts[w + 1]].sum()) + 2 * (starts[w + 1] - starts[w])
                     for w in range(1, NWARPS)]
            total += sum(loads)
            busiest += max(loads) * len(loads)
    # pattern rows (plus a unit's fixed part) per warp: within 20% of even
    assert total / busiest > 0.8


def three_shift_splits(tb):
    """Count the 32-word ranges of a pattern-row area that the plan built as
    several units whose patterns together span three or more shifts of some
    channel (each unit counts its shifts from its own smallest one, so the
    span is taken over element offset + code)."""
    nd = tb["nd_cta"]
    units_off = REC_HEADER + MAX_OCTETS_PER_CHUNK * nd
    n = 0
    for t in range(tb["ntiles"]):
        for c in range(tb["nchunks"]):
            rec = tb["recs"][t, c].astype(np.int64) & 0xFFFFFFFF
            units = rec[units_off:units_off + UNIT_WORDS * rec[3]].reshape(-1, UNIT_WORDS)
            ranges = {}
            for u in units:  # the reference channel's offset names the (octet, range)
                ranges.setdefault(int(u[2 + REF_CHAN // 2]) >> (16 * (REF_CHAN & 1)) & 0xFFFF,
                                  []).append(u)
            for us in ranges.values():
                if len(us) < 2:
                    continue
                span = 0
                for k in range(GROUP):
                    vals = [((int(u[2 + k // 2]) >> (16 * (k & 1))) & 0xFFFF)
                            + ((int(u[CODES_WORD + p // 2]) >> (16 * (p & 1) + 2 * k)) & 3)
                            for u in us for p in range(int(u[1]) & 0xFF)]
                    span = max(span, max(vals) - min(vals))
                n += span >= 2
    return n


@pytest.mark.parametrize("esize", [4, 2])
def test_octet_kernel_model_with_three_shift_units_split(esize):
    """Low in the L-band (256 channels from 1228.2 MHz down, DMs 38.4-51.1 in
    steps of 0.1, Sec. 2.1.1 delays) some octets' channels take three shifts
    over a unit's patterns; the plan builds those words as two units that
    each select between two candidates.  The kernel model on such tables
    must still equal the oracle exactly."""
    base = synth.workload("lband_f32")
    wl = synth.scaled(base, nchan=256, ndm=128)
    wl.chan_width_mhz = base.chan_width_mhz
    wl.f_top_mhz = 1228.2
    wl.dms = 38.4 + 0.1 * np.arange(128)
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    tb = octet_tables(delays, wl.nchan, wl.ndm, ND_THR, esize)
    assert tb is not None
    assert three_shift_splits(tb) > 0
    nsamp = mx + 700
    align = 16 // esize
    pitch = (nsamp + align - 1) // align * align
    rng = np.random.default_rng(11)
    block = rng.integers(-8, 9, size=(wl.nchan, pitch)).astype(np.float64)
    block[:, nsamp:] = 1e6  # row padding must never reach a stored output
    got = emulate(block, tb, wl.ndm, nsamp - mx)
    ref = oracle.dedisperse(block[:, :nsamp].astype(np.float32), delays, nsamp_in=nsamp)
    assert np.array_equal(got, ref)
