"""CPU checks of the staged u8 kernel's plan-time tables.

The tables (dd_quad_plan.cpp) tell the kernel which bytes to bulk-copy,
how to sum four channels into pattern rows of sample pairs (t, t + 256) and
where each DM trial reads.  A numpy model of the kernel's three phases (copy,
build, accumulate) runs on them here, asserting every shared-memory and global
index against the buffer it addresses and the 16-bit range of every packed
half between drains, and its result must equal the oracle bit for bit.
Uncopied / unbuilt bytes hold garbage so that a read of them shows up.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1401_8258_gb300 as dd
import synth

T_TILE = 512
HALF = T_TILE // 2
QUADS_PER_CHUNK = 4
FLUSH_CHUNKS = 64 // QUADS_PER_CHUNK
REC_HEADER = 4
UNIT_WORDS = 20
NWARPS = 12  # building warps
ND_THR = 4  # DM trials per thread of the 64-trial tile (16 warps x 4); 2 for the 32-trial one


@pytest.fixture(scope="module", autouse=True)
def built():
    dd.build()
    oracle.build()


def quad_tables(delays, nchan, ndm, nd_thr):
    lib = ctypes.CDLL(dd._native.library_path())
    fn = lib.ddi_quad_tables
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    info = np.zeros(9, dtype=np.int32)
    fn(delays.ctypes.data, nchan, ndm, nd_thr, info.ctypes.data, None, None)
    if not info[0]:
        return None
    ok, nd_cta, ntiles, nchunks, nchan_pad, rec_words, raw_stride, prow_words, smem = info.tolist()
    recs = np.zeros(ntiles * nchunks * rec_words, dtype=np.int32)
    meta = np.zeros(ntiles * nchan_pad * 2, dtype=np.int32)
    fn(delays.ctypes.data, nchan, ndm, nd_thr, info.ctypes.data, recs.ctypes.data, meta.ctypes.data)
    return dict(nd_cta=nd_cta, ntiles=ntiles, nchunks=nchunks, nchan_pad=nchan_pad,
                rec_words=rec_words, raw_stride=raw_stride, prow_words=prow_words, smem=smem,
                recs=recs.reshape(ntiles, nchunks, rec_words),
                meta=meta.reshape(ntiles, nchan_pad, 2))


def emulate(block, nsamp_in, tb, ndm, nsamp_out):
    """Model of dd_dedisperse_quad_u8 on the tables; asserts all indexes."""
    nchan, pitch = block.shape
    nd = tb["nd_cta"]
    rs = tb["raw_stride"]
    pw = tb["prow_words"]
    out = np.zeros((ndm, nsamp_out), dtype=np.int64)
    ntt = (nsamp_out + T_TILE - 1) // T_TILE
    garbage = np.uint8(0xA5)
    for tile in range(tb["ntiles"]):
        for tt in range(ntt):
            t_cta = tt * T_TILE
            acc = np.zeros((nd, T_TILE), dtype=np.int64)
            packed = np.zeros((nd, T_TILE), dtype=np.int64)  # the 16-bit halves
            for ch in range(tb["nchunks"]):
                rec = tb["recs"][tile, ch]
                raw = np.full((4 * QUADS_PER_CHUNK, rs), garbage, dtype=np.uint8)
                for s in range(4 * QUADS_PER_CHUNK):
                    c = ch * 4 * QUADS_PER_CHUNK + s
                    if c >= tb["nchan_pad"]:
                        continue
                    start, need = tb["meta"][tile, c]
                    if need <= 0:
                        assert c >= nchan
                        continue
                    off = t_cta + start
                    hi = min(off + (need + 15) // 16 * 16, pitch)
                    lo = max(off, 0)
                    assert off % 16 == 0 and off >= -16 and hi > lo
                    assert (hi - lo) % 16 == 0 and hi - off <= rs
                    raw[s, lo - off:hi - off] = block[c, lo:hi]
                nq, nunits = rec[2], rec[3]
                units_off = REC_HEADER + QUADS_PER_CHUNK * nd
                units = rec[units_off:units_off + UNIT_WORDS * nunits].reshape(-1, UNIT_WORDS)
                # per-warp unit ranges, int16 pairs after the unit array
                starts = rec[units_off + UNIT_WORDS * 32:].view(np.uint16)[:NWARPS + 1]
                assert starts[0] == 0 and starts[NWARPS] == nunits
                assert np.all(np.diff(starts.astype(int)) >= 0)
                raw_flat = raw.reshape(-1)
                # row words as (low half, high half); unbuilt words hold garbage
                prow = np.full((pw, 2), 77777, dtype=np.int64)
                written = np.zeros(pw, dtype=np.int64)
                for u in units.astype(np.int64) & 0xFFFFFFFF:  # one warp-wide step
                    items = (u[2] >> 20) & 63
                    npat = u[2] >> 26
                    dest0 = u[2] & 0xFFFFF
                    L = u[3] & 0xFFFF
                    assert 1 <= items <= 32 and 1 <= npat <= 8 and dest0 % 4 == 0 and L % 4 == 0
                    offs = [u[0] & 0xFFFF, u[0] >> 16, u[1] & 0xFFFF, u[1] >> 16]
                    lanes = np.arange(items)
                    for p in range(npat):
                        sels = [u[3] >> 16, u[4 + 2 * p] & 0xFFFF, u[4 + 2 * p] >> 16,
                                u[5 + 2 * p] & 0xFFFF]
                        words = (dest0 + p * L + 4 * lanes[:, None] + np.arange(4)[None, :]).reshape(-1)
                        assert words.max() < pw
                        written[words] += 1
                        prow[words] = 0
                        for k in range(4):
                            if offs[k] == 0xFFFF:
                                continue
                            sh = sels[k] & 0xF
                            # a 4-byte funnel inside the two loaded words
                            assert sels[k] == 0x3210 + 0x1111 * sh and sh <= 4
                            base = offs[k] + 4 * lanes
                            slot = offs[k] // rs
                            # two aligned words per half, all inside this channel's slot
                            assert base.min() % 4 == 0 and (base.max() + HALF + 7) // rs == slot
                            for h in range(2):
                                byte = (base[:, None] + h * HALF + sh + np.arange(4)[None, :]).reshape(-1)
                                prow[words, h] += raw_flat[byte]
                assert written.max() <= 1  # no row word is built twice
                A = rec[REC_HEADER:REC_HEADER + QUADS_PER_CHUNK * nd].reshape(QUADS_PER_CHUNK, nd)
                for q in range(nq):
                    for i in range(nd):
                        w = A[q, i] + np.arange(HALF)
                        assert w[0] >= 0 and w[-1] < pw
                        packed[i, :HALF] += prow[w, 0]
                        packed[i, HALF:] += prow[w, 1]
                assert packed.max() < 65536  # 16-bit halves never carry
                if (ch + 1) % FLUSH_CHUNKS == 0 or ch + 1 == tb["nchunks"]:
                    acc += packed
                    packed[:] = 0
            d0 = tile * nd
            dn = min(nd, ndm - d0)
            tn = min(T_TILE, nsamp_out - t_cta)
            out[d0:d0 + dn, t_cta:t_cta + tn] = acc[:dn, :tn]
    return out


CASES = [
    # (workload, nchan, ndm, extra samples past maxshift, pitch pad)
    ("full_block_u8", 1024, 128, 1100, 0),
    ("full_block_u8", 1021, 100, 700, 16),
    ("lband_f32", 512, 70, 600, 48),
    ("full_block_u8", 1036, 64, 900, 0),  # last chunk holds 3 quads
]

# Geometries whose first DM tile needs a row origin before sample 0 (the
# window of the band-top channel then starts at -16): (f_top MHz, channel
# width MHz, t_samp s, first DM, DM step, nchan, ndm)
SLACK_GEOMETRIES = [
    (559.74, 0.7752, 51.2e-6, 0.8816, 0.02105, 64, 100),
    (728.89, 5.5687, 64e-6, 0.917, 0.00745, 16, 40),
]


@pytest.mark.parametrize("name,nchan,ndm,extra,pad", CASES)
def test_quad_kernel_model_matches_oracle(name, nchan, ndm, extra, pad):
    wl = synth.scaled(synth.workload(name), nchan=nchan, ndm=ndm)
    # keep the channel width of the full band so that pattern counts are realistic
    wl.chan_width_mhz = synth.workload(name).chan_width_mhz
    delays, mx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    tb = quad_tables(delays, wl.nchan, wl.ndm, ND_THR) or quad_tables(delays, wl.nchan, wl.ndm, ND_THR // 2)
    assert tb is not None
    nsamp = mx + extra
    pitch = (nsamp + 15) // 16 * 16 + pad
    rng = np.random.default_rng(12)
    block = synth.random_block(rng, wl.nchan, nsamp, "u8", pitch)
    block[:, nsamp:] = 0xEE  # row padding must never reach a valid output
    nout = nsamp - mx
    got = emulate(block, nsamp, tb, wl.ndm, nout)
    ref = oracle.dedisperse(block, delays, nsamp_in=nsamp)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("geo", SLACK_GEOMETRIES)
def test_quad_kernel_model_with_row_origin_before_first_sample(geo):
    f_top, df, ts, dm0, step, nchan, ndm = geo
    dms = dm0 + step * np.arange(ndm)
    delays, mx = oracle.delay_table(nchan, f_top, df, ts, dms)
    tb = quad_tables(delays, nchan, ndm, ND_THR) or quad_tables(delays, nchan, ndm, ND_THR // 2)
    assert tb is not None and (tb["meta"][:, :, 0] < 0).any()
    nsamp = mx + 1300
    pitch = (nsamp + 15) // 16 * 16
    block = synth.random_block(np.random.default_rng(4), nchan, nsamp, "u8", pitch)
    got = emulate(block, nsamp, tb, ndm, nsamp - mx)
    assert np.array_equal(got, oracle.dedisperse(block, delays, nsamp_in=nsamp))


def test_tables_fit_shared_memory_for_the_workloads():
    for name in ("full_block_u8", "lband_f32"):
        wl = synth.workload(name)
        delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
        tb = quad_tables(delays, wl.nchan, wl.ndm, ND_THR)
        assert tb is not None and tb["nd_cta"] == 64, name
        meta = (tb["nchan_pad"] * 8 + 15) // 16 * 16
        smem = 64 + meta + 4 * tb["rec_words"] * 4 + 3 * 16 * tb["raw_stride"] + 2 * tb["prow_words"] * 4
        # (2 row stages, 4 record stages, 3 raw stages)
        assert smem == tb["smem"] <= 227 * 1024


def test_tables_refuse_geometries_with_too_many_patterns():
    # 64 channels of 0.25 MHz at DM step 1: relative delays change at almost
    # every trial, so the plan must fall back to the plain-load kernel
    wl = synth.workload("single_beam_f32")
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    assert quad_tables(delays, wl.nchan, wl.ndm, ND_THR) is None
    assert quad_tables(delays, wl.nchan, wl.ndm, ND_THR // 2) is None


@pytest.mark.parametrize("name", ["full_block_u8", "single_beam_f32"])
def test_shared_memory_per_staging_depth(name):
    """The kernel keeps copy_ahead + 1 window buffers and 2 + copy_ahead
    records (plus the barrier area, the window table and two pattern-row
    areas); depths outside 1..3 are refused."""
    wl = synth.scaled(synth.workload(name), nchan=256, ndm=128)
    wl.dtype = "u8"
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    lib = ctypes.CDLL(dd._native.library_path())
    fn = lib.ddi_quad_smem
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                   ctypes.c_int32, ctypes.c_void_p]
    d = np.ascontiguousarray(delays, dtype=np.int32)
    for nd_thr in (4, 2, 1):
        tb = quad_tables(d, wl.nchan, wl.ndm, nd_thr)
        if tb is None:
            continue
        meta = (tb["nchan_pad"] * 8 + 15) // 16 * 16
        for ca in (0, 1, 2, 3, 4):
            out = np.zeros(1, dtype=np.int32)
            fn(d.ctypes.data, wl.nchan, wl.ndm, nd_thr, ca, out.ctypes.data)
            want = (64 + meta + (2 + ca) * tb["rec_words"] * 4 + (ca + 1) * 16 * tb["raw_stride"]
                    + 2 * tb["prow_words"] * 4)
            if 1 <= ca <= 3 and want <= 227 * 1024:
                assert out[0] == want, (nd_thr, ca)
            else:
                assert out[0] == -1, (nd_thr, ca)
            if ca == 2:
                assert out[0] == tb["smem"]
