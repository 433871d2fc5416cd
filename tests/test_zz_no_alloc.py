"""dd_detect_noalloc against dd_detect.

dd_detect_noalloc serves callers that cannot allocate device memory at run
time (their memory is reserved up front by another allocator, or their loop
must never call cudaMalloc): it keeps its scratch in a static device array
instead of a plan's workspace.  Its candidates and count must equal those of
the plan-based dd_detect on the same dedispersed block -- exactly, as both run
the same passes -- on two calls in a row (the second call reuses the scratch
the first one left behind).  This file is collected last; it also passes on
its own in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1401_8258_gb300 as dd
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    dd.build()
    oracle.build()


def _dedispersed(dtype):
    base = synth.workload("full_block_u8" if dtype == "u8" else "lband_f32")
    wl = synth.scaled(base, nchan=256, nsamp=20000, ndm=96)
    wl.chan_width_mhz = base.chan_width_mhz
    wl.dtype = dtype
    delays, _ = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    block, _ = synth.make_block(wl, seed=9, delays=delays)
    plan = dd.Plan(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms, dtype)
    out = plan.execute(torch.from_numpy(block).cuda())
    return plan, out


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_noalloc_matches_plan_detect_twice(dtype):
    plan, out = _dedispersed(dtype)
    nsigma, cap = 3.5, 1 << 15
    ref, ref_total = plan.detect(out, nsigma, capacity=cap)
    assert 0 < ref_total <= cap
    for _ in range(2):
        cands = torch.full((cap, 16), 0xFF, dtype=torch.uint8, device="cuda")
        st, total = dd._native.dd_detect_noalloc(out, dtype, plan.ndm, out.shape[1], nsigma,
                                                 cands, cap)
        assert st == dd.DD_OK and total == ref_total
        got = cands[:total].cpu().numpy().view(dd.CANDIDATE_DTYPE).reshape(-1)
        assert np.array_equal(got, ref)
    plan.close()


def test_noalloc_overflow_and_size_limits():
    plan, out = _dedispersed("u8")
    _, ref_total = plan.detect(out, 2.0, capacity=0)
    cands = torch.empty((10, 16), dtype=torch.uint8, device="cuda")
    st, total = dd._native.dd_detect_noalloc(out, "u8", plan.ndm, out.shape[1], 2.0, cands, 10)
    assert st == dd.DD_ERR_OVERFLOW and total == ref_total
    with pytest.raises(dd.DDError) as e:  # more rows than the static scratch holds
        dd._native.dd_detect_noalloc(out, "u8", 16385, 16, 2.0, cands, 10)
    assert e.value.status == -2
    with pytest.raises(dd.DDError) as e:  # more (row, chunk) entries than it holds
        dd._native.dd_detect_noalloc(out, "u8", 4096, 4096 * 65, 2.0, cands, 10)
    assert e.value.status == -2
    plan.close()
