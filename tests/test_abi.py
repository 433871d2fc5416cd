"""CPU-side checks of the C ABI: the library builds and loads, exports every
symbol that include/*.h declares, and its host-side planner agrees with the
oracle.  No compute call reaches a GPU here."""
import glob
import os
import re

import numpy as np
import pytest

import oracle
import paper_1401_8258_gb300 as dd
import synth
from paper_1401_8258_gb300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    dd.build()
    oracle.build()


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(dd_[A-Za-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    lib = _native.load()
    names = _declared_functions()
    assert {"dd_plan_create", "dd_execute", "dd_detect", "dd_compute_delays"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    bound = {name for name, _, _ in _native.SIGNATURES}
    assert _declared_functions() <= bound


def test_status_strings():
    assert dd.dd_status_string(0) == "ok"
    assert "capacity" in dd.dd_status_string(-6)
    assert dd.dd_status_string(12345) == "unknown status"


@pytest.mark.parametrize("name", ["single_beam_f32", "full_block_u8", "lband_f32"])
def test_planner_delay_table_equals_oracle(name):
    wl = synth.workload(name)
    got, mx = dd.dd_compute_delays(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    ref, rmx = oracle.delay_table(wl.nchan, wl.f_top_mhz, wl.chan_width_mhz, wl.t_samp_s, wl.dms)
    assert mx == rmx
    assert np.array_equal(got, ref)


def test_planner_delay_table_equals_oracle_random_geometries():
    rng = np.random.default_rng(9)
    for _ in range(40):
        nchan = int(rng.integers(1, 600))
        f_top = float(rng.uniform(50, 3000))
        df = float(rng.uniform(1e-4, 0.9)) * f_top / nchan
        ts = float(rng.uniform(1e-6, 1e-3))
        dms = rng.uniform(0, 2000, int(rng.integers(1, 50)))
        got, mx = dd.dd_compute_delays(nchan, f_top, df, ts, dms)
        ref, rmx = oracle.delay_table(nchan, f_top, df, ts, dms)
        assert mx == rmx and np.array_equal(got, ref)


@pytest.mark.parametrize("args", [
    (0, 416.0, 0.25, 1e-4, [1.0]),          # no channels
    (64, 416.0, 0.0, 1e-4, [1.0]),          # zero width
    (64, 416.0, 0.25, -1e-4, [1.0]),        # negative sampling time
    (64, 10.0, 0.25, 1e-4, [1.0]),          # bottom channel below 0 MHz
    (64, 416.0, 0.25, 1e-4, [float("nan")]),
    (64, 416.0, 0.25, 1e-4, [-0.5]),
    (64, 416.0, 0.25, 1e-4, []),            # no DM trials
])
def test_compute_delays_rejects_bad_arguments(args):
    with pytest.raises(dd.DDError) as e:
        dd.dd_compute_delays(*args)
    assert e.value.status == -1


def test_compute_delays_reports_int32_overflow():
    with pytest.raises(dd.DDError) as e:
        dd.dd_compute_delays(16, 100.0, 6.0, 1e-9, [1e6])
    assert e.value.status == -8
