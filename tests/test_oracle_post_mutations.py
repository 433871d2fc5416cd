"""Plant plausible mistakes in a copy of ``oracle/post.py`` and check that the
pins in ``test_oracle_post_pins`` catch every one of them.

Each mutant is a textual edit of the module's source, loaded as a separate
module; a mutant is caught when some pin fails (assertion or exception).
"""
import importlib.util
import os

import pytest

import oracle
from tests import test_oracle_post_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "post.py")

MUTANTS = {
    "median of the sorted window off by one": ("return np.sort(windows, axis=-1)[..., h]",
                                               "return np.sort(windows, axis=-1)[..., h + 1]"),
    "median edges wrap around": ('mode="edge"', 'mode="wrap"'),
    "median window not centred": ("padded = np.pad(x, ((0, 0), (h, h)), mode=\"edge\")",
                                  "padded = np.pad(x, ((0, 0), (0, 2 * h)), mode=\"edge\")"),
    "slope without centring y": ("np.sum((t - t_mean) * (y[r] - y_mean)) / stt",
                                 "np.sum(t * y[r]) / stt"),
    "intercept sign flipped": ("a = y_mean - b * t_mean", "a = y_mean + b * t_mean"),
    "sample std (n-1)": ("s = np.sqrt(np.mean(res * res))",
                         "s = np.sqrt(np.sum(res * res) / max(n - 1, 1))"),
    "mean only, no trend removed": ("res = y[r] - (a + b * t)", "res = y[r] - y_mean"),
    "boxcar partner at t + 2w": ("s = s[:, :-half] + s[:, half:]",
                                 "s = s[:, :-2 * half] + s[:, 2 * half:] if s.shape[1] > 2 * half "
                                 "else s[:, :0]"),
    "boxcar noise grows as w": ("np.sqrt(np.float64(w))", "np.float64(w)"),
    "boxcar without the mean": ("sum_w.astype(np.float64) - w * mean[:, None]",
                                "sum_w.astype(np.float64) - mean[:, None]"),
    "threshold not strict": ("hit = (snr > thr)", "hit = (snr >= thr)"),
    "largest width kept on ties and beyond": ("better = hit & (snr > best[:, :m])",
                                              "better = hit"),
    "sigma zero rows not skipped": ("hit = (snr > thr) & ok[:, None]", "hit = (snr > thr)"),
}


def load_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    path = tmp_path / "post_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("post_mutant", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_post_pins_catch_planted_mistake(name, tmp_path):
    mod = load_mutant(name, tmp_path)
    caught = []
    for pin in pins.PINS:
        try:
            pin(mod)
        except pytest.skip.Exception:
            continue
        except Exception as e:  # an assertion or an error both count
            caught.append((pin.__name__, type(e).__name__))
    assert caught, f"no pin caught: {name}"
