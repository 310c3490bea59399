"""Host logic of the batched-solve autotuner (paper_2006_11267_b300/autotune.py):
the shape key, the persisted table, candidate timing and reuse, with the
library's batched call and the timer replaced by fakes (no GPU)."""
import json

import numpy as np

from paper_2006_11267_b300 import autotune


class _Arr:
    def __init__(self, *shape):
        self.shape = shape


def _probs(ns, t=8):
    return [dict(X=_Arr(n, 3), B=_Arr(t, n)) for n in ns]


def test_shape_key_bins_row_tiles_and_separates_settings():
    a = autotune.shape_key(_probs([256, 300, 5000]), 8, 1e-4, "fp16", "sqrt")
    b = autotune.shape_key(_probs([260, 290, 5100]), 8, 1e-4, "fp16", "sqrt")
    assert a == b                                      # same log2 row-tile histogram
    assert a != autotune.shape_key(_probs([256, 300, 9000]), 8, 1e-4, "fp16", "sqrt")
    assert a != autotune.shape_key(_probs([256, 300, 5000]), 8, 1e-4, "fp32", "sqrt")
    assert a != autotune.shape_key(_probs([256, 300, 5000], t=16), 8, 1e-4, "fp16", "sqrt")
    assert a != autotune.shape_key(_probs([256, 300, 5000]), 8, 1e-4, "fp16", "invsqrt")


def test_tune_measures_once_then_reuses_the_table(tmp_path, monkeypatch):
    calls = []
    cost = {(0, 1, 8): 5.0, (0, 1, 16): 4.0, (32, 2, 8): 3.0, (32, 2, 16): 3.5, (48, 4, 8): 6.0, (16, 2, 8): 3.2}

    def fake_batched(problems, Q, tol, **opts):
        calls.append(opts)
        return None, None

    def fake_time(fn):
        fn()
        o = calls[-1]
        return cost[(o["batch_split_rows"], o["batch_split"], o["check_every"])]

    monkeypatch.setattr(autotune._ciq, "ciq_sqrt_batched", fake_batched)
    monkeypatch.setattr(autotune, "_time_call", fake_time)
    path = str(tmp_path / "table.json")
    probs = _probs([256, 1000, 8000])
    best, timings = autotune.tune(probs, 8, 1e-4, path=path, precision="fp16")
    assert best == dict(batch_split_rows=32, batch_split=2, check_every=8)
    assert len(timings) == len(autotune.CANDIDATES) and len(calls) == len(autotune.CANDIDATES)
    assert all(c["precision"] == "fp16" for c in calls)
    table = json.load(open(path))
    assert list(table.values())[0]["best"] == best
    n = len(calls)
    best2, timings2 = autotune.tune(probs, 8, 1e-4, path=path, precision="fp16")
    assert best2 == best and timings2 == {} and len(calls) == n       # read from the table
    autotune.solve_batched_tuned(probs, 8, 1e-4, path=path, precision="fp16")
    assert calls[-1]["batch_split"] == 2 and len(calls) == n + 1
