"""Run-time autotuner of the batched solve's launch shape (no counterpart in
the paper: Algorithm "ciq" fixes the arithmetic, not how a GPU schedules
many problems).

The batched tensor-core solve runs one launch per phase over every live
problem; two choices shape those launches and leave the arithmetic of each
problem's iteration unchanged apart from summation order:

* ``batch_split_rows`` / ``batch_split``: problems with at least that many
  128-row tiles split each row tile's columns over ``batch_split`` CTAs.  A
  batch's tail is a few large, ill-conditioned problems; one CTA per row tile
  then leaves most of the 148 SMs idle.
* ``check_every``: iterations queued (as one CUDA graph) between reads of
  the device's convergence flags and rebuilds of the work lists.  Finished
  problems leave only at a rebuild.

On the first call for a batch *shape* (precision, T, Q, tolerance and a
histogram of the problems' row tiles) every candidate runs the whole batch
once, timed with CUDA events, and the fastest is stored in a JSON table
(``CIQ_AUTOTUNE_TABLE`` or ``~/.cache/ciq_autotune.json``); later calls
reuse it.  All numerical work is libciq's; this module only times calls.
"""
from __future__ import annotations

import json
import math
import os

from . import _ciq

DEFAULT = dict(batch_split_rows=0, batch_split=1, check_every=8)
CANDIDATES = [
    dict(batch_split_rows=0, batch_split=1, check_every=8),
    dict(batch_split_rows=0, batch_split=1, check_every=16),
    dict(batch_split_rows=32, batch_split=2, check_every=8),
    dict(batch_split_rows=32, batch_split=2, check_every=16),
    dict(batch_split_rows=48, batch_split=4, check_every=8),
    dict(batch_split_rows=16, batch_split=2, check_every=8),
]


def table_path():
    return os.environ.get("CIQ_AUTOTUNE_TABLE", os.path.join(os.path.expanduser("~"), ".cache",
                                                             "ciq_autotune.json"))


def shape_key(problems, Q, tol, precision, op):
    """Key of a batch: precision, op, T, Q, tol and a log2 histogram of the
    problems' 128-row tile counts."""
    hist = {}
    for p in problems:
        tiles = -(-int(p["X"].shape[0]) // 128)
        b = int(math.log2(tiles))
        hist[b] = hist.get(b, 0) + 1
    T = int(problems[0]["B"].shape[0])
    h = ",".join(f"{k}:{hist[k]}" for k in sorted(hist))
    return f"{precision}|{op}|T{T}|Q{Q}|tol{tol:g}|{h}"


def load_table(path=None):
    try:
        with open(path or table_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_table(table, path=None):
    path = path or table_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_call(fn):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def tune(problems, Q, tol, op="sqrt", candidates=None, path=None, **opts):
    """The fastest launch shape for this batch shape (measured now, or read
    from the table), as a dict of options, and the timings (ms) of the
    candidates measured now (empty when the table had the key)."""
    precision = opts.get("precision", "fp32")
    key = shape_key(problems, Q, tol, precision, op)
    table = load_table(path)
    if key in table:
        return dict(table[key]["best"]), {}
    fn = _ciq.ciq_sqrt_batched if op == "sqrt" else _ciq.ciq_invsqrt_batched
    timings = {}
    for cand in candidates or CANDIDATES:
        run = dict(opts, **cand)
        ms = _time_call(lambda: fn(problems, Q, tol, **run))
        timings[json.dumps(cand, sort_keys=True)] = ms
    best = json.loads(min(timings, key=timings.get))
    table[key] = {"best": best, "ms": timings}
    save_table(table, path)
    return best, timings


def solve_batched_tuned(problems, Q, tol, op="sqrt", path=None, **opts):
    """ciq_sqrt_batched / ciq_invsqrt_batched with the tuned launch shape."""
    best, _ = tune(problems, Q, tol, op=op, path=path, **opts)
    fn = _ciq.ciq_sqrt_batched if op == "sqrt" else _ciq.ciq_invsqrt_batched
    return fn(problems, Q, tol, **dict(opts, **best))
