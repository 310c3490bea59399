"""Host-side logic of the learned pipeline (no GPU): the batch schedule that
paper_2006_11267_b300.learned sizes ahead of time from predicted iterations."""
import numpy as np

from paper_2006_11267_b300 import learned


def test_batch_schedule_partitions_and_groups_long_problems():
    # The learned pipeline's schedule: every problem exactly once; problems
    # predicted to need >= long_iters iterations in one final batch; the rest
    # in batches of at most `batch` in order of predicted iterations.
    rng = np.random.default_rng(4)
    pred = np.log(rng.uniform(5, 1000, size=1300))
    batches = learned.batch_schedule(pred, batch=256, long_iters=500)
    flat = [i for b in batches for i in b]
    assert sorted(flat) == list(range(1300))
    long = [i for i in range(1300) if pred[i] >= np.log(500)]
    assert sorted(batches[-1]) == sorted(long)
    assert all(len(b) <= 256 for b in batches[:-1])
    order = [pred[i] for b in batches[:-1] for i in b]
    assert order == sorted(order)
    # no long problems: only batches of the short ones
    b2 = learned.batch_schedule(np.log(np.full(10, 3.0)), batch=4, long_iters=500)
    assert [len(b) for b in b2] == [4, 4, 2]
