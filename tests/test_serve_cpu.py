"""Admission policy of the continuous-batching server (host logic, no GPU):
FIFO, at most max_step requests per step, the HBM byte budget honoured
except for a head request larger than the whole budget when nothing is in
flight (so the queue never stalls)."""
from collections import deque

import numpy as np

from paper_2308_07173_gb300.serve import Request, admit


def reqs(sizes):
    return [Request(i, 0.0, np.zeros((n, 3), np.float32)) for i, n in enumerate(sizes)]


def nbytes(n):
    return 100 * n


def test_fifo_budget_and_step_limit():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        sizes = rng.integers(1, 50, size=int(rng.integers(0, 12))).tolist()
        q = deque(reqs(sizes))
        head = list(q)
        budget = int(rng.integers(100, 3000))
        used0 = int(rng.integers(0, budget + 1))
        max_step = int(rng.integers(1, 6))
        busy = bool(rng.integers(0, 2))
        batch, used = admit(q, used0, budget, max_step, busy, nbytes)
        assert batch == head[:len(batch)] and list(q) == head[len(batch):]  # FIFO prefix
        assert len(batch) <= max_step
        assert used == used0 + sum(nbytes(r.n) for r in batch)
        if len(batch) >= 2 or busy:
            assert used <= budget
        if batch and used > budget:  # only a lone head request over budget, nothing in flight
            assert len(batch) == 1 and not busy
        # greedy: the next request (if the step had room) would not have fit
        if q and len(batch) < max_step and (batch or busy):
            assert used + nbytes(q[0].n) > budget


def test_oversized_head_runs_alone_only_when_idle():
    q = deque(reqs([50, 1]))
    batch, used = admit(q, 0, 1000, 8, False, nbytes)  # 5000 B > budget, nothing in flight
    assert [r.rid for r in batch] == [0] and used == 5000 and [r.rid for r in q] == [1]
    q = deque(reqs([50, 1]))
    batch, used = admit(q, 0, 1000, 8, True, nbytes)  # something in flight: wait
    assert batch == [] and used == 0 and len(q) == 2


def test_empty_queue_and_full_step():
    batch, used = admit(deque(), 10, 1000, 4, False, nbytes)
    assert batch == [] and used == 10
    q = deque(reqs([1] * 10))
    batch, used = admit(q, 0, 10 ** 6, 4, False, nbytes)
    assert [r.rid for r in batch] == [0, 1, 2, 3] and len(q) == 6
