"""Admission policy of the continuous-batching server (host logic, no GPU):
FIFO, at most max_step requests per step, the step's points within the
slot capacity, except for a lone head request larger than the capacity (so
the queue never stalls)."""
from collections import deque

import numpy as np

from paper_2308_07173_gb300.serve import Request, admit


def reqs(sizes):
    return [Request(i, 0.0, np.zeros((n, 3), np.float32)) for i, n in enumerate(sizes)]


def test_fifo_capacity_and_step_limit():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        sizes = rng.integers(1, 50, size=int(rng.integers(0, 12))).tolist()
        q = deque(reqs(sizes))
        head = list(q)
        capacity = int(rng.integers(1, 200))
        max_step = int(rng.integers(1, 6))
        batch = admit(q, max_step, capacity)
        assert batch == head[:len(batch)] and list(q) == head[len(batch):]  # FIFO prefix
        assert len(batch) <= max_step
        pts = sum(r.n for r in batch)
        if len(batch) >= 2:
            assert pts <= capacity
        if pts > capacity:  # only a lone head request over the capacity
            assert len(batch) == 1
        if head:
            assert batch  # the head is always admitted
        # greedy: the next request (if the step had room) would not have fit
        if q and len(batch) < max_step and pts <= capacity:
            assert pts + q[0].n > capacity


def test_oversized_head_runs_alone():
    q = deque(reqs([50, 1]))
    batch = admit(q, 8, 10)
    assert [r.rid for r in batch] == [0] and [r.rid for r in q] == [1]
    batch = admit(q, 8, 10)
    assert [r.rid for r in batch] == [1] and not q


def test_empty_queue_and_full_step():
    assert admit(deque(), 4, 1000) == []
    q = deque(reqs([1] * 10))
    batch = admit(q, 4, 10 ** 6)
    assert [r.rid for r in batch] == [0, 1, 2, 3] and len(q) == 6
