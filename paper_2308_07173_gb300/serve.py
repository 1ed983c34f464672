"""Continuous-batching request loop for kNN + covariance over a resident map.

Scans arrive from many simulated LiDARs (the paper's estimator runs one
scan-match correction per scan, Sec. III-C3; here many sensors share one
GPU).  The map's grid stays resident on the device.  The loop:

* moves arrived requests to a pending queue (arrival times are replayed in
  real time, optionally sped up);
* admits pending requests while their device bytes (scan + idx + d2 + cov,
  each rounded up to the caching allocator's 512-byte blocks) fit in the
  HBM budget left after the step slots' fixed scratch, and a step slot is
  free;
* launches each admitted group as ONE batched kernel (pc_batch_run_scratch)
  on the slot's own stream: host-to-device copies into the slot's device
  buffers, the batched kernel and device-to-host copies into the slot's
  pinned buffers are queued on that stream, so a new step's copies and
  kernel overlap the steps already on the GPU (a slot's buffers grow to its
  largest step and are reused, so a step allocates nothing in the common
  case);
* retires steps whose completion event has fired, frees their bytes and
  slot, and stamps each request's completion time.

Latency is completion minus arrival.  ``serve_per_scan`` is the baseline:
one synchronous host-buffer call (pc_knn_cov_host) per scan in arrival
order.  Both paths run the same exact kernels, so every result is the same
alone and in the mix.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

from . import pc


@dataclass
class Request:
    rid: int
    t_arrival: float          # seconds from the start of the stream
    points: np.ndarray        # [n,3] float32
    t_sched: float = -1.0     # arrival time of this replay (t_arrival / speed)
    t_admit: float = -1.0
    t_done: float = -1.0
    q_host: object = None     # pinned input copy
    out_host: tuple = ()      # pinned idx, d2, cov
    dev: tuple = ()           # device q, idx, d2, cov while in flight

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.t_sched


def latency_report(reqs: Sequence[Request], wall: float) -> dict:
    lat = np.array([r.latency for r in reqs]) * 1e3
    pts = sum(r.n for r in reqs)
    return {
        "scans": len(reqs),
        "points": int(pts),
        "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()),
        "max_ms": float(lat.max()),
        "wall_s": wall,
        "throughput_pts_s": pts / wall if wall > 0 else float("nan"),
    }


def prepare(reqs: Sequence[Request]):
    """Pinned host copies of every request's points (a sensor driver would
    write into pinned buffers); done outside any timed region."""
    import torch

    for r in reqs:
        r.q_host = torch.from_numpy(np.ascontiguousarray(r.points, dtype=np.float32)).pin_memory()
        r.out_host = ()
        r.t_admit = r.t_done = r.t_sched = -1.0


def _pinned_outputs(n: int, k: int):
    import torch

    return (torch.empty((n, k), dtype=torch.int32, pin_memory=True),
            torch.empty((n, k), dtype=torch.float32, pin_memory=True),
            torch.empty((n, 6), dtype=torch.float32, pin_memory=True))


def admit(pending: deque, used: int, budget: int, max_step: int, busy: bool, nbytes) -> tuple:
    """One step's admission: take requests from the head of `pending` (FIFO)
    while the step has fewer than `max_step` and their device bytes
    (`nbytes(n)`) fit in `budget` beside the `used` bytes in flight.  A head
    request larger than the whole budget is admitted alone when nothing is
    in flight (`busy` false), so the queue never stalls; otherwise a request
    that does not fit waits for retirements.  Returns (batch, used)."""
    batch = []
    while pending and len(batch) < max_step:
        b = nbytes(pending[0].n)
        if used + b > budget and (batch or busy):
            break
        batch.append(pending.popleft())
        used += b
    return batch, used


ALLOC_BLOCK = 512  # torch's caching allocator rounds every block up to this


def _blocks(nbytes: int) -> int:
    return -(-int(nbytes) // ALLOC_BLOCK) * ALLOC_BLOCK


@dataclass
class _Step:
    slot: int
    reqs: List[Request]
    done: object
    nbytes: int


class Server:
    def __init__(self, target: "pc.Target", k: int, eps: float, hbm_budget: Optional[int] = None,
                 max_step_scans: int = 32, slots: int = 3, keep_results: bool = False):
        import torch

        self.t = target
        self.k = int(k)
        self.eps = float(eps)
        self.dev = target.device
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            hbm_budget = int(free * 0.5)
        self.budget = int(hbm_budget)
        self.max_step = int(max_step_scans)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(slots)]
        self.scratch_bytes = pc.pc_batch_scratch_bytes(self.max_step)
        self.scratch = [torch.empty(self.scratch_bytes, dtype=torch.uint8, device=self.dev)
                        for _ in range(slots)]
        # the slots' scan tables are held for the server's lifetime: the
        # requests share what is left of the budget
        self.fixed_bytes = slots * _blocks(self.scratch_bytes)
        self.request_budget = max(0, self.budget - self.fixed_bytes)
        self.steps_launched = 0
        self.keep = keep_results
        self.slot_buf = [None] * slots

    def request_bytes(self, n: int) -> int:
        """Device bytes one request holds while in flight: its scan, idx, d2
        and cov tensors, each rounded up to the allocator's block size."""
        return (_blocks(12 * n) + _blocks(4 * self.k * n) + _blocks(4 * self.k * n) + _blocks(24 * n))

    def _slot_buffers(self, slot: int, npts: int):
        """The slot's device and pinned host buffers, grown to hold npts
        points (q, idx, d2, cov each), so a step allocates nothing in the
        common case."""
        import torch

        have = self.slot_buf[slot]
        if have is not None and have[0] >= npts:
            return have
        cap = max(npts, 1 << 17)
        k = self.k
        dev = (torch.empty((cap, 3), dtype=torch.float32, device=self.dev),
               torch.empty((cap, k), dtype=torch.int32, device=self.dev),
               torch.empty((cap, k), dtype=torch.float32, device=self.dev),
               torch.empty((cap, 6), dtype=torch.float32, device=self.dev))
        host = _pinned_outputs(cap, k)
        self.slot_buf[slot] = (cap, dev, host)
        return self.slot_buf[slot]

    def _launch(self, slot: int, reqs: List[Request]) -> _Step:
        import torch

        s = self.streams[slot]
        npts = sum(r.n for r in reqs)
        _, (dq, di, dd, dc), (hi, hd, hc) = self._slot_buffers(slot, npts)
        descs = (pc.pc_scan * len(reqs))()
        with torch.cuda.stream(s):
            off = 0
            for j, r in enumerate(reqs):
                n = r.n
                dq[off:off + n].copy_(r.q_host, non_blocking=True)
                descs[j] = pc.pc_scan(dq[off].data_ptr() if n else 0, n, di[off].data_ptr() if n else 0,
                                      dd[off].data_ptr() if n else 0, dc[off].data_ptr() if n else 0)
                r.dev = (off, n)
                off += n
            rc = pc.pc_batch_run_scratch_array(self.t.handle, descs, len(reqs), self.k, self.eps,
                                               self.scratch[slot].data_ptr(), self.scratch_bytes,
                                               int(s.cuda_stream))
            if rc != pc.PC_OK:
                raise pc.PcError(rc, "pc_batch_run_scratch")
            if npts:
                hi[:npts].copy_(di[:npts], non_blocking=True)
                hd[:npts].copy_(dd[:npts], non_blocking=True)
                hc[:npts].copy_(dc[:npts], non_blocking=True)
            done = torch.cuda.Event()
            done.record(s)
        self.steps_launched += 1
        return _Step(slot, reqs, done, sum(self.request_bytes(r.n) for r in reqs))

    def _retire(self, st: _Step):
        """Results of a finished step: views of the slot's pinned buffers
        (copied out when the caller keeps them, since the slot is reused)."""
        _, _, (hi, hd, hc) = self.slot_buf[st.slot]
        for r in st.reqs:
            off, n = r.dev
            if self.keep:
                r.out_host = (hi[off:off + n].clone(), hd[off:off + n].clone(), hc[off:off + n].clone())
            r.dev = ()

    def serve(self, reqs: Sequence[Request], speed: float = 1.0) -> dict:
        """Replay the arrivals (times divided by `speed`) and serve them."""
        reqs = sorted(reqs, key=lambda r: r.t_arrival)
        for r in reqs:
            r.t_sched = r.t_arrival / speed
        self.steps_launched = 0
        waited = set()
        peak = 0
        pending: deque = deque()
        inflight: List[_Step] = []
        free_slots = list(range(len(self.streams)))
        used = 0
        nxt = 0
        done = 0
        t0 = time.perf_counter()
        while done < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].t_sched <= now:
                pending.append(reqs[nxt])
                nxt += 1
            for st in list(inflight):
                if st.done.query():
                    tdone = time.perf_counter() - t0
                    self._retire(st)
                    for r in st.reqs:
                        r.t_done = tdone
                    used -= st.nbytes
                    free_slots.append(st.slot)
                    inflight.remove(st)
                    done += len(st.reqs)
            if pending and free_slots:
                batch, used = admit(pending, used, self.request_budget, self.max_step, bool(inflight),
                                    self.request_bytes)
                peak = max(peak, used)
                for r in batch:
                    r.t_admit = now
                if not batch and pending[0].rid not in waited:
                    waited.add(pending[0].rid)  # the head request waits for bytes to be freed
                if batch:
                    inflight.append(self._launch(free_slots.pop(0), batch))
                    continue
            if not pending and not inflight and nxt < len(reqs):
                wait = reqs[nxt].t_sched - (time.perf_counter() - t0)
                if wait > 2e-4:
                    time.sleep(wait - 1e-4)
        wall = max(r.t_done for r in reqs) - reqs[0].t_sched
        out = latency_report(reqs, wall)
        out["steps"] = self.steps_launched
        out["mean_scans_per_step"] = len(reqs) / max(1, self.steps_launched)
        out["admission_waits"] = len(waited)  # requests that waited for budget
        out["peak_request_bytes"] = peak
        out["request_budget"] = self.request_budget
        return out


def serve_per_scan(target: "pc.Target", k: int, eps: float, reqs: Sequence[Request], speed: float = 1.0,
                   stream=None, keep_results: bool = False) -> dict:
    """Baseline: each scan in arrival order through one synchronous
    host-buffer call (copies in, kernel, copies out)."""
    import torch

    reqs = sorted(reqs, key=lambda r: r.t_arrival)
    for r in reqs:
        r.t_sched = r.t_arrival / speed
    stream = stream or torch.cuda.Stream(target.device)
    t0 = time.perf_counter()
    for r in reqs:
        wait = r.t_sched - (time.perf_counter() - t0)
        if wait > 2e-4:
            time.sleep(wait - 1e-4)
        while time.perf_counter() - t0 < r.t_sched:
            pass
        r.t_admit = time.perf_counter() - t0
        out = r.out_host if r.out_host else _pinned_outputs(r.n, k)
        target.knn_cov_host(r.q_host, k, eps, out=out, stream=stream)
        r.t_done = time.perf_counter() - t0
        r.out_host = out if keep_results else ()
    wall = max(r.t_done for r in reqs) - reqs[0].t_sched
    return latency_report(reqs, wall)


def requests_from_arrivals(arrivals) -> List[Request]:
    return [Request(i, a.t, a.points) for i, a in enumerate(arrivals)]
