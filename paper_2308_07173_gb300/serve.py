"""Continuous-batching request loop for kNN + covariance over a resident map.

Scans arrive from many simulated LiDARs (the paper's estimator runs one
scan-match correction per scan, Sec. III-C3; here many sensors share one
GPU).  The map's grid stays resident on the device.  The loop:

* moves arrived requests to a pending queue (arrival times are replayed in
  real time, optionally sped up);
* sizes each of its step slots once, from the HBM budget: a slot holds the
  scan, idx, d2 and cov of up to `capacity` points on the device and the
  same outputs in pinned host memory, allocated at start-up and reused by
  every step (so serving allocates nothing);
* admits pending requests into a step (FIFO) while the step has fewer than
  `max_step` scans and its points fit the slot's capacity, when a slot is
  free; a single scan larger than the capacity runs alone on buffers grown
  for it;
* launches each step as ONE batched kernel (pc_batch_run_scratch) on the
  slot's own stream: host-to-device copies, the batched kernel and
  device-to-host copies are queued on that stream, so a new step's copies
  and kernel overlap the steps already on the GPU;
* or, with ``in_place=True``, points the step's scan table at the requests'
  page-locked scans and the slot's page-locked outputs: the batched kernel
  reads the scans and writes the results in host memory itself (each warp
  its tile's rows as whole blocks), with no copies and no device buffers
  beyond the scan table;
* retires steps whose completion event has fired, frees their slot, and
  stamps each request's completion time.

Latency is completion minus arrival.  ``serve_per_scan`` is the baseline:
one synchronous host-buffer call (pc_knn_cov_host) per scan in arrival
order.  Both paths run the same exact kernels, so every result is the same
alone and in the mix.
"""
from __future__ import annotations

import gc
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
    worst = int(np.argmax(lat))
    return {
        "scans": len(reqs),
        "points": int(pts),
        "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()),
        "max_ms": float(lat.max()),
        "max_at_s": float(reqs[worst].t_sched),  # when (in the replay) the slowest scan arrived
        "over_10ms": int((lat > 10.0).sum()),
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


def admit(pending: deque, max_step: int, capacity: int) -> list:
    """One step's admission: take requests from the head of `pending` (FIFO)
    while the step has fewer than `max_step` and their points fit in
    `capacity`.  A head request larger than the whole capacity is admitted
    alone, so the queue never stalls.  Returns the step's requests."""
    batch = []
    pts = 0
    while pending and len(batch) < max_step:
        n = pending[0].n
        if batch and pts + n > capacity:
            break
        batch.append(pending.popleft())
        pts += n
        if pts > capacity:  # a lone oversized head
            break
    return batch


ALLOC_BLOCK = 512  # torch's caching allocator rounds every block up to this


def _blocks(nbytes: int) -> int:
    return -(-int(nbytes) // ALLOC_BLOCK) * ALLOC_BLOCK


@dataclass
class _Step:
    slot: int
    reqs: List[Request]
    done: object


class Server:
    """Continuous batching over a resident target.  hbm_budget (bytes; half
    the free device memory by default) sizes the slots: each slot's scan
    table and per-point buffers (12 + 8k + 24 bytes a point) share it, so a
    step holds up to capacity = (budget / slots - table) / point bytes
    points, capped by max_step_points.  With in_place the slots hold no
    per-point device buffers (the kernel reads the requests' page-locked
    scans and writes the slot's page-locked outputs), so the capacity is
    max_step_points and the budget covers the scan tables alone."""

    def __init__(self, target: "pc.Target", k: int, eps: float, hbm_budget: Optional[int] = None,
                 max_step_scans: int = 32, slots: int = 3, keep_results: bool = False,
                 max_step_points: int = 1 << 20, in_place: bool = False):
        import torch

        self.in_place = bool(in_place)
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
        # device bytes a point of a step holds (none in place: host memory)
        self.point_bytes = 0 if self.in_place else 12 + 8 * self.k + 24
        per_slot = self.budget // slots - _blocks(self.scratch_bytes) - 4 * ALLOC_BLOCK
        self.capacity = int(max(1, min(int(max_step_points), per_slot // max(1, self.point_bytes))))
        self.slot_buf = [self._alloc(self.capacity) for _ in range(slots)]
        self.steps_launched = 0
        self.keep = keep_results

    def device_bytes(self) -> int:
        """Device memory the server holds: the slots' tables and buffers."""
        return sum(_blocks(self.scratch_bytes) + sum(_blocks(x.numel() * x.element_size()) for x in (b[1] or ()))
                   for b in self.slot_buf)

    def _alloc(self, cap: int):
        import torch

        k = self.k
        if self.in_place:
            return (cap, None, _pinned_outputs(cap, k))
        dev = (torch.empty((cap, 3), dtype=torch.float32, device=self.dev),
               torch.empty((cap, k), dtype=torch.int32, device=self.dev),
               torch.empty((cap, k), dtype=torch.float32, device=self.dev),
               torch.empty((cap, 6), dtype=torch.float32, device=self.dev))
        return (cap, dev, _pinned_outputs(cap, k))

    def _slot_buffers(self, slot: int, npts: int):
        """The slot's buffers; a lone scan above the capacity gets buffers
        grown for it (kept for the slot's later steps)."""
        if self.slot_buf[slot][0] < npts:
            self.slot_buf[slot] = self._alloc(npts)
        return self.slot_buf[slot]

    def _launch(self, slot: int, reqs: List[Request]) -> _Step:
        import torch

        s = self.streams[slot]
        npts = sum(r.n for r in reqs)
        if self.in_place:
            return self._launch_in_place(slot, s, reqs, npts)
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
        return _Step(slot, reqs, done)

    def _launch_in_place(self, slot: int, s, reqs: List[Request], npts: int) -> _Step:
        import torch

        _, _, (hi, hd, hc) = self._slot_buffers(slot, npts)
        descs = (pc.pc_scan * len(reqs))()
        off = 0
        for j, r in enumerate(reqs):
            n = r.n
            descs[j] = pc.pc_scan(r.q_host.data_ptr() if n else 0, n, hi[off].data_ptr() if n else 0,
                                  hd[off].data_ptr() if n else 0, hc[off].data_ptr() if n else 0)
            r.dev = (off, n)
            off += n
        with torch.cuda.stream(s):
            rc = pc.pc_batch_run_scratch_array(self.t.handle, descs, len(reqs), self.k, self.eps,
                                               self.scratch[slot].data_ptr(), self.scratch_bytes,
                                               int(s.cuda_stream))
            if rc != pc.PC_OK:
                raise pc.PcError(rc, "pc_batch_run_scratch")
            done = torch.cuda.Event()
            done.record(s)
        self.steps_launched += 1
        return _Step(slot, reqs, done)

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
        """Replay the arrivals (times divided by `speed`) and serve them
        (the garbage collector is paused meanwhile, as in a latency-bound
        service loop)."""
        paused = gc.isenabled()
        gc.disable()
        try:
            return self._serve(reqs, speed)
        finally:
            if paused:
                gc.enable()

    def _serve(self, reqs: Sequence[Request], speed: float) -> dict:
        reqs = sorted(reqs, key=lambda r: r.t_arrival)
        for r in reqs:
            r.t_sched = r.t_arrival / speed
        self.steps_launched = 0
        waited = set()
        peak = 0
        pending: deque = deque()
        inflight: List[_Step] = []
        free_slots = list(range(len(self.streams)))
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
                    free_slots.append(st.slot)
                    inflight.remove(st)
                    done += len(st.reqs)
            if pending and free_slots:
                batch = admit(pending, self.max_step, self.capacity)
                peak = max(peak, sum(r.n for r in batch))
                for r in batch:
                    r.t_admit = now
                inflight.append(self._launch(free_slots.pop(0), batch))
                if pending and pending[0].rid not in waited:
                    waited.add(pending[0].rid)  # did not fit this step: waits for a slot
                continue
            if pending and not free_slots and pending[0].rid not in waited:
                waited.add(pending[0].rid)  # every slot busy
            if not pending and not inflight and nxt < len(reqs):
                wait = reqs[nxt].t_sched - (time.perf_counter() - t0)
                if wait > 2e-4:
                    time.sleep(wait - 1e-4)
        wall = max(r.t_done for r in reqs) - reqs[0].t_sched
        out = latency_report(reqs, wall)
        out["steps"] = self.steps_launched
        out["mean_scans_per_step"] = len(reqs) / max(1, self.steps_launched)
        out["admission_waits"] = len(waited)  # requests that waited for a slot or a step's room
        out["peak_step_points"] = peak
        out["capacity_points"] = self.capacity
        out["device_bytes"] = self.device_bytes()
        return out


def serve_per_scan(target: "pc.Target", k: int, eps: float, reqs: Sequence[Request], speed: float = 1.0,
                   stream=None, keep_results: bool = False) -> dict:
    """Baseline: each scan in arrival order through one synchronous
    host-buffer call (copies in, kernel, copies out)."""
    paused = gc.isenabled()
    gc.disable()
    try:
        return _per_scan(target, k, eps, reqs, speed, stream, keep_results)
    finally:
        if paused:
            gc.enable()


def _per_scan(target, k, eps, reqs, speed, stream, keep_results) -> dict:
    import torch

    reqs = sorted(reqs, key=lambda r: r.t_arrival)
    for r in reqs:
        r.t_sched = r.t_arrival / speed
    stream = stream or torch.cuda.Stream(target.device)
    # one set of pinned outputs for the largest scan, allocated before the
    # replay (a service would hold them), unless every result is kept
    shared = None if keep_results else _pinned_outputs(max(r.n for r in reqs), k)
    t0 = time.perf_counter()
    for r in reqs:
        wait = r.t_sched - (time.perf_counter() - t0)
        if wait > 2e-4:
            time.sleep(wait - 1e-4)
        while time.perf_counter() - t0 < r.t_sched:
            pass
        r.t_admit = time.perf_counter() - t0
        if shared is not None:
            out = tuple(x[:r.n] for x in shared)
        else:
            out = r.out_host if r.out_host else _pinned_outputs(r.n, k)
        target.knn_cov_host(r.q_host, k, eps, out=out, stream=stream)
        r.t_done = time.perf_counter() - t0
        r.out_host = out if keep_results else ()
    wall = max(r.t_done for r in reqs) - reqs[0].t_sched
    return latency_report(reqs, wall)


def requests_from_arrivals(arrivals) -> List[Request]:
    return [Request(i, a.t, a.points) for i, a in enumerate(arrivals)]
