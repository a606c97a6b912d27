"""Continuous-batching step server for many simulated RL environments, each owning one gelpad.

Every environment's gel state stays resident on the device inside one tx_batch handle.
Environments issue step requests (the next indenter pose of their trajectory); a request waits in
its environment's queue (at most one request per environment is in flight, as in an RL loop),
is admitted when the in-flight working set -- the sum of the admitted gels' device footprints
(tx_gel_footprint_bytes) -- stays within the HBM budget, and is then advanced by the library one
Newton iteration at a time together with every other admitted request (tx_batch_advance).  A
request that arrives while others are on the GPU joins at the next Newton-iteration boundary;
finished requests leave the batch and free their budget immediately.

Admission takes the oldest waiting requests first.  A request too large for the budget left over
may be passed by younger requests that fit, but only `max_bypass` times: after that no younger
request is admitted ahead of it until it fits, so a large gel cannot starve behind a stream of
small ones.

All numerical work runs in the CUDA library; this module is the host scheduling loop.
"""
from __future__ import annotations

import collections
import dataclasses
import heapq
import time

import numpy as np

from . import binding as B


@dataclasses.dataclass
class Request:
    env: int
    arrival: float
    step: int
    admitted: float = float("nan")
    done: float = float("nan")
    status: int = -1
    bypassed: int = 0  # younger requests admitted while this one waited at the head of its queue


def poisson_arrivals(n_envs: int, rate: float, duration: float, seed: int):
    """(time, env) pairs of a Poisson process of total rate `rate` over `duration` seconds,
    each arrival assigned to a uniformly random environment."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        out.append((t, int(rng.integers(0, n_envs))))


class GelServer:
    """Resident gels + admission by device footprint + continuous batching."""

    def __init__(self, workloads, budget_bytes: float, precision=B.TX_PREC_MIXED, stream=None, max_bypass=8,
                 **params):
        self.wls = list(workloads)
        self.max_bypass = int(max_bypass)
        self.descs = [B.GelDesc.from_workload(w, precision=precision, **params) for w in self.wls]
        self.footprint = np.array([B.tx_gel_footprint_bytes(d) for d in self.descs], dtype=np.float64)
        self.budget = float(budget_bytes)
        if self.footprint.max() > self.budget:
            raise ValueError("the HBM budget is smaller than a single gel's footprint")
        self.handle = B.tx_batch_create(self.descs, stream=stream)
        self.n = len(self.wls)
        self.cursor = np.zeros(self.n, dtype=np.int64)  # next trajectory step of every environment
        self.queues = [collections.deque() for _ in range(self.n)]
        self.inflight = {}
        self.inflight_bytes = 0.0
        self.max_inflight_bytes = 0.0
        self.max_inflight = 0
        self.completed = []

    def close(self):
        if self.handle:
            B.tx_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- scheduling
    def enqueue(self, env: int, now: float):
        step = int(self.cursor[env])
        self.cursor[env] += 1
        self.queues[env].append(Request(env, now, step))

    def _admit(self, now: float):
        # oldest waiting request first, among environments with nothing in flight
        heads = [(q[0].arrival, e) for e, q in enumerate(self.queues) if q and e not in self.inflight]
        heads.sort()
        ids, poses, dts = [], [], []
        waiting = []  # older heads that did not fit
        for _, e in heads:
            fp = self.footprint[e]
            if self.inflight_bytes + fp > self.budget:
                waiting.append(self.queues[e][0])
                if waiting[-1].bypassed >= self.max_bypass:
                    break  # it has been passed often enough: keep the rest of the budget for it
                continue
            for w in waiting:
                w.bypassed += 1
            req = self.queues[e].popleft()
            wl = self.wls[e]
            k = req.step % len(wl.poses)
            if k == 0 and req.step > 0:  # trajectory finished: the environment resets
                B.tx_batch_reset(self.handle, e)
            req.admitted = now
            self.inflight[e] = req
            self.inflight_bytes += fp
            ids.append(e)
            poses.append(wl.poses[k])
            dts.append(wl.dt)
        if ids:
            B.tx_batch_submit(self.handle, ids, np.stack(poses), np.array(dts))
        self.max_inflight_bytes = max(self.max_inflight_bytes, self.inflight_bytes)
        self.max_inflight = max(self.max_inflight, len(self.inflight))

    def advance(self, now_fn):
        done, statuses = B.tx_batch_advance(self.handle, self.n)
        t = now_fn()
        for e, st in zip(done, statuses):
            req = self.inflight.pop(int(e))
            req.done = t
            req.status = int(st)
            self.inflight_bytes -= self.footprint[int(e)]
            self.completed.append(req)
        return len(done)

    # ---------------------------------------------------------------- driver loops
    def serve(self, arrivals, drain=True, max_wall=None):
        """Replay (time, env) arrivals in wall-clock time.  Returns the completed requests."""
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        heap = list(arrivals)
        heapq.heapify(heap)
        while heap or (drain and (self.inflight or any(self.queues))):
            t = now()
            if max_wall is not None and t > max_wall:
                break
            while heap and heap[0][0] <= t:
                ta, e = heapq.heappop(heap)
                self.enqueue(e, ta)
            self._admit(t)
            if self.inflight:
                self.advance(now)
            elif heap:
                time.sleep(max(0.0, min(heap[0][0] - now(), 0.01)))
        return self.completed

    def run_schedule(self, schedule):
        """Deterministic driver for tests: schedule[k] lists the environments that issue a request
        just before Newton round k (no wall clock involved)."""
        for k in range(len(schedule)):
            for e in schedule[k]:
                self.enqueue(e, float(k))
            self._admit(float(k))
            if self.inflight:
                self.advance(lambda: float(k))
        r = len(schedule)
        while self.inflight or any(self.queues):
            self._admit(float(r))
            self.advance(lambda: float(r))
            r += 1
        return self.completed


def latency_summary(reqs):
    """Request latency (arrival to completion) and service time (admission to completion)
    percentiles over every completed request -- failed requests, often the slowest, included --
    and, beside them, over the successful ones only, with the failure count."""
    out = {"completed": len(reqs), "failed": sum(1 for r in reqs if r.status != 0)}
    for tag, sel in (("", lambda r: True), ("ok_", lambda r: r.status == 0)):
        lat = np.array([r.done - r.arrival for r in reqs if sel(r)])
        svc = np.array([r.done - r.admitted for r in reqs if sel(r)])
        if len(lat) == 0:
            continue
        out[tag + "p50_ms"] = float(np.percentile(lat, 50) * 1e3)
        out[tag + "p99_ms"] = float(np.percentile(lat, 99) * 1e3)
        out[tag + "service_p50_ms"] = float(np.percentile(svc, 50) * 1e3)
        out[tag + "service_p99_ms"] = float(np.percentile(svc, 99) * 1e3)
    return out
