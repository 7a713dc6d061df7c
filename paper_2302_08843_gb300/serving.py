"""Continuous-batching server for relax requests.

Requests are (arrival time, Workload) pairs with uniform materials.  A request
goes to the size bucket of its grid (shape and cell size); each bucket keeps
batch states (mm_batch, one CUDA stream each) whose tensor spectrum is built
once -- the bucket's cached plan -- and whose slots hold one request each.

Every loop iteration
  1. moves requests whose arrival time has passed to the waiting list,
  2. admits waiting requests into free slots, creating a new batch state for
     a bucket only while the summed device footprint of all batch states stays
     under the HBM cap (idle batch states of other buckets are released first;
     a request whose batch state alone is above the cap is rejected),
  3. enqueues one Dormand-Prince attempt on every batch state with running
     slots (all streams in flight together), then collects them all: each
     slot is accepted or rejected on its own, converged slots leave and free
     their slot for the next arrival.
So requests join and leave while others are on the GPU, and the attempts of
different buckets overlap on the device.  A request's result does not depend
on the requests it shares a batch with (per-slot arithmetic and reductions).
"""
import collections
import time

import numpy as np


class Server:
    REJECTED = 5

    def __init__(self, precision="fp32", hbm_cap=40e9, capacity=8, p=20, tol=1e-3, rtol=1e-5, max_steps=20000,
                 max_states_per_bucket=None):
        self.precision = precision
        self.hbm_cap = float(hbm_cap)
        self.capacity = int(capacity)
        self.max_states = max_states_per_bucket
        self.p = int(p)
        self.tol, self.rtol, self.max_steps = tol, rtol, max_steps
        self.buckets = collections.OrderedDict()     # key -> [Batch]
        self.used = 0
        self.peak_used = 0

    @staticmethod
    def bucket_key(w):
        return (tuple(w.n), tuple(w.dx))

    def _release_idle(self, need, busy):
        for key in list(self.buckets):
            for b in list(self.buckets[key]):
                if self.used + need <= self.hbm_cap:
                    return
                if id(b) not in busy:
                    self.buckets[key].remove(b)
                    self.used -= b.footprint
                    b.close()

    def _place(self, w, occupied, busy):
        """(batch, slot) for request w, (None, None) to wait, ("reject", None)
        when its batch state can never fit under the cap."""
        from . import binding
        key = self.bucket_key(w)
        states = self.buckets.get(key, [])
        for b in states:
            free = [s for s in range(b.capacity) if (id(b), s) not in occupied]
            if free:
                return b, free[0]
        if self.max_states is not None and len(states) >= self.max_states:
            return None, None
        need = binding.Batch.footprint_of(w.n, w.dx, self.precision, self.capacity)
        if need > self.hbm_cap:
            return "reject", None
        if self.used + need > self.hbm_cap:
            self._release_idle(need, busy)
        if self.used + need > self.hbm_cap:
            return None, None
        b = binding.Batch(w.n, w.dx, self.precision, self.capacity, self.p)
        self.buckets.setdefault(key, []).append(b)
        self.used += b.footprint
        self.peak_used = max(self.peak_used, self.used)
        return b, 0

    def run(self, requests, realtime=True, keep_m=False):
        """Serve `requests` [(arrival_s, Workload)]; returns one dict per request
        (index order) with arrival, admit and finish times (s, relative to the
        start), latency, steps, final torque, status and optionally the final m."""
        from .workloads import to_soa
        order = sorted(range(len(requests)), key=lambda i: requests[i][0])
        incoming = collections.deque(order)
        waiting = collections.deque()
        occupied = {}          # (id(batch), slot) -> request index
        where = {}             # request index -> (batch, slot)
        results = [None] * len(requests)
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else (lambda: float("inf"))
        iterations = 0
        while incoming or waiting or occupied:
            now = clock()
            while incoming and requests[incoming[0]][0] <= now:
                waiting.append(incoming.popleft())
            busy = {id(b) for (b, _) in where.values()}
            for idx in list(waiting):
                arr, w = requests[idx]
                b, slot = self._place(w, occupied, busy)
                if b is None:
                    continue
                if isinstance(b, str):
                    now = time.perf_counter() - t0
                    results[idx] = {"arrival": arr, "admitted": None, "finished": now,
                                    "latency": now - (arr if realtime else 0.0), "steps": 0,
                                    "torque": float("nan"), "status": self.REJECTED}
                    waiting.remove(idx)
                    continue
                b.set_slot(slot, w.Ms, w.A, w.alpha, to_soa(w.m0), 1e-13)
                occupied[(id(b), slot)] = idx
                where[idx] = (b, slot)
                busy.add(id(b))
                waiting.remove(idx)
                results[idx] = {"arrival": arr, "admitted": time.perf_counter() - t0}
            if not occupied:
                if incoming:
                    delay = requests[incoming[0]][0] - clock()
                    if delay > 0:
                        time.sleep(min(delay, 0.01))
                continue
            batches = list({id(b): b for (b, _) in where.values()}.values())
            for b in batches:
                b.begin(self.rtol)
            for b in batches:
                status, steps, torque = b.end(self.tol, self.max_steps)
                for slot in range(b.capacity):
                    idx = occupied.get((id(b), slot))
                    if idx is None or status[slot] <= 1:
                        continue
                    r = results[idx]
                    r["finished"] = time.perf_counter() - t0
                    r["latency"] = r["finished"] - (r["arrival"] if realtime else 0.0)
                    r["steps"] = int(steps[slot])
                    r["torque"] = float(torque[slot])
                    r["status"] = int(status[slot])
                    if keep_m:
                        r["m"] = b.get_m(slot)
                    b.clear_slot(slot)
                    del occupied[(id(b), slot)]
                    del where[idx]
            iterations += 1
        self.iterations = iterations
        self.elapsed = time.perf_counter() - t0
        return results

    def close(self):
        for key in list(self.buckets):
            for b in self.buckets[key]:
                b.close()
        self.buckets.clear()
        self.used = 0


def latency_summary(results, elapsed):
    """p50/p99/mean latency (arrival -> result, s) and throughput of served requests."""
    done = [r for r in results if r["status"] != Server.REJECTED]
    lat = np.array([r["latency"] for r in done])
    steps = np.array([r["steps"] for r in done])
    return {"requests": len(results), "rejected": len(results) - len(done), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "throughput_req_s": len(done) / elapsed,
            "steps_total": int(steps.sum()), "converged": int(sum(r["status"] == 2 for r in results)),
            "hit_max_steps": int(sum(r["status"] == 3 for r in results)),
            "failed": int(sum(r["status"] == 4 for r in results))}
