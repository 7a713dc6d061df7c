"""Continuous-batching server for relax requests.

Requests are (arrival time, Workload) pairs with uniform materials (and,
through Workload.extra, an optional uniform DMI "D" of kind "dmi" and the
"precession" switch, Sec. 4.3 and Sec. 3).  A request
goes to the size bucket of its grid (shape and cell size); each bucket keeps
batch states (mm_batch, one CUDA stream each) whose tensor spectrum is built
once -- the bucket's cached plan -- and whose slots hold one request each.
The number of slots of a bucket's state is sized to its grid (small grids get
more slots, so that every launch still fills the GPU).

The loop, repeated until every request is answered:
  1. requests whose arrival time has passed join the waiting list;
  2. waiting requests are admitted into free slots of idle batch states; a new
     batch state is created for a bucket only while the summed device
     footprint of all batch states stays under the HBM cap (idle states of
     other buckets are released first; a request whose state alone is above
     the cap is rejected);
  3. every idle batch state with running slots is given `attempts`
     Dormand-Prince attempts (one CUDA graph launch; each accept/reject and
     step-size decision is taken on the device, per slot);
  4. every batch state whose work has finished (a non-blocking event query)
     is collected: converged slots leave and free their slot for the next
     arrival, the others keep going.
Batch states advance independently on their own streams -- a bucket of small
grids is not held back by a bucket of large ones -- and their work overlaps on
the device.  A request's result does not depend on the requests it shares a
batch with (per-slot arithmetic and reductions, grids never share an FFT).
"""
import collections
import time

import numpy as np


def auto_capacity(n, target_cells=1 << 21, lo=4, hi=32):
    """Slots per batch state: about `target_cells` cells per launch, a power of
    two in [lo, hi]."""
    cells = int(n[0]) * int(n[1]) * int(n[2])
    c = lo
    while c * 2 <= hi and c * 2 * cells <= target_cells:
        c *= 2
    return c


class Server:
    REJECTED = 5

    def __init__(self, precision="fp32", hbm_cap=40e9, capacity=None, p=20, tol=1e-3, rtol=1e-5, max_steps=20000,
                 max_states_per_bucket=None, attempts=16):
        """capacity: slots per batch state, or None to size it per grid."""
        self.precision = precision
        self.hbm_cap = float(hbm_cap)
        self.capacity = capacity
        self.p = int(p)
        self.tol, self.rtol, self.max_steps = tol, rtol, max_steps
        self.max_states = max_states_per_bucket
        self.attempts = int(attempts)
        self.buckets = collections.OrderedDict()     # key -> [Batch]
        self.used = 0
        self.peak_used = 0

    @staticmethod
    def bucket_key(w):
        return (tuple(w.n), tuple(w.dx))

    def capacity_for(self, n):
        return int(self.capacity) if self.capacity is not None else auto_capacity(n)

    def _release_idle(self, need, busy):
        for key in list(self.buckets):
            for b in list(self.buckets[key]):
                if self.used + need <= self.hbm_cap:
                    return
                if id(b) not in busy:
                    self.buckets[key].remove(b)
                    self.used -= b.footprint
                    b.close()

    def _place(self, w, occupied, busy, pending):
        """(batch, slot) for request w, (None, None) to wait, ("reject", None)
        when its batch state can never fit under the cap."""
        from . import binding
        key = self.bucket_key(w)
        states = self.buckets.get(key, [])
        for b in states:
            if id(b) in pending:
                continue
            free = [s for s in range(b.capacity) if (id(b), s) not in occupied]
            if free:
                return b, free[0]
        if self.max_states is not None and len(states) >= self.max_states:
            return None, None
        cap = self.capacity_for(w.n)
        need = binding.Batch.footprint_of(w.n, w.dx, self.precision, cap)
        if need > self.hbm_cap:
            return "reject", None
        if self.used + need > self.hbm_cap:
            self._release_idle(need, busy)
        if self.used + need > self.hbm_cap:
            return None, None
        b = binding.Batch(w.n, w.dx, self.precision, cap, self.p)
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
        pending = {}           # id(batch) -> batch with attempts in flight
        results = [None] * len(requests)
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else (lambda: float("inf"))
        launches = 0
        while incoming or waiting or occupied:
            now = clock()
            while incoming and requests[incoming[0]][0] <= now:
                waiting.append(incoming.popleft())
            busy = {id(b) for (b, _) in where.values()}
            for idx in list(waiting):
                arr, w = requests[idx]
                b, slot = self._place(w, occupied, busy, pending)
                if b is None:
                    continue
                waiting.remove(idx)
                if isinstance(b, str):
                    now = time.perf_counter() - t0
                    results[idx] = {"arrival": arr, "admitted": None, "finished": now,
                                    "latency": now - (arr if realtime else 0.0), "steps": 0,
                                    "torque": float("nan"), "status": self.REJECTED}
                    continue
                b.set_slot(slot, w.Ms, w.A, w.alpha, to_soa(w.m0), 1e-13)
                ex = w.extra or {}
                if ex.get("D", 0.0) or not ex.get("precession", True):
                    b.set_slot_terms(slot, ex.get("dmi", "interface"), ex.get("D", 0.0), ex.get("precession", True))
                occupied[(id(b), slot)] = idx
                where[idx] = (b, slot)
                busy.add(id(b))
                results[idx] = {"arrival": arr, "admitted": time.perf_counter() - t0}
            if not occupied:
                if incoming:
                    delay = requests[incoming[0]][0] - clock()
                    if delay > 0:
                        time.sleep(min(delay, 0.01))
                continue
            for b in {id(b): b for (b, _) in where.values()}.values():
                if id(b) not in pending:
                    b.begin(self.attempts, self.rtol, self.tol, self.max_steps)
                    pending[id(b)] = b
                    launches += 1
            progressed = False
            for key, b in list(pending.items()):
                if not b.ready():
                    continue
                progressed = True
                del pending[key]
                status, steps, torque = b.end()
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
            if not progressed:
                time.sleep(2e-5)
        for b in pending.values():
            b.end()
        self.launches = launches
        self.elapsed = time.perf_counter() - t0
        return results

    def close(self):
        for key in list(self.buckets):
            for b in self.buckets[key]:
                b.close()
        self.buckets.clear()
        self.used = 0


def shard(requests, rank, world):
    """Requests rank, rank + world, ... of a stream (arrival times kept): the
    stream's share of one replica when each GPU runs its own server."""
    return [requests[i] for i in range(rank, len(requests), world)]


def unshard(parts, count):
    """Inverse of shard: per-rank result lists back in stream order."""
    world = len(parts)
    out = [None] * count
    for r, part in enumerate(parts):
        for k, res in enumerate(part):
            out[r + k * world] = res
    return out


def latency_summary(results, elapsed):
    """p50/p99/mean latency (arrival -> result, s) and throughput of served requests."""
    done = [r for r in results if r["status"] != Server.REJECTED]
    lat = np.array([r["latency"] for r in done])
    steps = np.array([r["steps"] for r in done])
    return {"requests": len(results), "rejected": len(results) - len(done),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "throughput_req_s": len(done) / elapsed,
            "steps_total": int(steps.sum()), "converged": int(sum(r["status"] == 2 for r in done)),
            "hit_max_steps": int(sum(r["status"] == 3 for r in done)),
            "failed": int(sum(r["status"] == 4 for r in done))}
