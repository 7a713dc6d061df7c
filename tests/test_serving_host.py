"""Host logic of the continuous-batching server, with a fake batch state in
place of the device one: every request is served, the summed footprint of
live batch states never exceeds the HBM cap, requests join batches that are
already running, a request whose batch state cannot fit is rejected, and a
request's outcome does not depend on what it was batched with."""
import numpy as np
import pytest

from paper_2302_08843_gb300 import binding
from paper_2302_08843_gb300.serving import Server, latency_summary
from paper_2302_08843_gb300.workloads import Workload


class FakeBatch:
    live = 0
    peak = 0
    created = 0
    joined_running = 0

    def __init__(self, n, dx, precision="fp32", capacity=8, p=20, stream=None):
        self.n, self.capacity = tuple(n), capacity
        self.footprint = FakeBatch.footprint_of(n, dx, precision, capacity)
        FakeBatch.live += self.footprint
        FakeBatch.peak = max(FakeBatch.peak, FakeBatch.live)
        FakeBatch.created += 1
        self.need = [0] * capacity
        self.steps = [0] * capacity
        self.status = [0] * capacity
        self.closed = False

    @staticmethod
    def footprint_of(n, dx, precision, capacity):
        return int(np.prod(n)) * capacity * 100

    def set_slot(self, slot, Ms, A, alpha, m0, dt0=1e-13):
        assert self.status[slot] == 0 and not self.closed
        if any(s == 1 for s in self.status):
            FakeBatch.joined_running += 1
        # the fake "relaxes" in a number of steps fixed by the request alone
        self.need[slot] = int(Ms // 1e5)
        self.steps[slot] = 0
        self.status[slot] = 1

    def set_slot_terms(self, slot, dmi=None, D=0.0, precession=True):
        assert self.status[slot] == 1 and self.steps[slot] == 0
        FakeBatch.terms.append((self.need[slot], dmi, D, precession))

    def begin(self, attempts=1, rtol=1e-5, tol=1e-3, max_steps=20000):
        self.attempts = attempts

    def ready(self):
        return True

    def end(self):
        for s in range(self.capacity):
            for _ in range(self.attempts):
                if self.status[s] == 1:
                    self.steps[s] += 1
                    if self.steps[s] >= self.need[s]:
                        self.status[s] = 2
        return (np.array(self.status, dtype=np.int32), np.array(self.steps, dtype=np.int32),
                np.zeros(self.capacity))

    def clear_slot(self, slot):
        self.status[slot] = 0

    def get_m(self, slot):
        return np.zeros((3,) + tuple(reversed(self.n)))

    def close(self):
        if not self.closed:
            FakeBatch.live -= self.footprint
            self.closed = True


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(binding, "Batch", FakeBatch)
    FakeBatch.live = FakeBatch.peak = FakeBatch.created = FakeBatch.joined_running = 0
    FakeBatch.terms = []
    return FakeBatch


def _requests(seed, count, grids):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = grids[int(rng.integers(len(grids)))]
        Ms = float(rng.uniform(2e5, 1.2e6))
        out.append((0.0, Workload("r%d" % i, n, (3e-9,) * 3, Ms=Ms, A=1e-11, alpha=1.0,
                                  m0=np.ones(n + (3,)) / np.sqrt(3.0))))
    return out


def test_all_served_under_cap(fake):
    grids = [(8, 8, 1), (16, 4, 2), (10, 10, 2)]
    reqs = _requests(1, 60, grids)
    cap = 2 * max(FakeBatch.footprint_of(g, None, "fp32", 4) for g in grids)   # at most two states live
    srv = Server(hbm_cap=cap, capacity=4)
    res = srv.run(reqs, realtime=False)
    assert all(r is not None and r["status"] == 2 for r in res)
    assert FakeBatch.peak <= cap and srv.peak_used <= cap
    # the fake's step count is fixed by the request alone
    for (_, w), r in zip(reqs, res):
        assert r["steps"] == int(w.Ms // 1e5)
    # buckets were evicted and rebuilt to stay under the cap
    assert FakeBatch.created > len(grids)
    s = latency_summary(res, srv.elapsed)
    assert s["converged"] == 60 and s["p99_s"] >= s["p50_s"] >= 0
    srv.close()
    assert FakeBatch.live == 0


def test_requests_join_running_batches(fake):
    reqs = _requests(2, 20, [(8, 8, 1)])
    srv = Server(hbm_cap=1e12, capacity=4, max_states_per_bucket=1)
    res = srv.run(reqs, realtime=False)
    assert all(r["status"] == 2 for r in res)
    assert FakeBatch.created == 1
    # slots freed by converged requests were refilled while others ran
    assert FakeBatch.joined_running > 0
    srv.close()


def test_oversize_request_rejected(fake):
    big = (64, 64, 4)
    reqs = _requests(3, 6, [(8, 8, 1)]) + [(0.0, Workload("big", big, (3e-9,) * 3, Ms=8e5, A=1e-11, alpha=1.0,
                                                        m0=np.ones(big + (3,))))]
    cap = FakeBatch.footprint_of(big, None, "fp32", 4) - 1
    srv = Server(hbm_cap=cap, capacity=4)
    res = srv.run(reqs, realtime=False)
    assert res[-1]["status"] == Server.REJECTED
    assert all(r["status"] == 2 for r in res[:-1])
    s = latency_summary(res, srv.elapsed)
    assert s["rejected"] == 1
    srv.close()


def test_auto_capacity():
    from paper_2302_08843_gb300.serving import auto_capacity
    assert auto_capacity((64, 64, 1)) == 32
    assert auto_capacity((100, 100, 8)) == 16
    assert auto_capacity((256, 256, 64)) == 4
    for n in [(1, 1, 1), (7, 5, 3), (512, 512, 8)]:
        c = auto_capacity(n)
        assert 4 <= c <= 32 and c & (c - 1) == 0


def test_realtime_arrivals_wait_for_their_time(fake):
    reqs = [(0.02 * i, w) for i, (_, w) in enumerate(_requests(4, 5, [(8, 8, 1)]))]
    srv = Server(hbm_cap=1e12, capacity=2)
    res = srv.run(reqs, realtime=True)
    for (arr, _), r in zip(reqs, res):
        assert r["admitted"] >= arr - 1e-9
        assert r["latency"] >= 0
    srv.close()


def test_request_terms_reach_their_slot(fake):
    """A request's DMI and precession switch (Workload.extra) are loaded into
    its own slot right after the slot's material, before any attempt; requests
    without them load none."""
    reqs = _requests(5, 12, [(8, 8, 1), (6, 4, 2)])
    want = []
    for i, (_, w) in enumerate(reqs):
        if i % 3 == 0:
            w.extra.update({"dmi": "bulk", "D": 1e-3 * (i + 1), "precession": i % 2 == 0})
            want.append((int(w.Ms // 1e5), "bulk", 1e-3 * (i + 1), i % 2 == 0))
    srv = Server(precision="fp32", capacity=4, tol=1e-3, max_steps=100)
    res = srv.run(reqs, realtime=False)
    srv.close()
    assert all(r["status"] == 2 for r in res)
    assert sorted(FakeBatch.terms) == sorted(want)
