"""Host logic of the serving loop (continuous batching, HBM-budget
admission, LRU eviction of idle sessions, slot reuse) with a stand-in for
the GPU tree, so that it runs without a device.  The GPU run of the same
loop, with every result compared bit for bit against a solo solve, is in
test_gpu_serving.py."""
import numpy as np
import pytest

from paper_2205_09411_gb300.serving import Request, Server, Session, poisson_arrivals, summarize


class FakeTree:
    """Stand-in with the tree interface: a slot's residual falls by `rate`
    per step from 1 (0 for a zero right-hand side); the 'solution' of a slot
    is its right-hand side times its step count."""

    live = 0

    def __init__(self, n, slots, nbytes, rate):
        self.n, self.slots, self.nbytes, self.rate = n, slots, nbytes, rate
        self.g = np.zeros((slots, n))
        self.rel = np.ones(slots)
        self.steps = np.zeros(slots, dtype=int)
        self.pending = None
        self.bound = False

    def workspace_bytes(self):
        return self.nbytes

    def bind(self):
        assert not self.bound
        self.bound = True
        FakeTree.live += self.nbytes

    def close(self):
        if self.bound:
            FakeTree.live -= self.nbytes
            self.bound = False

    def set_rhs_slots(self, slot, g, stream=None):
        self.g[slot] = g
        self.steps[slot] = 0

    def iterate_begin(self, precision, active, residual_only=False, stream=None):
        assert self.pending is None
        self.pending = (np.asarray(active).copy(), residual_only)

    def iterate_end(self):
        active, residual_only = self.pending
        self.pending = None
        for s in np.nonzero(active)[0]:
            if residual_only:
                self.rel[s] = 0.0 if not self.g[s].any() else 1.0
            else:
                self.steps[s] += 1
                self.rel[s] *= self.rate
        return self.rel.copy(), self.rel.copy()

    def solution_slots(self, slot, nslots=1, stream=None):
        return (self.g[slot] * self.steps[slot])[None, :]


def sessions(sizes, rate=0.1, n=16):
    return [Session(name, make=lambda slots, b=b: FakeTree(n, slots, b, rate)) for name, b in sizes.items()]


def requests(names, count, rate, seed, n=16):
    t = poisson_arrivals(rate, count, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    out = []
    for i in range(count):
        g = rng.standard_normal(n)
        out.append(Request(session=names[int(rng.integers(len(names)))], rhs=g, arrival=float(t[i])))
    return out


def test_every_request_completes_with_its_own_result():
    ss = sessions({"a": 100, "b": 200, "c": 300})
    reqs = requests(["a", "b", "c"], 60, 2000.0, 5)
    srv = Server(ss, budget_bytes=500, slots=3, tol=1e-8)
    done = srv.run(reqs, idle_sleep=None)
    assert len(done) == 60
    want, rel = 0, 1.0
    while rel > 1e-8:  # the stand-in's residual history
        rel *= 0.1
        want += 1
    for r in done:
        assert r.cycles == want
        assert np.array_equal(r.result, r.rhs * want)
        assert r.done >= r.start >= r.arrival - 1e-9
    assert srv.peak_bytes <= 500


def test_budget_forces_eviction_of_idle_sessions_only():
    ss = sessions({"a": 300, "b": 300, "c": 300})
    reqs = requests(["a", "b", "c"], 40, 5000.0, 7)
    srv = Server(ss, budget_bytes=600, slots=2, tol=1e-8)
    FakeTree.live = 0
    done = srv.run(reqs, idle_sleep=None)
    assert len(done) == 40
    assert srv.peak_bytes <= 600
    assert any(e[0] == "evict" for e in srv.log)
    srv.close()
    assert FakeTree.live == 0


def test_fifo_within_a_session_and_slot_reuse():
    ss = sessions({"a": 100})
    reqs = requests(["a"], 25, 10000.0, 9)
    srv = Server(ss, budget_bytes=100, slots=4, tol=1e-8)
    done = srv.run(reqs, idle_sleep=None)
    starts = sorted(done, key=lambda r: r.arrival)
    assert all(x.start <= y.start for x, y in zip(starts, starts[1:]))
    assert ss[0].loads == 1


def test_zero_rhs_finishes_without_a_cycle_and_oversize_session_rejected():
    ss = sessions({"a": 100, "big": 1000})
    srv = Server(ss, budget_bytes=200, slots=2, tol=1e-8)
    done = srv.run([Request("a", np.zeros(16), 0.0)], idle_sleep=None)
    assert done[0].cycles == 0
    srv2 = Server(sessions({"big": 1000}), budget_bytes=200, slots=2)
    with pytest.raises(ValueError):
        srv2.run([Request("big", np.ones(16), 0.0)], idle_sleep=None)


def test_poisson_arrivals_and_summary():
    t = poisson_arrivals(100.0, 4000, 3)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.01) < 0.001
    ss = sessions({"a": 100})
    done = Server(ss, budget_bytes=100, slots=2).run(requests(["a"], 10, 1e4, 4), idle_sleep=None)
    s = summarize(done)
    assert s["requests"] == 10 and s["p99_ms"] >= s["p50_ms"] >= 0
