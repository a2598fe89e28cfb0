"""Host logic of the continuous-batching server (no GPU): admission against
the memory budget, head-of-line order, chunk lengths, failure isolation and
site-update accounting, driven through a fake batch backend that only
counts sweeps."""
import pytest

from paper_2302_14720_gb300 import SWError
from paper_2302_14720_gb300.serving import Request, Server, latency_summary


class FakeBackend:
    """Stands in for sw_batch_*: slots, counters, limits and footprints."""

    def __init__(self, bytes_per_site=10):
        self.bps = bytes_per_site
        self.slots = {}          # slot -> [L, count, limit]
        self.sweep_calls = []
        self.peak_sites = 0

    def footprint(self, L, sweeps):
        if L < 2:
            raise SWError(-1, "sw_batch_footprint", "L outside 2 <= L")
        return self.bps * L * L + 16 * max(1024, sweeps)

    def add(self, L, beta, seed, init):
        if not beta >= 0:
            raise SWError(-1, "sw_batch_add", "beta must be finite and >= 0")
        slot = next(i for i in range(len(self.slots) + 1) if i not in self.slots)
        self.slots[slot] = [L, 0, None]
        self.peak_sites = max(self.peak_sites, sum(v[0] ** 2 for v in self.slots.values()))
        return slot

    def set_limit(self, slot, sweeps):
        self.slots[slot][2] = self.slots[slot][1] + sweeps

    def sweep(self, n):
        self.sweep_calls.append(n)
        for v in self.slots.values():
            v[1] = min(v[1] + n, v[2])

    def sweep_count(self, slot):
        return self.slots[slot][1]

    def observables(self, slot, count):
        import numpy as np
        assert count == self.slots[slot][1]
        return np.arange(count, dtype=np.int64), -np.arange(count, dtype=np.int64)

    def spins(self, slot, L):
        raise AssertionError("not requested")

    def remove(self, slot):
        del self.slots[slot]

    def close(self):
        pass


def test_every_chunk_has_the_configured_length():
    # a request about to finish does not shorten the chunk of the others:
    # its sweep limit stops it inside the chunk
    fb = FakeBackend()
    reqs = [Request(0, L=8, beta=0.4, seed=0, sweeps=3), Request(1, L=8, beta=0.4, seed=1, sweeps=200)]
    with Server(budget_bytes=10 ** 9, chunk=64, backend=fb) as srv:
        res = {r.rid: r for r in srv.run(reqs, realtime=False)}
    assert fb.sweep_calls == [64, 64, 64, 64]
    assert len(res[0].E) == 3 and len(res[1].E) == 200


def test_every_request_gets_exactly_its_sweeps():
    fb = FakeBackend()
    reqs = [Request(i, L=8 + 4 * i, beta=0.4, seed=i, sweeps=s) for i, s in enumerate([5, 0, 130, 64, 1, 77])]
    with Server(budget_bytes=10 ** 9, chunk=64, backend=fb) as srv:
        res = srv.run(reqs, realtime=False)
    assert sorted(r.rid for r in res) == list(range(6))
    for r in res:
        assert r.error is None
        n = reqs[r.rid].sweeps
        assert len(r.E) == n and list(r.E) == list(range(n))
    assert srv.site_updates == sum(q.L * q.L * q.sweeps for q in reqs)
    assert all(n == 64 for n in fb.sweep_calls)
    assert not fb.slots and srv.used == 0


def test_budget_is_never_exceeded_and_order_is_kept():
    fb = FakeBackend(bytes_per_site=1)
    # Each request needs 64*64 + 16*1024 = 20480 bytes; the budget admits 2.
    reqs = [Request(i, L=64, beta=0.4, seed=i, sweeps=10 + i) for i in range(5)]
    srv = Server(budget_bytes=2 * 20480 + 100, chunk=8, backend=fb)
    admitted_order = []
    orig_add = fb.add

    def add(L, beta, seed, init):
        assert srv.used + fb.footprint(L, 0) <= srv.budget
        admitted_order.append(seed)
        return orig_add(L, beta, seed, init)

    fb.add = add
    res = srv.run(reqs, realtime=False)
    assert admitted_order == [0, 1, 2, 3, 4]
    assert fb.peak_sites <= 2 * 64 * 64
    assert all(r.error is None for r in res) and len(res) == 5


def test_failures_are_isolated():
    fb = FakeBackend()
    reqs = [Request(0, L=16, beta=0.4, seed=1, sweeps=9),
            Request(1, L=1, beta=0.4, seed=2, sweeps=9),        # invalid L
            Request(2, L=16, beta=-1.0, seed=3, sweeps=9),      # invalid beta
            Request(3, L=4000, beta=0.4, seed=4, sweeps=9),     # larger than the budget
            Request(4, L=16, beta=0.4, seed=5, sweeps=-2),      # invalid count
            Request(5, L=20, beta=0.5, seed=6, sweeps=33)]
    with Server(budget_bytes=10 ** 6, chunk=16, backend=fb) as srv:
        res = {r.rid: r for r in srv.run(reqs, realtime=False)}
    assert set(res) == set(range(6))
    assert [rid for rid, r in sorted(res.items()) if r.error] == [1, 2, 3, 4]
    assert "budget" in res[3].error
    assert len(res[0].E) == 9 and len(res[5].E) == 33


def test_latency_summary():
    from paper_2302_14720_gb300.serving import Result
    rs = [Result(i, arrival=0.0, finished=float(i + 1)) for i in range(100)] + [Result(100, error="x")]
    s = latency_summary(rs)
    assert s["served"] == 100 and s["failed"] == 1
    assert s["p50_s"] == pytest.approx(50.5) and s["max_s"] == 100.0
