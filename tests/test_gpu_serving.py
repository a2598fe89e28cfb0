"""Continuous-batching server on the GPU: every served chain equals the
same chain run alone (sw_sweep on its own handle) and the oracle's chain,
bit for bit, while requests join and leave mid-flight, memory runs short
and invalid requests fail beside them."""
import numpy as np
import pytest

import oracle
from workloads import serving_requests

pytestmark = pytest.mark.gpu

BETA_C = 0.44068679


@pytest.fixture(scope="module")
def sw():
    from conftest import build_libsw
    build_libsw()
    import paper_2302_14720_gb300 as sw
    return sw


def test_served_chains_equal_oracle_chains(sw):
    from paper_2302_14720_gb300.serving import Request, Server
    specs = [(2, 0.3, 31, 7, 0), (17, BETA_C, 32, 40, 0), (64, 0.6, 33, 1, 1), (33, 0.2, 34, 0, 0),
             (100, 0.45, 35, 23, 0), (5, 0.9, 36, 64, 1), (129, BETA_C, 37, 17, 0), (48, 0.5, 38, 65, 0),
             (1, 0.4, 39, 5, 0), (40, -0.5, 40, 5, 0)]
    reqs = [Request(i, L=L, beta=b, seed=s, sweeps=n, init=init, want_spins=True)
            for i, (L, b, s, n, init) in enumerate(specs)]
    with Server(budget_bytes=0, chunk=16) as srv:
        # Room for the largest request and a little more: later requests
        # wait for earlier ones to leave.
        srv.budget = srv.backend.footprint(129, 17) + 60_000
        res = {r.rid: r for r in srv.run(reqs, realtime=False)}
        assert srv.used == 0
    assert set(res) == set(range(len(specs)))
    for i, (L, beta, seed, n, init) in enumerate(specs):
        r = res[i]
        if L < 2 or beta < 0:
            assert r.error is not None
            continue
        assert r.error is None, r.error
        want_s, want_E, want_M, _ = oracle.run(L, beta, seed, n, cold=bool(init))
        assert np.array_equal(r.E, want_E) and np.array_equal(r.M, want_M), i
        assert np.array_equal(r.spins, want_s), i


def test_solo_equals_mix_on_a_poisson_stream(sw):
    # A short Poisson stream with the serving mix (L log-uniform, beta
    # uniform in [0.30, 0.60]) scaled to seconds; every 4th request is rerun
    # alone and compared in full (tolerance 0).
    from paper_2302_14720_gb300.serving import Request, Server, latency_summary
    stream = serving_requests(n=24, rate_per_s=40.0, seed=5, L_min=32, L_max=512, sweeps_min=10,
                              sweeps_max=120)
    reqs = [Request(i, L=q["L"], beta=q["beta"], seed=q["seed"], sweeps=q["sweeps"], arrival=q["arrival"],
                    want_spins=True) for i, q in enumerate(stream)]
    with Server(budget_bytes=64 << 20, chunk=32) as srv:
        res = {r.rid: r for r in srv.run(reqs, realtime=True)}
        assert srv.site_updates == sum(q.L * q.L * q.sweeps for q in reqs)
    summary = latency_summary(list(res.values()))
    assert summary["served"] == len(reqs) and summary["failed"] == 0
    for i in range(0, len(reqs), 4):
        q = reqs[i]
        with sw.Lattice(q.L, q.beta, q.seed) as lat:
            lat.sweep(q.sweeps)
            E, M = lat.observables(0, q.sweeps)
            assert np.array_equal(res[i].E, E) and np.array_equal(res[i].M, M), i
            assert np.array_equal(res[i].spins, lat.spins()), i
