"""q-state Potts sweeps on the GPU (the paper's §6 generalisation), on the
tiled path (128 x 64 tiles): chains bit-exact against the oracle's Potts
chain -- one tile, ragged tiles, many tiles with rows on and off 16-byte
boundaries, clusters spanning the lattice (large beta), q up to 127 --
labels against the oracle's labels of the same bonds, q = 2 against the
Ising assignment chain."""
import numpy as np
import pytest

import oracle
from workloads import random_spins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    from conftest import build_libsw
    build_libsw()
    import paper_2302_14720_gb300 as sw
    return sw


@pytest.mark.parametrize("L,q,beta,cold", [(2, 3, 0.7, False), (5, 4, 1.2, True), (33, 3, 1.0050833, False),
                                           (64, 2, 0.88137, False), (100, 5, 1.1, False), (257, 3, 1.3, False),
                                           (130, 10, 1.4, True), (512, 3, 1.0050833, False),
                                           (1000, 3, 1.0050833, False), (256, 4, 4.0, False),
                                           (200, 127, 2.0, False), (129, 2, 0.1, False)])
def test_potts_chain_parity(sw, L, q, beta, cold):
    seed, n = 600 + L + q, 7
    with sw.Potts(L, q, beta, seed, sw.SW_INIT_COLD if cold else sw.SW_INIT_HOT) as p:
        p.sweep(3)
        p.sweep(4)
        want_s, want_E, want_M = oracle.potts_run(L, q, beta, seed, n, cold=cold)
        E, M = p.observables(0, n)
        assert np.array_equal(E, want_E) and np.array_equal(M, want_M)
        assert np.array_equal(p.states(), want_s)


def test_potts_bench_configuration(sw):
    """The benchmark's Potts run (L = 1024, q = 3 at its critical coupling
    ln(1 + sqrt 3), hot start, seed 4), ten sweeps, element by element."""
    L, q, beta, seed, n = 1024, 3, 1.0050833, 4, 10
    with sw.Potts(L, q, beta, seed) as p:
        p.sweep(n)
        E, M = p.observables(0, n)
        want_s, want_E, want_M = oracle.potts_run(L, q, beta, seed, n)
        assert np.array_equal(E, want_E) and np.array_equal(M, want_M)
        assert np.array_equal(p.states(), want_s)


def test_potts_q2_equals_ising_assign(sw):
    L, beta, seed, n = 96, 0.43, 21, 6
    with sw.Potts(L, 2, 2 * beta, seed) as p, sw.Lattice(L, beta, seed) as lat:
        lat.set_rule(sw.SW_RULE_ASSIGN)
        p.sweep(n)
        lat.sweep(n)
        assert np.array_equal(p.states(), (lat.spins() < 0).astype(np.int8))
        E, M = p.observables(0, n)
        Ei, Mi = lat.observables(0, n)
        assert np.array_equal(E, Ei // 2 - L * L) and np.array_equal(M, (L * L + Mi) // 2)


def test_potts_labels_and_set_state(sw):
    L, q, beta, seed, t = 150, 4, 1.1, 8, 40
    rng = np.random.default_rng(3)
    s0 = rng.integers(0, q, (L, L)).astype(np.int8)
    with sw.Potts(L, q, beta, seed) as p:
        p.set_state(s0, t)
        lab = p.labels()
        want, _ = oracle.labels(oracle.bonds(s0, seed, t, oracle.potts_threshold(beta)))
        assert np.array_equal(lab, want)
        p.sweep(3)
        want_s, want_E, _ = oracle.potts_run(L, q, beta, seed, 3, states=s0, t0=t)
        assert np.array_equal(p.states(), want_s)
        assert np.array_equal(p.observables(t, 3)[0], want_E)
        bad = s0.copy()
        bad[3, 4] = q
        with pytest.raises(sw.SWError) as ei:
            p.set_state(bad, 0)
        assert ei.value.status == sw.SW_EINVAL
        assert np.array_equal(p.states(), want_s)   # state kept


def test_potts_threshold_matches_oracle(sw):
    for beta in [0.0, 0.3, 1.0050833, 5.0, 40.0]:
        assert sw.sw_potts_threshold(beta) == oracle.potts_threshold(beta)
