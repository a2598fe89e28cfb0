"""The assignment rule (§2.4 as printed, C6b) on the GPU: chains equal the
oracle's assignment chains bit for bit, alone, in a batch beside flip-rule
replicas, and after switching rules mid-chain."""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

BETA_C = 0.44068679


@pytest.fixture(scope="module")
def sw():
    from conftest import build_libsw
    build_libsw()
    import paper_2302_14720_gb300 as sw
    return sw


@pytest.mark.parametrize("shape", [2, 6])
@pytest.mark.parametrize("L,beta", [(2, 0.3), (7, 0.9), (33, BETA_C), (130, 0.5), (200, 0.35)])
def test_assign_chain_parity(sw, shape, L, beta):
    seed, n = 900 + L, 6
    os.environ["SW_TILE_SHAPE"] = str(shape)
    try:
        lat = sw.Lattice(L, beta, seed)
    finally:
        os.environ.pop("SW_TILE_SHAPE", None)
    with lat:
        lat.set_rule(sw.SW_RULE_ASSIGN)
        lat.sweep(n)
        want_s, want_E, want_M, _ = oracle.run(L, beta, seed, n, rule="assign")
        E, M = lat.observables(0, n)
        assert np.array_equal(E, want_E) and np.array_equal(M, want_M)
        assert np.array_equal(lat.spins(), want_s)


def test_assign_with_histogram_parity(sw):
    L, beta, seed, n = 70, BETA_C, 77, 4
    with sw.Lattice(L, beta, seed) as lat:
        lat.set_rule(sw.SW_RULE_ASSIGN)
        lat.histogram(True)
        lat.sweep(n)
        want_s, want_E, _, want_H = oracle.run(L, beta, seed, n, rule="assign", hist=True)
        assert np.array_equal(lat.histograms(0, n), want_H)
        assert np.array_equal(lat.observables(0, n)[0], want_E)
        assert np.array_equal(lat.spins(), want_s)


def test_rule_switch_mid_chain(sw):
    L, beta, seed = 50, 0.42, 31
    with sw.Lattice(L, beta, seed) as lat:
        lat.sweep(3)
        lat.set_rule(sw.SW_RULE_ASSIGN)
        lat.sweep(2)
        lat.set_rule(sw.SW_RULE_FLIP)
        lat.sweep(2)
        s, E1, _, _ = oracle.run(L, beta, seed, 3)
        s, E2, _, _ = oracle.run(L, beta, seed, 2, spins=s, t0=3, rule="assign")
        s, E3, _, _ = oracle.run(L, beta, seed, 2, spins=s, t0=5)
        assert np.array_equal(lat.observables(0, 7)[0], np.concatenate([E1, E2, E3]))
        assert np.array_equal(lat.spins(), s)
        with pytest.raises(sw.SWError):
            lat.set_rule(7)


def test_batch_mixed_rules(sw):
    reps = [(40, 0.5, 1, 1), (64, BETA_C, 2, 0), (17, 0.3, 3, 1), (100, 0.45, 4, 0)]
    b = sw.sw_batch_create([r[0] for r in reps], [r[1] for r in reps], [r[2] for r in reps])
    try:
        for slot, r in enumerate(reps):
            sw.sw_batch_set_rule(b, slot, r[3])
        sw.sw_batch_sweep(b, 5)
        for slot, (L, beta, seed, rule) in enumerate(reps):
            want_s, want_E, want_M, _ = oracle.run(L, beta, seed, 5, rule="assign" if rule else "flip")
            assert np.array_equal(sw.sw_batch_spins(b, slot, L), want_s), slot
            E, M = sw.sw_batch_observables(b, slot, 0, 5)
            assert np.array_equal(E, want_E) and np.array_equal(M, want_M), slot
    finally:
        sw.sw_batch_destroy(b)


# ------------------------------------------------ whole-lattice CTA path

@pytest.mark.parametrize("rule", ["flip", "assign"])
@pytest.mark.parametrize("L", [2, 3, 5, 17, 31, 32, 33, 64, 100, 128, 144, 145, 181])
def test_small_lattice_path_parity(sw, L, rule):
    # sw_sweep runs every sweep of a call in one CTA for L <= 144; 145 is the
    # first tiled size (the one-CTA kernel itself goes up to 181: see the
    # allocation-free entry point's tests)
    beta = [0.3, 0.44068679, 0.6][L % 3]
    seed, n = 4000 + L, 9
    with sw.Lattice(L, beta, seed) as lat:
        if rule == "assign":
            lat.set_rule(sw.SW_RULE_ASSIGN)
        lat.sweep(4)
        lat.sweep(5)
        want_s, want_E, want_M, _ = oracle.run(L, beta, seed, n, rule=rule)
        E, M = lat.observables(0, n)
        assert np.array_equal(E, want_E) and np.array_equal(M, want_M)
        assert np.array_equal(lat.spins(), want_s)


def test_small_lattice_path_from_set_state(sw):
    from workloads import random_spins
    L, beta, seed, t0 = 150, 0.41, 12, 33
    s0 = random_spins(L, seed=2, p_minus=0.7)
    with sw.Lattice(L, beta, seed) as lat:
        lat.set_state(s0, t0)
        lat.sweep(6)
        want_s, want_E, _, _ = oracle.run(L, beta, seed, 6, spins=s0, t0=t0)
        assert np.array_equal(lat.observables(t0, 6)[0], want_E)
        assert np.array_equal(lat.spins(), want_s)
