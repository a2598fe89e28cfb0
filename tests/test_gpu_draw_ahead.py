"""Bond draws taken one sweep ahead.

The C5 bond draws of sweep t depend on the seed, the counter and the site,
not on the spins (§2.1 draws a number per edge; only the comparison with
the spins' equality needs the state). Inside one sw_sweep call, where phase 3
of sweep t and phase 1 of sweep t + 1 run as one launch, the merge phases of
sweep t draw the bonds of sweep t + 1 and the launch's phase 1 part reads
them; a later call whose counter meets the drawn one reads them as well.
These tests run chains whose calls do and do not meet the drawn counter
(set_state to the same counter with other spins, to another counter, and
back), on tile shapes with and without the fused launch, odd and ragged
sides, and compare every result with the oracle exactly (C5, C8).
"""
import os

import numpy as np
import pytest

import oracle
from workloads import random_spins

pytestmark = pytest.mark.gpu

BETA_C = 0.44068679


@pytest.fixture(scope="module")
def sw():
    from conftest import build_libsw
    build_libsw()
    import paper_2302_14720_gb300 as sw
    return sw


def make(sw, L, beta, seed, shape):
    os.environ["SW_TILE_SHAPE"] = str(shape)
    try:
        return sw.Lattice(L, beta, seed, 0)
    finally:
        os.environ.pop("SW_TILE_SHAPE", None)


# 6: 128x64 (the fused launch between the sweeps of a call; one-sweep calls
# never fuse and draw in phase 1), 0: 128x64 with four-row strips and 7:
# 128x32 (no fused launch)
@pytest.mark.parametrize("shape", [6, 0, 7])
@pytest.mark.parametrize("L", [129, 200, 257])
def test_one_sweep_calls_equal_the_oracle_chain(sw, shape, L):
    seed, n = 600 + L, 8
    with make(sw, L, BETA_C, seed, shape) as lat:
        for _ in range(n):
            lat.sweep(1)
        spins = lat.spins()
        E, M = lat.observables(0, n)
    want_s, want_E, want_M, _ = oracle.run(L, BETA_C, seed, n)
    assert np.array_equal(spins, want_s)
    assert np.array_equal(E, want_E) and np.array_equal(M, want_M)


@pytest.mark.parametrize("shape", [6, 0])
@pytest.mark.parametrize("asynchronous", [False, True])
def test_state_replaced_at_the_drawn_counter(sw, shape, asynchronous):
    # on the fused shape, sweep(3) leaves the draws of sweep 2; they serve
    # other spins at counter 2, not counter 10; sweep(2) from counter 10
    # leaves those of 11, which a state set at 11 reads, and a state set at 3
    # draws afresh
    L, seed, beta = 190, 31, 0.5
    thr = oracle.threshold(beta)
    states = {k: random_spins(L, seed=k, p_minus=0.3 + 0.1 * k) for k in range(4)}
    put = (lambda lat, s, t: lat.set_state_async(s, t)) if asynchronous else (lambda lat, s, t: lat.set_state(s, t))
    got = []
    with make(sw, L, beta, seed, shape) as lat:
        lat.sweep(3)
        put(lat, states[0], 2)
        assert np.array_equal(lat.bonds(), oracle.bonds(states[0], seed, 2, thr))
        for k, (t0, n) in enumerate(((2, 1), (10, 2), (11, 1), (3, 1))):
            if k:
                put(lat, states[k], t0)
            lat.sweep(n)
            E, M = lat.observables(t0, n)
            got.append((lat.spins(), E, M, states[k], t0, n))
    for spins, E, M, s0, t0, n in got:
        want_s, want_E, want_M, _ = oracle.run(L, beta, seed, n, spins=s0, t0=t0)
        assert np.array_equal(spins, want_s)
        assert np.array_equal(E, want_E) and np.array_equal(M, want_M)


def test_labels_at_the_drawn_counter(sw):
    # sw_labels and sw_bonds run phase 1 for the current counter, here the
    # one whose bonds the previous call's merge drew
    L, seed = 300, 8
    thr = oracle.threshold(BETA_C)
    with make(sw, L, BETA_C, seed, 6) as lat:
        lat.sweep(2)
        lat.set_state(lat.spins(), 1)
        s = lat.spins()
        lab = lat.labels()
        bonds = lat.bonds()
        lat.sweep(2)
        spins = lat.spins()
    want_bonds = oracle.bonds(s, seed, 1, thr)
    assert np.array_equal(bonds, want_bonds)
    want_lab, _ = oracle.labels(want_bonds)
    assert np.array_equal(lab, want_lab)
    want_s, _, _, _ = oracle.run(L, BETA_C, seed, 2, spins=s, t0=1)
    assert np.array_equal(spins, want_s)


def test_statistics_between_fused_calls(sw):
    # statistics sweeps run unfused: the draws of a fused call are not
    # carried into them unless the counter meets
    L, seed = 256, 19
    with make(sw, L, BETA_C, seed, 6) as lat:
        lat.sweep(3)
        lat.histogram(True)
        lat.sweep(2)
        lat.histogram(False)
        lat.sweep(3)
        H = lat.histograms(3, 2)
        E, M = lat.observables(0, 8)
        spins = lat.spins()
    want_s, want_E, want_M, want_H = oracle.run(L, BETA_C, seed, 8, hist=True)
    assert np.array_equal(spins, want_s)
    assert np.array_equal(E, want_E) and np.array_equal(M, want_M)
    for k in (0, 1):
        assert np.array_equal(H[k], want_H[3 + k])
