"""The sweep with phase 3 and the next sweep's phase 1 in one launch.

On tile shapes whose phases 1 and 3 take the same block, the sweeps of one
sw_sweep call without statistics run phase 3 of sweep t and phase 1 of sweep
t + 1 as one launch; a call's last sweep runs phase 3 alone. These tests
split chains into calls of every length (one-sweep calls never fuse, longer
ones do), put the operations that change the state or run phase 1 themselves
between them (labels, bonds, the equivalence labels, statistics on and off,
set_state, set_state_async) and check every result against the oracle
exactly (C8, §2).
"""
import os

import numpy as np
import pytest

import oracle
from workloads import random_spins

pytestmark = pytest.mark.gpu

BETA_C = 0.44068679
FUSED_SHAPES = [4, 6]  # 128x128 and 128x64 tiles


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


def oracle_states(L, beta, seed, n):
    """The oracle's state after each of sweeps 1..n from the C7 hot start."""
    s = oracle.init(L, seed)
    out = [s]
    for k in range(n):
        s, _, _, _ = oracle.run(L, beta, seed, 1, spins=s, t0=k)
        out.append(s)
    return out


@pytest.mark.parametrize("shape", FUSED_SHAPES)
@pytest.mark.parametrize("L", [33, 130, 257, 500])
def test_split_calls_with_queries_between(sw, shape, L):
    seed, beta = 4100 + L, BETA_C
    thr = oracle.threshold(beta)
    want = oracle_states(L, beta, seed, 12)
    with make(sw, L, beta, seed, shape) as lat:
        lat.sweep(1)
        assert np.array_equal(lat.spins(), want[1])
        lat.sweep(2)  # one fused launch
        assert np.array_equal(lat.spins(), want[3])
        want_lab, _ = oracle.labels(oracle.bonds(want[3], seed, 3, thr))
        assert np.array_equal(lat.labels(), want_lab)
        lat.sweep(1)
        assert np.array_equal(lat.spins(), want[4])
        assert np.array_equal(lat.bonds(), oracle.bonds(want[4], seed, 4, thr))
        lat.sweep(2)
        assert np.array_equal(lat.spins(), want[6])
        lab_eq, _ = lat.labels_equivalence()
        want_lab, _ = oracle.labels(oracle.bonds(want[6], seed, 6, thr))
        assert np.array_equal(lab_eq, want_lab)
        lat.histogram(True)
        lat.sweep(1)
        lat.histogram(False)
        lat.sweep(2)
        lat.sweep(1)
        lat.sweep(2)
        assert np.array_equal(lat.spins(), want[12])
        E, M = lat.observables(0, 12)
        H = lat.histograms(6, 1)
    _, want_E, want_M, want_H = oracle.run(L, beta, seed, 12, hist=True)
    assert np.array_equal(E, want_E) and np.array_equal(M, want_M)
    assert np.array_equal(H[0], want_H[6])


@pytest.mark.parametrize("shape", FUSED_SHAPES)
@pytest.mark.parametrize("asynchronous", [False, True])
def test_set_state_between_fused_calls(sw, shape, asynchronous):
    L, seed, beta = 257, 77, 0.6
    s = random_spins(L, seed=9, p_minus=0.3)
    with make(sw, L, beta, seed, shape) as lat:
        lat.sweep(3)
        if asynchronous:
            lat.set_state_async(s, 40)
        else:
            lat.set_state(s, 40)
        lat.sweep(2)
        lat.sweep(3)
        spins = lat.spins()
        E, M = lat.observables(40, 5)
    want_s, want_E, want_M, _ = oracle.run(L, beta, seed, 5, spins=s, t0=40)
    assert np.array_equal(spins, want_s)
    assert np.array_equal(E, want_E) and np.array_equal(M, want_M)


@pytest.mark.parametrize("shape", FUSED_SHAPES)
def test_every_call_length(sw, shape):
    L, seed = 193, 12
    calls = [1, 1, 2, 1, 3, 1, 4, 5]
    n = sum(calls)
    with make(sw, L, BETA_C, seed, shape) as a, make(sw, L, BETA_C, seed, shape) as b:
        for c in calls:
            a.sweep(c)
        b.sweep(n)
        sa, sb = a.spins(), b.spins()
        Ea, Ma = a.observables(0, n)
        Eb, Mb = b.observables(0, n)
    want_s, want_E, want_M, _ = oracle.run(L, BETA_C, seed, n)
    assert np.array_equal(sa, want_s) and np.array_equal(sb, want_s)
    for E, M in ((Ea, Ma), (Eb, Mb)):
        assert np.array_equal(E, want_E) and np.array_equal(M, want_M)


def test_trace_growth_across_fused_calls(sw):
    # the trace holds 1024 sweeps at first: the next calls grow it while the
    # fused launches zero each next sweep's E/M row
    L, seed, n1 = 130, 21, 1023
    with make(sw, L, BETA_C, seed, 6) as lat:
        lat.sweep(n1)
        lat.sweep(1)
        lat.sweep(5)
        E, M = lat.observables(0, n1 + 6)
        spins = lat.spins()
    want_s, want_E, want_M, _ = oracle.run(L, BETA_C, seed, n1 + 6)
    assert np.array_equal(E, want_E) and np.array_equal(M, want_M)
    assert np.array_equal(spins, want_s)


def test_assignment_rule_on_the_fused_launch(sw):
    L, seed = 300, 5
    with make(sw, L, BETA_C, seed, 6) as lat:
        lat.set_rule(sw.SW_RULE_ASSIGN)
        lat.sweep(2)
        lat.sweep(3)
        spins = lat.spins()
        E, M = lat.observables(0, 5)
    want_s, want_E, want_M, _ = oracle.run(L, BETA_C, seed, 5, rule="assign")
    assert np.array_equal(spins, want_s)
    assert np.array_equal(E, want_E) and np.array_equal(M, want_M)
