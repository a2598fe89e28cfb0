"""Pins of the oracle's assignment rule (§2.4 as the paper prints it: every
cluster gets a fresh spin, +1 or -1 with probability 1/2), the alternative
to the flip rule (C6).

What fixes it independently of its own code: the exact one-sweep transition
matrix on the 2x2 torus equals the flip rule's (the two rules agree in
distribution because clusters are monochrome) and satisfies detailed
balance; the chain's moments on the 4x4 torus equal the exact Boltzmann
moments; the result does not depend on the old spins; a flip and an
assignment that differ exactly where the old spin differs give the same
state; and the per-cluster values are fair coins.
"""
import numpy as np
import pytest

import exact_ising as ex
import oracle

BETA_C_LIT = 0.44068679


@pytest.mark.parametrize("beta", [0.2, BETA_C_LIT, 0.9])
def test_assign_kernel_equals_flip_kernel_2x2(beta):
    Ta = ex.sw_transition_matrix(2, beta, oracle, rule="assign")
    Tf = ex.sw_transition_matrix(2, beta, oracle, rule="flip")
    pi = ex.boltzmann(2, beta)
    assert np.allclose(Ta.sum(axis=1), 1.0, atol=1e-13)
    assert np.abs(Ta - Tf).max() < 1e-14
    assert np.abs(pi @ Ta - pi).max() < 1e-14


def _labels(s, seed, t, beta):
    b = oracle.bonds(s, seed, t, oracle.threshold(beta))
    return oracle.labels(b)


def test_assign_is_monochrome_and_ignores_old_spins():
    L, seed, t, beta = 40, 9, 3, BETA_C_LIT
    s = oracle.init(L, seed)
    lab, nc = _labels(s, seed, t, beta)
    a = oracle.assign(L, lab, seed, t)
    assert set(np.unique(a)) <= {-1, 1}
    for r in np.unique(lab)[:200]:
        vals = a[lab == r]
        assert (vals == vals[0]).all()
    # the same labels with the opposite old state give the same new state
    # (the step reads only the labels); compare with a flip of -s as well
    f = (oracle.flip(-s, lab, seed, t) == oracle.flip(s, lab, seed, t))
    assert not f.all()  # the flip rule does depend on the old spins
    assert np.array_equal(a, oracle.assign(L, lab.copy(), seed, t))


def test_assign_equals_flip_by_the_difference():
    L, seed, t, beta = 24, 5, 8, 0.6
    s0 = oracle.init(L, seed)
    lab, _ = _labels(s0, seed, t, beta)
    # a state whose clusters are monochrome: one assignment step from s0
    m0 = np.random.default_rng(1).integers(0, 2, L * L).astype(np.uint8)
    s = oracle.apply_assign(L, lab, m0)
    m = np.random.default_rng(2).integers(0, 2, L * L).astype(np.uint8)
    old_minus = (s.reshape(-1) < 0).astype(np.uint8)
    f = m ^ old_minus          # flip exactly where the new value differs
    roots = np.unique(lab)
    f_at = np.zeros(L * L, np.uint8)
    f_at[roots] = f[roots]
    assert np.array_equal(oracle.apply_flips(s, lab, f_at), oracle.apply_assign(L, lab, m))


def test_assign_values_follow_philox_tag_3():
    # convention pin: the value of root r is bit 31 of x0 of block (r, t, 3, 0)
    L, seed, t = 16, 0xDEADBEEF12345, 77
    lab = np.arange(L * L, dtype=np.int32).reshape(L, L)   # every site its own cluster
    a = oracle.assign(L, lab, seed, t)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    want = np.array([1 - 2 * (int(oracle.philox([r, t, 3, 0], key)[0]) >> 31) for r in range(L * L)])
    assert np.array_equal(a.reshape(-1), want)
    # fair coins: about half of 256 singletons are -1
    assert 90 < (a < 0).sum() < 166


@pytest.mark.parametrize("beta", [0.25, BETA_C_LIT, 0.6])
def test_assign_chain_moments_4x4(beta):
    exm = ex.exact_moments(4, beta)
    Es, Ms = [], []
    for k in range(3):
        _, E, M, _ = oracle.run(4, beta, 300 + k, 6000, rule="assign")
        Es.append(E[500:])
        Ms.append(M[500:])
    E = np.concatenate(Es).astype(float)
    aM = np.abs(np.concatenate(Ms)).astype(float)
    # batch-means errors (20 blocks per chain)
    def err(x):
        b = x[: len(x) // 60 * 60].reshape(60, -1).mean(axis=1)
        return b.std(ddof=1) / np.sqrt(len(b))
    assert abs(E.mean() - exm["E"]) < 5 * err(E)
    assert abs(aM.mean() - exm["absM"]) < 5 * err(aM)
