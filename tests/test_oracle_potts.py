"""Pins of the oracle's q-state Potts sweep (the paper's §6 generalisation:
H = -sum over edges of delta(s_i, s_j), bonds between equal states with
probability 1 - exp(-beta), each cluster assigned a state uniform in q).

What fixes it independently of its own code: for q = 2 it is exactly the
(pinned) Ising chain with the assignment rule at half the coupling
(delta(s, s') = (1 + s s') / 2); on the 2x2 torus with q = 3 its exact
one-sweep transition matrix satisfies detailed balance with the Potts
Boltzmann weights; on the 3x3 torus with q = 3 its chain reproduces the
exact moments of E and of the state-0 count; the threshold equals the Ising
threshold at half the argument; hot-start and new states are uniform.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle


@pytest.mark.parametrize("L,beta,seed,cold", [(2, 0.3, 1, False), (7, 0.44068679, 2, False),
                                               (16, 0.6, 3, True), (33, 0.2, 4, False)])
def test_q2_is_the_ising_assignment_chain(L, beta, seed, cold):
    n = 12
    sp, Ep, Mp = oracle.potts_run(L, 2, 2 * beta, seed, n, cold=cold)
    si, Ei, Mi, _ = oracle.run(L, beta, seed, n, cold=cold, rule="assign")
    N = L * L
    assert np.array_equal(sp, (si < 0).astype(np.int8))
    assert np.array_equal(Ep, Ei // 2 - N)
    assert np.array_equal(Mp, (N + Mi) // 2)


def test_threshold_is_ising_threshold_at_half_argument():
    for beta in np.linspace(0, 6, 301):
        assert oracle.potts_threshold(2 * beta) == oracle.threshold(beta)
    for beta in [0.1, 1.0, 1.0050833]:
        assert abs(oracle.potts_threshold(beta) - 2**32 * (-math.expm1(-beta))) <= 1.0


def _potts_states(L, q):
    N = L * L
    idx = np.arange(q**N)
    return np.stack([(idx // q**k) % q for k in range(N)], axis=1).astype(np.int8).reshape(-1, L, L)


def _energy_n0(states):
    s = states.astype(np.int64)
    eq = (s == np.roll(s, -1, axis=2)).sum(axis=(1, 2)) + (s == np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    return -eq, (s == 0).sum(axis=(1, 2))


@pytest.mark.parametrize("beta", [0.4, 1.0050833, 2.0])
def test_exact_kernel_detailed_balance_2x2_q3(beta):
    L, q = 2, 3
    states = _potts_states(L, q)
    N = L * L
    code = lambda s: int((s.reshape(-1).astype(np.int64) * q ** np.arange(N)).sum())
    p = -math.expm1(-beta)
    T = np.zeros((len(states), len(states)))
    for a, s in enumerate(states):
        east, south = np.roll(s, -1, axis=1), np.roll(s, -1, axis=0)
        sat = [(y, x, 1) for y in range(L) for x in range(L) if s[y, x] == east[y, x]]
        sat += [(y, x, 2) for y in range(L) for x in range(L) if s[y, x] == south[y, x]]
        for mask in itertools.product((0, 1), repeat=len(sat)):
            b = np.zeros((L, L), np.uint8)
            for on, (y, x, bit) in zip(mask, sat):
                if on:
                    b[y, x] |= bit
            nb = sum(mask)
            wB = p**nb * (1 - p) ** (len(sat) - nb)
            lab, nc = oracle.labels(b)
            roots = np.unique(lab)
            for vals in itertools.product(range(q), repeat=nc):
                v = np.zeros(N, np.uint8)
                v[roots] = vals
                T[a, code(oracle.potts_apply(L, lab, v))] += wB / q**nc
    E, _ = _energy_n0(states)
    w = np.exp(-beta * (E - E.min()))
    pi = w / w.sum()
    assert np.allclose(T.sum(axis=1), 1.0, atol=1e-13)
    assert np.abs(pi @ T - pi).max() < 1e-14
    F = pi[:, None] * T
    assert np.abs(F - F.T).max() < 1e-14


@pytest.mark.parametrize("beta", [0.5, 1.0050833, 1.6])
def test_chain_moments_3x3_q3(beta):
    L, q = 3, 3
    E_all, n0_all = _energy_n0(_potts_states(L, q))
    w = np.exp(-beta * (E_all - E_all.min()))
    w /= w.sum()
    exE, exN0 = float((w * E_all).sum()), float((w * n0_all).sum())
    Es, Ns = [], []
    for k in range(3):
        _, E, M = oracle.potts_run(L, q, beta, 700 + k, 8000)
        Es.append(E[500:])
        Ns.append(M[500:])
    E, n0 = np.concatenate(Es).astype(float), np.concatenate(Ns).astype(float)

    def err(x):
        b = x[: len(x) // 60 * 60].reshape(60, -1).mean(axis=1)
        return b.std(ddof=1) / np.sqrt(len(b))

    assert abs(E.mean() - exE) < 5 * err(E)
    assert abs(n0.mean() - exN0) < 5 * err(n0)


def test_states_follow_the_uniform_map_and_are_uniform():
    L, q, seed = 64, 5, 0xABCDEF0123
    s = oracle.potts_init(L, q, seed)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in [0, 1, 77, 4095]:
        x0 = int(oracle.philox([i, 0, 2, 0], key)[0])
        assert s.reshape(-1)[i] == (x0 * q) >> 32
    counts = np.bincount(s.reshape(-1), minlength=q)
    assert stats.chisquare(counts).pvalue > 1e-4
    lab = np.arange(L * L, dtype=np.int32).reshape(L, L)
    a = oracle.potts_assign(L, q, lab, seed, 9)
    x0 = int(oracle.philox([123, 9, 3, 0], key)[0])
    assert a.reshape(-1)[123] == (x0 * q) >> 32
    assert stats.chisquare(np.bincount(a.reshape(-1), minlength=q)).pvalue > 1e-4
    assert (oracle.potts_init(8, q, seed, cold=True) == 0).all()
