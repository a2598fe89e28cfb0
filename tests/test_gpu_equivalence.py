"""The paper's label-equivalence labelling (§2.3), kept as a comparator:
its labels equal the oracle's BFS labels and the union-find path's labels
on the same bond graph, bit for bit."""
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


@pytest.mark.parametrize("L,beta", [(2, 0.4), (5, 0.9), (33, BETA_C), (130, 0.3), (257, 0.6), (300, BETA_C)])
def test_equivalence_labels_match_oracle_and_union_find(sw, L, beta):
    seed, t = 77 + L, 5
    s0 = random_spins(L, seed=L, p_minus=0.4)
    with sw.Lattice(L, beta, seed) as lat:
        lat.set_state(s0, t)
        lab_le, its = lat.labels_equivalence()
        lab_uf = lat.labels()
    want, _ = oracle.labels(oracle.bonds(s0, seed, t, oracle.threshold(beta)))
    assert its >= 1
    assert np.array_equal(lab_le, want)
    assert np.array_equal(lab_uf, want)


def test_equivalence_at_L1024(sw):
    L, beta, seed = 1024, BETA_C, 2
    with sw.Lattice(L, beta, seed, sw.SW_INIT_COLD) as lat:
        lat.sweep(20)
        lab_le, its = lat.labels_equivalence()
        lab_uf = lat.labels()
    assert np.array_equal(lab_le, lab_uf)
    assert (lab_le <= np.arange(L * L).reshape(L, L)).all()
