"""O(4) phi^4 multicluster updates (§3, Eqs. 2 and 3) on the GPU: the field
equals the oracle's bit for bit (floating point decides the bonds, and both
sides take each decision with the same operations), labels equal the
oracle's BFS labels, directions equal the oracle's, and E and M agree with
the oracle's serial sums to rounding."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
KAPPA = 0.304


@pytest.fixture(scope="module")
def sw():
    from conftest import build_libsw
    build_libsw()
    import paper_2302_14720_gb300 as sw
    return sw


def test_direction_matches_oracle(sw):
    for seed, t in [(1, 0), (99, 3), (2**40 + 7, 12345)]:
        assert np.array_equal(sw.sw_phi4_direction(seed, t), oracle.phi4_direction(seed, t))


@pytest.mark.parametrize("L,kappa,cold", [(2, 0.3, False), (3, KAPPA, False), (5, 0.5, True), (8, KAPPA, False),
                                          (11, 0.2, False)])
def test_phi4_chain_parity(sw, L, kappa, cold):
    seed, n = 40 + L, 6
    with sw.Phi4(L, kappa, seed, sw.SW_INIT_COLD if cold else sw.SW_INIT_HOT) as f:
        f.sweep(2)
        f.sweep(4)
        want, wE, wM = oracle.phi4_run(L, kappa, seed, n, cold=cold)
        got = f.field()
        assert np.array_equal(got, want)
        E, M = f.observables(0, n)
        scale = 4 * L**4 * np.abs(want).max() ** 2 + 1.0
        assert np.abs(E - wE).max() <= 1e-12 * scale
        assert np.abs(M - wM).max() <= 1e-12 * scale


@pytest.mark.parametrize("L,n", [(16, 5), (28, 5), (64, 1)])
def test_phi4_bench_configuration(sw, L, n):
    """The benchmark's runs (kappa = 0.304, hot start, seed 6) at the
    smallest and largest L of the paper's table, five updates, and its
    L = 64 run (a field larger than L2), one update."""
    seed = 6
    with sw.Phi4(L, KAPPA, seed) as f:
        f.sweep(n)
        want, wE, wM = oracle.phi4_run(L, KAPPA, seed, n)
        assert np.array_equal(f.field(), want)
        E, M = f.observables(0, n)
        scale = 4 * L**4 * np.abs(want).max() ** 2 + 1.0
        assert np.abs(E - wE).max() <= 1e-12 * scale
        assert np.abs(M - wM).max() <= 1e-12 * scale


def test_phi4_labels_and_set_field(sw):
    L, seed, t = 6, 5, 9
    rng = np.random.default_rng(2)
    phi = rng.normal(size=(L, L, L, L, 4))
    with sw.Phi4(L, KAPPA, seed) as f:
        f.set_field(phi, t)
        lab = f.labels()
        r = oracle.phi4_direction(seed, t)
        want, _ = oracle.phi4_labels(oracle.phi4_bonds(phi, KAPPA, seed, t, r))
        assert np.array_equal(lab, want)
        f.sweep(3)
        wf, wE, _ = oracle.phi4_run(L, KAPPA, seed, 3, phi=phi, t0=t)
        assert np.array_equal(f.field(), wf)
