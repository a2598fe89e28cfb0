"""Pin the oracle's chain as a whole against exact Ising results.

  - Kaufman's exact finite-torus partition function is itself pinned to
    brute-force enumeration, then used for finite-L energies.
  - The exact Swendsen-Wang kernel on 2x2 (oracle labelling + flip on
    enumerated bond sets) satisfies detailed balance with the Boltzmann
    weights of Eq. 1.
  - One Philox-driven oracle sweep started from an exact Boltzmann sample on
    3x3 leaves the Boltzmann distribution invariant (chi-square).
  - Long oracle runs reproduce exact 4x4 moments, Kaufman energies at beta_c,
    Yang's spontaneous magnetisation, and the identity E[M^2 | clusters] =
    sum |C|^2 of the cluster statistics.
Statistical checks use batch means and |z| < 4.5.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import exact_ising as ex

BETA_C_LIT = 0.44068679


def zscore(samples: np.ndarray, target: float, n_batches: int = 50) -> float:
    x = np.asarray(samples, dtype=float)
    x = x[: len(x) // n_batches * n_batches].reshape(n_batches, -1).mean(axis=1)
    se = x.std(ddof=1) / math.sqrt(n_batches)
    return (x.mean() - target) / max(se, 1e-300)


# ------------------------------------------------------- exact formulas

@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("beta", [0.05, 0.3, ex.BETA_C, 0.7, 1.5])
def test_kaufman_equals_enumeration(L, beta):
    assert abs(float(ex.kaufman_logZ(L, L, beta)) - ex.exact_moments(L, beta)["logZ"]) < 1e-11


def test_kaufman_energy_by_enumeration_derivative():
    for L in (3, 4):
        for beta in (0.2, ex.BETA_C, 0.6):
            assert abs(ex.kaufman_energy_per_site(L, beta) - ex.exact_moments(L, beta)["E"] / (L * L)) < 1e-10


def test_large_torus_reaches_onsager():
    # Away from beta_c finite-size corrections are exponentially small.
    for beta in (0.3, 0.6):
        assert abs(ex.kaufman_energy_per_site(64, beta) - ex.onsager_energy_per_site(beta)) < 1e-8
    # At beta_c the correction is O(1/L) and the limit is -sqrt(2).
    assert abs(ex.onsager_energy_per_site(ex.BETA_C) + math.sqrt(2)) < 1e-12
    e128 = ex.kaufman_energy_per_site(128, ex.BETA_C)
    e256 = ex.kaufman_energy_per_site(256, ex.BETA_C)
    assert 0 < (-math.sqrt(2) - e256) < (-math.sqrt(2) - e128) < 2.0 / 128


def test_yang_values():
    assert abs(ex.yang_magnetisation(0.45) - 0.7493) < 1e-4
    assert abs(ex.yang_magnetisation(0.48) - 0.8775) < 1e-4
    assert abs(ex.yang_magnetisation(0.50) - 0.91132) < 1e-5


# ----------------------------------------------------- exact SW kernel

@pytest.mark.parametrize("beta", [0.2, BETA_C_LIT, 0.9])
def test_sw_kernel_detailed_balance_2x2(beta):
    T = ex.sw_transition_matrix(2, beta, oracle)
    pi = ex.boltzmann(2, beta)
    assert np.allclose(T.sum(axis=1), 1.0, atol=1e-13)
    assert np.abs(pi @ T - pi).max() < 1e-14
    F = pi[:, None] * T
    assert np.abs(F - F.T).max() < 1e-14
    # ergodic and aperiodic: every entry of T^2 positive
    assert (np.linalg.matrix_power(T, 2) > 0).all()


def test_one_sweep_preserves_boltzmann_3x3():
    L, beta = 3, 0.3
    pi = ex.boltzmann(L, beta)
    states = ex.all_states(L)
    rng = np.random.default_rng(123)
    n = 60_000
    start = rng.choice(len(pi), size=n, p=pi)
    weights = 1 << np.arange(L * L)
    counts = np.zeros(len(pi))
    for i, a in enumerate(start):
        s, _, _, _ = oracle.run(L, beta, seed=10_000 + i, n=1, spins=states[a], t0=i)
        counts[int((((1 - s.reshape(-1).astype(np.int64)) // 2) * weights).sum())] += 1
    expected = n * pi
    keep = expected >= 5
    obs, exp_ = counts[keep], expected[keep]
    if (~keep).any():
        obs = np.append(obs, counts[~keep].sum())
        exp_ = np.append(exp_, expected[~keep].sum())
    chi2 = ((obs - exp_) ** 2 / exp_).sum()
    pval = stats.chi2.sf(chi2, len(obs) - 1)
    assert pval > 1e-4, (chi2, len(obs), pval)


# ------------------------------------------------------- long oracle runs

@pytest.mark.parametrize("beta", [0.2, BETA_C_LIT, 0.6])
def test_oracle_moments_4x4(beta):
    L, n = 4, 200_000
    ex_m = ex.exact_moments(L, beta)
    _, E, M, _ = oracle.run(L, beta, seed=int(beta * 1e6), n=n)
    E = E.astype(float)
    M = M.astype(float)
    for name, x in (("E", E), ("E2", E**2), ("absM", np.abs(M)), ("M2", M**2)):
        z = zscore(x, ex_m[name])
        assert abs(z) < 4.5, (beta, name, z)


@pytest.mark.parametrize("L", [12, 16])
def test_oracle_energy_matches_kaufman(L):
    n, burn = 20_000, 200
    _, E, _, _ = oracle.run(L, BETA_C_LIT, seed=L, n=n + burn)
    e = E[burn:] / (L * L)
    z = zscore(e, ex.kaufman_energy_per_site(L, BETA_C_LIT))
    assert abs(z) < 4.5, z


def test_oracle_spontaneous_magnetisation():
    L, n, burn, beta = 64, 1500, 100, 0.5
    _, _, M, _ = oracle.run(L, beta, seed=9, n=n + burn, cold=True)
    m = np.abs(M[burn:]) / (L * L)
    target = ex.yang_magnetisation(beta)
    z = zscore(m, target, n_batches=30)
    assert abs(z) < 4.5 or abs(m.mean() - target) < 1e-3, (m.mean(), target, z)


def test_cluster_statistics_improved_estimator():
    # Given the clusters of a sweep every cluster's new sign is a fair coin,
    # so E[M^2 | clusters] = sum |C|^2, hence sum|C|^2 - M^2 has mean zero.
    L, n = 32, 6000
    _, _, M, H = oracle.run(L, BETA_C_LIT, seed=77, n=n, hist=True)
    d = H[:, 1].astype(float) - M.astype(float) ** 2
    z = zscore(d, 0.0)
    assert abs(z) < 4.5, z
    assert (H[:, 2:].sum(axis=1) == H[:, 0]).all()
