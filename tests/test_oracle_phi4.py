"""Pins of the oracle's O(4) phi^4 multicluster update (the paper's §3,
Eqs. 2 and 3) on an L^4 torus.

What fixes it independently of its own code: its exponential against the C
library's within one ulp; the direction's norm and isotropy; labels against
scipy's connected components of the same 4D bond graph; bonds only between
same-sign projections, with frequencies matching p = 1 - exp(-4 kappa a_x a_y)
computed with the library exponential; reflections keep |phi|, flip the
projection and keep the orthogonal part, and are involutions; whole clusters
flip together, half of them on average; and with every field parallel to
the update direction the update is the Swendsen-Wang update of an Ising
model at beta = 2 kappa c^2, which leaves that model's exact Boltzmann
distribution on the 2^4 torus invariant.
"""
import math

import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.csgraph
from scipy import stats

import oracle

KAPPA = 0.304


def test_exp_neg_within_one_ulp():
    rng = np.random.default_rng(0)
    zs = np.concatenate([np.linspace(0, 40, 8001), rng.uniform(0, 40, 8000), [1e-300, 5e-324, 0.5 * math.log(2)]])
    for z in zs:
        got, want = oracle.phi4_exp_neg(z), math.exp(-z)
        assert abs(got - want) <= 2.3e-16 * want, z
        # what a bond decision uses: 1 - e^-z scaled to 2^32
        assert abs((1.0 - got) - (-math.expm1(-z))) <= 2.3e-16 * max(1.0 - got, 1e-300) + 1.2e-16, z
    assert oracle.phi4_exp_neg(0.0) == 1.0
    # beyond z = 40, 1 - e^-z is 1 in binary64 and the function returns 0
    for z in [40.5, 100.0, 800.0]:
        assert oracle.phi4_exp_neg(z) == 0.0 and 1.0 - math.exp(-z) == 1.0
    v = [oracle.phi4_exp_neg(z) for z in np.linspace(0, 30, 3001)]
    assert all(a >= b for a, b in zip(v, v[1:]))


def test_direction_unit_and_isotropic():
    rs = np.array([oracle.phi4_direction(99, t) for t in range(4000)])
    assert np.abs((rs ** 2).sum(axis=1) - 1.0).max() < 1e-15
    assert np.abs(rs.mean(axis=0)).max() < 0.05
    C = rs.T @ rs / len(rs)
    assert np.abs(C - np.eye(4) / 4).max() < 0.03


def _graph_labels(bonds):
    L = bonds.shape[0]
    N = L**4
    idx = np.arange(N).reshape(L, L, L, L)
    rows, cols = [], []
    for mu in range(4):
        # site index x = x0 + L (x1 + L (x2 + L x3)): axis mu of the array is
        # dimension 3 - mu
        nbr = np.roll(idx, -1, axis=3 - mu)
        m = ((bonds >> mu) & 1).astype(bool)
        rows.append(idx[m])
        cols.append(nbr[m])
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    g = scipy.sparse.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(N, N))
    n, comp = scipy.sparse.csgraph.connected_components(g, directed=False)
    mins = np.full(n, N)
    np.minimum.at(mins, comp, np.arange(N))
    return mins[comp].reshape(L, L, L, L), n


@pytest.mark.parametrize("L,kappa,seed", [(2, 0.3, 1), (3, KAPPA, 2), (4, 0.5, 3), (5, 0.2, 4)])
def test_labels_match_connected_components(L, kappa, seed):
    phi = oracle.phi4_init(L, seed)
    r = oracle.phi4_direction(seed, 3)
    b = oracle.phi4_bonds(phi, kappa, seed, 3, r)
    lab, n = oracle.phi4_labels(b)
    want, nw = _graph_labels(b)
    assert n == nw and np.array_equal(lab, want)


def test_bonds_only_between_same_sign_projections_with_the_right_frequency():
    L, seed = 8, 11
    phi = oracle.phi4_init(L, seed)
    hits = np.zeros(10)
    tries = np.zeros(10)
    expect = np.zeros(10)
    for t in range(6):
        r = oracle.phi4_direction(seed, t)
        a = phi @ r
        b = oracle.phi4_bonds(phi, KAPPA, seed, t, r)
        for mu in range(4):
            ay = np.roll(a, -1, axis=3 - mu)
            bit = ((b >> mu) & 1).astype(bool)
            q = a * ay
            assert not bit[q <= 0].any()
            p = -np.expm1(-4 * KAPPA * np.where(q > 0, q, 0))
            k = np.minimum((p * 10).astype(int), 9)
            for j in range(10):
                sel = (q > 0) & (k == j)
                tries[j] += sel.sum()
                hits[j] += bit[sel].sum()
                expect[j] += p[sel].sum()
    for j in range(10):
        if tries[j] < 50:
            continue
        var = expect[j] * (1 - expect[j] / tries[j])
        assert abs(hits[j] - expect[j]) < 5 * math.sqrt(var) + 1, (j, hits[j], expect[j])


def test_reflection_geometry_and_coherent_clusters():
    L, seed, t = 5, 21, 4
    phi = oracle.phi4_init(L, seed)
    r = oracle.phi4_direction(seed, t)
    lab, n = oracle.phi4_labels(oracle.phi4_bonds(phi, KAPPA, seed, t, r))
    new = oracle.phi4_reflect(phi, lab, seed, t, r)
    assert np.allclose(np.linalg.norm(new, axis=-1), np.linalg.norm(phi, axis=-1), rtol=1e-15, atol=0)
    a, a2 = phi @ r, new @ r
    flipped = ~np.all(new == phi, axis=-1)
    assert np.allclose(a2[flipped], -a[flipped], atol=1e-15)
    perp, perp2 = phi - a[..., None] * r, new - a2[..., None] * r
    assert np.allclose(perp, perp2, atol=1e-14)
    for root in np.unique(lab)[:300]:
        f = flipped[lab == root]
        assert f.all() or not f.any()
    frac = np.mean([flipped[lab == root][0] for root in np.unique(lab)])
    assert 0.35 < frac < 0.65
    # a reflection undone: reflecting every site twice in the same direction
    twice = oracle.phi4_reflect(oracle.phi4_reflect(phi, np.zeros_like(lab), 0, 0, r), np.zeros_like(lab), 0, 0, r)
    assert np.allclose(twice, phi, atol=1e-14)


def _ising_energies(L):
    N = L**4
    idx = np.arange(2**N)[:, None]
    s = (1 - 2 * ((idx >> np.arange(N)) & 1)).astype(np.int8).reshape(-1, L, L, L, L)
    E = np.zeros(len(s), np.int64)
    for mu in range(4):
        E -= (s.astype(np.int64) * np.roll(s, -1, axis=4 - mu)).sum(axis=(1, 2, 3, 4))
    return s, E


def test_aligned_fields_follow_the_embedded_ising_chain():
    # phi_x = sigma_x c e_0 and r = e_0: the update is SW for an Ising model at
    # beta = 2 kappa c^2 (bond probability 1 - exp(-4 kappa c^2)), whose exact
    # Boltzmann distribution on the 2^4 torus it must leave invariant.
    L, kappa, c = 2, 0.25, 0.6
    beta = 2 * kappa * c * c
    s, E = _ising_energies(L)
    w = np.exp(-beta * (E - E.min()))
    w /= w.sum()
    levels, inv = np.unique(E, return_inverse=True)
    p_level = np.bincount(inv, weights=w)
    rng = np.random.default_rng(5)
    n = 20000
    start = rng.choice(len(w), size=n, p=w)
    r = np.array([1.0, 0.0, 0.0, 0.0])
    counts = np.zeros(len(levels))
    for i, k in enumerate(start):
        phi = np.zeros((L, L, L, L, 4))
        phi[..., 0] = c * s[k]
        lab, _ = oracle.phi4_labels(oracle.phi4_bonds(phi, kappa, 1000 + i, 0, r))
        new = oracle.phi4_reflect(phi, lab, 1000 + i, 0, r)
        sig = np.sign(new[..., 0]).astype(np.int64)
        e = sum(-(sig * np.roll(sig, -1, axis=3 - mu)).sum() for mu in range(4))
        counts[np.searchsorted(levels, e)] += 1
    exp_ = n * p_level
    keep = exp_ >= 5
    obs, ex = counts[keep], exp_[keep]
    if (~keep).any():
        obs, ex = np.append(obs, counts[~keep].sum()), np.append(ex, exp_[~keep].sum())
    chi2 = ((obs - ex) ** 2 / ex).sum()
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-4, chi2
