"""Parity of the headline workload's own chain, at full size (L = 8192).

The benchmark's lattice (L = 8192, hot start from seed 3) is run on the GPU
through the C ABI in the launch configuration the benchmark times, and on
the CPU oracle from the same seeded start:

* the first 20 sweeps at beta_c and at beta = 0.50, compared sweep by sweep
  (E and M), then the final spins and the canonical labels of the next
  sweep's bonds element by element. From a hot start the clusters grow to
  the critical (beta_c) or spanning (0.50) shapes within these sweeps, so
  the cross-tile merge meets clusters that span many tiles;
* later sweeps (t = 500 and t = 1999 of the same chain) are too far for the
  serial oracle (about 3.5 s per sweep), so there the GPU's own state is
  checked through properties that hold at any size and sampled outputs the
  oracle computes one by one: bonds only join equal spins, each sampled
  bond and each sampled cluster's flip equals its Philox draw (C5, C6), the
  labels are the connected components of the exported bond graph
  (scipy) with the minimum site as label (C9), every cluster flips as a
  whole, and E and M equal their definitions on the new spins.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

BETA_C = 0.44068679
L, SEED = 8192, 3


@pytest.fixture(scope="module")
def sw():
    from conftest import build_libsw
    build_libsw()
    import paper_2302_14720_gb300 as sw
    return sw


@pytest.mark.parametrize("beta", [BETA_C, 0.50])
def test_first_sweeps_of_the_headline_chain(sw, beta):
    n = 20
    with sw.Lattice(L, beta, SEED, sw.SW_INIT_HOT) as lat:
        lat.sweep(n)
        E, M = lat.observables(0, n)
        spins = lat.spins()
        lab = lat.labels()  # clusters of sweep n's bonds from the current state
    want_s, want_E, want_M, _ = oracle.run(L, beta, SEED, n)
    assert np.array_equal(E, want_E), np.flatnonzero(E != want_E)[:5]
    assert np.array_equal(M, want_M), np.flatnonzero(M != want_M)[:5]
    assert np.array_equal(spins, want_s)
    del spins
    want_lab, ncl = oracle.labels(oracle.bonds(want_s, SEED, n, oracle.threshold(beta)))
    assert np.array_equal(lab, want_lab)
    # the clusters compared are large: the biggest covers more sites than ten
    # 128 x 64 tiles hold
    sizes = np.bincount(want_lab.reshape(-1))
    assert sizes.max() > 10 * 128 * 64


def _components(bonds: np.ndarray) -> np.ndarray:
    """Minimum-site label of every site's component in the bond graph, by
    scipy's connected components (independent of the oracle and the GPU)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    n = bonds.size
    idx = np.arange(n, dtype=np.int64).reshape(L, L)
    e = (bonds & 1).astype(bool)
    s = (bonds & 2).astype(bool)
    src = np.concatenate([idx[e], idx[s]])
    dst = np.concatenate([np.roll(idx, -1, axis=1)[e], np.roll(idx, -1, axis=0)[s]])
    g = coo_matrix((np.ones(src.size, np.uint8), (src.astype(np.int32), dst.astype(np.int32))), shape=(n, n))
    _, comp = connected_components(g, directed=False)
    _, first = np.unique(comp, return_index=True)  # smallest site of each component
    return first[comp].reshape(L, L).astype(np.int32)


def _philox_key(seed):
    return (seed & 0xFFFFFFFF, seed >> 32)


@pytest.mark.parametrize("beta", [BETA_C, 0.50])
def test_late_sweeps_of_the_headline_chain(sw, beta):
    thr = oracle.threshold(beta)
    key = _philox_key(SEED)
    rng = np.random.default_rng(8192)
    with sw.Lattice(L, beta, SEED, sw.SW_INIT_HOT) as lat:
        for t in (500, 1999):
            lat.sweep(t - lat.t)
            old = lat.spins()
            bonds = lat.bonds()
            lab = lat.labels()
            lat.sweep(1)
            E, M = lat.observables(t, 1)
            new = lat.spins()

            # bonds join equal spins only; sampled draws equal C5's Philox words
            east_eq = old == np.roll(old, -1, axis=1)
            south_eq = old == np.roll(old, -1, axis=0)
            assert not ((bonds & 1).astype(bool) & ~east_eq).any()
            assert not ((bonds & 2).astype(bool) & ~south_eq).any()
            for i in rng.integers(0, L * L, 400):
                y, x = divmod(int(i), L)
                q = oracle.philox((int(i) >> 1, t, 0, 0), key)
                want_e = bool(east_eq[y, x]) and int(q[2 * (int(i) & 1)]) < thr
                want_s = bool(south_eq[y, x]) and int(q[2 * (int(i) & 1) + 1]) < thr
                assert bool(bonds[y, x] & 1) == want_e and bool(bonds[y, x] & 2) == want_s, (t, y, x)

            # labels: the components of that bond graph, named by their minimum site
            assert np.array_equal(lab, _components(bonds))
            del bonds

            # each cluster flips as a whole; sampled clusters flip by their C6 bit
            flipped = (old != new).reshape(-1)
            labf = lab.reshape(-1)
            size = np.bincount(labf, minlength=L * L)
            nflip = np.bincount(labf, weights=flipped, minlength=L * L)
            roots = np.flatnonzero(size)
            assert np.all((nflip[roots] == 0) | (nflip[roots] == size[roots]))
            for r in rng.choice(roots, 400, replace=False):
                r = int(r)
                q = oracle.philox((r >> 7, t, 1, 0), key)
                want = (int(q[(r >> 5) & 3]) >> (r & 31)) & 1
                assert int(nflip[r] > 0) == want, (t, r)
            assert abs(np.mean(nflip[roots] > 0) - 0.5) < 6 * 0.5 / np.sqrt(roots.size)

            # E and M of the new state, from their definitions
            n64 = new.astype(np.int64)
            want_E = -int((n64 * np.roll(n64, -1, axis=1)).sum() + (n64 * np.roll(n64, -1, axis=0)).sum())
            assert E[0] == want_E and M[0] == int(n64.sum())
            del old, new, lab, n64
