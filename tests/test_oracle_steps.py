"""Pin each step of the oracle's sweep (§2.1 bonds, §2.3 labels, §2.4 flips,
end of §2 observables, cluster statistics) against mathematics and library
routines that share nothing with the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import oracle
from workloads import random_spins

SIZES = [2, 3, 4, 5, 7, 16, 17, 33]


def bond_edges(b: np.ndarray):
    """Edge list (i, j) of a bond array: bit0 east, bit1 south (C1)."""
    L = b.shape[0]
    y, x = np.nonzero(b & 1)
    e1 = np.stack([y * L + x, y * L + (x + 1) % L], 1)
    y, x = np.nonzero(b & 2)
    e2 = np.stack([y * L + x, ((y + 1) % L) * L + x], 1)
    return np.concatenate([e1, e2]).astype(np.int64)


def scipy_canonical_labels(b: np.ndarray) -> np.ndarray:
    """Components by scipy, relabelled to the minimum site of each component."""
    L = b.shape[0]
    N = L * L
    e = bond_edges(b)
    A = sp.coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(N, N))
    _, comp = connected_components(A, directed=False)
    mins = np.full(comp.max() + 1, N, dtype=np.int64)
    np.minimum.at(mins, comp, np.arange(N))
    return mins[comp].reshape(L, L).astype(np.int32)


def union_find_labels(b: np.ndarray) -> np.ndarray:
    """A second, differently written labelling: union by smaller index with
    full path compression, processed edge by edge."""
    L = b.shape[0]
    parent = list(range(L * L))

    def root(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for i, j in bond_edges(b):
        ri, rj = root(int(i)), root(int(j))
        if ri != rj:
            parent[max(ri, rj)] = min(ri, rj)
    return np.array([root(a) for a in range(L * L)], dtype=np.int32).reshape(L, L)


# ------------------------------------------------------------------ init

def test_init_cold_and_hot():
    assert (oracle.init(9, 5, cold=True) == 1).all()
    s = oracle.init(256, 1)
    assert set(np.unique(s)) <= {-1, 1}
    frac = (s == -1).mean()
    n = s.size
    assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(n)
    assert not np.array_equal(s, oracle.init(256, 2))
    assert np.array_equal(s, oracle.init(256, 1))


# ----------------------------------------------------------------- bonds

@pytest.mark.parametrize("L", SIZES)
def test_bonds_only_between_equal_spins(L):
    s = random_spins(L, seed=L)
    b = oracle.bonds(s, seed=9, t=3, thr=oracle.threshold(0.7))
    east = np.roll(s, -1, axis=1)
    south = np.roll(s, -1, axis=0)
    assert not ((b & 1).astype(bool) & (s != east)).any()
    assert not ((b & 2).astype(bool) & (s != south)).any()


def test_bond_frequency_matches_threshold():
    # Among equal-spin pairs a bond forms with probability thr / 2^32.
    L = 256
    for beta in (0.2, 0.44068679, 0.5):
        thr = oracle.threshold(beta)
        p = thr / 2.0**32
        s = random_spins(L, seed=77)
        n_eq = 0
        n_b = 0
        for t in range(4):
            b = oracle.bonds(s, seed=1234, t=t, thr=thr)
            eq_e = s == np.roll(s, -1, axis=1)
            eq_s = s == np.roll(s, -1, axis=0)
            n_eq += eq_e.sum() + eq_s.sum()
            n_b += (b & 1).astype(bool).sum() + (b & 2).astype(bool).sum()
        z = (n_b - n_eq * p) / np.sqrt(n_eq * p * (1 - p))
        assert abs(z) < 5, (beta, z)
        assert abs(p - (-np.expm1(-2 * beta))) < 2.0**-32


def test_bonds_limits():
    s = np.ones((8, 8), dtype=np.int8)
    assert (oracle.bonds(s, 1, 0, 0) == 0).all()
    full = oracle.bonds(s, 1, 0, 0xFFFFFFFF)
    assert (full == 3).mean() > 0.99


def test_bonds_depend_on_sweep_and_seed():
    s = np.ones((32, 32), dtype=np.int8)
    thr = oracle.threshold(0.44068679)
    a = oracle.bonds(s, 1, 0, thr)
    assert not np.array_equal(a, oracle.bonds(s, 1, 1, thr))
    assert not np.array_equal(a, oracle.bonds(s, 2, 0, thr))
    assert np.array_equal(a, oracle.bonds(s, 1, 0, thr))


# ---------------------------------------------------------------- labels

@pytest.mark.parametrize("L", SIZES)
@pytest.mark.parametrize("beta", [0.0, 0.3, 0.44068679, 0.6, 3.0])
def test_labels_match_scipy_and_union_find(L, beta):
    s = random_spins(L, seed=3 * L + 1)
    b = oracle.bonds(s, seed=5, t=7, thr=oracle.threshold(beta))
    lab, n = oracle.labels(b)
    want = scipy_canonical_labels(b)
    assert np.array_equal(lab, want)
    assert np.array_equal(lab, union_find_labels(b))
    assert n == len(np.unique(lab))


def test_labels_invariants_and_degenerate_cases():
    L = 17
    flat_idx = np.arange(L * L).reshape(L, L)
    # no bonds: every site is its own cluster
    lab, n = oracle.labels(np.zeros((L, L), np.uint8))
    assert np.array_equal(lab, flat_idx) and n == L * L
    # all bonds: one cluster rooted at 0
    lab, n = oracle.labels(np.full((L, L), 3, np.uint8))
    assert (lab == 0).all() and n == 1
    # only the periodic wrap edges of row 3 and column 5 are bonded
    b = np.zeros((L, L), np.uint8)
    b[3, L - 1] |= 1
    b[L - 1, 5] |= 2
    lab, n = oracle.labels(b)
    assert lab[3, 0] == lab[3, L - 1] == 3 * L
    assert lab[0, 5] == lab[L - 1, 5] == 5
    # invariants on a random state
    s = random_spins(L, seed=1)
    b = oracle.bonds(s, 2, 0, oracle.threshold(0.5))
    lab, _ = oracle.labels(b)
    f = lab.reshape(-1)
    assert (f[f] == f).all()
    assert (f <= np.arange(L * L)).all()
    e = bond_edges(b)
    assert (f[e[:, 0]] == f[e[:, 1]]).all()


def test_labels_double_edges_L2():
    # L = 2: the east and west neighbour are the same site; each edge counts.
    b = np.zeros((2, 2), np.uint8)
    b[0, 1] = 1  # east bond of (0,1) wraps to (0,0)
    lab, n = oracle.labels(b)
    assert lab.tolist() == [[0, 0], [2, 3]] and n == 3


# ------------------------------------------------------------------ flip

@pytest.mark.parametrize("L", [2, 5, 16, 33])
def test_flip_keeps_clusters_monochrome(L):
    s = random_spins(L, seed=L)
    b = oracle.bonds(s, 11, 0, oracle.threshold(0.5))
    lab, n = oracle.labels(b)
    s2 = oracle.flip(s, lab, 11, 0)
    f = lab.reshape(-1)
    new = s2.reshape(-1)
    old = s.reshape(-1)
    for r in np.unique(f):
        m = f == r
        assert len(np.unique(new[m])) == 1
        assert len(np.unique(old[m])) == 1
        # a cluster either flips as a whole or not at all
        assert (new[m] == old[m]).all() or (new[m] == -old[m]).all()


def test_flip_fraction_is_half():
    L = 128
    s = random_spins(L, seed=4)
    b = oracle.bonds(s, 3, 0, oracle.threshold(0.3))
    lab, n = oracle.labels(b)
    s2 = oracle.flip(s, lab, 3, 0)
    roots = np.unique(lab)
    flipped = (s2.reshape(-1)[roots] != s.reshape(-1)[roots]).sum()
    assert abs(flipped - n / 2) < 5 * np.sqrt(n) / 2


def test_apply_flips_explicit():
    L = 4
    lab = np.arange(L * L, dtype=np.int32).reshape(L, L)
    lab[0, :] = 0
    s = np.ones((L, L), np.int8)
    f = np.zeros(L * L, np.uint8)
    f[0] = 1
    out = oracle.apply_flips(s, lab, f)
    assert (out[0] == -1).all() and (out[1:] == 1).all()


# ------------------------------------------------------------- chain-level

@pytest.mark.parametrize("L", [2, 3, 8, 17])
def test_spin_reversal_symmetry(L):
    # Bonds depend only on spin equality and the flip is relative, so the
    # chain from -s is exactly minus the chain from s.
    s = random_spins(L, seed=L + 100)
    a, Ea, Ma, _ = oracle.run(L, 0.44068679, 21, 6, spins=s)
    b, Eb, Mb, _ = oracle.run(L, 0.44068679, 21, 6, spins=-s)
    assert np.array_equal(a, -b)
    assert np.array_equal(Ea, Eb) and np.array_equal(Ma, -Mb)


def test_sweep_composition():
    L = 12
    s0 = oracle.init(L, 8)
    a, Ea, Ma, _ = oracle.run(L, 0.4, 8, 7, spins=s0)
    m, E1, M1, _ = oracle.run(L, 0.4, 8, 3, spins=s0)
    b, E2, M2, _ = oracle.run(L, 0.4, 8, 4, spins=m, t0=3)
    assert np.array_equal(a, b)
    assert np.array_equal(Ea, np.concatenate([E1, E2]))
    assert np.array_equal(Ma, np.concatenate([M1, M2]))


def test_beta_zero_is_independent_coin_flips():
    # thr = 0: no bonds, every site is a cluster, each flips with prob 1/2.
    L = 64
    s = np.ones((L, L), np.int8)
    out, E, M, H = oracle.run(L, 0.0, 5, 1, spins=s, hist=True)
    assert H[0, 0] == L * L and H[0, 1] == L * L and H[0, 2] == L * L
    assert abs((out == -1).mean() - 0.5) < 5 * 0.5 / L


# ----------------------------------------------------------- observables

@pytest.mark.parametrize("L", [2, 3, 4, 6, 9])
def test_observe_closed_forms(L):
    N = L * L
    up = np.ones((L, L), np.int8)
    assert oracle.observe(up) == (-2 * N, N)
    assert oracle.observe(-up) == (-2 * N, -N)
    one = up.copy()
    one[1 % L, 0] = -1
    assert oracle.observe(one) == (-2 * N + 8, N - 2)
    if L % 2 == 0:
        y, x = np.indices((L, L))
        cb = np.where((x + y) % 2 == 0, 1, -1).astype(np.int8)
        assert oracle.observe(cb) == (2 * N, 0)
        stripes = np.where(x % 2 == 0, 1, -1).astype(np.int8)
        assert oracle.observe(stripes) == (0, 0)


# ------------------------------------------------------------- histogram

@pytest.mark.parametrize("L", [3, 16, 31])
def test_histogram_matches_scipy_sizes(L):
    s = random_spins(L, seed=L)
    b = oracle.bonds(s, 2, 0, oracle.threshold(0.6))
    lab = scipy_canonical_labels(b)
    sizes = np.bincount(lab.reshape(-1))
    sizes = sizes[sizes > 0]
    h = oracle.histogram(oracle.labels(b)[0])
    assert h[0] == len(sizes)
    assert h[1] == int((sizes.astype(np.int64) ** 2).sum())
    bins = np.bincount(np.floor(np.log2(sizes)).astype(int), minlength=32)
    assert np.array_equal(h[2:], bins)
    assert (h[2:] * 0 + 1).sum() == 32


# ------------------------------------------ conventions C5-C7 word by word
# The statistics above cannot tell which Philox word or bit a convention
# uses, nor '<' from '<=' at the threshold. These checks take the Philox
# block from oracle.philox (pinned to cuRAND's generator) and the
# conventions as stated in include/sw.h.

def _key(seed):
    return (seed & 0xFFFFFFFF, seed >> 32)


def test_hot_start_word_and_bit():
    L, seed = 9, 0xABCDEF0123
    s = oracle.init(L, seed)
    for i in range(L * L):
        x0 = oracle.philox((i, 0, 2, 0), _key(seed))[0]
        assert s.reshape(-1)[i] == (-1 if x0 >> 31 else 1)


@pytest.mark.parametrize("L", [4, 5])
def test_bond_words_and_strict_threshold(L):
    seed, t = 0x1234_5678_9ABC, 17
    s = np.ones((L, L), np.int8)
    for i in range(L * L):
        blk = oracle.philox((i >> 1, t, 0, 0), _key(seed))
        for d in (0, 1):
            u = int(blk[2 * (i & 1) + d])
            below = oracle.bonds(s, seed, t, u).reshape(-1)[i]
            assert (below >> d) & 1 == 0  # u < u is false: strict comparison
            if u < 0xFFFFFFFF:
                above = oracle.bonds(s, seed, t, u + 1).reshape(-1)[i]
                assert (above >> d) & 1 == 1


@pytest.mark.parametrize("L", [7, 16, 23])
def test_flip_word_and_bit(L):
    # beta = 0: no bonds, every site is its own root, so the flips of sites
    # 0 .. N-1 are the bit stream of blocks (0, t, 1, 0), (1, t, 1, 0), ...:
    # words x0..x3 of each block in order, bit 0 of a word first.
    seed, t = 99, 5
    s = random_spins(L, seed=3)
    out, _, _, _ = oracle.run(L, 0.0, seed, 1, spins=s, t0=t)
    N = L * L
    words = np.concatenate([oracle.philox((b, t, 1, 0), _key(seed)) for b in range((N + 127) // 128)])
    stream = np.unpackbits(words.astype("<u4").view(np.uint8), bitorder="little")[:N]
    want = np.where(stream == 1, -s.reshape(-1), s.reshape(-1))
    assert np.array_equal(out.reshape(-1), want)
