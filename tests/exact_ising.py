"""Exact results for the 2D Ising model on small periodic lattices, used to
pin the oracle. Nothing here calls the oracle except `sw_transition_matrix`,
which uses the oracle's labelling and flip steps on explicitly enumerated
bond sets (no random numbers) so that the transition kernel can be checked
against detailed balance.

References (restated from the literature, not from the paper under build):
  - brute-force sums over all 2^N states (the partition function Z, Eq. 1 of
    the paper's §2, with H = -sum_<ij> s_i s_j and k_B T = 1/beta);
  - B. Kaufman, Phys. Rev. 76, 1232 (1949): exact Z of an m x n torus;
  - L. Onsager, Phys. Rev. 65, 117 (1944): energy per site of the infinite
    lattice; C. N. Yang, Phys. Rev. 85, 808 (1952): spontaneous
    magnetisation (1 - sinh(2 beta)^-4)^(1/8).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.special

BETA_C = math.log1p(math.sqrt(2.0)) / 2.0


# ----------------------------------------------------------- enumeration

def all_states(L: int) -> np.ndarray:
    """Every configuration of an L x L lattice, int8 [2^N, L, L]."""
    N = L * L
    assert N <= 20
    idx = np.arange(2**N, dtype=np.int64)[:, None]
    bits = (idx >> np.arange(N)) & 1
    return (1 - 2 * bits).astype(np.int8).reshape(-1, L, L)


def energy_magnetisation(states: np.ndarray):
    s = states.astype(np.int64)
    E = -(s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)) - (s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    M = s.sum(axis=(1, 2))
    return E, M


def exact_moments(L: int, beta: float) -> dict:
    """Z and Boltzmann averages of E, E^2, |M|, M^2 by summing all states."""
    E, M = energy_magnetisation(all_states(L))
    w = np.exp(-beta * (E - E.min()))
    Z = w.sum()
    avg = lambda a: float((w * a).sum() / Z)
    return dict(logZ=float(np.log(Z) - beta * E.min()), E=avg(E), E2=avg(E.astype(float) ** 2),
                absM=avg(np.abs(M)), M2=avg(M.astype(float) ** 2))


def boltzmann(L: int, beta: float) -> np.ndarray:
    E, _ = energy_magnetisation(all_states(L))
    w = np.exp(-beta * (E - E.min()))
    return w / w.sum()


# --------------------------------------------------------------- Kaufman

def kaufman_logZ(m: int, n: int, K) -> mpmath.mpf:
    """log Z of the m-row, n-column periodic lattice at coupling K = beta J.

    Z = 1/2 (2 sinh 2K)^(mn/2) (Z1 + Z2 + Z3 + Z4), with
    Z1, Z2 = prod_{r=0}^{n-1} 2 cosh, 2 sinh (m g_{2r+1} / 2),
    Z3, Z4 = prod_{r=0}^{n-1} 2 cosh, 2 sinh (m g_{2r} / 2),
    cosh g_l = cosh 2K coth 2K - cos(pi l / n) for l > 0, and
    g_0 = 2K + log tanh K (which changes sign at K_c).
    """
    import mpmath  # only the Kaufman checks need arbitrary precision
    K = mpmath.mpf(K)
    c = mpmath.cosh(2 * K) / mpmath.tanh(2 * K)

    def gamma(l):
        if l == 0:
            return 2 * K + mpmath.log(mpmath.tanh(K))
        return mpmath.acosh(c - mpmath.cos(mpmath.pi * l / n))

    z1 = z2 = z3 = z4 = mpmath.mpf(1)
    for r in range(n):
        go = gamma(2 * r + 1)
        ge = gamma(2 * r)
        z1 *= 2 * mpmath.cosh(m * go / 2)
        z2 *= 2 * mpmath.sinh(m * go / 2)
        z3 *= 2 * mpmath.cosh(m * ge / 2)
        z4 *= 2 * mpmath.sinh(m * ge / 2)
    return mpmath.log(mpmath.mpf("0.5")) + (m * n / mpmath.mpf(2)) * mpmath.log(2 * mpmath.sinh(2 * K)) \
        + mpmath.log(z1 + z2 + z3 + z4)


def kaufman_energy_per_site(L: int, beta: float) -> float:
    """<E>/N = -(1/N) d log Z / d beta on the L x L torus (exact)."""
    import mpmath  # only the Kaufman checks need arbitrary precision
    with mpmath.workdps(40):
        d = mpmath.diff(lambda k: kaufman_logZ(L, L, k), mpmath.mpf(beta))
        return float(-d / (L * L))


# --------------------------------------------------- Onsager and Yang

def onsager_energy_per_site(beta: float) -> float:
    """Infinite-lattice energy per site, u = -coth(2b)[1 + (2/pi)(2 tanh^2(2b) - 1) K(k)],
    k = 2 sinh(2b) / cosh^2(2b); K the complete elliptic integral of the first kind."""
    t = 2.0 * beta
    k = 2.0 * math.sinh(t) / math.cosh(t) ** 2
    c = 2.0 * math.tanh(t) ** 2 - 1.0
    # At beta_c, k = 1 and K(k) diverges only logarithmically while c -> 0
    # linearly, so the product vanishes there.
    term = 0.0 if abs(c) < 1e-15 else c * scipy.special.ellipk(k * k)
    return -(1.0 / math.tanh(t)) * (1.0 + (2.0 / math.pi) * term)


def yang_magnetisation(beta: float) -> float:
    """Spontaneous magnetisation per site (1 - sinh(2 beta)^-4)^(1/8), beta > beta_c."""
    return (1.0 - math.sinh(2.0 * beta) ** -4) ** 0.125


# --------------------------------------------- exact Swendsen-Wang kernel

def sw_transition_matrix(L: int, beta: float, oracle, rule: str = "flip") -> np.ndarray:
    """T[a, b] = probability that one Swendsen-Wang update takes state a to b.

    Every bond set B among the satisfied edges of a (each bonded with
    probability p = 1 - exp(-2 beta), independently) and every flip (or,
    with rule="assign", new-spin) pattern of the clusters of B (each pattern
    with probability 2^-#clusters) is enumerated. The clusters come from the
    oracle's labelling and the new state from the oracle's flip (assign)
    step, so T is the kernel the oracle applies when its random words are
    replaced by exact probabilities.
    """
    states = all_states(L)
    nS = len(states)
    N = L * L
    p = -math.expm1(-2.0 * beta)
    code = lambda s: int((((1 - s.reshape(-1).astype(np.int64)) // 2) << np.arange(N)).sum())
    T = np.zeros((nS, nS))
    for a, s in enumerate(states):
        east = np.roll(s, -1, axis=1)
        south = np.roll(s, -1, axis=0)
        sat = [(y, x, 1) for y in range(L) for x in range(L) if s[y, x] == east[y, x]]
        sat += [(y, x, 2) for y in range(L) for x in range(L) if s[y, x] == south[y, x]]
        for mask in itertools.product((0, 1), repeat=len(sat)):
            b = np.zeros((L, L), np.uint8)
            nb = 0
            for on, (y, x, bit) in zip(mask, sat):
                if on:
                    b[y, x] |= bit
                    nb += 1
            wB = p**nb * (1 - p) ** (len(sat) - nb)
            if wB == 0.0:
                continue
            lab, nc = oracle.labels(b)
            roots = np.unique(lab)
            for flips in itertools.product((0, 1), repeat=nc):
                f = np.zeros(N, np.uint8)
                f[roots] = flips
                s2 = oracle.apply_assign(L, lab, f) if rule == "assign" else oracle.apply_flips(s, lab, f)
                T[a, code(s2)] += wB / 2**nc
    return T
