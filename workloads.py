"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
runs. This module holds none of the method's arithmetic: it only draws spin
configurations and workload parameters (lattice sides, inverse temperatures,
seeds, sweep counts, arrival times) from numpy's seeded generators.

The workloads follow the paper's own benchmark (§5, Table 1: square lattices
of side 128 to 4096, 10^4 iterations) scaled to the five configurations this
library is measured on; no dataset is involved (the paper uses none).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BETA_C_LITERAL = 0.44068679  # the beta the configurations quote for beta_c


def random_spins(L: int, seed: int, p_minus: float = 0.5) -> np.ndarray:
    """int8 [L, L] of +1/-1, each -1 with probability p_minus."""
    rng = np.random.default_rng(seed)
    return np.where(rng.random((L, L)) < p_minus, -1, 1).astype(np.int8)


def striped_spins(L: int, width: int) -> np.ndarray:
    """Vertical stripes of the given width: long straight cluster borders."""
    x = np.arange(L)
    row = np.where((x // max(width, 1)) % 2 == 0, 1, -1).astype(np.int8)
    return np.tile(row, (L, 1))


@dataclass(frozen=True)
class Config:
    name: str
    L: int
    beta: float
    seed: int
    init: str  # "hot" or "cold"
    sweeps: int
    histogram: bool = False


CONFIGS = {
    "L64": Config("L64 beta_c hot seed1", 64, BETA_C_LITERAL, 1, "hot", 1000),
    "L1024": Config("L1024 beta_c cold seed2 histogram", 1024, BETA_C_LITERAL, 2, "cold", 10_000, True),
    "L8192": Config("L8192 beta_c hot seed3", 8192, BETA_C_LITERAL, 3, "hot", 2000),
    "L8192b05": Config("L8192 beta0.50 hot seed3", 8192, 0.50, 3, "hot", 2000),
}


def batch_replicas():
    """256 replicas r = 4b + k: beta on a 64-point grid in [0.40, 0.48],
    4 seeds each, L drawn uniformly from {64,128,256,512,1024}.
    Returns lists (L, beta, seed)."""
    rng = np.random.default_rng(4)
    Ls = rng.choice([64, 128, 256, 512, 1024], 256)
    out_L, out_b, out_s = [], [], []
    for r in range(256):
        b, k = divmod(r, 4)
        out_L.append(int(Ls[r]))
        out_b.append(0.40 + 0.08 * b / 63)
        out_s.append(1000 + r)
    return out_L, out_b, out_s


def serving_requests(n: int = 2000, rate_per_s: float = 1.0, seed: int = 5,
                     L_min: int = 32, L_max: int = 4096,
                     sweeps_min: int = 100, sweeps_max: int = 10_000):
    """Poisson request stream: arrival times (s), L log-uniform in
    [L_min, L_max], beta uniform in [0.30, 0.60], sweeps uniform integers in
    [sweeps_min, sweeps_max], one random 64-bit seed each."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n)
    arrivals = np.cumsum(gaps) - gaps[0]
    Ls = np.round(np.exp(rng.uniform(np.log(L_min), np.log(L_max), n))).astype(int)
    betas = rng.uniform(0.30, 0.60, n)
    sweeps = rng.integers(sweeps_min, sweeps_max + 1, n)
    seeds = rng.integers(0, 2**63, n, dtype=np.int64).astype(np.uint64)
    return [dict(arrival=float(a), L=int(L), beta=float(b), sweeps=int(k), seed=int(s))
            for a, L, b, k, s in zip(arrivals, Ls, betas, sweeps, seeds)]
