"""Temperature scans: energy, specific heat and magnetisation against
temperature (the quantities the paper plots in §4, Results), measured by running one
Swendsen-Wang chain per (temperature, seed) together in one sw_batch.

Per temperature, from the per-sweep traces after `n_equil` sweeps:
  e   = <E> / N                         energy per site (the Hamiltonian that closes §2, J = 1)
  c   = beta^2 (<E^2> - <E>^2) / N      specific heat per site
  m   = <|M|> / N                       magnetisation per site
  chi = beta (<M^2> - <|M|>^2) / N      susceptibility per site
  u4  = 1 - <M^4> / (3 <M^2>^2)         Binder cumulant
with standard errors from batch means (blocks of consecutive sweeps within
each chain, pooled over seeds) and a jackknife over the same blocks for c,
chi and u4. The sweeps run in libsw's kernels; this module launches them
and reduces the int64 traces on the host.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import SW_INIT_HOT, sw_batch_create, sw_batch_destroy, sw_batch_observables, sw_batch_sweep


@dataclasses.dataclass
class Point:
    beta: float
    L: int
    samples: int
    e: float
    e_err: float
    c: float
    c_err: float
    m: float
    m_err: float
    chi: float
    chi_err: float
    u4: float
    u4_err: float

    @property
    def T(self) -> float:
        return 1.0 / self.beta if self.beta > 0 else float("inf")


def _block_means(x: np.ndarray, n_blocks: int) -> np.ndarray:
    """Means of n_blocks equal consecutive blocks along the last axis of
    x[chains, sweeps] (a ragged tail is dropped), flattened over chains."""
    per = x.shape[-1] // n_blocks
    if per < 1:
        raise ValueError("fewer measurement sweeps than blocks")
    return x[..., :per * n_blocks].reshape(*x.shape[:-1], n_blocks, per).mean(axis=-1).reshape(-1)


def point_from_traces(E: np.ndarray, M: np.ndarray, beta: float, L: int, n_blocks: int = 16) -> Point:
    """Estimates at one temperature from E, M traces [chains, sweeps] (int64)."""
    E = np.asarray(E, dtype=np.float64)
    M = np.abs(np.asarray(M, dtype=np.float64))
    if E.ndim == 1:
        E, M = E[None], M[None]
    N = float(L * L)
    moments = np.stack([_block_means(E, n_blocks), _block_means(E * E, n_blocks), _block_means(M, n_blocks),
                        _block_means(M * M, n_blocks), _block_means(M ** 4, n_blocks)])  # [5, B]
    B = moments.shape[1]

    def derived(mo):
        e1, e2, m1, m2, m4 = mo
        return np.array([e1 / N, beta * beta * (e2 - e1 * e1) / N, m1 / N, beta * (m2 - m1 * m1) / N,
                         1.0 - m4 / (3.0 * m2 * m2) if m2 > 0 else 0.0])

    full = derived(moments.mean(axis=1))
    # jackknife over blocks: leave one block out
    tot = moments.sum(axis=1, keepdims=True)
    jk = np.stack([derived(((tot - moments[:, [b]]) / (B - 1))[:, 0]) for b in range(B)])  # [B, 5]
    err = np.sqrt((B - 1) / B * ((jk - jk.mean(axis=0)) ** 2).sum(axis=0))
    return Point(beta=float(beta), L=int(L), samples=int(E.size), e=full[0], e_err=err[0], c=full[1], c_err=err[1],
                 m=full[2], m_err=err[2], chi=full[3], chi_err=err[3], u4=full[4], u4_err=err[4])


def scan(L: int, betas, n_equil: int, n_meas: int, seeds_per_beta: int = 1, seed0: int = 1,
         init: int = SW_INIT_HOT, chunk: int = 100, n_blocks: int = 16, shape: int = -1,
         stream: int | None = None, traces: bool = False):
    """Run len(betas) * seeds_per_beta chains of side L in one batch.

    Chain (i, k) has inverse temperature betas[i] and seed
    seed0 + i * seeds_per_beta + k. Returns a Point per beta (and, with
    traces=True, the raw E, M traces [beta, seed, sweep] as well).
    """
    betas = [float(b) for b in betas]
    nb = len(betas)
    Ls = [L] * (nb * seeds_per_beta)
    bs = [b for b in betas for _ in range(seeds_per_beta)]
    ss = [seed0 + i for i in range(nb * seeds_per_beta)]
    total = n_equil + n_meas
    h = sw_batch_create(Ls, bs, ss, [init] * len(Ls), shape=shape, stream=stream)
    try:
        done = 0
        while done < total:
            n = min(chunk, total - done)
            sw_batch_sweep(h, n)
            done += n
        E = np.zeros((nb, seeds_per_beta, n_meas), np.int64)
        M = np.zeros_like(E)
        for i in range(nb):
            for k in range(seeds_per_beta):
                E[i, k], M[i, k] = sw_batch_observables(h, i * seeds_per_beta + k, n_equil, n_meas)
    finally:
        sw_batch_destroy(h)
    pts = [point_from_traces(E[i], M[i], betas[i], L, n_blocks) for i in range(nb)]
    return (pts, E, M) if traces else pts
