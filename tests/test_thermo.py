"""Estimators of the temperature scan (host reductions of E/M traces):
closed forms on constructed traces, and the oracle's chains on a 4x4 torus
against the exact Boltzmann moments."""
import numpy as np
import pytest

import oracle
from exact_ising import exact_moments
from paper_2302_14720_gb300.thermo import point_from_traces


def test_constant_traces():
    E = np.full((2, 64), -20, np.int64)
    M = np.full((2, 64), -7, np.int64)
    p = point_from_traces(E, M, beta=0.5, L=4, n_blocks=8)
    assert p.e == -20 / 16 and p.c == 0 and p.m == 7 / 16 and p.chi == 0
    assert p.u4 == pytest.approx(2 / 3)
    assert p.e_err == 0 and p.m_err == 0


def test_two_level_traces():
    # E alternates -a, +a: <E> = 0, var = a^2 -> c = beta^2 a^2 / N.
    # |M| alternates 2, 4: <|M|> = 3, <M^2> = 10, <M^4> = 136.
    a, beta, L = 6, 0.3, 3
    E = np.tile([-a, a], 32)[None]
    M = np.tile([2, -4], 32)[None]
    p = point_from_traces(E, M, beta, L, n_blocks=4)
    assert p.e == 0 and p.c == pytest.approx(beta * beta * a * a / 9)
    assert p.m == pytest.approx(3 / 9) and p.chi == pytest.approx(beta * (10 - 9) / 9)
    assert p.u4 == pytest.approx(1 - 136 / 300)


def test_error_bars_of_independent_samples():
    rng = np.random.default_rng(0)
    E = rng.normal(-100.0, 5.0, (4, 4096)).round().astype(np.int64)
    M = rng.normal(0, 3.0, (4, 4096)).round().astype(np.int64)
    p = point_from_traces(E, M, beta=1.0, L=10, n_blocks=32)
    want = 5.0 / np.sqrt(E.size) / 100
    assert 0.6 * want < p.e_err < 1.5 * want


@pytest.mark.parametrize("beta", [0.3, 0.44068679, 0.6])
def test_oracle_chain_estimates_match_exact_4x4(beta):
    ex = exact_moments(4, beta)
    chains = [oracle.run(4, beta, 100 + k, 6000)[1:3] for k in range(3)]
    E = np.stack([c[0][500:] for c in chains])
    M = np.stack([c[1][500:] for c in chains])
    p = point_from_traces(E, M, beta, 4, n_blocks=20)
    c_exact = beta * beta * (ex["E2"] - ex["E"] ** 2) / 16
    assert abs(p.e - ex["E"] / 16) < 5 * p.e_err + 1e-12
    assert abs(p.m - ex["absM"] / 16) < 5 * p.m_err + 1e-12
    assert abs(p.c - c_exact) < 5 * p.c_err + 1e-12
