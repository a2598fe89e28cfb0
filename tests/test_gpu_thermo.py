"""Temperature scans on the GPU: the scan's chains are the oracle's chains
bit for bit; on a 4x4 torus its estimates agree with the exact Boltzmann
moments; at L=64 the specific heat peaks at the grid point nearest the
critical temperature and the magnetisation follows Onsager-Yang below it."""
import math

import numpy as np
import pytest

import oracle
from exact_ising import exact_moments

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def thermo():
    from conftest import build_libsw
    build_libsw()
    from paper_2302_14720_gb300 import thermo
    return thermo


def test_scan_traces_are_the_oracle_chains(thermo):
    betas = [0.2, 0.44068679, 0.7]
    pts, E, M = thermo.scan(6, betas, n_equil=10, n_meas=40, seeds_per_beta=2, seed0=50, traces=True, n_blocks=4)
    for i, b in enumerate(betas):
        for k in range(2):
            _, want_E, want_M, _ = oracle.run(6, b, 50 + 2 * i + k, 50)
            assert np.array_equal(E[i, k], want_E[10:]) and np.array_equal(M[i, k], want_M[10:])
    assert [p.beta for p in pts] == betas


def test_scan_4x4_matches_exact_moments(thermo):
    betas = [0.25, 0.44068679, 0.65]
    pts = thermo.scan(4, betas, n_equil=200, n_meas=20000, seeds_per_beta=4, n_blocks=20)
    for p in pts:
        ex = exact_moments(4, p.beta)
        assert abs(p.e - ex["E"] / 16) < 5 * p.e_err
        assert abs(p.m - ex["absM"] / 16) < 5 * p.m_err
        assert abs(p.c - p.beta ** 2 * (ex["E2"] - ex["E"] ** 2) / 16) < 5 * p.c_err


def test_scan_L64_specific_heat_peak_and_magnetisation(thermo):
    betas = [0.36, 0.40, 0.44, 0.48, 0.52]
    pts = thermo.scan(64, betas, n_equil=200, n_meas=2000, seeds_per_beta=2, n_blocks=20)
    c = [p.c for p in pts]
    assert int(np.argmax(c)) == 2
    for p in pts[3:]:
        yang = (1 - math.sinh(2 * p.beta) ** -4) ** 0.125
        assert abs(p.m - yang) < 0.02 + 5 * p.m_err
    assert pts[0].m < 0.3
