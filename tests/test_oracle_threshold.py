"""Pin the bond threshold (conventions C2/C3, bond probability of §2.1).

thr must equal floor(2^32 * (1 - exp(-2 beta))) for the exact binary64 value
of beta, capped at 2^32 - 1. The test evaluates that closed form with 60
significant digits (mpmath), independently of the oracle's expm1/ldexp
route. Where the exact product lies within 1e-6 of an integer the binary64
route may round to the neighbour; elsewhere it must agree exactly.
"""
import math

import mpmath
import numpy as np
import pytest

import oracle

mpmath.mp.dps = 60


def exact_thr(beta: float):
    b = mpmath.mpf(beta)  # exact value of the double
    v = mpmath.ldexp(1 - mpmath.exp(-2 * b), 32)
    fl = int(mpmath.floor(v))
    near = abs(v - mpmath.nint(v)) < mpmath.mpf("1e-6")
    return min(fl, 0xFFFFFFFF), near


def test_threshold_grid_exact():
    rng = np.random.default_rng(11)
    betas = list(np.linspace(0.0, 2.0, 401)) + list(rng.uniform(0, 1, 300)) + [
        0.44068679, math.log1p(math.sqrt(2)) / 2, 0.4, 0.5, 0.45, 0.48, 1e-300, 5e-324, 1e-10]
    for beta in betas:
        want, near = exact_thr(float(beta))
        got = oracle.threshold(float(beta))
        if near:
            assert abs(got - want) <= 1
        else:
            assert got == want, beta


def test_threshold_limits():
    assert oracle.threshold(0.0) == 0
    assert oracle.threshold(-0.0) == 0
    # p rounds to 1 in binary64 once exp(-2 beta) < 2^-53; thr saturates.
    assert oracle.threshold(30.0) == 0xFFFFFFFF
    assert oracle.threshold(1e300) == 0xFFFFFFFF
    # Monotone in beta.
    vals = [oracle.threshold(b) for b in np.linspace(0, 5, 2001)]
    assert all(a <= b for a, b in zip(vals, vals[1:]))


@pytest.mark.parametrize("bad", [-1e-12, -1.0, float("nan"), float("inf"), float("-inf")])
def test_threshold_rejects(bad):
    with pytest.raises(ValueError):
        oracle.threshold(bad)


def test_threshold_config_values():
    # Literal beta of the L=64/1024/8192 configurations versus exact beta_c.
    assert oracle.threshold(0.44068679) == exact_thr(0.44068679)[0] == 2515933579
    bc = math.log1p(math.sqrt(2)) / 2
    assert oracle.threshold(bc) == exact_thr(bc)[0] == 2515933592
