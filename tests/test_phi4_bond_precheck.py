"""The binary32 first test of the phi^4 bond kernel, checked on the CPU.

The bond kernel decides an edge of Eq. 2 first from the projections
rounded to binary32 and expf, and leaves to the binary64 test (the
oracle's rule: w < (1 - e^{-z}) 2^32 with z = 4 kappa a_x a_y and the
pinned exponential) every word within 2^18 of its binary32 threshold,
every projection below 2^-60 and every z within 0.01 of 40. This test
restates that first test in numpy binary32 arithmetic (round to nearest,
as the kernel's intrinsics) with expf taken anywhere within 2 ulp of the
exact value (its documented bound), and checks on random and adversarial
edges -- words right at the binary64 threshold, z near 40, tiny and zero
projections -- that every decision the first test takes equals the
binary64 one.
"""
import numpy as np

import oracle

K4 = 4.0 * 0.304
MARGIN = np.float32(2.0 ** 18)


def exact_bond(ax, ay, w):
    q = ax * ay
    if not q > 0.0:
        return False
    e = oracle.phi4_exp_neg(K4 * q)
    return float(w) < (1.0 - e) * 2.0 ** 32


def first_test(ax, ay, w, ulps):
    """The kernel's binary32 decision, or None where it defers to binary64."""
    fx, fy = np.float32(ax), np.float32(ay)
    mx, my = abs(fx), abs(fy)
    if not (mx >= np.float32(2.0 ** -60) and my >= np.float32(2.0 ** -60)):
        return None
    if np.signbit(fx) != np.signbit(fy):
        return False
    zf = np.float32(np.float32(np.float32(K4) * mx) * my)
    if zf > np.float32(40.01):
        return True
    if not zf < np.float32(39.99):
        return None
    ef = np.float32(np.exp(-np.float64(zf)))      # exp of the binary32 argument, rounded once
    for _ in range(abs(ulps)):                     # then moved by up to 2 ulp, as expf may be
        ef = np.nextafter(ef, np.float32(np.inf if ulps > 0 else 0.0), dtype=np.float32)
    tf = np.float32(np.float32(np.float32(1.0) - ef) * np.float32(2.0 ** 32))
    wf = np.float32(w)
    if wf < tf - MARGIN:
        return True
    if wf > tf + MARGIN:
        return False
    return None


def check(ax, ay, w):
    want = exact_bond(ax, ay, w)
    for ulps in (-2, -1, 0, 1, 2):
        got = first_test(ax, ay, w, ulps)
        assert got is None or got == want, (ax, ay, w, ulps, got, want)


def test_random_edges():
    rng = np.random.default_rng(11)
    n = 4000
    mag = np.exp(rng.uniform(np.log(1e-3), np.log(8.0), size=(n, 2)))
    sgn = rng.choice([-1.0, 1.0], size=(n, 2))
    a = mag * sgn
    w = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64)
    decided = 0
    for (ax, ay), wk in zip(a, w):
        check(float(ax), float(ay), int(wk))
        decided += first_test(float(ax), float(ay), int(wk), 0) is not None
    assert decided >= 0.99 * n  # the binary32 test decides almost every edge


def test_words_at_the_threshold():
    # the adversarial case: words within a few 2^18 of the binary64 threshold
    rng = np.random.default_rng(12)
    n = 3000
    a = np.exp(rng.uniform(np.log(1e-2), np.log(6.0), size=(n, 2)))
    deltas = rng.integers(-(2 ** 20), 2 ** 20, size=n)
    for (ax, ay), d in zip(a, deltas):
        q = ax * ay
        T = (1.0 - oracle.phi4_exp_neg(K4 * q)) * 2.0 ** 32
        w = int(min(max(round(T) + int(d), 0), 2 ** 32 - 1))
        check(float(ax), float(ay), w)
        check(-float(ax), -float(ay), w)


def test_z_near_40_and_tiny_projections():
    rng = np.random.default_rng(13)
    for z in np.concatenate([np.linspace(39.9, 40.1, 401), [40.0, np.nextafter(40.0, 0), np.nextafter(40.0, 50)]]):
        ax = float(rng.uniform(1.0, 6.0))
        ay = float(z / K4 / ax)
        for w in (0, 1, 2 ** 31, 2 ** 32 - 2 ** 18, 2 ** 32 - 1):
            check(ax, ay, w)
    for ax in (0.0, -0.0, 2.0 ** -70, -(2.0 ** -61), 2.0 ** -60, 1e-30):
        for ay in (0.5, -0.5, 3.0, 2.0 ** -65):
            for w in (0, 12345, 2 ** 31, 2 ** 32 - 1):
                check(ax, ay, w)
