"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

All results are integer, so every comparison is exact: spins, bonds, labels,
E, M and cluster statistics must be bit-identical. Both sides start from the
same seeded input -- the C7 hot/cold start that each computes itself, or a
spin array drawn by workloads.random_spins and handed to both -- and the
oracle never consumes anything the GPU produced.

Sizes span one tile to several tiles with ragged right and bottom tiles,
odd L (Philox pairs straddle rows), L = 2 (double edges) and the three
compiled tile shapes; the full-size cases run the bench's configuration
(L = 8192, default tile shape) on one sweep from a generated state.
"""
import os

import numpy as np
import pytest

import oracle
from workloads import random_spins, striped_spins

pytestmark = pytest.mark.gpu

BETA_C = 0.44068679
SHAPES = [0, 2, 6, 8]  # 4-row strips, 64-wide tiles, the default 128x64, 256x32 tiles
SMALL_L = [2, 3, 5, 17, 31, 32, 33, 64, 65, 100, 127, 128, 129, 191, 257]


@pytest.fixture(scope="module")
def sw():
    from conftest import build_libsw
    build_libsw()
    import paper_2302_14720_gb300 as sw
    return sw


def make(sw, L, beta, seed, init=0, shape=None):
    if shape is not None:
        os.environ["SW_TILE_SHAPE"] = str(shape)
    try:
        return sw.Lattice(L, beta, seed, init)
    finally:
        os.environ.pop("SW_TILE_SHAPE", None)


# ------------------------------------------------------------- init (C7)

@pytest.mark.parametrize("L", [2, 3, 17, 64, 130, 257, 1000])
@pytest.mark.parametrize("init", [0, 1])
def test_init_parity(sw, L, init):
    with make(sw, L, 0.4, 12345 + L, init) as lat:
        assert np.array_equal(lat.spins(), oracle.init(L, 12345 + L, cold=bool(init)))


# ------------------------------------------------ bonds and labels (§2.1, §2.3)

@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("L", SMALL_L)
def test_bonds_and_labels_parity(sw, shape, L):
    seed, t = 0xC0FFEE + L, 11
    for beta_i, beta in enumerate([0.0, 0.3, BETA_C, 0.6, 5.0]):
        with make(sw, L, beta, seed, shape=shape) as lat:
            for k, s in enumerate([random_spins(L, seed=L * 7 + beta_i),
                                   random_spins(L, seed=L * 7 + beta_i, p_minus=0.04),
                                   striped_spins(L, 3)]):
                lat.set_state(s, t + k)
                b = lat.bonds()
                want_b = oracle.bonds(s, seed, t + k, oracle.threshold(beta))
                assert np.array_equal(b, want_b), (shape, L, beta, k)
                want_lab, _ = oracle.labels(want_b)
                assert np.array_equal(lat.labels(), want_lab), (shape, L, beta, k)
                # the queries leave the state alone
                assert np.array_equal(lat.spins(), s)


# -------------------------------------------------------- chains (§2, C8)

@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("L", [2, 3, 17, 64, 129, 257])
@pytest.mark.parametrize("beta", [0.3, BETA_C, 0.6])
def test_chain_parity(sw, shape, L, beta):
    seed, n = 1000 + L, 8
    with make(sw, L, beta, seed, shape=shape) as lat:
        lat.sweep(n)
        E, M = lat.observables(0, n)
        spins = lat.spins()
    want_s, want_E, want_M, _ = oracle.run(L, beta, seed, n)
    assert np.array_equal(E, want_E) and np.array_equal(M, want_M)
    assert np.array_equal(spins, want_s)


def test_config_L64_every_sweep(sw):
    # L=64, beta_c, hot start seed 1, 1000 sweeps: state and E/M after every sweep.
    L, beta, seed, n = 64, BETA_C, 1, 1000
    s_or = oracle.init(L, seed)
    with make(sw, L, beta, seed) as lat:
        for k in range(n):
            lat.sweep(1)
            s_or, e1, m1, _ = oracle.run(L, beta, seed, 1, spins=s_or, t0=k)
            assert np.array_equal(lat.spins(), s_or), k
        E, M = lat.observables(0, n)
    _, want_E, want_M, _ = oracle.run(L, beta, seed, n)
    assert np.array_equal(E, want_E) and np.array_equal(M, want_M)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("L", [5, 33, 130, 257])
def test_histogram_parity_small(sw, shape, L):
    seed, n = 77 + L, 6
    for beta in (0.2, BETA_C, 0.7):
        with make(sw, L, beta, seed, shape=shape) as lat:
            lat.histogram(True)
            lat.sweep(n)
            H = lat.histograms(0, n)
        _, _, _, want_H = oracle.run(L, beta, seed, n, hist=True)
        assert np.array_equal(H, want_H), (shape, L, beta)


def test_config_L1024_cold_histogram(sw):
    # L=1024, beta_c, cold start, seed 2: E, M and cluster statistics of each
    # of the first 1000 sweeps (the oracle needs about a minute).
    L, beta, seed, n = 1024, BETA_C, 2, 1000
    with make(sw, L, beta, seed, init=1) as lat:
        lat.histogram(True)
        lat.sweep(n)
        E, M = lat.observables(0, n)
        H = lat.histograms(0, n)
        spins = lat.spins()
    want_s, want_E, want_M, want_H = oracle.run(L, beta, seed, n, cold=True, hist=True)
    assert np.array_equal(E, want_E) and np.array_equal(M, want_M)
    assert np.array_equal(H, want_H)
    assert np.array_equal(spins, want_s)


def test_histogram_toggle_rows(sw):
    L, seed = 40, 5
    with make(sw, L, BETA_C, seed) as lat:
        lat.sweep(2)
        lat.histogram(True)
        lat.sweep(2)
        lat.histogram(False)
        lat.sweep(1)
        H = lat.histograms(0, 5)
    _, _, _, want_H = oracle.run(L, BETA_C, seed, 5, hist=True)
    assert (H[:2] == 0).all() and (H[4] == 0).all()
    assert np.array_equal(H[2:4], want_H[2:4])


# --------------------------------------------- full size, bench configuration

@pytest.mark.parametrize("beta,p_minus", [(BETA_C, 0.5), (0.50, 0.03)])
def test_full_size_spot_sweep(sw, beta, p_minus):
    L, seed, t = 8192, 3, 1000
    s = random_spins(L, seed=2024, p_minus=p_minus)
    with make(sw, L, beta, seed) as lat:
        lat.set_state(s, t)
        lab = lat.labels()
        lat.sweep(1)
        E, M = lat.observables(t, 1)
        spins = lat.spins()
    thr = oracle.threshold(beta)
    want_lab, _ = oracle.labels(oracle.bonds(s, seed, t, thr))
    assert np.array_equal(lab, want_lab)
    del want_lab, lab
    want_s, want_E, want_M, _ = oracle.run(L, beta, seed, 1, spins=s, t0=t)
    assert np.array_equal(spins, want_s)
    assert E[0] == want_E[0] and M[0] == want_M[0]


def test_maximum_size_sweep(sw):
    """The largest lattice the ABI accepts (L*L < 2^31): 2.1 G sites, tiles
    4 columns wide on the right and 4 rows high at the bottom, site keys
    near 2^31. Both sides take the C7 hot start themselves; one sweep's
    spins, E and M must agree exactly (the oracle needs about two minutes)."""
    L, seed = 46340, 11
    assert L * L < 2**31 <= (L + 1) * (L + 1)
    with make(sw, L, BETA_C, seed) as lat:
        lat.sweep(1)
        E, M = lat.observables(0, 1)
        spins = lat.spins()
    want_s, want_E, want_M, _ = oracle.run(L, BETA_C, seed, 1)
    assert E[0] == want_E[0] and M[0] == want_M[0]
    assert np.array_equal(spins, want_s)


# ---------------------------------------------------------------- invariants

def test_sweep_composition(sw):
    L, seed = 97, 31
    with make(sw, L, BETA_C, seed) as a, make(sw, L, BETA_C, seed) as b:
        a.sweep(3)
        a.sweep(4)
        b.sweep(7)
        assert np.array_equal(a.spins(), b.spins())
        assert all(np.array_equal(x, y) for x, y in zip(a.observables(0, 7), b.observables(0, 7)))
        assert a.t == b.t == 7


def test_spin_reversal(sw):
    L, seed = 150, 8
    s = random_spins(L, seed=1)
    with make(sw, L, BETA_C, seed) as a, make(sw, L, BETA_C, seed) as b:
        a.set_state(s, 0)
        b.set_state(-s, 0)
        a.sweep(5)
        b.sweep(5)
        assert np.array_equal(a.spins(), -b.spins())


def test_deterministic_under_atomics(sw):
    L, seed = 1024, 4
    outs = []
    for _ in range(3):
        with make(sw, L, 0.5, seed) as lat:
            lat.sweep(5)
            outs.append((lat.spins(), lat.labels()))
    for s, lab in outs[1:]:
        assert np.array_equal(s, outs[0][0]) and np.array_equal(lab, outs[0][1])


def test_resume_equals_uninterrupted(sw):
    L, seed = 200, 17
    with make(sw, L, BETA_C, seed) as a:
        a.sweep(10)
        ref = a.spins()
        E_ref, M_ref = a.observables(0, 10)
    with make(sw, L, BETA_C, seed) as b:
        b.sweep(4)
        ckpt, t = b.spins(), b.t
    with make(sw, L, BETA_C, seed) as c:
        c.set_state(ckpt, t)
        c.sweep(6)
        assert np.array_equal(c.spins(), ref)
        E, M = c.observables(4, 6)
        assert np.array_equal(E, E_ref[4:]) and np.array_equal(M, M_ref[4:])


# --------------------------------------------------------- device pointers

def test_device_pointer_paths(sw):
    import torch
    L, seed = 130, 3
    s = random_spins(L, seed=9)
    d_in = torch.from_numpy(s).cuda()
    d_spins = torch.empty((L, L), dtype=torch.int8, device="cuda")
    d_lab = torch.empty((L, L), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    lat = sw.Lattice(L, BETA_C, seed, 0, stream=stream)
    try:
        sw.sw_set_state(lat.h, d_in.data_ptr(), 5, in_device_ptr=True)
        sw.sw_labels(lat.h, L, out_device_ptr=d_lab.data_ptr())
        lat.sweep(1)
        sw.sw_spins(lat.h, L, out_device_ptr=d_spins.data_ptr())
        torch.cuda.synchronize()
        want_lab, _ = oracle.labels(oracle.bonds(s, seed, 5, oracle.threshold(BETA_C)))
        assert np.array_equal(d_lab.cpu().numpy(), want_lab)
        want_s, _, _, _ = oracle.run(L, BETA_C, seed, 1, spins=s, t0=5)
        assert np.array_equal(d_spins.cpu().numpy(), want_s)
    finally:
        lat.close()


# ------------------------------------------------------------------ errors

def test_error_statuses(sw):
    L = 16
    with make(sw, L, 0.4, 1) as lat:
        lat.sweep(2)
        with pytest.raises(sw.SWError) as ei:
            lat.observables(0, 3)
        assert ei.value.status == sw.SW_EINVAL
        with pytest.raises(sw.SWError) as ei:
            sw.sw_sweep(lat.h, -1)
        assert ei.value.status == sw.SW_EINVAL
        bad = np.ones((L, L), np.int8)
        bad[3, 4] = 0
        with pytest.raises(sw.SWError) as ei:
            lat.set_state(bad, 0)
        assert ei.value.status == sw.SW_EINVAL
        # the failed call left the state untouched
        assert lat.t == 2
        import torch
        dbad = torch.from_numpy(bad).cuda()
        sw.sw_set_state(lat.h, dbad.data_ptr(), 0, in_device_ptr=True)
        with pytest.raises(sw.SWError) as ei:
            lat.spins()
        assert ei.value.status == sw.SW_EINVAL
        # a valid state clears the flag
        lat.set_state(np.ones((L, L), np.int8), 0)
        lat.sweep(1)
        lat.observables(0, 1)


@pytest.mark.parametrize("L", [16, 17, 33, 1000])
@pytest.mark.parametrize("where", ["first", "middle", "last"])
@pytest.mark.parametrize("value", [0, 2, -2, 127, -128])
def test_set_state_rejects_every_invalid_spin(sw, L, where, value):
    # the check reads 16 bytes at a time with a byte-wise tail: a bad value
    # in the first byte, inside a vector, and in the last byte (the tail
    # when L*L is not a multiple of 16) must all be caught
    s = np.ones((L, L), np.int8)
    s[::3] = -1
    idx = {"first": 0, "middle": (L * L) // 2 + 5, "last": L * L - 1}[where]
    s.reshape(-1)[idx] = value
    with make(sw, L, 0.4, 1) as lat:
        lat.sweep(1)
        with pytest.raises(sw.SWError) as ei:
            lat.set_state(s, 0)
        assert ei.value.status == sw.SW_EINVAL
        assert lat.t == 1


def test_default_tile_shapes(sw):
    # built-in defaults (no tuning installed, SW_TILE_SHAPE unset): a lone
    # lattice takes 128x32 tiles up to L = 1024 and 128x64 above; a batch
    # keeps 128x64 (results never depend on the shape; the parity tests
    # above run every shape)
    assert "SW_TILE_SHAPE" not in os.environ
    for L, want in ((200, 7), (1024, 7), (1025, 6), (4096, 6)):
        with sw.Lattice(L, BETA_C, 1, sw.SW_INIT_HOT) as lat:
            got = sw.sw_lattice_shape(lat.h)
        assert got == want, (L, got)
        assert sw.sw_shape_info(got)["tile_w"] == 128
