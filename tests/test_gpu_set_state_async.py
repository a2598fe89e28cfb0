"""sw_set_state_async: host-input state replacement queued on the handle's
stream. The chain it starts is the chain sw_set_state starts (and the
oracle's); an invalid input is reported by the next synchronising call and
leaves the previous spins in place."""
import numpy as np
import pytest

import oracle
from workloads import random_spins

pytestmark = pytest.mark.gpu
BETA_C = 0.44068679


@pytest.fixture(scope="module")
def sw():
    from conftest import build_libsw
    build_libsw()
    import paper_2302_14720_gb300 as sw
    return sw


@pytest.mark.parametrize("L", [64, 300])
def test_async_state_starts_the_same_chain(sw, L):
    seed, t0, n = 21, 40, 5
    s0 = random_spins(L, seed=5, p_minus=0.4)
    with sw.Lattice(L, BETA_C, seed) as a, sw.Lattice(L, BETA_C, seed) as b:
        a.sweep(3)
        b.sweep(2)
        a.set_state_async(s0, t0)
        b.set_state(s0, t0)
        a.sweep(n)
        b.sweep(n)
        assert a.t == b.t == t0 + n
        Ea, Ma = a.observables(t0, n)
        sa = a.spins()
        assert np.array_equal(sa, b.spins())
        Eb, Mb = b.observables(t0, n)
        assert np.array_equal(Ea, Eb) and np.array_equal(Ma, Mb)
    want_s, want_E, want_M, _ = oracle.run(L, BETA_C, seed, n, spins=s0, t0=t0)
    assert np.array_equal(sa, want_s)
    assert np.array_equal(Ea, want_E) and np.array_equal(Ma, want_M)


def test_async_state_rejects_an_invalid_value_and_keeps_the_spins(sw):
    import torch
    L, seed = 64, 3
    with sw.Lattice(L, 0.5, seed) as lat:
        lat.sweep(2)
        before = lat.spins()
        bad = np.ones((L, L), np.int8)
        bad[5, 7] = 3
        lat.set_state_async(bad, 0)
        out = torch.empty((L, L), dtype=torch.int8, device="cuda")
        sw.sw_spins(lat.h, L, out.data_ptr())   # device copy: queued, no error check
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), before)
        with pytest.raises(sw.SWError) as ei:
            lat.spins()
        assert ei.value.status == sw.SW_EINVAL
        # a valid state clears the error and the lattice runs on
        good = random_spins(L, seed=9)
        lat.set_state_async(good, 7)
        lat.sweep(2)
        want_s, _, _, _ = oracle.run(L, 0.5, seed, 2, spins=good, t0=7)
        assert np.array_equal(lat.spins(), want_s)


def test_a_pending_bad_state_survives_a_second_async_call(sw):
    """An invalid state queued first and a valid one queued right after: the
    second call must not wipe the first one's error, so the next synchronising
    call still reports SW_EINVAL; the valid state is then in place."""
    L, seed = 64, 4
    with sw.Lattice(L, 0.45, seed) as lat:
        lat.sweep(1)
        bad = np.ones((L, L), np.int8)
        bad[0, 0] = 0
        good = random_spins(L, seed=11)
        lat.set_state_async(bad, 3)
        lat.set_state_async(good, 5)
        with pytest.raises(sw.SWError) as ei:
            lat.spins()
        assert ei.value.status == sw.SW_EINVAL
        assert np.array_equal(lat.spins(), good)   # reported once; the valid state stands
        lat.sweep(2)
        want_s, want_E, want_M, _ = oracle.run(L, 0.45, seed, 2, spins=good, t0=5)
        E, M = lat.observables(5, 2)
        assert np.array_equal(lat.spins(), want_s)
        assert np.array_equal(E, want_E) and np.array_equal(M, want_M)


def test_async_state_needs_an_int8_array(sw):
    with sw.Lattice(16, 0.4, 1) as lat:
        with pytest.raises(TypeError):
            lat.set_state_async(np.ones((16, 16), np.int32), 0)
