"""sw_sweep_noalloc: the allocation-free sweep, called through the C ABI.

This entry point serves callers that cannot allocate device memory (a host
framework whose allocator already owns the GPU's memory, a plugin host that
forbids device allocation, a latency-critical loop that cannot take
cudaMalloc's device-wide synchronisation). It must give exactly what the
handle-based sw_sweep gives -- results are integer, so the comparison is
bit-exact -- on two calls in a row, since every call reuses the same
file-scope device scratch array. This file is named so that pytest collects
it last.
"""
import numpy as np
import pytest

from workloads import random_spins

pytestmark = pytest.mark.gpu

BETA_C = 0.44068679


@pytest.fixture(scope="module")
def sw():
    from conftest import build_libsw
    build_libsw()
    import paper_2302_14720_gb300 as sw
    return sw


@pytest.mark.parametrize("L,beta", [(5, 0.6), (130, BETA_C), (181, 0.41), (1000, 0.5), (1024, BETA_C)])
def test_noalloc_matches_sw_sweep_on_two_calls(sw, L, beta):
    import torch
    seed, t0, n = 4242 + L, 17, 4
    s0 = random_spins(L, seed=L, p_minus=0.3)
    stream = torch.cuda.Stream()
    spins = torch.from_numpy(s0).cuda()
    em = torch.zeros((2, n, 2), dtype=torch.int64, device="cuda")
    err = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    got = []
    for call in range(2):
        sw.sw_sweep_noalloc(spins.data_ptr(), L, beta, seed, t0 + call * n, n, em[call].data_ptr(),
                            err[call:call + 1].data_ptr(), stream.cuda_stream)
        stream.synchronize()
        got.append(spins.cpu().numpy().copy())
    assert err.cpu().tolist() == [0, 0]
    em_h = em.cpu().numpy()

    with sw.Lattice(L, beta, seed) as lat:
        lat.set_state(s0, t0)
        for call in range(2):
            lat.sweep(n)
            assert np.array_equal(got[call], lat.spins()), call
            E, M = lat.observables(t0 + call * n, n)
            assert np.array_equal(em_h[call, :, 0], E) and np.array_equal(em_h[call, :, 1], M), call


def test_noalloc_rejects_bad_arguments(sw):
    import torch
    spins = torch.ones((8, 8), dtype=torch.int8, device="cuda")
    em = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for L, beta, n in [(sw.SW_NOALLOC_MAX_L + 1, 0.4, 1), (1, 0.4, 1), (8, -1.0, 1), (8, 0.4, -1)]:
        with pytest.raises(sw.SWError) as ei:
            sw.sw_sweep_noalloc(spins.data_ptr(), L, beta, 1, 0, n, em.data_ptr(), err.data_ptr())
        assert ei.value.status == sw.SW_EINVAL
    assert "1024" in sw.sw_last_error() or "n must" in sw.sw_last_error() or "beta" in sw.sw_last_error()
    with pytest.raises(sw.SWError) as ei:
        sw.sw_sweep_noalloc(0, 8, 0.4, 1, 0, 1, em.data_ptr(), err.data_ptr())
    assert ei.value.status == sw.SW_EINVAL
