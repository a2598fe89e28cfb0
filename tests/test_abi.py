"""CPU-side checks of the C ABI: the library builds, loads, exports every
symbol include/sw.h declares, computes the host threshold like the oracle,
validates arguments, and refuses to run without a GPU (no CPU fallback)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(sw_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from conftest import build_libsw
    build_libsw()
    import paper_2302_14720_gb300 as sw
    return sw


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("sw_create", "sw_sweep", "sw_observables", "sw_labels", "sw_threshold", "sw_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIBRARY_PATH)
    for name in declared_functions():
        assert hasattr(so, name), name
    assert set(declared_functions()) == set(lib.SIGNATURES), "binding and header disagree"


def test_threshold_matches_oracle(lib):
    import oracle
    for beta in list(np.linspace(0, 3, 301)) + [0.44068679, 0.5, 30.0, 1e-300]:
        assert lib.sw_threshold(beta) == oracle.threshold(beta)
    assert lib.sw_threshold(-1.0) == 0 and "beta" in lib.sw_last_error()
    assert lib.sw_threshold(float("nan")) == 0


@pytest.mark.parametrize("L,beta,init", [(1, 0.4, 0), (0, 0.4, 0), (46341, 0.4, 0), (-5, 0.4, 0),
                                         (64, -0.1, 0), (64, float("nan"), 0), (64, float("inf"), 0),
                                         (64, 0.4, 2)])
def test_create_rejects_bad_arguments(lib, L, beta, init):
    with pytest.raises(lib.SWError) as ei:
        lib.sw_create(L, beta, 1, init)
    assert ei.value.status == lib.SW_EINVAL


def test_no_cpu_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.SWError) as ei:
        lib.sw_create(64, 0.4, 1, 0)
    assert ei.value.status == lib.SW_ECUDA


def test_async_set_state_checks_its_host_array(lib):
    # the array is read after the call returns, so the binding takes only an
    # int8 C-contiguous numpy array (checked before the library is called)
    for bad in (np.ones((4, 4), np.int32), np.ones((4, 8), np.int8)[:, ::2], [[1, -1], [1, 1]]):
        with pytest.raises(TypeError):
            lib.sw_set_state_async(0, bad, 0)
    # a NULL handle with a valid array is the library's SW_EINVAL
    with pytest.raises(lib.SWError) as ei:
        lib.sw_set_state_async(0, np.ones((4, 4), np.int8), 0)
    assert ei.value.status == lib.SW_EINVAL
