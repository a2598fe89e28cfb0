"""Swendsen-Wang dynamics of the 2D Ising model on one GB300 (sm_103a).

Thin ctypes binding of libsw (include/sw.h). Every function below has the
name of the C entry point it marshals; it converts arguments and statuses
and nothing else -- all sweep arithmetic runs in the library's CUDA kernels.
There is no CPU fallback: importing the binding raises if libsw.so has not
been built (``paper_2302_14720_gb300.build.build()``), and ``sw_create``
fails without a GPU.

Device buffers and streams may come from PyTorch: pass ``tensor.data_ptr()``
with ``*_is_device=True`` and ``torch.cuda.current_stream().cuda_stream`` as
the stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB_PATH

SW_OK = 0
SW_EINVAL = -1
SW_ENOMEM = -2
SW_ECUDA = -3
SW_EDEVICE = -4
SW_ETIMEOUT = -5
SW_INIT_HOT = 0
SW_INIT_COLD = 1
SW_RULE_FLIP = 0
SW_RULE_ASSIGN = 1
SW_SCHEDULE_PHASES = 0
SW_SCHEDULE_FUSED = 1
SW_TIMING_PHASES = 5
SW_HIST_WORDS = 34

_STATUS_NAMES = {SW_EINVAL: "SW_EINVAL", SW_ENOMEM: "SW_ENOMEM", SW_ECUDA: "SW_ECUDA",
                 SW_EDEVICE: "SW_EDEVICE", SW_ETIMEOUT: "SW_ETIMEOUT"}

# Every symbol include/sw.h declares, with its ctypes signature.
_P = ctypes.c_void_p
SIGNATURES = {
    "sw_threshold": (ctypes.c_uint32, [ctypes.c_double]),
    "sw_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, ctypes.c_int32, _P,
                                 ctypes.POINTER(_P)]),
    "sw_destroy": (ctypes.c_int, [_P]),
    "sw_sweep": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sw_get_sweep": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint32)]),
    "sw_observables": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P]),
    "sw_histogram": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sw_set_rule": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sw_histograms": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P]),
    "sw_labels": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "sw_labels_equivalence": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "sw_spins": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "sw_set_state": (ctypes.c_int, [_P, _P, ctypes.c_uint32, ctypes.c_int32]),
    "sw_set_state_async": (ctypes.c_int, [_P, _P, ctypes.c_uint32]),
    "sw_bonds": (ctypes.c_int, [_P, _P]),
    "sw_timing": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sw_timing_read": (ctypes.c_int, [_P, _P, _P]),
    "sw_batch_create": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int32, _P, ctypes.POINTER(_P)]),
    "sw_batch_add": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int32)]),
    "sw_batch_remove": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sw_batch_sweep": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sw_batch_footprint": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "sw_batch_set_rule": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "sw_batch_set_schedule": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sw_batch_set_small": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sw_batch_set_limit": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64]),
    "sw_batch_get_sweep": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint32)]),
    "sw_batch_observables": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _P, _P]),
    "sw_batch_spins": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    "sw_batch_info": (ctypes.c_int, [_P, _P, _P, _P]),
    "sw_batch_destroy": (ctypes.c_int, [_P]),
    "sw_sweep_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_int32, _P, _P, _P]),
    "sw_num_shapes": (ctypes.c_int, []),
    "sw_shape_info": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P]),
    "sw_tune_shape": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32]),
    "sw_lattice_shape": (ctypes.c_int, [ctypes.c_void_p, _P]),
    "sw_last_error": (ctypes.c_char_p, []),
    "sw_potts_threshold": (ctypes.c_uint32, [ctypes.c_double]),
    "sw_potts_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                                       ctypes.c_int32, _P, ctypes.POINTER(_P)]),
    "sw_potts_sweep": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sw_potts_observables": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P]),
    "sw_potts_states": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "sw_potts_set_state": (ctypes.c_int, [_P, _P, ctypes.c_uint32, ctypes.c_int32]),
    "sw_potts_labels": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "sw_potts_get_sweep": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint32)]),
    "sw_potts_destroy": (ctypes.c_int, [_P]),
    "sw_phi4_direction": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, _P]),
    "sw_phi4_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, ctypes.c_int32, _P,
                                      ctypes.POINTER(_P)]),
    "sw_phi4_sweep": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sw_phi4_observables": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P]),
    "sw_phi4_field": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "sw_phi4_set_field": (ctypes.c_int, [_P, _P, ctypes.c_uint32, ctypes.c_int32]),
    "sw_phi4_labels": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "sw_phi4_get_sweep": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint32)]),
    "sw_phi4_destroy": (ctypes.c_int, [_P]),
}
SW_NOALLOC_MAX_L = 1024


class SWError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsw is not built ({LIB_PATH} missing); run paper_2302_14720_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
LIBRARY_PATH = LIB_PATH


def _check(rc: int, where: str) -> None:
    if rc != SW_OK:
        raise SWError(rc, where, _lib.sw_last_error().decode())


def _host_ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------- functions

def sw_threshold(beta: float) -> int:
    return int(_lib.sw_threshold(float(beta)))


def sw_create(L: int, beta: float, seed: int, init: int = SW_INIT_HOT, stream: int | None = None) -> int:
    """stream: a cudaStream_t handle; None lets the library create its own. The
    legacy default stream (handle 0) cannot be passed: it reads as None."""
    h = ctypes.c_void_p()
    _check(_lib.sw_create(int(L), float(beta), int(seed) & 0xFFFFFFFFFFFFFFFF, int(init),
                          ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)), "sw_create")
    return h.value


def sw_destroy(h: int) -> None:
    _check(_lib.sw_destroy(h), "sw_destroy")


def sw_sweep(h: int, n: int) -> None:
    _check(_lib.sw_sweep(h, int(n)), "sw_sweep")


def sw_get_sweep(h: int) -> int:
    t = ctypes.c_uint32()
    _check(_lib.sw_get_sweep(h, ctypes.byref(t)), "sw_get_sweep")
    return t.value


def sw_observables(h: int, first: int, count: int):
    E = np.zeros(max(count, 0), np.int64)
    M = np.zeros(max(count, 0), np.int64)
    _check(_lib.sw_observables(h, int(first), int(count), _host_ptr(E), _host_ptr(M)), "sw_observables")
    return E, M


def sw_histogram(h: int, enable: bool) -> None:
    _check(_lib.sw_histogram(h, 1 if enable else 0), "sw_histogram")


def sw_set_rule(h: int, rule: int) -> None:
    _check(_lib.sw_set_rule(h, int(rule)), "sw_set_rule")


def sw_histograms(h: int, first: int, count: int) -> np.ndarray:
    out = np.zeros((max(count, 0), SW_HIST_WORDS), np.int64)
    _check(_lib.sw_histograms(h, int(first), int(count), _host_ptr(out)), "sw_histograms")
    return out


def sw_labels(h: int, L: int, out_device_ptr: int | None = None):
    """Host int32 [L, L] labels, or write to a device pointer when given."""
    if out_device_ptr is not None:
        _check(_lib.sw_labels(h, ctypes.c_void_p(out_device_ptr), 1), "sw_labels")
        return None
    out = np.zeros((L, L), np.int32)
    _check(_lib.sw_labels(h, _host_ptr(out), 0), "sw_labels")
    return out


def sw_labels_equivalence(h: int, L: int, out=None):
    """Labels by the paper's label-equivalence iteration; returns (labels, iterations).
    With out a device pointer (int), the labels go there and None is returned for them."""
    its = ctypes.c_int32(0)
    if out is None:
        lab = np.zeros((L, L), np.int32)
        _check(_lib.sw_labels_equivalence(h, _host_ptr(lab), 0, ctypes.byref(its)), "sw_labels_equivalence")
        return lab, its.value
    _check(_lib.sw_labels_equivalence(h, ctypes.c_void_p(out), 1, ctypes.byref(its)), "sw_labels_equivalence")
    return None, its.value


def sw_spins(h: int, L: int, out_device_ptr: int | None = None):
    if out_device_ptr is not None:
        _check(_lib.sw_spins(h, ctypes.c_void_p(out_device_ptr), 1), "sw_spins")
        return None
    out = np.zeros((L, L), np.int8)
    _check(_lib.sw_spins(h, _host_ptr(out), 0), "sw_spins")
    return out


def sw_set_state(h: int, spins, t: int, in_device_ptr: bool = False) -> None:
    """spins: int8 numpy array (host) or an integer device pointer with in_device_ptr=True."""
    if in_device_ptr:
        _check(_lib.sw_set_state(h, ctypes.c_void_p(int(spins)), int(t) & 0xFFFFFFFF, 1), "sw_set_state")
        return
    s = np.ascontiguousarray(spins, dtype=np.int8)
    _check(_lib.sw_set_state(h, _host_ptr(s), int(t) & 0xFFFFFFFF, 0), "sw_set_state")


def sw_set_state_async(h: int, spins: np.ndarray, t: int) -> None:
    """spins: C-contiguous int8 host array (pinned for an asynchronous copy); it
    must stay unchanged until the handle's stream has copied it."""
    if not (isinstance(spins, np.ndarray) and spins.dtype == np.int8 and spins.flags["C_CONTIGUOUS"]):
        raise TypeError("sw_set_state_async needs a C-contiguous int8 numpy array (it is read after the call)")
    _check(_lib.sw_set_state_async(h, _host_ptr(spins), int(t) & 0xFFFFFFFF), "sw_set_state_async")


def sw_bonds(h: int, L: int) -> np.ndarray:
    out = np.zeros((L, L), np.uint8)
    _check(_lib.sw_bonds(h, _host_ptr(out)), "sw_bonds")
    return out


def sw_timing(h: int, enable: bool) -> None:
    _check(_lib.sw_timing(h, 1 if enable else 0), "sw_timing")


def sw_timing_read(h: int):
    """(ms per phase float64[5], launches per phase int64[5]) since sw_timing(h, True);
    phase 4 is a sweep's flips together with the next sweep's bonds and tile clusters."""
    ms = np.zeros(SW_TIMING_PHASES, np.float64)
    n = np.zeros(SW_TIMING_PHASES, np.int64)
    _check(_lib.sw_timing_read(h, _host_ptr(ms), _host_ptr(n)), "sw_timing_read")
    return ms, n


def sw_sweep_noalloc(spins_dev: int, L: int, beta: float, seed: int, t0: int, n: int, em_dev: int,
                     err_dev: int, stream: int | None = None) -> None:
    """Allocation-free sweep on caller-owned device buffers (see include/sw.h):
    spins int8 [L][L] updated in place, em int64 [n][2] and err int32 [1]
    outputs, all device pointers; asynchronous on `stream`."""
    _check(_lib.sw_sweep_noalloc(ctypes.c_void_p(spins_dev), int(L), float(beta), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                 int(t0) & 0xFFFFFFFF, int(n), ctypes.c_void_p(em_dev), ctypes.c_void_p(err_dev),
                                 ctypes.c_void_p(stream) if stream else None), "sw_sweep_noalloc")


def sw_num_shapes() -> int:
    return int(_lib.sw_num_shapes())


def sw_shape_info(shape: int) -> dict:
    v = np.zeros(4, np.int32)
    ptrs = [ctypes.c_void_p(v.ctypes.data + 4 * i) for i in range(4)]
    _check(_lib.sw_shape_info(int(shape), *ptrs), "sw_shape_info")
    return dict(tile_w=int(v[0]), tile_h=int(v[1]), strip_h=int(v[2]), threads=int(v[3]))


def sw_tune_shape(log2_bucket: int, shape: int) -> None:
    _check(_lib.sw_tune_shape(int(log2_bucket), int(shape)), "sw_tune_shape")


def sw_lattice_shape(h: int) -> int:
    v = np.zeros(1, np.int32)
    _check(_lib.sw_lattice_shape(h, _host_ptr(v)), "sw_lattice_shape")
    return int(v[0])


def sw_last_error() -> str:
    return _lib.sw_last_error().decode()


# ------------------------------------------------------------------ batch

def sw_batch_create(L, beta, seed, init=None, shape: int = -1, stream: int | None = None) -> int:
    n = len(L)
    Ls = np.ascontiguousarray(L, dtype=np.int32)
    bs = np.ascontiguousarray(beta, dtype=np.float64)
    ss = np.ascontiguousarray(np.asarray(seed, dtype=np.uint64))
    ins = None if init is None else np.ascontiguousarray(init, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(_lib.sw_batch_create(n, _host_ptr(Ls) if n else None, _host_ptr(bs) if n else None,
                                _host_ptr(ss) if n else None, _host_ptr(ins) if ins is not None and n else None,
                                int(shape), ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)),
           "sw_batch_create")
    return h.value


def sw_batch_add(b: int, L: int, beta: float, seed: int, init: int = SW_INIT_HOT) -> int:
    slot = ctypes.c_int32()
    _check(_lib.sw_batch_add(b, int(L), float(beta), int(seed) & 0xFFFFFFFFFFFFFFFF, int(init), ctypes.byref(slot)),
           "sw_batch_add")
    return slot.value


def sw_batch_remove(b: int, slot: int) -> None:
    _check(_lib.sw_batch_remove(b, int(slot)), "sw_batch_remove")


def sw_batch_sweep(b: int, n: int) -> None:
    _check(_lib.sw_batch_sweep(b, int(n)), "sw_batch_sweep")


def sw_batch_set_rule(b: int, slot: int, rule: int) -> None:
    _check(_lib.sw_batch_set_rule(b, int(slot), int(rule)), "sw_batch_set_rule")


def sw_batch_set_schedule(b: int, schedule: int) -> None:
    _check(_lib.sw_batch_set_schedule(b, int(schedule)), "sw_batch_set_schedule")


def sw_batch_set_small(b: int, max_L: int) -> None:
    _check(_lib.sw_batch_set_small(b, int(max_L)), "sw_batch_set_small")


def sw_batch_set_limit(b: int, slot: int, sweeps_left: int) -> None:
    _check(_lib.sw_batch_set_limit(b, int(slot), int(sweeps_left)), "sw_batch_set_limit")


def sw_batch_get_sweep(b: int, slot: int) -> int:
    t = ctypes.c_uint32()
    _check(_lib.sw_batch_get_sweep(b, int(slot), ctypes.byref(t)), "sw_batch_get_sweep")
    return t.value


def sw_batch_observables(b: int, slot: int, first: int, count: int):
    E = np.zeros(max(count, 0), np.int64)
    M = np.zeros(max(count, 0), np.int64)
    _check(_lib.sw_batch_observables(b, int(slot), int(first), int(count), _host_ptr(E), _host_ptr(M)),
           "sw_batch_observables")
    return E, M


def sw_batch_spins(b: int, slot: int, L: int) -> np.ndarray:
    out = np.zeros((L, L), np.int8)
    _check(_lib.sw_batch_spins(b, int(slot), _host_ptr(out), 0), "sw_batch_spins")
    return out


def sw_batch_info(b: int):
    n = np.zeros(1, np.int32)
    sites = np.zeros(1, np.int64)
    nbytes = np.zeros(1, np.int64)
    _check(_lib.sw_batch_info(b, _host_ptr(n), _host_ptr(sites), _host_ptr(nbytes)), "sw_batch_info")
    return int(n[0]), int(sites[0]), int(nbytes[0])


def sw_batch_footprint(b: int, L: int, sweeps: int) -> int:
    out = ctypes.c_int64(0)
    _check(_lib.sw_batch_footprint(b, int(L), int(sweeps), ctypes.byref(out)), "sw_batch_footprint")
    return out.value


def sw_batch_destroy(b: int) -> None:
    _check(_lib.sw_batch_destroy(b), "sw_batch_destroy")


# ------------------------------------------------------------ convenience

class Lattice:
    """Owning wrapper of one sw_lattice handle."""

    def __init__(self, L: int, beta: float, seed: int, init: int = SW_INIT_HOT, stream: int | None = None):
        self.L = int(L)
        self.beta = float(beta)
        self.seed = int(seed)
        self.h = sw_create(L, beta, seed, init, stream)

    def sweep(self, n: int = 1) -> None:
        sw_sweep(self.h, n)

    @property
    def t(self) -> int:
        return sw_get_sweep(self.h)

    def observables(self, first: int, count: int):
        return sw_observables(self.h, first, count)

    def histograms(self, first: int, count: int) -> np.ndarray:
        return sw_histograms(self.h, first, count)

    def histogram(self, enable: bool) -> None:
        sw_histogram(self.h, enable)

    def set_rule(self, rule: int) -> None:
        sw_set_rule(self.h, rule)

    def spins(self) -> np.ndarray:
        return sw_spins(self.h, self.L)

    def labels(self) -> np.ndarray:
        return sw_labels(self.h, self.L)

    def labels_equivalence(self):
        return sw_labels_equivalence(self.h, self.L)

    def bonds(self) -> np.ndarray:
        return sw_bonds(self.h, self.L)

    def set_state(self, spins, t: int) -> None:
        sw_set_state(self.h, spins, t)

    def set_state_async(self, spins: np.ndarray, t: int) -> None:
        sw_set_state_async(self.h, spins, t)

    def close(self) -> None:
        if self.h:
            sw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------ q-state Potts

def sw_potts_threshold(beta: float) -> int:
    return int(_lib.sw_potts_threshold(float(beta)))


class Potts:
    """Owning wrapper of one sw_potts handle (q-state Potts, states 0..q-1)."""

    def __init__(self, L: int, q: int, beta: float, seed: int, init: int = SW_INIT_HOT, stream: int | None = None):
        self.L, self.q = int(L), int(q)
        h = ctypes.c_void_p()
        _check(_lib.sw_potts_create(int(L), int(q), float(beta), int(seed) & 0xFFFFFFFFFFFFFFFF, int(init),
                                    ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)), "sw_potts_create")
        self.h = h.value

    def sweep(self, n: int = 1) -> None:
        _check(_lib.sw_potts_sweep(self.h, int(n)), "sw_potts_sweep")

    @property
    def t(self) -> int:
        t = ctypes.c_uint32()
        _check(_lib.sw_potts_get_sweep(self.h, ctypes.byref(t)), "sw_potts_get_sweep")
        return t.value

    def observables(self, first: int, count: int):
        E = np.zeros(max(count, 0), np.int64)
        M = np.zeros(max(count, 0), np.int64)
        _check(_lib.sw_potts_observables(self.h, int(first), int(count), _host_ptr(E), _host_ptr(M)),
               "sw_potts_observables")
        return E, M

    def states(self) -> np.ndarray:
        out = np.zeros((self.L, self.L), np.int8)
        _check(_lib.sw_potts_states(self.h, _host_ptr(out), 0), "sw_potts_states")
        return out

    def set_state(self, states, t: int) -> None:
        a = np.ascontiguousarray(states, dtype=np.int8)
        assert a.shape == (self.L, self.L)
        _check(_lib.sw_potts_set_state(self.h, _host_ptr(a), int(t) & 0xFFFFFFFF, 0), "sw_potts_set_state")

    def labels(self) -> np.ndarray:
        out = np.zeros((self.L, self.L), np.int32)
        _check(_lib.sw_potts_labels(self.h, _host_ptr(out), 0), "sw_potts_labels")
        return out

    def close(self) -> None:
        if self.h:
            _lib.sw_potts_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# --------------------------------------------------- O(4) phi^4 multicluster

def sw_phi4_direction(seed: int, t: int) -> np.ndarray:
    r = np.zeros(4)
    _check(_lib.sw_phi4_direction(int(seed) & 0xFFFFFFFFFFFFFFFF, int(t) & 0xFFFFFFFF, _host_ptr(r)),
           "sw_phi4_direction")
    return r


class Phi4:
    """Owning wrapper of one sw_phi4 handle (field double [L, L, L, L, 4])."""

    def __init__(self, L: int, kappa: float, seed: int, init: int = SW_INIT_HOT, stream: int | None = None):
        self.L = int(L)
        h = ctypes.c_void_p()
        _check(_lib.sw_phi4_create(int(L), float(kappa), int(seed) & 0xFFFFFFFFFFFFFFFF, int(init),
                                   ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)), "sw_phi4_create")
        self.h = h.value

    def sweep(self, n: int = 1) -> None:
        _check(_lib.sw_phi4_sweep(self.h, int(n)), "sw_phi4_sweep")

    @property
    def t(self) -> int:
        t = ctypes.c_uint32()
        _check(_lib.sw_phi4_get_sweep(self.h, ctypes.byref(t)), "sw_phi4_get_sweep")
        return t.value

    def observables(self, first: int, count: int):
        E = np.zeros(max(count, 0))
        M = np.zeros((max(count, 0), 4))
        _check(_lib.sw_phi4_observables(self.h, int(first), int(count), _host_ptr(E), _host_ptr(M)),
               "sw_phi4_observables")
        return E, M

    def field(self) -> np.ndarray:
        L = self.L
        out = np.zeros((L, L, L, L, 4))
        _check(_lib.sw_phi4_field(self.h, _host_ptr(out), 0), "sw_phi4_field")
        return out

    def set_field(self, phi, t: int) -> None:
        a = np.ascontiguousarray(phi, dtype=np.float64)
        assert a.shape == (self.L,) * 4 + (4,)
        _check(_lib.sw_phi4_set_field(self.h, _host_ptr(a), int(t) & 0xFFFFFFFF, 0), "sw_phi4_set_field")

    def labels(self) -> np.ndarray:
        out = np.zeros((self.L,) * 4, np.int32)
        _check(_lib.sw_phi4_labels(self.h, _host_ptr(out), 0), "sw_phi4_labels")
        return out

    def close(self) -> None:
        if self.h:
            _lib.sw_phi4_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
