"""Serial CPU oracle for Swendsen-Wang dynamics of the 2D Ising model.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark load this package; the library in ``paper_2302_14720_gb300``
never does, and the two share no code. The C source ``sw_oracle.c`` states one
sweep exactly in the order of the paper's §2 (bonds §2.1, clusters §2.3 by
breadth-first search, new spins §2.4, then E and M); this module compiles it
with the host C compiler and wraps it with ctypes and numpy.

Every function cites the passage it follows in the C source. Parity status of
each function (what pins it, in tests/test_oracle_*.py):
  philox      -- cuRAND's host Philox-4x32-10 generator (library pin)
  threshold   -- closed form in exact arithmetic, limits beta=0 and beta->inf
  init        -- statistics of a fair coin, cold start all +1
  bonds       -- only between equal spins; frequency p = thr/2^32 (binomial)
  labels      -- scipy.sparse.csgraph.connected_components and a union-find
                 written differently in the test; canonical-min invariants
  flip        -- clusters stay monochrome; spin-reversal symmetry
  assign      -- clusters end monochrome; the result ignores the old spins;
                 equals a flip by the old-vs-new difference; exact 2x2
                 transition matrix and 4x4 moments of the assign chain
  observe     -- closed forms of ordered, checkerboard and striped states
  histogram   -- against cluster sizes from scipy's labelling
  potts_*     -- q = 2 equals the Ising assignment chain at twice beta (state 1
                 <-> spin -1, E and M mapped); exact 2x2 q = 3 transition
                 matrix (detailed balance); 3x3 q = 3 exact moments
  run         -- exact 2x2 transition matrix (detailed balance), 3x3 state
                 histogram vs Boltzmann, 4x4 exact moments, Kaufman's exact
                 finite-torus energy, Onsager-Yang magnetisation
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sw_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "phi4_oracle.c")]
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

HIST_WORDS = 34


def build(force: bool = False) -> str:
    """Compile sw_oracle.c into _build/liboracle.so (plain C, -O2)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    # ISO C mode: no floating-point contraction beyond the explicit fma calls
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.oracle_philox.argtypes = [P, P, P]
        lib.oracle_philox.restype = None
        lib.oracle_threshold.argtypes = [ctypes.c_double]
        lib.oracle_threshold.restype = ctypes.c_uint32
        lib.oracle_init.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, P]
        lib.oracle_init.restype = None
        lib.oracle_bonds.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, P, P]
        lib.oracle_bonds.restype = None
        lib.oracle_labels.argtypes = [ctypes.c_int, P, P, P]
        lib.oracle_labels.restype = ctypes.c_int64
        lib.oracle_flip.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, P, P]
        lib.oracle_flip.restype = None
        lib.oracle_apply_flips.argtypes = [ctypes.c_int, P, P, P]
        lib.oracle_apply_flips.restype = None
        lib.oracle_assign.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, P, P]
        lib.oracle_assign.restype = None
        lib.oracle_apply_assign.argtypes = [ctypes.c_int, P, P, P]
        lib.oracle_apply_assign.restype = None
        lib.oracle_observe.argtypes = [ctypes.c_int, P, P, P]
        lib.oracle_observe.restype = None
        lib.oracle_histogram.argtypes = [ctypes.c_int, P, P, P]
        lib.oracle_histogram.restype = None
        lib.oracle_run.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_int, P, P, P, P, ctypes.c_int]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_potts_threshold.argtypes = [ctypes.c_double]
        lib.oracle_potts_threshold.restype = ctypes.c_uint32
        lib.oracle_potts_init.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, P]
        lib.oracle_potts_init.restype = None
        lib.oracle_potts_assign.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, P, P]
        lib.oracle_potts_assign.restype = None
        lib.oracle_potts_apply.argtypes = [ctypes.c_int, P, P, P]
        lib.oracle_potts_apply.restype = None
        lib.oracle_potts_observe.argtypes = [ctypes.c_int, P, P, P]
        lib.oracle_potts_observe.restype = None
        lib.oracle_potts_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_uint32, ctypes.c_int, P, P, P]
        lib.oracle_potts_run.restype = ctypes.c_int
        D = ctypes.c_double
        lib.phi4_exp_neg.argtypes = [D]
        lib.phi4_exp_neg.restype = D
        lib.phi4_direction.argtypes = [ctypes.c_uint64, ctypes.c_uint32, P]
        lib.phi4_direction.restype = ctypes.c_int
        lib.phi4_init.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, P]
        lib.phi4_init.restype = None
        lib.phi4_bonds.argtypes = [ctypes.c_int, D, ctypes.c_uint64, ctypes.c_uint32, P, P, P]
        lib.phi4_bonds.restype = None
        lib.phi4_labels.argtypes = [ctypes.c_int, P, P, P]
        lib.phi4_labels.restype = ctypes.c_int64
        lib.phi4_reflect.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, P, P, P]
        lib.phi4_reflect.restype = None
        lib.phi4_observe.argtypes = [ctypes.c_int, P, P, P]
        lib.phi4_observe.restype = None
        lib.phi4_run.argtypes = [ctypes.c_int, D, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, P, P, P]
        lib.phi4_run.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _check_L(L: int):
    if not (2 <= L and L * L < 2**31):
        raise ValueError(f"L={L} outside 2 <= L, L*L < 2^31")


def philox(ctr, key) -> np.ndarray:
    """Philox-4x32-10 block for counter ctr[4] and key key[2] (uint32 words)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def threshold(beta: float) -> int:
    """Bond threshold floor(2^32 (1 - exp(-2 beta))) capped at 2^32-1 (§2.1)."""
    b = float(beta)
    if not (b >= 0.0) or np.isinf(b):
        raise ValueError("beta must be finite and >= 0")
    return int(_load().oracle_threshold(b))


def init(L: int, seed: int, cold: bool = False) -> np.ndarray:
    """Initial spins int8 [L, L]: hot start from Philox (Fig. 1) or all +1."""
    _check_L(L)
    s = np.zeros((L, L), dtype=np.int8)
    _load().oracle_init(L, seed, 1 if cold else 0, _ptr(s))
    return s


def bonds(spins: np.ndarray, seed: int, t: int, thr: int) -> np.ndarray:
    """Bonds of sweep t from spins (§2.1): uint8 [L, L], bit0 east, bit1 south."""
    s = np.ascontiguousarray(spins, dtype=np.int8)
    L = s.shape[0]
    out = np.zeros((L, L), dtype=np.uint8)
    _load().oracle_bonds(L, seed, t & 0xffffffff, thr, _ptr(s), _ptr(out))
    return out


def labels(bond_bits: np.ndarray):
    """Canonical cluster labels (§2.3) by BFS: (int32 [L, L], n_clusters)."""
    b = np.ascontiguousarray(bond_bits, dtype=np.uint8)
    L = b.shape[0]
    lab = np.zeros((L, L), dtype=np.int32)
    queue = np.zeros(L * L, dtype=np.int32)
    n = _load().oracle_labels(L, _ptr(b), _ptr(lab), _ptr(queue))
    return lab, int(n)


def flip(spins: np.ndarray, lab: np.ndarray, seed: int, t: int) -> np.ndarray:
    """New spins (§2.4): cluster rooted at r flips iff bit r % 32 of word
    (r // 32) % 4 of Philox block (r // 128, t, 1, 0) is set."""
    s = np.array(spins, dtype=np.int8, copy=True, order="C")
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    _load().oracle_flip(s.shape[0], seed, t & 0xffffffff, _ptr(lab), _ptr(s))
    return s


def apply_flips(spins: np.ndarray, lab: np.ndarray, flip_of_root: np.ndarray) -> np.ndarray:
    """New spins with an explicit 0/1 flip decision stored at each root."""
    s = np.array(spins, dtype=np.int8, copy=True, order="C")
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    f = np.ascontiguousarray(flip_of_root, dtype=np.uint8).reshape(-1)
    _load().oracle_apply_flips(s.shape[0], _ptr(lab), _ptr(f), _ptr(s))
    return s


def assign(spins_shape_L: int, lab: np.ndarray, seed: int, t: int) -> np.ndarray:
    """New spins by §2.4's assignment: cluster rooted at r gets -1 iff
    Philox (r,t,3,0).x0 >> 31, whatever its old spin."""
    L = int(spins_shape_L)
    s = np.zeros((L, L), dtype=np.int8)
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    _load().oracle_assign(L, seed, t & 0xffffffff, _ptr(lab), _ptr(s))
    return s


def apply_assign(L: int, lab: np.ndarray, minus_of_root: np.ndarray) -> np.ndarray:
    """New spins with an explicit 0/1 (1 = -1) value stored at each root."""
    s = np.zeros((L, L), dtype=np.int8)
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    m = np.ascontiguousarray(minus_of_root, dtype=np.uint8).reshape(-1)
    _load().oracle_apply_assign(L, _ptr(lab), _ptr(m), _ptr(s))
    return s


def observe(spins: np.ndarray):
    """(E, M) of a state: E over the 2N edges, M = sum of spins (end of §2)."""
    s = np.ascontiguousarray(spins, dtype=np.int8)
    E = np.zeros(1, dtype=np.int64)
    M = np.zeros(1, dtype=np.int64)
    _load().oracle_observe(s.shape[0], _ptr(s), _ptr(E), _ptr(M))
    return int(E[0]), int(M[0])


def histogram(lab: np.ndarray) -> np.ndarray:
    """Cluster statistics of a labelling: [n_clusters, sum |C|^2, 32 log2 bins]."""
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    L = lab.shape[0]
    hist = np.zeros(HIST_WORDS, dtype=np.int64)
    count = np.zeros(L * L, dtype=np.int64)
    _load().oracle_histogram(L, _ptr(lab), _ptr(hist), _ptr(count))
    return hist


RULES = {"flip": 0, "assign": 1}


def run(L: int, beta: float, seed: int, n: int, *, spins: np.ndarray | None = None,
        cold: bool = False, t0: int = 0, hist: bool = False, rule: str = "flip"):
    """Run n sweeps (counters t0..t0+n-1) from spins (or the C7 start);
    rule "flip" (C6) or "assign" (§2.4 as printed).

    Returns (final spins int8 [L, L], E int64 [n], M int64 [n], hist int64
    [n, 34] or None).
    """
    _check_L(L)
    thr_check = float(beta)
    if not (thr_check >= 0.0) or np.isinf(thr_check):
        raise ValueError("beta must be finite and >= 0")
    s = init(L, seed, cold) if spins is None else np.array(spins, dtype=np.int8, copy=True, order="C")
    assert s.shape == (L, L)
    E = np.zeros(max(n, 1), dtype=np.int64)
    M = np.zeros(max(n, 1), dtype=np.int64)
    H = np.zeros((max(n, 1), HIST_WORDS), dtype=np.int64) if hist else None
    rc = _load().oracle_run(L, float(beta), seed, t0 & 0xffffffff, n, _ptr(s), _ptr(E), _ptr(M),
                            _ptr(H) if hist else None, RULES[rule])
    if rc != 0:
        raise MemoryError("oracle_run: allocation failed")
    return s, E[:n], M[:n], (H[:n] if hist else None)


# ------------------------------------------------------------ q-state Potts
# §6's generalisation: H = -sum over edges of delta(s_i, s_j), states
# 0..q-1 (int8); bonds between equal states with p = 1 - exp(-beta) (the
# Ising bond draws C5 otherwise); each cluster assigned a state uniform in q
# from word x0 of block (root, t, 3, 0) as floor(x0 q / 2^32).

def _check_q(q: int):
    if not (2 <= q <= 127):
        raise ValueError("q must be in 2..127")


def potts_threshold(beta: float) -> int:
    return int(_load().oracle_potts_threshold(float(beta)))


def potts_init(L: int, q: int, seed: int, cold: bool = False) -> np.ndarray:
    _check_L(L)
    _check_q(q)
    s = np.zeros((L, L), dtype=np.int8)
    _load().oracle_potts_init(L, q, seed, 1 if cold else 0, _ptr(s))
    return s


def potts_assign(L: int, q: int, lab: np.ndarray, seed: int, t: int) -> np.ndarray:
    s = np.zeros((L, L), dtype=np.int8)
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    _load().oracle_potts_assign(L, q, seed, t & 0xffffffff, _ptr(lab), _ptr(s))
    return s


def potts_apply(L: int, lab: np.ndarray, state_of_root: np.ndarray) -> np.ndarray:
    s = np.zeros((L, L), dtype=np.int8)
    lab = np.ascontiguousarray(lab, dtype=np.int32)
    v = np.ascontiguousarray(state_of_root, dtype=np.uint8).reshape(-1)
    _load().oracle_potts_apply(L, _ptr(lab), _ptr(v), _ptr(s))
    return s


def potts_observe(states: np.ndarray):
    """(E, M): E = -(edges joining equal states), M = sites in state 0."""
    s = np.ascontiguousarray(states, dtype=np.int8)
    E = np.zeros(1, dtype=np.int64)
    M = np.zeros(1, dtype=np.int64)
    _load().oracle_potts_observe(s.shape[0], _ptr(s), _ptr(E), _ptr(M))
    return int(E[0]), int(M[0])


def potts_run(L: int, q: int, beta: float, seed: int, n: int, *, states: np.ndarray | None = None,
              cold: bool = False, t0: int = 0):
    """n Potts sweeps; returns (final states int8 [L, L], E int64 [n], M int64 [n])."""
    _check_L(L)
    _check_q(q)
    if not (float(beta) >= 0.0) or np.isinf(beta):
        raise ValueError("beta must be finite and >= 0")
    s = potts_init(L, q, seed, cold) if states is None else np.array(states, dtype=np.int8, copy=True, order="C")
    E = np.zeros(max(n, 1), dtype=np.int64)
    M = np.zeros(max(n, 1), dtype=np.int64)
    if _load().oracle_potts_run(L, q, float(beta), seed, t0 & 0xffffffff, n, _ptr(s), _ptr(E), _ptr(M)) != 0:
        raise MemoryError("oracle_potts_run: allocation failed")
    return s, E[:n], M[:n]


# ------------------------------------------------- O(4) phi^4 multicluster
# §3's update (Eqs. 2 and 3) on an L^4 torus; see phi4_oracle.c (O1-O5).

def phi4_exp_neg(z: float) -> float:
    return float(_load().phi4_exp_neg(float(z)))


def phi4_direction(seed: int, t: int) -> np.ndarray:
    r = np.zeros(4)
    if _load().phi4_direction(seed, t & 0xffffffff, _ptr(r)) != 0:
        raise RuntimeError("phi4_direction: no direction found")
    return r


def phi4_init(L: int, seed: int, cold: bool = False) -> np.ndarray:
    phi = np.zeros((L, L, L, L, 4))
    _load().phi4_init(L, seed, 1 if cold else 0, _ptr(phi))
    return phi


def phi4_bonds(phi: np.ndarray, kappa: float, seed: int, t: int, r: np.ndarray) -> np.ndarray:
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    L = phi.shape[0]
    b = np.zeros((L, L, L, L), np.uint8)
    _load().phi4_bonds(L, float(kappa), seed, t & 0xffffffff, _ptr(phi), _ptr(np.ascontiguousarray(r, np.float64)),
                       _ptr(b))
    return b


def phi4_labels(bonds: np.ndarray):
    b = np.ascontiguousarray(bonds, dtype=np.uint8)
    L = b.shape[0]
    lab = np.zeros(b.shape, np.int32)
    queue = np.zeros(b.size, np.int32)
    n = _load().phi4_labels(L, _ptr(b), _ptr(lab), _ptr(queue))
    return lab, int(n)


def phi4_reflect(phi: np.ndarray, lab: np.ndarray, seed: int, t: int, r: np.ndarray) -> np.ndarray:
    out = np.array(phi, dtype=np.float64, copy=True, order="C")
    L = out.shape[0]
    _load().phi4_reflect(L, seed, t & 0xffffffff, _ptr(np.ascontiguousarray(lab, np.int32)),
                         _ptr(np.ascontiguousarray(r, np.float64)), _ptr(out))
    return out


def phi4_observe(phi: np.ndarray):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    E = np.zeros(1)
    M = np.zeros(4)
    _load().phi4_observe(phi.shape[0], _ptr(phi), _ptr(E), _ptr(M))
    return float(E[0]), M


def phi4_run(L: int, kappa: float, seed: int, n: int, *, phi: np.ndarray | None = None, cold: bool = False,
             t0: int = 0):
    """n multicluster updates; returns (field [L,L,L,L,4], E [n], M [n,4])."""
    if not (2 <= L and L**4 < 2**31):
        raise ValueError("L outside 2 <= L, L^4 < 2^31")
    f = phi4_init(L, seed, cold) if phi is None else np.array(phi, dtype=np.float64, copy=True, order="C")
    E = np.zeros(max(n, 1))
    M = np.zeros((max(n, 1), 4))
    rc = _load().phi4_run(L, float(kappa), seed, t0 & 0xffffffff, n, _ptr(f), _ptr(E), _ptr(M))
    if rc != 0:
        raise RuntimeError(f"phi4_run failed ({rc})")
    return f, E[:n], M[:n]
