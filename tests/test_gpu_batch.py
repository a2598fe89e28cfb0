"""Batched form (sw_batch_*): every replica of a batch must follow exactly
the chain it follows alone -- same spins, E and M, bit for bit -- whatever
the other replicas are, across graph re-captures, and while replicas join
and leave between sweep calls (continuous batching)."""
import numpy as np
import pytest

import oracle
from workloads import batch_replicas

pytestmark = pytest.mark.gpu

BETA_C = 0.44068679


@pytest.fixture(scope="module")
def sw():
    from conftest import build_libsw
    build_libsw()
    import paper_2302_14720_gb300 as sw
    return sw


def oracle_chain(L, beta, seed, n, cold=False):
    s, E, M, _ = oracle.run(L, beta, seed, n, cold=cold)
    return s, E, M


@pytest.mark.parametrize("shape", [-1, 0, 6])
def test_mixed_batch_matches_oracle(sw, shape):
    reps = [(2, 0.3, 11, 0), (5, 0.6, 12, 1), (17, BETA_C, 13, 0), (64, 0.2, 14, 0),
            (100, BETA_C, 15, 1), (128, 0.5, 16, 0), (257, 0.45, 17, 0), (64, BETA_C, 18, 0)]
    L, beta, seed, init = (list(x) for x in zip(*reps))
    b = sw.sw_batch_create(L, beta, seed, init, shape=shape)
    try:
        sw.sw_batch_sweep(b, 3)
        sw.sw_batch_sweep(b, 4)   # a different n: the graph is captured again
        sw.sw_batch_sweep(b, 3)   # same n as before: replay
        for slot, (Lr, br, sr, ir) in enumerate(reps):
            want_s, want_E, want_M = oracle_chain(Lr, br, sr, 10, cold=bool(ir))
            assert sw.sw_batch_get_sweep(b, slot) == 10
            assert np.array_equal(sw.sw_batch_spins(b, slot, Lr), want_s), slot
            E, M = sw.sw_batch_observables(b, slot, 0, 10)
            assert np.array_equal(E, want_E) and np.array_equal(M, want_M), slot
    finally:
        sw.sw_batch_destroy(b)


def test_continuous_batching_join_and_leave(sw):
    b = sw.sw_batch_create([33, 64, 80], [0.4, BETA_C, 0.55], [1, 2, 3])
    try:
        sw.sw_batch_sweep(b, 5)
        s3 = sw.sw_batch_add(b, 48, 0.35, 4)
        s4 = sw.sw_batch_add(b, 130, BETA_C, 5, sw.SW_INIT_COLD)
        sw.sw_batch_sweep(b, 4)
        sw.sw_batch_remove(b, 1)
        sw.sw_batch_sweep(b, 3)
        s5 = sw.sw_batch_add(b, 20, 0.8, 6)      # reuses the freed slot
        assert s5 == 1
        sw.sw_batch_sweep(b, 2)
        n_active, sites, nbytes = sw.sw_batch_info(b)
        assert n_active == 5 and sites == 33 * 33 + 80 * 80 + 48 * 48 + 130 * 130 + 20 * 20 and nbytes > sites
        expect = {0: (33, 0.4, 1, 14, False), 2: (80, 0.55, 3, 14, False), s3: (48, 0.35, 4, 9, False),
                  s4: (130, BETA_C, 5, 9, True), s5: (20, 0.8, 6, 2, False)}
        for slot, (L, beta, seed, n, cold) in expect.items():
            want_s, want_E, want_M = oracle_chain(L, beta, seed, n, cold)
            assert sw.sw_batch_get_sweep(b, slot) == n
            assert np.array_equal(sw.sw_batch_spins(b, slot, L), want_s), slot
            E, M = sw.sw_batch_observables(b, slot, 0, n)
            assert np.array_equal(E, want_E) and np.array_equal(M, want_M), slot
        with pytest.raises(sw.SWError):
            sw.sw_batch_spins(b, 7, 10)
    finally:
        sw.sw_batch_destroy(b)


def test_batch_equals_solo_lattices_config_mix(sw):
    # The 256-replica mix (L in {64..1024}, beta grid in [0.40, 0.48]); every
    # replica is compared with the same replica run alone with sw_sweep.
    L, beta, seed = batch_replicas()
    b = sw.sw_batch_create(L, beta, seed)
    try:
        sw.sw_batch_sweep(b, 4)
        for slot in range(256):
            with sw.Lattice(L[slot], beta[slot], seed[slot]) as lat:
                lat.sweep(4)
                assert np.array_equal(sw.sw_batch_spins(b, slot, L[slot]), lat.spins()), slot
                Eb, Mb = sw.sw_batch_observables(b, slot, 0, 4)
                E, M = lat.observables(0, 4)
                assert np.array_equal(Eb, E) and np.array_equal(Mb, M), slot
    finally:
        sw.sw_batch_destroy(b)


def test_empty_batch_and_errors(sw):
    b = sw.sw_batch_create([], [], [])
    try:
        sw.sw_batch_sweep(b, 3)
        assert sw.sw_batch_info(b)[0] == 0
        with pytest.raises(sw.SWError) as ei:
            sw.sw_batch_add(b, 1, 0.4, 1)
        assert ei.value.status == sw.SW_EINVAL
        with pytest.raises(sw.SWError):
            sw.sw_batch_remove(b, 0)
    finally:
        sw.sw_batch_destroy(b)


def test_sweep_limit_stops_each_replica_at_its_target(sw):
    # Three replicas with targets 3, 7 and unlimited advance in chunks of 4:
    # each stops exactly at its target, its chain equal to the oracle's,
    # while the others go on; lifting a limit resumes the same chain.
    reps = [(40, 0.5, 21, 3), (64, BETA_C, 22, 7), (33, 0.3, 23, None)]
    b = sw.sw_batch_create([r[0] for r in reps], [r[1] for r in reps], [r[2] for r in reps])
    try:
        for slot, (_, _, _, target) in enumerate(reps):
            if target is not None:
                sw.sw_batch_set_limit(b, slot, target)
        sw.sw_batch_sweep(b, 4)
        sw.sw_batch_sweep(b, 4)
        for slot, (L, beta, seed, target) in enumerate(reps):
            n = 8 if target is None else target
            assert sw.sw_batch_get_sweep(b, slot) == n
            want_s, want_E, want_M = oracle_chain(L, beta, seed, n)
            assert np.array_equal(sw.sw_batch_spins(b, slot, L), want_s), slot
            E, M = sw.sw_batch_observables(b, slot, 0, n)
            assert np.array_equal(E, want_E) and np.array_equal(M, want_M), slot
        sw.sw_batch_set_limit(b, 0, -1)
        sw.sw_batch_sweep(b, 4)
        assert [sw.sw_batch_get_sweep(b, s) for s in range(3)] == [7, 7, 12]
        want_s, want_E, _ = oracle_chain(40, 0.5, 21, 7)
        assert np.array_equal(sw.sw_batch_spins(b, 0, 40), want_s)
        assert np.array_equal(sw.sw_batch_observables(b, 0, 0, 7)[0], want_E)
    finally:
        sw.sw_batch_destroy(b)


def test_autotune_installs_a_measured_shape(sw):
    from paper_2302_14720_gb300 import autotune
    table = autotune.tune([300], shapes=[2, 6])
    b = autotune.bucket_of(300)
    assert table[b]["shape"] in (2, 6) and all(v > 0 for v in table[b]["ms"].values())
    # results do not depend on the shape chosen
    with sw.Lattice(300, 0.44, 5) as lat:
        lat.sweep(3)
        want_s, want_E, _, _ = oracle.run(300, 0.44, 5, 3)
        assert np.array_equal(lat.spins(), want_s)
    sw.sw_tune_shape(b, -1)


# ------------------------------------------------- fused schedule (one launch per chunk)

@pytest.mark.parametrize("shape", [6, 4])
def test_fused_schedule_matches_oracle(sw, shape):
    """The persistent cooperative launch runs every sweep of a chunk; each
    replica still follows its own chain bit for bit (ragged tiles, cold and
    hot starts, both rules), across graph re-captures and limits."""
    reps = [(2, 0.3, 11, 0), (5, 0.6, 12, 1), (17, BETA_C, 13, 0), (64, 0.2, 14, 0),
            (100, BETA_C, 15, 1), (128, 0.5, 16, 0), (257, 0.45, 17, 0), (300, BETA_C, 18, 0)]
    L, beta, seed, init = (list(x) for x in zip(*reps))
    b = sw.sw_batch_create(L, beta, seed, init, shape=shape)
    try:
        sw.sw_batch_set_schedule(b, sw.SW_SCHEDULE_FUSED)
        sw.sw_batch_set_limit(b, 3, 6)            # replica 3 stops after 6 sweeps
        sw.sw_batch_sweep(b, 3)
        sw.sw_batch_sweep(b, 4)                   # another n: captured again
        sw.sw_batch_sweep(b, 3)                   # replayed
        for slot, (Lr, br, sr, ir) in enumerate(reps):
            n = 6 if slot == 3 else 10
            want_s, want_E, want_M = oracle_chain(Lr, br, sr, n, cold=bool(ir))
            assert sw.sw_batch_get_sweep(b, slot) == n
            assert np.array_equal(sw.sw_batch_spins(b, slot, Lr), want_s), slot
            E, M = sw.sw_batch_observables(b, slot, 0, n)
            assert np.array_equal(E, want_E) and np.array_equal(M, want_M), slot
    finally:
        sw.sw_batch_destroy(b)


def test_fused_schedule_joins_leaves_and_switches(sw):
    """Replicas join and leave between fused chunks, the assignment rule runs
    beside the flip rule, and switching schedules mid-chain changes nothing."""
    b = sw.sw_batch_create([33, 64, 80], [0.4, BETA_C, 0.55], [1, 2, 3], shape=6)
    try:
        sw.sw_batch_set_schedule(b, sw.SW_SCHEDULE_FUSED)
        sw.sw_batch_set_rule(b, 2, sw.SW_RULE_ASSIGN)
        sw.sw_batch_sweep(b, 5)
        s3 = sw.sw_batch_add(b, 140, BETA_C, 4)
        sw.sw_batch_sweep(b, 4)
        sw.sw_batch_set_schedule(b, sw.SW_SCHEDULE_PHASES)
        sw.sw_batch_remove(b, 1)
        sw.sw_batch_sweep(b, 3)
        sw.sw_batch_set_schedule(b, sw.SW_SCHEDULE_FUSED)
        sw.sw_batch_sweep(b, 2)
        expect = {0: (33, 0.4, 1, 14, "flip"), 2: (80, 0.55, 3, 14, "assign"), s3: (140, BETA_C, 4, 9, "flip")}
        for slot, (Lr, br, sr, n, rule) in expect.items():
            want_s, want_E, want_M, _ = oracle.run(Lr, br, sr, n, rule=rule)
            assert sw.sw_batch_get_sweep(b, slot) == n
            assert np.array_equal(sw.sw_batch_spins(b, slot, Lr), want_s), slot
            E, M = sw.sw_batch_observables(b, slot, 0, n)
            assert np.array_equal(E, want_E) and np.array_equal(M, want_M), slot
    finally:
        sw.sw_batch_destroy(b)


def test_fused_schedule_on_the_replica_mix(sw):
    """The 256-replica mix under the fused schedule equals the per-phase
    schedule replica by replica (spins and whole traces)."""
    L, beta, seed = batch_replicas()
    out = []
    for sched in (sw.SW_SCHEDULE_PHASES, sw.SW_SCHEDULE_FUSED):
        b = sw.sw_batch_create(L, beta, seed)
        try:
            sw.sw_batch_set_schedule(b, sched)
            sw.sw_batch_sweep(b, 6)
            sw.sw_batch_sweep(b, 6)
            out.append([(sw.sw_batch_spins(b, r, int(L[r])), *sw.sw_batch_observables(b, r, 0, 12))
                        for r in range(len(L))])
        finally:
            sw.sw_batch_destroy(b)
    for r, (a, f) in enumerate(zip(*out)):
        assert all(np.array_equal(x, y) for x, y in zip(a, f)), r


def test_fused_schedule_needs_a_matching_shape(sw):
    b = sw.sw_batch_create([64], [0.4], [1], shape=0)   # 4-row strips in 64-row tiles
    try:
        with pytest.raises(sw.SWError) as ei:
            sw.sw_batch_set_schedule(b, sw.SW_SCHEDULE_FUSED)
        assert ei.value.status == sw.SW_EINVAL
        with pytest.raises(sw.SWError):
            sw.sw_batch_set_schedule(b, 7)
    finally:
        sw.sw_batch_destroy(b)


# ------------------------------------------- small replicas on the one-CTA path

@pytest.mark.parametrize("schedule", [0, 1])
def test_small_replicas_on_the_one_cta_path(sw, schedule):
    """Replicas up to the threshold run whole chunks in one CTA each, beside
    tiled replicas; every chain stays the oracle's (limits, both rules,
    cold and hot starts, ragged sides, a threshold change mid-run)."""
    reps = [(2, 0.3, 21, 0), (17, BETA_C, 22, 1), (64, 0.2, 23, 0), (100, BETA_C, 24, 0),
            (181, 0.45, 25, 0), (182, BETA_C, 26, 0), (300, 0.5, 27, 1)]
    L, beta, seed, init = (list(x) for x in zip(*reps))
    b = sw.sw_batch_create(L, beta, seed, init, shape=6)
    try:
        sw.sw_batch_set_schedule(b, schedule)
        sw.sw_batch_set_small(b, 181)
        sw.sw_batch_set_rule(b, 3, sw.SW_RULE_ASSIGN)
        sw.sw_batch_set_limit(b, 1, 5)
        sw.sw_batch_sweep(b, 4)
        sw.sw_batch_sweep(b, 3)
        sw.sw_batch_set_small(b, 64)             # 100 and 181 move back to the tiles
        sw.sw_batch_sweep(b, 3)
        for slot, (Lr, br, sr, ir) in enumerate(reps):
            n = 5 if slot == 1 else 10
            rule = "assign" if slot == 3 else "flip"
            want_s, want_E, want_M, _ = oracle.run(Lr, br, sr, n, cold=bool(ir), rule=rule)
            assert sw.sw_batch_get_sweep(b, slot) == n
            assert np.array_equal(sw.sw_batch_spins(b, slot, Lr), want_s), slot
            E, M = sw.sw_batch_observables(b, slot, 0, n)
            assert np.array_equal(E, want_E) and np.array_equal(M, want_M), slot
        with pytest.raises(sw.SWError):
            sw.sw_batch_set_small(b, 182)
    finally:
        sw.sw_batch_destroy(b)


def test_only_small_replicas(sw):
    b = sw.sw_batch_create([16, 40], [BETA_C, 0.5], [31, 32], shape=6)
    try:
        sw.sw_batch_set_small(b, 64)
        sw.sw_batch_sweep(b, 7)
        for slot, (Lr, br, sr) in enumerate([(16, BETA_C, 31), (40, 0.5, 32)]):
            want_s, want_E, want_M = oracle_chain(Lr, br, sr, 7)
            assert np.array_equal(sw.sw_batch_spins(b, slot, Lr), want_s)
            E, M = sw.sw_batch_observables(b, slot, 0, 7)
            assert np.array_equal(E, want_E) and np.array_equal(M, want_M)
    finally:
        sw.sw_batch_destroy(b)
