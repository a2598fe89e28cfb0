"""Host logic of the tile-shape autotuner: bucket arithmetic (the library's
ceil(log2 L)), the choice of the fastest shape, and the JSON table round
trip, with a fake timer (no GPU)."""
import json

import paper_2302_14720_gb300 as sw
from paper_2302_14720_gb300 import autotune


def test_bucket_is_ceil_log2():
    assert [autotune.bucket_of(L) for L in (2, 3, 4, 5, 64, 65, 1024, 1025, 8192)] == [1, 2, 2, 3, 6, 7, 10, 11, 13]


def test_choose_fastest_with_ties_to_lower_index():
    assert autotune.choose({0: 2.0, 3: 1.0, 5: 1.0}) == 3
    assert autotune.choose({6: 0.5}) == 6


def test_tune_and_table_round_trip(tmp_path, monkeypatch):
    installed = {}
    monkeypatch.setattr(autotune, "sw_tune_shape", lambda b, s: installed.__setitem__(b, s))
    monkeypatch.setattr(autotune, "sw_shape_info", lambda s: {"shape": s})
    fake = {(1024, 0): 3.0, (1024, 1): 2.0, (8192, 0): 5.0, (8192, 1): 9.0}
    table = autotune.tune([1024, 8192], shapes=[0, 1], timer=lambda L, s: fake[(L, s)])
    assert installed == {10: 1, 13: 0}
    assert table[10]["shape"] == 1 and table[13]["shape"] == 0
    path = tmp_path / "shapes.json"
    autotune.save(table, str(path), device="GB300-test")
    assert json.load(open(path))["GB300-test"]["10"]["shape"] == 1
    installed.clear()
    monkeypatch.setattr(autotune, "sw_num_shapes", lambda: 10)
    got = autotune.load(str(path), device="GB300-test")
    assert installed == {10: 1, 13: 0} and got[13]["L"] == 8192
    assert autotune.load(str(path), device="other") == {}


def test_batch_candidates_offer_the_fused_schedule_only_where_it_exists():
    c = autotune.batch_candidates([6, 0], small=(0, 64))
    assert (6, sw.SW_SCHEDULE_FUSED, 64) in c and (6, sw.SW_SCHEDULE_PHASES, 0) in c
    assert all(sched == sw.SW_SCHEDULE_PHASES for sh, sched, _ in c if sh == 0)   # 4-row strips in 64-row tiles
    assert len(c) == 2 * 2 + 1 * 2


def test_tune_batch_picks_the_fastest_and_skips_refused_candidates():
    fake = {(6, 0, 0): 0.48, (6, 1, 0): 0.61, (6, 0, 64): 0.47, (4, 0, 0): 0.50}

    def timer(sh, sc, sm):
        if (sh, sc, sm) not in fake:
            raise sw.SWError(sw.SW_EINVAL, "sw_batch_set_schedule", "refused")
        return fake[(sh, sc, sm)]
    got = autotune.tune_batch([64], [0.4], [1], candidates=list(fake) + [(0, 1, 0)], timer=timer)
    assert (got["shape"], got["schedule"], got["small_max_L"]) == (6, 0, 64)
    assert got["ms_per_sweep"] == 0.47 and len(got["ms"]) == 4


def test_apply_batch_sets_schedule_and_threshold(monkeypatch):
    calls = []
    monkeypatch.setattr(autotune, "sw_batch_set_schedule", lambda b, s: calls.append(("schedule", b, s)))
    monkeypatch.setattr(autotune, "sw_batch_set_small", lambda b, m: calls.append(("small", b, m)))
    autotune.apply_batch(7, {"shape": 6, "schedule": 1, "small_max_L": 64})
    assert calls == [("schedule", 7, 1), ("small", 7, 64)]
