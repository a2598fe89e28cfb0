"""Host-side helpers of bench.py, on the CPU: the code-only source hash that
keys the committed counter record, and the clock sampler's reading of
nvidia-smi lines (fed from a file; no GPU and no nvidia-smi needed)."""
import json
import os

import bench


def test_code_only_ignores_comments_and_layout():
    a = "int f(int x) {  // twice\n  return 2 * x; /* doubled */\n}\n"
    b = "/* header */\nint f(int x) {\n    return 2 * x;\n}"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(a.replace("2 * x", "3 * x"))


def test_source_hash_follows_code_only(tmp_path):
    for f in bench.TILED_SOURCES:
        (tmp_path / f).write_text("int v = 1; // note\n")
    h0 = bench.sw_source_hash(str(tmp_path))
    (tmp_path / bench.TILED_SOURCES[0]).write_text("int v = 1; /* another note */\n")
    assert bench.sw_source_hash(str(tmp_path)) == h0
    (tmp_path / bench.TILED_SOURCES[0]).write_text("int v = 2;\n")
    assert bench.sw_source_hash(str(tmp_path)) != h0


def test_counter_record_is_consistent():
    # traffic = read + write of one launch; the hash has the form bench.py writes
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "dram_traffic_L8192.json")))
    assert rec["bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    assert len(rec["source_hash"]) == 16 and int(rec["source_hash"], 16) >= 0
    assert rec["kernel"] in bench.PHASE_NAMES.values()


def _sampler_from(lines, window):
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    import tempfile
    fd, s.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    s.fh = open(os.devnull, "w")

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s.proc = _Done()
    s.window = window
    return s


def test_clock_sampler_keeps_samples_inside_the_window():
    t = bench.ClockSampler._epoch
    lines = ["2026/12/03 10:00:00.000, 0, 1200, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "2026/12/03 10:00:00.050, 0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Active",
             "2026/12/03 10:00:00.100, 0, 2055, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "2026/12/03 10:00:00.150, 0, 1100, 2070, 200.0, 0x4, Not Active, Active, Not Active, Not Active"]
    w = (t("2026/12/03 10:00:00.040"), t("2026/12/03 10:00:00.120"))
    out = _sampler_from(lines, w).stop()
    assert out["samples_in_timed_region"] == 2 and out["samples"] == 2
    assert out["sm_mhz"] == (2070.0 + 2055.0) / 2 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]          # the thermal sample lies outside


def test_clock_sampler_falls_back_to_all_samples():
    lines = ["2026/12/03 10:00:00.000, 0, 2070, 2070, 800.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage line",
             "2026/12/03 10:00:00.050, 0, 2060, 2070, 810.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    out = _sampler_from(lines, (0.0, 1.0)).stop()
    assert out["samples_in_timed_region"] == 0 and out["samples"] == 2
    assert out["sm_mhz"] == 2065.0 and out["reasons"] == []


def test_cpu_model_names_the_host():
    m = bench.cpu_model()
    assert str(os.cpu_count()) in m and "cores" in m


def test_oracle_replica_share_counts_its_site_updates():
    # one process's share of the replica mix: n sweeps of each of its replicas
    sites, dt = bench._oracle_replicas(([(16, 0.44, 1000), (8, 0.40, 1001)], 2))
    assert sites == 2 * (16 * 16 + 8 * 8) and dt >= 0.0


def test_phase_byte_models_cover_every_sweep_kernel():
    for p in (0, 1, 2):
        assert bench.PHASE_BYTES_PER_TILE[p] > 0
    # phase 1 moves at least the spins in and the 16-bit labels out
    assert bench.PHASE_BYTES_PER_TILE[0] >= 3 * bench.TW * bench.TH


def test_byte_model_per_site():
    # the per-kernel algorithmic bytes of the 128x64 tile, per site, as the
    # layout states them: phase 1 reads 1 B of spins (+ halo) and writes the
    # masks (0.375 B), 16-bit labels (2 B), border-root and root masks
    # (0.25 B) and border tables; phase 3 reads masks, labels and root masks
    # and writes 1 B of spins
    pb = bench.phase_bytes_per_tile(128, 64)
    per = {k: v / (128 * 64) for k, v in pb.items()}
    assert abs(per[0] - 3.7485) < 1e-3
    assert abs(per[2] - 3.5532) < 1e-3
    assert abs(per[1] - 1.2720) < 1e-3
    # the fused launch: both, less the spins and halo handed over on chip,
    # plus the pre-drawn bond masks (8 B per 32 sites)
    assert pb[4] == pb[0] + pb[2] - (128 * 64 + 64 + 128) + 8 * 4 * 64
    assert bench.PHASE_BYTES_PER_TILE == pb
    # the border terms grow per site as the tile shrinks
    small = bench.phase_bytes_per_tile(128, 32)
    assert small[1] / (128 * 32) > per[1] and small[0] / (128 * 32) > per[0]
