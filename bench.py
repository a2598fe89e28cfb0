#!/usr/bin/env python3
"""Benchmark of one Swendsen-Wang sweep of the 2D Ising model on GB300.

Workload: L = 8192 periodic lattice (67,108,864 sites), beta = 0.44068679
(beta_c), hot start from seed 3; one step = one full sweep (bonds, tile-local
and cross-tile cluster labelling, per-cluster flips, E/M reduction).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Our arm prints one JSON line with site-updates/s measured on the device
(CUDA events on the library's stream, L2 flushed between steps by writing a
256 MiB buffer; the K timed steps are repeated until they span 0.25 s and
the median repeat is reported), the roofline of every kernel of the sweep,
the end-to-end rate through the C ABI with host buffers, the oracle's CPU
rates (one core on the headline lattice, every core on the 256-replica mix),
and the SM clocks seen during the timed repeats. Under torchrun every rank runs its own replica
(independent chains, no data-path collective: "replicas only"), and rank 0
reports the whole-job rate.

The reference arm (--impl reference) times the serial CPU oracle on the
host cores on the same workload, one oracle sweep per step.

Rank 0 also reports the 256-replica batch against the same replicas run one
by one ("batched_vs_plain") and a bounded Poisson serving run through the
continuous-batching server ("serving": p50/p99 latency, aggregate rate).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SW site-updates/s at L=8192, β_c; % of HBM roofline; batched vs plain"
UNIT = "site-updates/s"
L = 8192
BETA = 0.44068679
SEED = 3
N_SITES = L * L
FLUSH_BYTES = 256 << 20
MIN_CLOCK_WINDOW_S = 0.25  # timed repeats span at least this long (>= 10 clock samples)
MAX_REPEATS = 200
# Tile shape of the default configuration at this L (128 x 64 sites).
TW, TH = 128, 64
NB = 2 * TH + 2 * TW
BBW = 2 * (TH // 32) + 2 * (TW // 32)
RW = (TW // 32) * TH  # 32-site row-words per tile
# Algorithmic bytes per full tile: what each kernel must read and write for
# the stored layout (bit masks, 16-bit tile roots, border tables); slot nodes
# (8 bytes per border component) are data dependent and not counted.
def phase_bytes_per_tile(tw: int, th: int) -> dict:
    """Algorithmic bytes of each kernel for one full tile of tw x th sites:
    what it must read and write for the stored layout (bit masks, 16-bit
    tile roots, border-root and root masks, border tables); slot nodes (8
    bytes per border component) are data dependent and not counted."""
    nb = 2 * th + 2 * tw                    # border sites
    bbw = 2 * (th // 32) + 2 * (tw // 32)   # border bit words
    rw = (tw // 32) * th                    # 32-site row words
    d = {
        # spins + halo in; spin/east/south masks, 16-bit tile roots,
        # border-root and root masks, border slots, tile bits, slot count out
        # (a one-sweep call: phase 1 draws its own bonds)
        0: (tw * th + th + tw) + (3 * rw * 4 + 2 * tw * th + 2 * 4 * rw + 2 * nb + 4 * bbw + 4),
        # spin/east masks, roots, border-root and root masks, slot count,
        # tile bits, neighbours' halo slots in; spins out
        2: (2 * rw * 4 + 2 * tw * th + 2 * 4 * rw + 4 + 4 * bbw + 2 * (th + tw)) + tw * th,
    }
    # Phase 2 + resolve touch O(tile perimeter): the tile's border bits and
    # the border slots of the tile and of its east and south neighbours, and
    # per border slot its node (read in the union walks, rewritten by the
    # resolve pass); the slot count is data dependent, so the model counts
    # every border site as a slot (an upper bound of the algorithmic bytes).
    d[1] = 4 * bbw + 2 * (nb + th + tw) + 4 + 3 * 8 * nb
    # Phase 3 of a sweep with phase 1 of the next in one launch: both
    # kernels' bytes, less the spins and halo that phase 1 then takes from
    # shared memory, plus the bond draws (two 32-bit masks per row word) that
    # the merge phases before it drew (in such calls the merge phases write
    # them: 8 bytes per row word more than d[1]).
    d[4] = d[0] + d[2] - (tw * th + th + tw) + 8 * rw
    return d


PHASE_BYTES_PER_TILE = phase_bytes_per_tile(TW, TH)
PHASE_NAMES = {0: "phase1_bonds_tile_ccl", 1: "phase2_merge_resolve", 2: "phase3_flip_em", 3: "phase4_hist",
               4: "phase3_with_next_phase1"}
SWEEP_MODEL_BYTES_PER_SITE = 10  # read spins, write+read int32 labels, write spins
# q-state Potts sweep (§6) on the same tiles: phase 1 and phase 2 + resolve
# as for Ising (the state bytes take the place of the spins); phase 3 reads
# the 16-bit tile roots, border-root and root masks, slot count, the tile's
# slot states and the halo's slots and slot states, and writes the states.
MS = 2 * (TW + TH)
POTTS_BYTES_PER_TILE = (PHASE_BYTES_PER_TILE[0] + PHASE_BYTES_PER_TILE[1]
                        + 2 * TW * TH + 2 * 4 * RW + 4 + MS + 3 * (TH + TW) + TW * TH)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples every 10 ms from construction to stop(); stop()
    reports the samples whose timestamps fall inside the marked window (the
    timed region) and, when the window is shorter than the sampling period,
    the samples of the whole busy span around it."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="sw_clocks_", suffix=".csv")
        self.proc = None
        self.window = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark(self, t0: float, t1: float) -> None:
        """The timed region, as time.time() values."""
        self.window = (t0, t1)

    @staticmethod
    def _epoch(stamp: str):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(stamp, fmt).timestamp()
            except ValueError:
                pass
        return None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                sm, smax = float(f[2]), float(f[3])
            except ValueError:
                continue
            active = {n for n, v in zip(names, f[6:10]) if v.lower().startswith("active")}
            rows.append((self._epoch(f[0]), sm, smax, active))
        os.unlink(self.path)
        inside = rows
        if self.window is not None:
            t0, t1 = self.window
            inside = [r for r in rows if r[0] is not None and t0 <= r[0] <= t1]
        use = inside if inside else rows
        return {"sm_mhz": statistics.median(r[1] for r in use) if use else None,
                "sm_max_mhz": max(r[2] for r in use) if use else None,
                "samples": len(use), "samples_in_timed_region": len(inside),
                "sampled": "timed region" if inside else "warm-up through timed region (no sample fell inside it)",
                "reasons": sorted(set().union(*(r[3] for r in use))) if use else []}


# ---------------------------------------------------------------- helpers

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), and its core count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                name = line.split(":", 1)[1].strip()
                break
    return f"{name or 'unknown'} ({platform.machine()}, {os.cpu_count()} cores)"


def cpu_oracle_rate(n_sweeps: int, label: str):
    """Time the serial oracle as it stands on n_sweeps of the workload."""
    import oracle
    oracle.build()
    s0 = oracle.init(L, SEED)
    t0 = time.perf_counter()
    oracle.run(L, BETA, SEED, n_sweeps, spins=s0)
    dt = time.perf_counter() - t0
    return {"value": N_SITES * n_sweeps / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{n_sweeps} {label} of L={L} beta={BETA} from the oracle's own hot start "
                      f"({dt:.1f} s, serial C, {platform.machine()})"}


def _oracle_replicas(job):
    """One process's share of the 256-replica mix: n sweeps of each replica."""
    import oracle
    items, n = job
    t0 = time.perf_counter()
    sites = 0
    for Lr, br, sr in items:
        oracle.run(int(Lr), float(br), int(sr), n)
        sites += int(Lr) * int(Lr) * n
    return sites, time.perf_counter() - t0


def cpu_oracle_batch_rate(n_sweeps: int):
    """The oracle on the 256-replica mix, one process per host core (a spawn
    pool: no process is forked from this CUDA-using one). Each process takes
    every nproc-th replica; the rate is all site-updates over the wall time."""
    import multiprocessing as mp
    import oracle
    from workloads import batch_replicas
    oracle.build()
    Ls, betas, seeds = batch_replicas()
    reps = list(zip(Ls, betas, seeds))
    order = sorted(range(len(reps)), key=lambda i: -int(reps[i][0]))   # big replicas first, dealt round robin
    nproc = os.cpu_count() or 1
    jobs = [([reps[i] for i in order[k::nproc]], n_sweeps) for k in range(nproc)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(nproc) as pool:
        res = pool.map(_oracle_replicas, jobs)
    wall = time.perf_counter() - t0
    sites = sum(r[0] for r in res)
    return {"value": sites / wall, "unit": UNIT, "cores": nproc, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{n_sweeps} oracle sweeps of each of the 256 replicas from their hot starts, "
                      f"{nproc} processes ({wall:.1f} s wall, pool start-up included)"}


def dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank: int) -> int:
    """Rank 0 runs the configured chain; the others independent replicas."""
    return SEED + rank


def whole_job_rate(units_per_rank: int, local_ms: float, world: int, device: str = "cuda") -> tuple[float, float]:
    """Units all ranks processed / the slowest rank's time: (rate, max ms)."""
    max_ms = max_over_ranks(local_ms, world, device)
    return world * units_per_rank / (max_ms / 1e3), max_ms


# -------------------------------------------------------------- reference

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    # Each step is one oracle sweep of the L = 8192 lattice (about 3.4 s on a
    # Grace core), the same lattice our arm sweeps; the run takes K + W such
    # sweeps.
    Ls = L
    s, _, _, _ = oracle.run(L, BETA, SEED, 1, spins=oracle.init(L, SEED), t0=0)
    t = 1
    for _ in range(args.warmup):
        s, _, _, _ = oracle.run(Ls, BETA, SEED, 1, spins=s, t0=t)
        t += 1
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        s, _, _, _ = oracle.run(Ls, BETA, SEED, 1, spins=s, t0=t)
        times.append(time.perf_counter() - t0)
        t += 1
    total = sum(times)
    value = Ls * Ls * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8/u32",
        "data": "synthetic (Philox hot start, seed 3)",
        "config": {"workload": f"L{L} beta_c={BETA} hot start seed {SEED}, one SW sweep per step",
                   "L": L, "beta": BETA, "seed": SEED},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": cpu_model(),
                         "sample": f"{args.steps} oracle sweeps of L={Ls} (serial C, one host core, "
                                   f"{platform.machine()})"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- ours

def run_ours(args):
    import torch
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    import paper_2302_14720_gb300 as sw

    hbm_peak, peak_kind = peaks()
    # One non-default stream carries the library's kernels, the L2 flushes and
    # the timing events, so the events bracket exactly the sweep's kernels.
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    seed = replica_seed(rank)
    lat = sw.Lattice(L, BETA, seed, sw.SW_INIT_HOT, stream=stream.cuda_stream)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    clocks = ClockSampler(local) if rank == 0 else None
    # warm-up (each step preceded by an L2 flush, as in the timed loop)
    for k in range(args.warmup):
        flush.fill_(k & 0xFF)
        lat.sweep(1)
    torch.cuda.synchronize()

    # The timed region: exactly K steps, each an L2 flush and one sweep,
    # bracketed by CUDA events on the library's stream. It is repeated until
    # the repeats span at least MIN_CLOCK_WINDOW_S, so that the SM clock
    # sampler (one sample per 10 ms) sees the timed work itself; `value` is
    # the repeat with the median time, and every repeat is listed.
    t_first = lat.t
    sw.sw_timing(lat.h, True)
    barrier(world)
    torch.cuda.synchronize()
    t_region0 = time.time()
    repeats = []
    while True:
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_((k + 7) & 0xFF)
            starts[k].record(stream)
            lat.sweep(1)
            ends[k].record(stream)
        torch.cuda.synchronize()
        repeats.append(sum(s.elapsed_time(e) for s, e in zip(starts, ends)))
        if time.time() - t_region0 >= MIN_CLOCK_WINDOW_S or len(repeats) >= MAX_REPEATS:
            break
    t_region1 = time.time()
    barrier(world)
    if clocks:
        clocks.mark(t_region0, t_region1)
    clock_info = clocks.stop() if clocks else None
    phase_ms, phase_n = sw.sw_timing_read(lat.h)
    sw.sw_timing(lat.h, False)
    total_ms = sorted(repeats)[len(repeats) // 2]
    E, M = lat.observables(t_first, args.steps * len(repeats))
    assert (np.abs(E) <= 2 * N_SITES).all() and (np.abs(M) <= N_SITES).all()
    value, max_ms = whole_job_rate(N_SITES * args.steps, total_ms, world)

    # ---- roofline of the dominant kernel (largest summed device time)
    ntiles = (L // TW) * (L // TH)
    dom = max((0, 1, 2, 4), key=lambda p: phase_ms[p])
    dom_avg_ms = phase_ms[dom] / max(phase_n[dom], 1)
    dom_bytes = PHASE_BYTES_PER_TILE.get(dom, 0) * ntiles
    achieved = dom_bytes / (dom_avg_ms / 1e3) / 1e9
    traffic = warp_instr = None
    tpath = os.path.join(ROOT, "profiles", "dram_traffic_L8192.json")
    if os.path.exists(tpath):
        tr = json.load(open(tpath))
        if tr.get("kernel") == PHASE_NAMES[dom] and tr.get("source_hash") == sw_source_hash():
            traffic = tr.get("bytes_per_launch")
            warp_instr = tr.get("warp_instructions_per_launch")
    roofline = {"bound": "hbm", "kernel": PHASE_NAMES[dom], "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": traffic,
                "peak_kind": peak_kind, "bytes_per_launch": dom_bytes, "avg_launch_ms": dom_avg_ms}
    # What binds the dominant kernel: instruction issue. Its warp instructions
    # per launch (ncu, same sources) over its live launch time, against one
    # warp instruction per cycle on each of an SM's 4 schedulers.
    if warp_instr:
        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = (clock_info or {}).get("sm_mhz") or (clock_info or {}).get("sm_max_mhz") or 2070.0
        issue_peak = n_sm * 4 * mhz * 1e6
        issue_rate = warp_instr / (dom_avg_ms / 1e3)
        roofline["issue"] = {"warp_instructions_per_launch": warp_instr, "achieved": issue_rate,
                             "peak": issue_peak, "unit": "warp instructions/s", "frac": issue_rate / issue_peak,
                             "peak_from": f"{n_sm} SMs x 4 schedulers x {mhz:.0f} MHz"}
    phases = {PHASE_NAMES[p]: {"ms_per_launch": phase_ms[p] / max(phase_n[p], 1), "launches": int(phase_n[p])}
              for p in range(5) if phase_n[p]}
    # every kernel of the sweep against the same HBM peak: algorithmic bytes
    # per launch (the model above) over its average CUDA-event time
    roofline_phases = {}
    for p in (0, 1, 2, 4):
        if not phase_n[p]:
            continue
        ms_p = phase_ms[p] / phase_n[p]
        by = PHASE_BYTES_PER_TILE[p] * ntiles
        gbs = by / (ms_p / 1e3) / 1e9
        roofline_phases[PHASE_NAMES[p]] = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                                           "bytes_per_launch": by, "avg_launch_ms": ms_p,
                                           "bytes_per_site": PHASE_BYTES_PER_TILE[p] / (TW * TH)}
    sweep_roofline_su_s = hbm_peak * 1e9 / SWEEP_MODEL_BYTES_PER_SITE

    # ---- end to end through the C ABI with host buffers (pinned). Two
    # lattices on two streams take the steps in turn, so one step's input
    # copy and check overlap the other lattice's sweep; every step still
    # copies its whole input state host -> device (sw_set_state_async, whose
    # check the next sw_observables of that lattice reads back) and reads its
    # E and M back (sw_observables).
    host = torch.empty((L, L), dtype=torch.int8, pin_memory=True)
    host_np = host.numpy()
    host_np[...] = lat.spins()
    stream2 = torch.cuda.Stream()
    lat2 = sw.Lattice(L, BETA, seed + 1000, sw.SW_INIT_HOT, stream=stream2.cuda_stream)
    pair = [lat, lat2]
    # Each lattice's steps take consecutive counters (a chain whose state
    # goes through host memory between sweeps).
    e2e_steps = max(4, min(args.steps, 20))
    t = lat.t
    for k in range(2):  # warm-up of both lattices (allocates their staging buffers)
        sw.sw_set_state_async(pair[k].h, host_np, t)
        pair[k].sweep(1)
        pair[k].observables(t, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pending = None
    for k in range(e2e_steps):
        h, tk = pair[k % 2], t + 1 + k // 2
        sw.sw_set_state_async(h.h, host_np, tk)        # H2D: the step's input state (checked on the GPU)
        h.sweep(1)
        if pending is not None:
            pending[0].observables(pending[1], 1)      # D2H: the previous step's E and M
        pending = (h, tk)
    pending[0].observables(pending[1], 1)
    e2e_total = time.perf_counter() - t0
    e2e_value = world * N_SITES * e2e_steps / max_over_ranks(e2e_total, world)
    lat2.close()
    lat.close()

    if rank != 0:
        return 0
    others = None
    if not args.no_configs:
        others = measure_other_configs(sw, torch, stream, flush)
        log("configs:", json.dumps(others))
    batched = serving = None
    if args.batched_sweeps > 0:
        batched = measure_batched(sw, torch, stream, args.batched_sweeps, args.plain_sweeps)
        log("batched:", json.dumps(batched))
        if args.serving_requests > 0:
            serving = measure_serving(sw, stream, args.serving_requests, batched["batched_su_s"],
                                      args.serving_budget_gib)
            log("serving:", json.dumps(serving))
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(args.cpu_sweeps, "sweeps")
        if batched is not None:
            batched["cpu_oracle_nproc"] = cpu_oracle_batch_rate(args.cpu_batch_sweeps)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8/u32",
        "data": "synthetic (Philox hot start, seed 3 + rank)",
        "config": {"workload": f"L{L} beta_c={BETA} hot start seed {SEED}, one SW sweep per step",
                   "L": L, "beta": BETA, "seed": SEED, "tile": f"{TW}x{TH}, one warp per 32-column band",
                   "l2": "flushed between steps (256 MiB write), inputs 64 MiB < L2",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "roofline_phases": roofline_phases,
        "timed_repeats": {"count": len(repeats), "ms": repeats, "value_from": "median repeat",
                          "why": "the K timed steps are repeated until they span >= 0.25 s, so the clock "
                                 "sampler sees them"},
        "sweep_vs_10B_per_site_hbm_model": {"roofline_su_s": sweep_roofline_su_s, "frac": value / world / sweep_roofline_su_s},
        "phases": phases,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": N_SITES, "d2h_bytes_per_step": 16,
                "steps": e2e_steps, "ms_per_step": 1e3 * e2e_total / e2e_steps,
                "how": "public C ABI: sw_set_state_async from pinned host memory (copy, check, buffer "
                       "exchange queued on the lattice's stream), sw_sweep, sw_observables; two lattices on "
                       "two streams alternate steps so copies overlap sweeps"},
        # phase 2 is two launches (the merge and the resolve pass)
        "gpu_launches": int(phase_n[0] + 2 * phase_n[1] + phase_n[2] + phase_n[3] + phase_n[4]),
        "clocks": clock_info,
        "other_configs": others,
        "batched_vs_plain": batched,
        "serving": serving,
    }
    print(json.dumps(line), flush=True)
    return 0


def timed_sweeps(torch, stream, fn, n: int) -> float:
    """Device milliseconds of fn() (which issues n sweeps) on `stream`."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def l2_copy_gbs(torch, stream) -> float:
    """Copy bandwidth (read + write bytes per second) between two 24 MiB
    device buffers that stay in L2: 40 copies back and forth replayed from
    one CUDA graph (no launch gaps), best of 5 replays."""
    a = torch.empty(24 << 20, dtype=torch.uint8, device="cuda")
    b = torch.empty_like(a)
    a.fill_(1)
    b.copy_(a)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for k in range(40):
            (b.copy_(a) if k % 2 == 0 else a.copy_(b))
    best = 0.0
    with torch.cuda.stream(stream):
        g.replay()
        for _ in range(5):
            ms = timed_sweeps(torch, stream, g.replay, 40)
            best = max(best, 2 * (24 << 20) * 40 / (ms / 1e3) / 1e9)
    del g
    return best


def measure_other_configs(sw, torch, stream, flush):
    """The smaller configurations and the second temperature of the headline
    lattice: per-sweep latency at L=64, the L2-resident rate with per-sweep
    cluster histograms at L=1024, and L=8192 at beta=0.50."""
    out = {}
    # L=64, beta_c, hot start seed 1: 1000 sweeps, plain launches and as a
    # one-replica batch (one CUDA graph of 100 sweeps per call)
    with sw.Lattice(64, BETA, 1, stream=stream.cuda_stream) as lat:
        lat.sweep(10)
        ms = timed_sweeps(torch, stream, lambda: lat.sweep(1000), 1000)
        lat.observables(0, 1)
    b = sw.sw_batch_create([64], [BETA], [1], stream=stream.cuda_stream)
    try:
        sw.sw_batch_sweep(b, 100)
        ms_g = timed_sweeps(torch, stream, lambda: [sw.sw_batch_sweep(b, 100) for _ in range(10)], 1000)
        sw.sw_batch_observables(b, 0, 0, 1)
    finally:
        sw.sw_batch_destroy(b)
    out["L64_betac"] = {"us_per_sweep": 1e3 * ms / 1000, "us_per_sweep_graph": 1e3 * ms_g / 1000,
                        "su_s": 64 * 64 * 1000 / (ms / 1e3), "sweeps": 1000,
                        "how": "sw_sweep(1000) launches; and a one-replica batch replaying a 100-sweep graph"}
    # L=1024, beta_c, cold start seed 2, histogram every sweep (L2-resident)
    with sw.Lattice(1024, BETA, 2, sw.SW_INIT_COLD, stream=stream.cuda_stream) as lat:
        shape1024 = sw.sw_lattice_shape(lat.h)
        lat.histogram(True)
        lat.sweep(20)
        n = 1000
        ms = timed_sweeps(torch, stream, lambda: lat.sweep(n), n)
        h = lat.histograms(20, n)
        assert (h[:, 1] > 0).all()
        lat.histogram(False)
        ms_nh = timed_sweeps(torch, stream, lambda: lat.sweep(n), n)
    # The L=1024 state and its tables (about 9 MB) stay in L2, so its rate is
    # set against the L2 copy bandwidth measured here (two 24 MiB buffers,
    # L2-resident, copied back and forth), not against HBM. Algorithmic bytes
    # per site: with statistics the one-sweep phases (phase 4's O(clusters)
    # not counted); without, the merge phases (with their bond draws) and the
    # fused launch of a multi-sweep call.
    l2_gbs = l2_copy_gbs(torch, stream)
    info = sw.sw_shape_info(shape1024)
    tw1, th1 = info["tile_w"], info["tile_h"]
    pb = phase_bytes_per_tile(tw1, th1)
    tiles = (1024 // tw1) * (1024 // th1)
    by_hist = (pb[0] + pb[1] + pb[2]) * tiles
    # without statistics: the fused launch where the shape has it, else the
    # one-sweep phases
    by_fused = ((pb[1] + 8 * (tw1 // 32) * th1 + pb[4]) if shape1024 in (4, 6) else (pb[0] + pb[1] + pb[2])) * tiles
    g_hist = by_hist / (ms / n / 1e3) / 1e9
    g_fused = by_fused / (ms_nh / n / 1e3) / 1e9
    out["L1024_betac_cold_hist"] = {"su_s": 1024 * 1024 * n / (ms / 1e3), "us_per_sweep": 1e3 * ms / n,
                                    "su_s_without_hist": 1024 * 1024 * n / (ms_nh / 1e3), "sweeps": n,
                                    "l2": "state L2-resident (1 MiB spins), no flush",
                                    "tile": f"{tw1}x{th1}",
                                    "l2_roofline": {"peak": l2_gbs, "unit": "GB/s",
                                                    "peak_kind": "measured live: L2-resident copy, 2 x 24 MiB",
                                                    "bytes_per_site_hist": by_hist / 1024**2,
                                                    "achieved_hist": g_hist, "frac_hist": g_hist / l2_gbs,
                                                    "bytes_per_site_no_hist": by_fused / 1024**2,
                                                    "achieved_no_hist": g_fused, "frac_no_hist": g_fused / l2_gbs}}
    # L=8192, beta=0.50, hot start seed 3, L2 flushed between sweeps
    with sw.Lattice(L, 0.50, SEED, stream=stream.cuda_stream) as lat:
        for k in range(3):
            flush.fill_(k)
            lat.sweep(1)
        tot = 0.0
        for k in range(10):
            flush.fill_(k + 3)
            tot += timed_sweeps(torch, stream, lambda: lat.sweep(1), 1)
        lat.observables(3, 10)
    out["L8192_beta0.50"] = {"su_s": N_SITES * 10 / (tot / 1e3), "ms_per_sweep": tot / 10, "sweeps": 10}
    # The headline lattice as a chain: 200 consecutive sweeps in one
    # sw_sweep call (phase 3 and the next sweep's phase 1 in one launch, the
    # merge phases drawing the next sweep's bonds); a sweep moves ~0.5 GB,
    # well above L2, so no flush is needed between sweeps.
    with sw.Lattice(L, BETA, SEED, stream=stream.cuda_stream) as lat:
        lat.sweep(20)
        n = 200
        ms = timed_sweeps(torch, stream, lambda: lat.sweep(n), n)
        lat.observables(20, n)
    out["L8192_betac_chain"] = {"su_s": N_SITES * n / (ms / 1e3), "ms_per_sweep": ms / n, "sweeps": n,
                                "how": "one sw_sweep(200) call, CUDA events around it"}
    # the paper's label-equivalence labelling (§2.3) against the tile
    # union-find, both from the same state (each includes drawing the bonds)
    out["labels_union_find_vs_equivalence"] = {}
    for Lc in (1024, 4096):
        with sw.Lattice(Lc, BETA, 2, sw.SW_INIT_COLD, stream=stream.cuda_stream) as lat:
            lat.sweep(30)
            buf = torch.empty((Lc, Lc), dtype=torch.int32, device="cuda")
            sw.sw_labels(lat.h, Lc, buf.data_ptr())
            ms_uf = timed_sweeps(torch, stream, lambda: sw.sw_labels(lat.h, Lc, buf.data_ptr()), 1)
            its = sw.sw_labels_equivalence(lat.h, Lc, buf.data_ptr())[1]
            ms_le = timed_sweeps(torch, stream, lambda: sw.sw_labels_equivalence(lat.h, Lc, buf.data_ptr()), 1)
        out["labels_union_find_vs_equivalence"][f"L{Lc}"] = {
            "union_find_ms": ms_uf, "label_equivalence_ms": ms_le, "iterations": its, "speedup": ms_le / ms_uf}
    # q = 3 Potts at its critical coupling ln(1 + sqrt 3), on the tiled path
    peak_gbs, peak_kind = peaks()
    for Lq, n in ((1024, 200), (8192, 40)):
        with sw.Potts(Lq, 3, 1.0050833, 4, stream=stream.cuda_stream) as pt:
            pt.sweep(10)
            ms = timed_sweeps(torch, stream, lambda: pt.sweep(n), n)
            pt.observables(10, n)
        ntiles = -(-Lq // TW) * -(-Lq // TH)
        gbs = POTTS_BYTES_PER_TILE * ntiles / (ms / n / 1e3) / 1e9
        out[f"potts_q3_L{Lq}_betac"] = {
            "su_s": Lq * Lq * n / (ms / 1e3), "us_per_sweep": 1e3 * ms / n, "sweeps": n,
            "bytes_per_site": POTTS_BYTES_PER_TILE / (TW * TH), "achieved_gbs": gbs,
            "frac_of_hbm": gbs / peak_gbs, "peak": f"{peak_gbs:.0f} GB/s ({peak_kind})"}
    # O(4) phi^4 multicluster updates at the paper's kappa = 0.304 (§5's
    # second table: L = 16..28, 10^4 updates), and L = 64 (16.8 M sites,
    # 0.5 GB of field) where the update's arrays no longer fit in L2.
    # Algorithmic bytes per site of one update: project (field 32 in,
    # projection 8 and parent 4 out), bonds (projection 8 in, bond bits 1
    # out), unite (bond bits 1 in; the parent walks are data dependent and
    # not counted), roots (parent 4 in and 4 out), reflect (parent 4, flip 1,
    # projection 8 in; the field of the half of the sites that flip, 32 in
    # and 32 out), observables (field 32 in).
    phi4_bytes = (32 + 8 + 4) + (8 + 1) + 1 + (4 + 4) + (4 + 1 + 8 + 0.5 * 64) + 32
    out["phi4_kappa0.304"] = {}
    for Lp in (16, 28, 64):
        with sw.Phi4(Lp, 0.304, 6, stream=stream.cuda_stream) as f4:
            f4.sweep(5)
            n4 = 200
            ms4 = timed_sweeps(torch, stream, lambda: f4.sweep(n4), n4)
            f4.observables(5, n4)
        gbs = phi4_bytes * Lp**4 / (ms4 / n4 / 1e3) / 1e9
        out["phi4_kappa0.304"][f"L{Lp}"] = {"ms_per_update": ms4 / n4, "site_updates_s": Lp**4 * n4 / (ms4 / 1e3),
                                            "updates": n4, "minutes_per_1e4_updates": ms4 / n4 * 1e4 / 6e4,
                                            "bytes_per_site": phi4_bytes, "achieved_gbs": gbs,
                                            "frac_of_hbm": gbs / peak_gbs,
                                            "peak": f"{peak_gbs:.0f} GB/s ({peak_kind})",
                                            "l2": "fits in L2" if 46 * Lp**4 < 100e6 else "exceeds L2"}
    return out


def measure_batched(sw, torch, stream, n_batched: int, n_plain: int):
    """The 256-replica mix (L in {64..1024}, beta grid in [0.40, 0.48], hot
    starts): one batched sweep over all replicas per graph node group versus
    every replica swept alone on its own handle, one after the other."""
    from workloads import batch_replicas
    from paper_2302_14720_gb300 import autotune
    Ls, betas, seeds = batch_replicas()
    sites = int(sum(int(x) * int(x) for x in Ls))
    chunk = 50
    # tile shape, schedule (per-phase launches or one fused launch per chunk)
    # and one-CTA threshold chosen by measurement on a scratch batch
    choice = autotune.tune_batch(Ls, betas, seeds)
    b = sw.sw_batch_create(Ls, betas, seeds, shape=choice["shape"], stream=stream.cuda_stream)
    try:
        autotune.apply_batch(b, choice)
        sw.sw_batch_sweep(b, chunk)             # warm-up: captures the graph
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_b = max(chunk, n_batched // chunk * chunk)
        e0.record(stream)
        for _ in range(n_b // chunk):
            sw.sw_batch_sweep(b, chunk)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_b = e0.elapsed_time(e1)
        E, _ = sw.sw_batch_observables(b, 0, 0, 1)  # also checks the device error flag
    finally:
        sw.sw_batch_destroy(b)
    lats = [sw.Lattice(int(Lr), float(br), int(sr), stream=stream.cuda_stream) for Lr, br, sr in zip(Ls, betas, seeds)]
    try:
        for lat in lats:
            lat.sweep(2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for lat in lats:
            lat.sweep(n_plain)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_p = e0.elapsed_time(e1)
        lats[0].observables(0, 1)
    finally:
        for lat in lats:
            lat.close()
    batched = sites * n_b / (ms_b / 1e3)
    plain = sites * n_plain / (ms_p / 1e3)
    return {"workload": "256 replicas, L_r from default_rng(4) over {64,128,256,512,1024}, "
                        "beta_b = 0.40 + 0.08 b/63, seed 1000 + r, hot start",
            "sites": sites, "batched_su_s": batched, "batched_sweeps": n_b,
            "batched_ms_per_sweep": ms_b / n_b, "plain_su_s": plain, "plain_sweeps": n_plain,
            "plain_ms_per_sweep": ms_p / n_plain, "ratio": batched / plain,
            "tuned": {"shape": choice["shape"], "schedule": ["per-phase launches", "fused persistent launch"][choice["schedule"]],
                      "small_max_L": choice["small_max_L"], "ms_per_sweep_by_candidate": choice["ms"]},
            "how": "batched: sw_batch_sweep graph replays of 50 sweeps under the autotuned shape, schedule and "
                   "one-CTA threshold; plain: sw_sweep(n) on each of the 256 "
                   "handles in turn; CUDA events on one stream; working set > L2 (batched), each plain "
                   "replica <= 1 MiB of spins (L2-resident)"}


def measure_serving(sw, stream, n_requests: int, capacity_su_s: float, budget_gib: int):
    """Poisson stream of requests with the serving mix (L log-uniform in
    [32, 4096], beta uniform in [0.30, 0.60], sweeps uniform in [100, 10000],
    seeds from default_rng(5)) at 80% of the batched capacity; latency from
    arrival to result on the host."""
    from workloads import serving_requests
    from paper_2302_14720_gb300.serving import Request, Server, latency_summary
    mean_su = 8.73e9   # E[L^2] * E[sweeps] of the mix
    rate = 0.8 * capacity_su_s / mean_su
    stream_reqs = serving_requests(n=n_requests, rate_per_s=rate, seed=5)
    reqs = [Request(i, L=q["L"], beta=q["beta"], seed=q["seed"], sweeps=q["sweeps"], arrival=q["arrival"])
            for i, q in enumerate(stream_reqs)]
    with Server(budget_bytes=budget_gib << 30, chunk=64, stream=stream.cuda_stream) as srv:
        t0 = time.perf_counter()
        res = srv.run(reqs, realtime=True)
        wall = time.perf_counter() - t0
        su = srv.site_updates
        steps = srv.steps
    for r in res:
        if r.error is None:
            assert (np.abs(r.E) <= 2 * reqs[r.rid].L ** 2).all()
    summary = latency_summary(res)
    summary.update({"requests": n_requests, "rate_per_s": rate, "budget_gib": budget_gib,
                    "aggregate_su_s": su / wall, "site_updates": su, "wall_s": wall, "chunks": steps,
                    "workload": "Poisson arrivals at 0.8 x batched capacity / 8.73e9 SU per request; "
                                "L = round(exp(U[ln 32, ln 4096])), beta ~ U[0.30, 0.60], "
                                "sweeps ~ U{100..10000}, default_rng(5)"})
    return summary


def code_only(text: str) -> str:
    """C/CUDA source without its comments and with whitespace runs collapsed,
    so that the hash below follows the code and not its commentary."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


# The sources that compile into the tiled sweep kernels (phases 1-4).
TILED_SOURCES = ("sw_kernels.cu", "sw_internal.h", "sw_philox.cuh")


def sw_source_hash(csrc: str | None = None) -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = csrc or os.path.join(ROOT, "paper_2302_14720_gb300", "csrc")
    for f in TILED_SOURCES:
        h.update(f.encode())
        h.update(code_only(open(os.path.join(csrc, f), encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sweeps", type=int, default=3)
    ap.add_argument("--cpu-batch-sweeps", type=int, default=10,
                    help="oracle sweeps of each replica in the nproc-process baseline of the 256-replica mix")
    ap.add_argument("--no-configs", action="store_true", help="skip the L=64, L=1024 and beta=0.50 lines")
    ap.add_argument("--batched-sweeps", type=int, default=500,
                    help="sweeps of the 256-replica batch (0 skips the batched and serving measurements)")
    ap.add_argument("--plain-sweeps", type=int, default=100, help="sweeps of each replica run alone")
    ap.add_argument("--serving-requests", type=int, default=100, help="requests of the serving run (0 skips it)")
    ap.add_argument("--serving-budget-gib", type=int, default=64)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
