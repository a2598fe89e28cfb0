// sw_batch.cu -- many independent lattices advanced together (the batched
// and serving forms of the sweep). Every phase of a sweep is one launch over
// the tiles of all active replicas; a replica's tiles find its descriptor
// (geometry, threshold, key schedule, buffers, counter, trace row) in a
// device table. An n-sweep sequence (3 phases + a counter advance per sweep)
// is captured once per n as a CUDA graph and replayed until the power-of-two
// bucket of the tile count or a table's capacity changes.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include <climits>

#include <cstdio>
#include <new>
#include <utility>
#include <vector>

#include "sw.h"
#include "sw_internal.h"

namespace {

struct Replica {
  bool active = false;
  int L = 0;
  double beta = 0.0;
  uint64_t seed = 0;
  uint32_t thr = 0;
  int rule = SW_RULE_FLIP;
  int64_t t = 0;       // counter of the next sweep (host mirror of the device value)
  int64_t t_end = INT64_MAX;  // the replica stops before this counter
  int64_t t_base = 0;  // first sweep in the trace
  int64_t cap = 0;     // trace capacity in sweeps
  int ntiles = 0;
  int tile0 = 0;
  bool small = false;  // on the one-CTA path (L <= the batch's small_max_L)
  int8_t* spins = nullptr;
  sw::TileBuffers tb{};
  int64_t* em = nullptr;
};

uint32_t thr_of(double beta) {
  const double p = -expm1(-2.0 * beta);
  const double scaled = floor(ldexp(p, 32));
  if (scaled >= 4294967295.0) return 0xffffffffu;
  return (uint32_t)scaled;
}

void free_replica(Replica& r) {
  void* ptrs[] = {r.spins, r.tb.tbits, r.tb.roots, r.tb.bmask, r.tb.rbits, r.tb.nodes, r.tb.bslot, r.tb.bbits, r.tb.nslots, r.em};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  r = Replica{};
}

}  // namespace

struct sw_batch {
  int shape = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int* d_err = nullptr;
  std::vector<Replica> reps;
  sw::ReplicaDesc* d_descs = nullptr;
  int desc_cap = 0;
  int* d_tile_rep = nullptr;
  int tile_cap = 0;
  int ntiles = 0;       // tiles of the active replicas
  int grid_tiles = 0;   // launch width: ntiles rounded up to a power of two
  bool dirty = true;        // tile map and descriptors must be rebuilt
  bool descs_stale = true;  // descriptors must be uploaded
  // Captured n-sweep graphs, one per n in use (a server runs a few chunk
  // lengths); all are dropped when a launch width, a table or the schedule
  // moves.
  std::vector<std::pair<int, cudaGraphExec_t>> graphs;
  // SW_SCHEDULE_PHASES: a sweep is four launches (phases 1-3 + a counter
  // advance); SW_SCHEDULE_FUSED: one cooperative launch runs a whole chunk.
  int schedule = SW_SCHEDULE_PHASES;
  sw::GridBarrier* d_gbar = nullptr;  // the fused kernel's grid barrier
  bool fused_capture = true;          // false once capturing the cooperative launch has failed
  // Replicas of side <= small_max_L run whole chunks on the one-CTA path
  // (one CTA each, launched before the tiled work of a chunk); 0: none.
  int small_max_L = 0;
  int* d_small = nullptr;  // slots of the small replicas
  int small_cap = 0;
  int nsmall = 0;
  int small_L = 0;  // largest side among them (sizes the launch's shared memory)
};

namespace {

int bfail(int code, const char* msg) { return sw::record_error(code, msg); }

int cuda_bfail(cudaError_t e, const char* what) {
  static thread_local char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  return bfail(e == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA, buf);
}

#define B_CUDA(call, what)                             \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_bfail(e_, what); \
  } while (0)

constexpr size_t kMaxGraphs = 16;

void drop_graph(sw_batch* b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
  b->graphs.clear();
}

sw::ReplicaDesc desc_of(const sw_batch* b, const Replica& r) {
  sw::ReplicaDesc d{};
  if (!r.active) return d;
  const sw::TileShape ts = sw::shape_of(b->shape);
  d.a.g.L = r.L;
  d.a.g.tiles_x = (r.L + ts.tw() - 1) / ts.tw();
  d.a.g.tiles_y = (r.L + ts.th - 1) / ts.th;
  d.a.g.aligned16 = (r.L % 16) == 0;
  d.a.thr = r.thr;
  d.a.rule = (uint32_t)r.rule;
  d.a.ks = sw::make_key_schedule(r.seed);
  d.a.tb = r.tb;
  d.a.spins_in = r.spins;
  d.a.spins_out = r.spins;
  d.tile0 = r.tile0;
  d.active = 1;
  d.t = (uint32_t)r.t;
  d.t_left = r.t_end - r.t;
  d.em_base = r.em;
  d.em_next = r.t - r.t_base;
  d.small = r.small ? 1 : 0;
  return d;
}

// Rebuild the tile numbering and upload the descriptor table when needed.
int sync_tables(sw_batch* b) {
  if (!b->dirty && !b->descs_stale) return SW_OK;
  B_CUDA(cudaStreamSynchronize(b->stream), "stream synchronize");
  if (b->dirty) {
    std::vector<int> tile_rep, small;
    int small_L = 0;
    for (size_t i = 0; i < b->reps.size(); ++i) {
      Replica& r = b->reps[i];
      if (!r.active) continue;
      r.small = r.L <= b->small_max_L;
      if (r.small) {
        small.push_back((int)i);
        small_L = r.L > small_L ? r.L : small_L;
        continue;
      }
      r.tile0 = (int)tile_rep.size();
      tile_rep.insert(tile_rep.end(), r.ntiles, (int)i);
    }
    if ((int)small.size() > b->small_cap) {
      if (b->d_small) cudaFree(b->d_small);
      b->d_small = nullptr;
      b->small_cap = 0;
      int cap = 64;
      while (cap < (int)small.size()) cap *= 2;
      B_CUDA(cudaMalloc(&b->d_small, (size_t)cap * sizeof(int)), "small replica list");
      b->small_cap = cap;
      drop_graph(b);
    }
    if ((int)small.size() != b->nsmall || small_L != b->small_L) drop_graph(b);  // the launch's width and size
    b->nsmall = (int)small.size();
    b->small_L = small_L;
    if (!small.empty())
      B_CUDA(cudaMemcpy(b->d_small, small.data(), small.size() * sizeof(int), cudaMemcpyHostToDevice),
             "small replica list upload");
    b->ntiles = (int)tile_rep.size();
    // The captured graph launches grid_tiles CTAs per phase; the tiles past
    // ntiles map to no replica and exit at once. Membership changes inside
    // the same power-of-two bucket therefore keep the graph.
    int grid = 64;
    while (grid < b->ntiles) grid *= 2;
    if (grid > b->tile_cap) {
      if (b->d_tile_rep) cudaFree(b->d_tile_rep);
      b->d_tile_rep = nullptr;
      b->tile_cap = 0;
      B_CUDA(cudaMalloc(&b->d_tile_rep, (size_t)grid * sizeof(int)), "tile map");
      b->tile_cap = grid;
      drop_graph(b);
    }
    if (grid != b->grid_tiles) drop_graph(b);
    b->grid_tiles = grid;
    tile_rep.resize(grid, -1);
    B_CUDA(cudaMemcpy(b->d_tile_rep, tile_rep.data(), (size_t)grid * sizeof(int), cudaMemcpyHostToDevice),
           "tile map upload");
  }
  // The descriptor table also grows by doubling; entries past the last
  // replica are inactive, and the graph's counter-advance launch covers the
  // whole table.
  const int n = (int)b->reps.size();
  if (n > b->desc_cap) {
    int cap = 64;
    while (cap < n) cap *= 2;
    if (b->d_descs) cudaFree(b->d_descs);
    b->d_descs = nullptr;
    b->desc_cap = 0;
    B_CUDA(cudaMalloc(&b->d_descs, (size_t)cap * sizeof(sw::ReplicaDesc)), "descriptor table");
    b->desc_cap = cap;
    drop_graph(b);
  }
  std::vector<sw::ReplicaDesc> descs(b->desc_cap);
  for (int i = 0; i < n; ++i) descs[i] = desc_of(b, b->reps[i]);
  B_CUDA(cudaMemcpy(b->d_descs, descs.data(), (size_t)b->desc_cap * sizeof(sw::ReplicaDesc), cudaMemcpyHostToDevice),
         "descriptor upload");
  b->dirty = false;
  b->descs_stale = false;
  return SW_OK;
}

// Trace capacity (sweeps) that grow_trace reaches for `needed` sweeps.
int64_t trace_cap_for(int64_t needed) {
  int64_t cap = 1024;
  while (cap < needed) cap *= 2;
  return cap;
}

int grow_trace(Replica& r, int64_t needed, cudaStream_t st) {
  if (needed <= r.cap) return SW_OK;
  const int64_t ncap = trace_cap_for(needed);
  int64_t* em = nullptr;
  B_CUDA(cudaMalloc(&em, (size_t)ncap * 2 * sizeof(int64_t)), "trace growth");
  if (r.cap) {
    cudaError_t e = cudaMemcpyAsync(em, r.em, (size_t)r.cap * 2 * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaFree(em);
      return cuda_bfail(e, "trace growth");
    }
    cudaFree(r.em);
  }
  r.em = em;
  r.cap = ncap;
  return SW_OK;
}

// Device bytes one replica of side L holds with a trace of cap sweeps.
int64_t replica_bytes(const sw::TileShape& ts, int L, int64_t cap) {
  const int64_t nt = (int64_t)((L + ts.tw() - 1) / ts.tw()) * ((L + ts.th - 1) / ts.th);
  return (int64_t)L * L +
         nt * (3 * ts.row_words() * 4 + ts.sites() * 2 + 2 * ts.row_words() * 4 + ts.max_slots() * 8 +
               ts.boundary_sites() * 2 + ts.bbits_words() * 4 + 4) +
         cap * 16;
}

int check_slot(sw_batch* b, int32_t slot) {
  if (!b) return bfail(SW_EINVAL, "batch is NULL");
  if (slot < 0 || slot >= (int32_t)b->reps.size() || !b->reps[slot].active)
    return bfail(SW_EINVAL, "no active replica in this slot");
  return SW_OK;
}

int sync_and_check_batch(sw_batch* b) {
  B_CUDA(cudaStreamSynchronize(b->stream), "stream synchronize");
  int flag = 0;
  B_CUDA(cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error flag read");
  if (flag == sw::kErrUnionCap) return bfail(SW_ETIMEOUT, "device union-find retry loop reached its cap");
  if (flag == sw::kErrCopyTimeout) return bfail(SW_ETIMEOUT, "device bulk copy into shared memory did not complete");
  if (flag == sw::kErrBarrierTimeout) return bfail(SW_ETIMEOUT, "a grid barrier of the fused batch kernel did not open");
  if (flag != 0) return bfail(SW_EDEVICE, "device error flag set");
  return SW_OK;
}

}  // namespace

extern "C" {

int sw_batch_create(int32_t n, const int32_t* L, const double* beta, const uint64_t* seed, const int32_t* init,
                    int32_t shape, void* stream, sw_batch** out) {
  if (!out) return bfail(SW_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 0 || (n > 0 && (!L || !beta || !seed))) return bfail(SW_EINVAL, "bad replica arrays");
  if (shape < -1 || shape >= sw::kNumShapes) return bfail(SW_EINVAL, "unknown tile shape");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return bfail(SW_ECUDA, "no CUDA device available (libsw has no CPU fallback)");
  }
  sw_batch* b = new (std::nothrow) sw_batch();
  if (!b) return bfail(SW_ENOMEM, "host allocation failed");
  if (shape < 0) {
    int lmax = 2;
    for (int32_t i = 0; i < n; ++i) lmax = L[i] > lmax ? L[i] : lmax;
    shape = sw::default_shape(lmax);
  }
  b->shape = shape;
  cudaError_t e = cudaSuccess;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_gbar, sizeof(sw::GridBarrier));
  if (e == cudaSuccess) e = cudaMemset(b->d_gbar, 0, sizeof(sw::GridBarrier));
  if (e != cudaSuccess) {
    const int rc = cuda_bfail(e, "sw_batch_create");
    sw_batch_destroy(b);
    return rc;
  }
  for (int32_t i = 0; i < n; ++i) {
    int32_t slot = 0;
    const int rc = sw_batch_add(b, L[i], beta[i], seed[i], init ? init[i] : SW_INIT_HOT, &slot);
    if (rc != SW_OK) {
      sw_batch_destroy(b);
      return rc;
    }
  }
  *out = b;
  return SW_OK;
}

int sw_batch_add(sw_batch* b, int32_t L, double beta, uint64_t seed, int32_t init, int32_t* slot_out) {
  if (!b || !slot_out) return bfail(SW_EINVAL, "NULL argument");
  if (L < 2 || (int64_t)L * L >= ((int64_t)1 << 31)) return bfail(SW_EINVAL, "L outside 2 <= L, L*L < 2^31");
  if (!(beta >= 0.0) || isinf(beta)) return bfail(SW_EINVAL, "beta must be finite and >= 0");
  if (init != SW_INIT_HOT && init != SW_INIT_COLD) return bfail(SW_EINVAL, "init must be SW_INIT_HOT or SW_INIT_COLD");
  const sw::TileShape ts = sw::shape_of(b->shape);
  Replica r;
  r.L = L;
  r.beta = beta;
  r.seed = seed;
  r.thr = thr_of(beta);
  r.ntiles = ((L + ts.tw() - 1) / ts.tw()) * ((L + ts.th - 1) / ts.th);
  const size_t nt = (size_t)r.ntiles, N = (size_t)L * L;
  cudaError_t e = cudaMalloc(&r.spins, N);
  if (e == cudaSuccess) e = cudaMalloc(&r.tb.tbits, nt * 3 * ts.row_words() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&r.tb.roots, nt * ts.sites() * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMalloc(&r.tb.bmask, nt * ts.row_words() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&r.tb.rbits, nt * ts.row_words() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&r.tb.nodes, nt * ts.max_slots() * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&r.tb.bslot, nt * ts.boundary_sites() * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMalloc(&r.tb.bbits, nt * ts.bbits_words() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&r.tb.nslots, nt * sizeof(int32_t));
  if (e == cudaSuccess) e = sw::launch_init(r.spins, L, seed, init == SW_INIT_COLD, b->stream);
  if (e != cudaSuccess) {
    free_replica(r);
    return cuda_bfail(e, "sw_batch_add");
  }
  r.tb.err = b->d_err;
  const int rc = grow_trace(r, 1024, b->stream);
  if (rc != SW_OK) {
    free_replica(r);
    return rc;
  }
  r.active = true;
  int slot = -1;
  for (size_t i = 0; i < b->reps.size(); ++i)
    if (!b->reps[i].active) {
      slot = (int)i;
      break;
    }
  if (slot < 0) {
    slot = (int)b->reps.size();
    b->reps.push_back(Replica{});
  }
  b->reps[slot] = r;
  b->dirty = true;
  *slot_out = slot;
  return SW_OK;
}

int sw_batch_remove(sw_batch* b, int32_t slot) {
  int rc = check_slot(b, slot);
  if (rc != SW_OK) return rc;
  B_CUDA(cudaStreamSynchronize(b->stream), "stream synchronize");
  free_replica(b->reps[slot]);
  b->dirty = true;
  return SW_OK;
}

int sw_batch_sweep(sw_batch* b, int32_t n) {
  // an NVTX range over the call for profilers (a no-op without one)
  struct Range {
    Range() { nvtxRangePushA("sw_batch_sweep"); }
    ~Range() { nvtxRangePop(); }
  } range;
  if (!b) return bfail(SW_EINVAL, "batch is NULL");
  if (n < 0) return bfail(SW_EINVAL, "n must be >= 0");
  if (n == 0) return SW_OK;
  for (Replica& r : b->reps) {
    if (!r.active) continue;
    const int64_t cap0 = r.cap;
    const int64_t run = r.t_end - r.t < n ? r.t_end - r.t : n;
    const int rc = grow_trace(r, r.t - r.t_base + run, b->stream);
    if (rc != SW_OK) return rc;
    if (r.cap != cap0) b->descs_stale = true;
  }
  int rc = sync_tables(b);
  if (rc != SW_OK) return rc;
  if (b->ntiles == 0 && b->nsmall == 0) return SW_OK;
  sw::BatchArgs ba{b->d_descs, b->d_tile_rep, b->desc_cap, b->d_err, b->d_gbar};
  const bool fused = b->schedule == SW_SCHEDULE_FUSED;
  // The n-sweep sequence: the barrier reset and one cooperative launch
  // (fused), or per sweep the three phases and the counter advance. The
  // fused kernel walks the whole power-of-two bucket of batch tiles (spare
  // tiles map to no replica), like the per-phase launches.
  auto enqueue = [&]() -> cudaError_t {
    cudaError_t es = sw::launch_small_batch(ba, b->d_small, b->nsmall, b->small_L, n, b->stream);
    if (es != cudaSuccess || b->ntiles == 0) return es;
    if (fused) {
      cudaError_t e = cudaMemsetAsync(b->d_gbar, 0, sizeof(sw::GridBarrier), b->stream);
      if (e == cudaSuccess) e = sw::launch_batch_fused(b->shape, ba, b->grid_tiles, n, b->stream);
      return e;
    }
    cudaError_t e = cudaSuccess;
    for (int32_t k = 0; k < n && e == cudaSuccess; ++k) {
      e = sw::launch_batch_phase(b->shape, 1, ba, b->grid_tiles, b->stream);
      if (e == cudaSuccess) e = sw::launch_batch_phase(b->shape, 2, ba, b->grid_tiles, b->stream);
      if (e == cudaSuccess) e = sw::launch_batch_phase(b->shape, 3, ba, b->grid_tiles, b->stream);
      if (e == cudaSuccess) e = sw::launch_batch_advance(ba, b->stream);
    }
    return e;
  };
  if (fused && !b->fused_capture) {
    // the cooperative launch could not be captured on this system: launch it
    B_CUDA(enqueue(), "fused batch launch");
    for (Replica& r : b->reps)
      if (r.active) r.t += (r.t_end - r.t < n ? r.t_end - r.t : n);
    return SW_OK;
  }
  cudaGraphExec_t exec = nullptr;
  for (auto& g : b->graphs)
    if (g.first == n) exec = g.second;
  if (!exec) {
    if (b->graphs.size() >= kMaxGraphs) {
      cudaGraphExecDestroy(b->graphs.front().second);
      b->graphs.erase(b->graphs.begin());
    }
    cudaGraph_t g = nullptr;
    B_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
    cudaError_t e = enqueue();
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess && fused) {
      // capture of the cooperative launch refused: launch it directly from now on
      cudaGetLastError();
      b->fused_capture = false;
      return sw_batch_sweep(b, n);
    }
    if (e != cudaSuccess) return cuda_bfail(e, "graph capture of the batch sweep");
    b->graphs.emplace_back(n, exec);
  }
  B_CUDA(cudaGraphLaunch(exec, b->stream), "graph launch");
  for (Replica& r : b->reps)
    if (r.active) r.t += (r.t_end - r.t < n ? r.t_end - r.t : n);
  return SW_OK;
}

int sw_batch_set_limit(sw_batch* b, int32_t slot, int64_t sweeps_left) {
  int rc = check_slot(b, slot);
  if (rc != SW_OK) return rc;
  Replica& r = b->reps[slot];
  r.t_end = sweeps_left < 0 ? INT64_MAX : r.t + sweeps_left;
  b->descs_stale = true;
  return SW_OK;
}

int sw_batch_set_schedule(sw_batch* b, int32_t schedule) {
  if (!b) return bfail(SW_EINVAL, "batch is NULL");
  if (schedule != SW_SCHEDULE_PHASES && schedule != SW_SCHEDULE_FUSED)
    return bfail(SW_EINVAL, "schedule must be SW_SCHEDULE_PHASES or SW_SCHEDULE_FUSED");
  if (schedule == SW_SCHEDULE_FUSED && !sw::batch_fused_supported(b->shape))
    return bfail(SW_EINVAL, "the fused schedule needs a tile shape whose phases 1 and 3 take the same block");
  if (schedule != b->schedule) {
    B_CUDA(cudaStreamSynchronize(b->stream), "stream synchronize");
    drop_graph(b);
    b->schedule = schedule;
  }
  return SW_OK;
}

int sw_batch_set_small(sw_batch* b, int32_t max_L) {
  if (!b) return bfail(SW_EINVAL, "batch is NULL");
  if (max_L != 0 && (max_L < 2 || max_L > sw::kSmallMaxL))
    return bfail(SW_EINVAL, "max_L must be 0 or in 2..181 (a lattice the one-CTA path holds)");
  if (max_L != b->small_max_L) {
    B_CUDA(cudaStreamSynchronize(b->stream), "stream synchronize");
    b->small_max_L = max_L;
    b->dirty = true;
  }
  return SW_OK;
}

int sw_batch_set_rule(sw_batch* b, int32_t slot, int32_t rule) {
  int rc = check_slot(b, slot);
  if (rc != SW_OK) return rc;
  if (rule != SW_RULE_FLIP && rule != SW_RULE_ASSIGN) return bfail(SW_EINVAL, "rule must be SW_RULE_FLIP or SW_RULE_ASSIGN");
  b->reps[slot].rule = rule;
  b->descs_stale = true;
  return SW_OK;
}

int sw_batch_get_sweep(sw_batch* b, int32_t slot, uint32_t* t_out) {
  int rc = check_slot(b, slot);
  if (rc != SW_OK) return rc;
  if (!t_out) return bfail(SW_EINVAL, "t_out is NULL");
  *t_out = (uint32_t)b->reps[slot].t;
  return SW_OK;
}

int sw_batch_observables(sw_batch* b, int32_t slot, int64_t first, int64_t count, int64_t* E_host, int64_t* M_host) {
  int rc = check_slot(b, slot);
  if (rc != SW_OK) return rc;
  const Replica& r = b->reps[slot];
  if (count < 0 || first < r.t_base || first + count > r.t) return bfail(SW_EINVAL, "sweeps outside the trace");
  rc = sync_and_check_batch(b);
  if (rc != SW_OK) return rc;
  if (count == 0) return SW_OK;
  std::vector<int64_t> tmp((size_t)count * 2);
  B_CUDA(cudaMemcpy(tmp.data(), r.em + 2 * (first - r.t_base), (size_t)count * 2 * sizeof(int64_t),
                    cudaMemcpyDeviceToHost),
         "trace copy");
  for (int64_t k = 0; k < count; ++k) {
    if (E_host) E_host[k] = tmp[2 * k];
    if (M_host) M_host[k] = tmp[2 * k + 1];
  }
  return SW_OK;
}

int sw_batch_spins(sw_batch* b, int32_t slot, int8_t* out, int32_t out_is_device) {
  int rc = check_slot(b, slot);
  if (rc != SW_OK) return rc;
  if (!out) return bfail(SW_EINVAL, "out is NULL");
  const Replica& r = b->reps[slot];
  B_CUDA(cudaMemcpyAsync(out, r.spins, (size_t)r.L * r.L, out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                         b->stream),
         "spins copy");
  if (out_is_device) return SW_OK;
  return sync_and_check_batch(b);
}

int sw_batch_info(sw_batch* b, int32_t* n_active, int64_t* sites, int64_t* device_bytes) {
  if (!b) return bfail(SW_EINVAL, "batch is NULL");
  int32_t na = 0;
  int64_t st = 0, bytes = 0;
  const sw::TileShape ts = sw::shape_of(b->shape);
  for (const Replica& r : b->reps) {
    if (!r.active) continue;
    ++na;
    st += (int64_t)r.L * r.L;
    bytes += replica_bytes(ts, r.L, r.cap);
  }
  if (n_active) *n_active = na;
  if (sites) *sites = st;
  if (device_bytes) *device_bytes = bytes;
  return SW_OK;
}

int sw_batch_footprint(sw_batch* b, int32_t L, int64_t sweeps, int64_t* bytes) {
  if (!b || !bytes) return bfail(SW_EINVAL, "NULL argument");
  if (L < 2 || (int64_t)L * L >= ((int64_t)1 << 31)) return bfail(SW_EINVAL, "L outside 2 <= L, L*L < 2^31");
  if (sweeps < 0) return bfail(SW_EINVAL, "sweeps must be >= 0");
  *bytes = replica_bytes(sw::shape_of(b->shape), L, trace_cap_for(sweeps));
  return SW_OK;
}

int sw_batch_destroy(sw_batch* b) {
  if (!b) return SW_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (Replica& r : b->reps)
    if (r.active) free_replica(r);
  if (b->d_descs) cudaFree(b->d_descs);
  if (b->d_tile_rep) cudaFree(b->d_tile_rep);
  if (b->d_err) cudaFree(b->d_err);
  if (b->d_gbar) cudaFree(b->d_gbar);
  if (b->d_small) cudaFree(b->d_small);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return SW_OK;
}

}  // extern "C"
