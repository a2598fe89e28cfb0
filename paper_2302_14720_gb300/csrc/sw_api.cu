// sw_api.cu -- the C ABI of libsw (include/sw.h): handles, device memory,
// the per-sweep trace, argument checks and error reporting. All arithmetic
// of a sweep runs in the kernels of sw_kernels.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <cstdarg>
#include <mutex>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "sw.h"
#include "sw_internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SW_CUDA(call, what)                          \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

bool beta_ok(double beta) { return isfinite(beta) && beta >= 0.0; }

uint32_t threshold_of(double beta) {
  // C3: thr = floor(2^32 * (1 - exp(-2 beta))), capped at 2^32 - 1
  const double p = -expm1(-2.0 * beta);
  const double scaled = floor(ldexp(p, 32));
  if (scaled >= 4294967295.0) return 0xffffffffu;
  return (uint32_t)scaled;
}

constexpr int kBuckets = 17;  // ceil(log2 L) for 2 <= L <= 46340
std::atomic<int> g_tuned[kBuckets];
std::once_flag g_tuned_once;

int bucket_of(int L) {
  int b = 0;
  while ((1 << b) < L) ++b;
  return b < kBuckets ? b : kBuckets - 1;
}

// lattice: the shape of a lone lattice (sw_create); else of a batch whose
// largest side is L.
int shape_for(int L, bool lattice) {
  if (const char* env = getenv("SW_TILE_SHAPE")) {
    const int v = atoi(env);
    if (v >= 0 && v < sw::kNumShapes) return v;
  }
  std::call_once(g_tuned_once, [] {
    for (auto& x : g_tuned) x.store(-1);
  });
  const int t = g_tuned[bucket_of(L)].load();
  if (t >= 0) return t;
  if (L <= 64) return 2;
  // A lone lattice of side <= 1024 has at most 128 tiles of 128 x 64, less
  // than one wave of 152 SMs; with 128 x 32 tiles twice as many CTAs share
  // each phase's latency (measured on GB300 at L = 256 .. 1024: one-sweep
  // calls 12 %, sweeps with statistics 9 % faster, chains even). Batches keep
  // 128 x 64, whose fused schedule the 128 x 32 shape does not have.
  return lattice && L <= 1024 ? 7 : 6;
}

}  // namespace

namespace sw {
int default_shape(int L) { return shape_for(L, false); }
}  // namespace sw

namespace sw {
int record_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace sw

struct sw_lattice {
  int L = 0;
  double beta = 0.0;
  uint64_t seed = 0;
  uint32_t thr = 0;
  int64_t t = 0;       // next sweep counter (absolute)
  int64_t t_base = 0;  // first sweep held in the trace
  int64_t cap = 0;     // trace capacity in sweeps
  int shape = 0;
  int device = 0;
  bool hist_on = false;
  bool tiles_only = false;  // SW_TILE_SHAPE was set: always the tiled path
  int rule = SW_RULE_FLIP;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  sw::Geometry g{};
  sw::KeySchedule ks{};
  sw::TileBuffers tb{};
  // A second set of the tables that neighbouring tiles read (border slots,
  // slot counts, slot nodes): sweep t uses set t & 1, so that phase 3 of
  // sweep t and phase 1 of sweep t + 1 can run in one launch (phase31).
  uint16_t* bslot2 = nullptr;
  int32_t* nslots2 = nullptr;
  uint64_t* nodes2 = nullptr;
  bool fuse = false;       // the tile shape has the phase31 launch
  // The bond draws of sweep draws_t (C5 depends on the seed, the counter and
  // the site, not on the spins): the merge phases of a sweep leave those of
  // the next sweep here when the two run in one call with the fused launch;
  // any later phase 1 of counter draws_t may read them too; -1: none held.
  uint2* draws = nullptr;
  int64_t draws_t = -1;
  int8_t* spins = nullptr;
  uint32_t* csize = nullptr;
  int64_t* em = nullptr;    // [cap][2]
  int64_t* hist = nullptr;  // [cap][SW_HIST_WORDS]
  int32_t* label_buf = nullptr;
  uint8_t* bond_buf = nullptr;
  int32_t* ref_buf = nullptr;  // label-equivalence references
  int* le_flag = nullptr;
  int8_t* staging = nullptr;  // host sw_set_state lands here and is checked first
  int* check_flag = nullptr;
  // per-phase timing (sw_timing)
  bool timing_on = false;
  struct Mark {
    int phase;
    cudaEvent_t start, stop;
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> event_pool;
  double phase_ms[SW_TIMING_PHASES] = {0, 0, 0, 0, 0};
  int64_t phase_launches[SW_TIMING_PHASES] = {0, 0, 0, 0, 0};
};

namespace {

void free_all(sw_lattice* h) {
  void* ptrs[] = {h->spins, h->tb.tbits, h->tb.roots, h->tb.bmask, h->tb.rbits, h->tb.nodes, h->tb.bslot, h->tb.bbits, h->tb.nslots, h->tb.err,
                  h->bslot2, h->nslots2, h->nodes2, h->draws,
                  h->csize, h->em, h->hist, h->label_buf, h->bond_buf, h->ref_buf, h->le_flag, h->staging,
                  h->check_flag};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& m : h->marks) {
    cudaEventDestroy(m.start);
    cudaEventDestroy(m.stop);
  }
  for (cudaEvent_t ev : h->event_pool) cudaEventDestroy(ev);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

cudaError_t take_event(sw_lattice* h, cudaEvent_t* ev) {
  if (!h->event_pool.empty()) {
    *ev = h->event_pool.back();
    h->event_pool.pop_back();
    return cudaSuccess;
  }
  return cudaEventCreate(ev);
}

// An NVTX range over a scope: profilers (ncu --nvtx, nsys) see each phase
// launch and each call under its name; without an attached tool the calls
// are no-ops.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
const char* const kPhaseRange[SW_TIMING_PHASES] = {"sw phase 1: bonds + tile clusters",
                                                   "sw phase 2: cross-tile merge + resolve",
                                                   "sw phase 3: new spins + E/M",
                                                   "sw phase 4: cluster statistics",
                                                   "sw phase 3 + next phase 1"};

// Launch one phase, bracketed by timing events when sw_timing is on.
template <typename F>
cudaError_t timed_phase(sw_lattice* h, int phase, F&& launch) {
  NvtxRange range(kPhaseRange[phase]);
  if (!h->timing_on) return launch();
  sw_lattice::Mark m{phase, nullptr, nullptr};
  cudaError_t e = take_event(h, &m.start);
  if (e == cudaSuccess) e = take_event(h, &m.stop);
  if (e == cudaSuccess) e = cudaEventRecord(m.start, h->stream);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(m.stop, h->stream);
  if (e == cudaSuccess) h->marks.push_back(m);
  return e;
}

// Fold recorded event pairs into the per-phase sums (events must be complete).
cudaError_t drain_marks(sw_lattice* h) {
  for (auto& m : h->marks) {
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, m.start, m.stop);
    if (e != cudaSuccess) return e;
    h->phase_ms[m.phase] += ms;
    h->phase_launches[m.phase] += 1;
    h->event_pool.push_back(m.start);
    h->event_pool.push_back(m.stop);
  }
  h->marks.clear();
  return cudaSuccess;
}

// The arguments of sweep t (default: the current counter); an odd sweep uses
// the second set of neighbour-read tables when the handle has one.
sw::SweepArgs args_of(const sw_lattice* h, int64_t t = -1) {
  if (t < 0) t = h->t;
  sw::SweepArgs a{};
  a.g = h->g;
  a.thr = h->thr;
  a.t = (uint32_t)t;
  a.rule = (uint32_t)h->rule;
  a.ks = h->ks;
  a.tb = h->tb;
  if (h->fuse && (t & 1)) {
    a.tb.bslot = h->bslot2;
    a.tb.nslots = h->nslots2;
    a.tb.nodes = h->nodes2;
  }
  a.spins_in = h->spins;
  a.spins_out = h->spins;
  if (h->draws && h->draws_t == t) a.draws_in = h->draws;
  return a;
}

int ensure_trace(sw_lattice* h, int64_t sweeps_needed) {
  if (sweeps_needed <= h->cap) return SW_OK;
  int64_t ncap = h->cap ? h->cap : 1024;
  while (ncap < sweeps_needed) ncap *= 2;
  int64_t *em = nullptr, *hist = nullptr;
  cudaError_t e = cudaMalloc(&em, (size_t)ncap * 2 * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&hist, (size_t)ncap * SW_HIST_WORDS * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, (size_t)ncap * SW_HIST_WORDS * sizeof(int64_t), h->stream);
  if (e == cudaSuccess && h->cap) {
    e = cudaMemcpyAsync(em, h->em, (size_t)h->cap * 2 * sizeof(int64_t), cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hist, h->hist, (size_t)h->cap * SW_HIST_WORDS * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                          h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    if (em) cudaFree(em);
    if (hist) cudaFree(hist);
    return cuda_fail(e, "trace growth");
  }
  if (h->em) cudaFree(h->em);
  if (h->hist) cudaFree(h->hist);
  h->em = em;
  h->hist = hist;
  h->cap = ncap;
  return SW_OK;
}

// Synchronise the handle's stream and turn the device error flag into a status.
int sync_and_check(sw_lattice* h) {
  SW_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
  int flag = 0;
  SW_CUDA(cudaMemcpy(&flag, h->tb.err, sizeof(int), cudaMemcpyDeviceToHost), "error flag read");
  switch (flag) {
    case sw::kErrNone: return SW_OK;
    case sw::kErrUnionCap: return fail(SW_ETIMEOUT, "device union-find retry loop reached its cap");
    case sw::kErrBadSpin:
      // the state is valid again (the previous spins were kept): report once
      SW_CUDA(cudaMemset(h->tb.err, 0, sizeof(int)), "error flag reset");
      return fail(SW_EINVAL, "sw_set_state: spins contain values other than +1/-1");
    case sw::kErrSlotOverflow: return fail(SW_EDEVICE, "device: tile border slots overflowed");
    case sw::kErrCopyTimeout: return fail(SW_ETIMEOUT, "device: a bulk copy into shared memory did not complete");
    default: return fail(SW_EDEVICE, "device error flag %d", flag);
  }
}

int range_ok(const sw_lattice* h, int64_t first, int64_t count) {
  if (count < 0 || first < h->t_base || first + count > h->t)
    return fail(SW_EINVAL, "sweeps [%lld, %lld) outside the trace [%lld, %lld)", (long long)first,
                (long long)(first + count), (long long)h->t_base, (long long)h->t);
  return SW_OK;
}

// Phases 1-2 for the current state and counter (bonds, tile clusters, merge).
int run_clusters(sw_lattice* h, sw::SweepArgs& a) {
  a.em = nullptr;
  a.hist = nullptr;
  a.csize = nullptr;
  SW_CUDA(sw::launch_phase1(h->shape, a, h->stream), "phase 1 launch");
  SW_CUDA(sw::launch_phase2(h->shape, a, h->stream), "phase 2 launch");
  return SW_OK;
}

}  // namespace

extern "C" {

uint32_t sw_threshold(double beta) {
  if (!beta_ok(beta)) {
    fail(SW_EINVAL, "beta must be finite and >= 0");
    return 0u;
  }
  return threshold_of(beta);
}

const char* sw_last_error(void) { return g_last_error.c_str(); }

int sw_create(int32_t L, double beta, uint64_t seed, int32_t init, void* stream, sw_lattice** out) {
  if (!out) return fail(SW_EINVAL, "out is NULL");
  *out = nullptr;
  if (L < 2 || (int64_t)L * L >= ((int64_t)1 << 31)) return fail(SW_EINVAL, "L=%d outside 2 <= L, L*L < 2^31", L);
  if (!beta_ok(beta)) return fail(SW_EINVAL, "beta must be finite and >= 0");
  if (init != SW_INIT_HOT && init != SW_INIT_COLD) return fail(SW_EINVAL, "init must be SW_INIT_HOT or SW_INIT_COLD");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(SW_ECUDA, "no CUDA device available (libsw has no CPU fallback)");
  }
  sw_lattice* h = new (std::nothrow) sw_lattice();
  if (!h) return fail(SW_ENOMEM, "host allocation failed");
  h->L = L;
  h->beta = beta;
  h->seed = seed;
  h->thr = threshold_of(beta);
  h->shape = shape_for(L, true);
  h->tiles_only = getenv("SW_TILE_SHAPE") != nullptr;
  h->ks = sw::make_key_schedule(seed);
  cudaGetDevice(&h->device);
  const sw::TileShape ts = sw::shape_of(h->shape);
  h->g.L = L;
  h->g.tiles_x = (L + ts.tw() - 1) / ts.tw();
  h->g.tiles_y = (L + ts.th - 1) / ts.th;
  h->g.aligned16 = (L % 16) == 0;
  const size_t ntiles = (size_t)h->g.tiles_x * h->g.tiles_y;
  const size_t N = (size_t)L * L;
  cudaError_t e = cudaSuccess;
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    h->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaMalloc(&h->spins, N);
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.tbits, ntiles * 3 * ts.row_words() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.roots, ntiles * ts.sites() * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.bmask, ntiles * ts.row_words() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.rbits, ntiles * ts.row_words() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.nodes, ntiles * ts.max_slots() * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.bslot, ntiles * ts.boundary_sites() * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.bbits, ntiles * ts.bbits_words() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.nslots, ntiles * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->csize, ntiles * ts.max_slots() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->draws, ntiles * ts.row_words() * sizeof(uint2));
  h->fuse = sw::batch_fused_supported(h->shape);
  if (e == cudaSuccess && h->fuse) e = cudaMalloc(&h->nodes2, ntiles * ts.max_slots() * sizeof(uint64_t));
  if (e == cudaSuccess && h->fuse) e = cudaMalloc(&h->bslot2, ntiles * ts.boundary_sites() * sizeof(uint16_t));
  if (e == cudaSuccess && h->fuse) e = cudaMalloc(&h->nslots2, ntiles * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->tb.err, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) e = sw::launch_init(h->spins, L, seed, init == SW_INIT_COLD, h->stream);
  if (e != cudaSuccess) {
    const int rc = cuda_fail(e, "sw_create");
    free_all(h);
    delete h;
    return rc;
  }
  const int rc = ensure_trace(h, 1024);
  if (rc != SW_OK) {
    free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return SW_OK;
}

int sw_destroy(sw_lattice* h) {
  if (!h) return SW_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
  return SW_OK;
}

int sw_sweep(sw_lattice* h, int32_t n) {
  NvtxRange range("sw_sweep");
  if (!h) return fail(SW_EINVAL, "handle is NULL");
  if (n < 0) return fail(SW_EINVAL, "n must be >= 0");
  if (n == 0) return SW_OK;
  int rc = ensure_trace(h, h->t - h->t_base + n);
  if (rc != SW_OK) return rc;
  const sw::TileShape ts = sw::shape_of(h->shape);
  (void)ts;
  if (h->L <= sw::kSmallSweepMaxL && !h->hist_on && !h->tiles_only) {
    // the whole lattice fits one CTA: all n sweeps in one launch
    sw::SmallArgs s{};
    s.L = h->L;
    s.thr = h->thr;
    s.rule = (uint32_t)h->rule;
    s.t0 = (uint32_t)h->t;
    s.n = n;
    s.ks = h->ks;
    s.spins = h->spins;
    s.em = h->em + 2 * (h->t - h->t_base);
    s.err = h->tb.err;
    SW_CUDA(timed_phase(h, 0, [&] { return sw::launch_small(s, h->stream); }), "small-lattice sweep launch");
    h->t += n;
    return SW_OK;
  }
  // Without statistics and on a shape that has it, phase 3 of a sweep and
  // phase 1 of the next sweep of this call run as one launch (phase31); the
  // call's last sweep runs phase 3 alone, so no work is carried from one
  // call to the next (the caller may change the state in between).
  const bool fused = h->fuse && !h->hist_on;
  bool carried = false;  // phase 1 of the current sweep ran in the previous launch
  for (int32_t k = 0; k < n; ++k) {
    sw::SweepArgs a = args_of(h);
    const int64_t row = h->t - h->t_base;
    a.em = h->em + 2 * row;
    a.hist = h->hist + SW_HIST_WORDS * row;
    a.csize = h->hist_on ? h->csize : nullptr;
    if (!carried)
      SW_CUDA(timed_phase(h, 0, [&] { return sw::launch_phase1(h->shape, a, h->stream); }), "phase 1 launch");
    carried = false;
    // Before the fused launch, the merge phases also draw the next sweep's
    // bonds, which the launch's phase 1 part then reads (phase 1 alone is
    // faster drawing them itself: measured at L = 8192).
    const bool fuse_next = fused && k + 1 < n;
    if (fuse_next) a.draws_out = h->draws;
    SW_CUDA(timed_phase(h, 1, [&] { return sw::launch_phase2(h->shape, a, h->stream); }), "phase 2 launch");
    if (fuse_next) h->draws_t = h->t + 1;
    a.draws_out = nullptr;
    if (!h->hist_on) a.hist = nullptr;
    if (fuse_next) {
      sw::SweepArgs a1 = args_of(h, h->t + 1);
      a1.em = h->em + 2 * (row + 1);  // zeroed by the next sweep's phase 1
      a1.hist = nullptr;
      a1.csize = nullptr;
      SW_CUDA(timed_phase(h, 4, [&] { return sw::launch_phase31(h->shape, a, a1, h->stream); }),
              "phase 3 + next phase 1 launch");
      carried = true;
    } else {
      SW_CUDA(timed_phase(h, 2, [&] { return sw::launch_phase3(h->shape, a, false, h->stream); }), "phase 3 launch");
      if (h->hist_on)
        SW_CUDA(timed_phase(h, 3, [&] { return sw::launch_phase4(h->shape, a, h->stream); }), "phase 4 launch");
    }
    h->t += 1;
  }
  return SW_OK;
}

int sw_get_sweep(sw_lattice* h, uint32_t* t_out) {
  if (!h || !t_out) return fail(SW_EINVAL, "NULL argument");
  *t_out = (uint32_t)h->t;
  return SW_OK;
}

int sw_observables(sw_lattice* h, int64_t first, int64_t count, int64_t* E_host, int64_t* M_host) {
  if (!h) return fail(SW_EINVAL, "handle is NULL");
  int rc = range_ok(h, first, count);
  if (rc != SW_OK) return rc;
  rc = sync_and_check(h);
  if (rc != SW_OK) return rc;
  if (count == 0) return SW_OK;
  int64_t* tmp = (int64_t*)malloc((size_t)count * 2 * sizeof(int64_t));
  if (!tmp) return fail(SW_ENOMEM, "host allocation failed");
  cudaError_t e = cudaMemcpy(tmp, h->em + 2 * (first - h->t_base), (size_t)count * 2 * sizeof(int64_t),
                             cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    free(tmp);
    return cuda_fail(e, "trace copy");
  }
  for (int64_t k = 0; k < count; ++k) {
    if (E_host) E_host[k] = tmp[2 * k];
    if (M_host) M_host[k] = tmp[2 * k + 1];
  }
  free(tmp);
  return SW_OK;
}

int sw_set_rule(sw_lattice* h, int32_t rule) {
  if (!h) return fail(SW_EINVAL, "handle is NULL");
  if (rule != SW_RULE_FLIP && rule != SW_RULE_ASSIGN) return fail(SW_EINVAL, "rule must be SW_RULE_FLIP or SW_RULE_ASSIGN");
  h->rule = rule;
  return SW_OK;
}

int sw_histogram(sw_lattice* h, int32_t enable) {
  if (!h) return fail(SW_EINVAL, "handle is NULL");
  h->hist_on = enable != 0;
  return SW_OK;
}

int sw_histograms(sw_lattice* h, int64_t first, int64_t count, int64_t* out_host) {
  if (!h) return fail(SW_EINVAL, "handle is NULL");
  int rc = range_ok(h, first, count);
  if (rc != SW_OK) return rc;
  if (count > 0 && !out_host) return fail(SW_EINVAL, "out_host is NULL");
  rc = sync_and_check(h);
  if (rc != SW_OK) return rc;
  if (count == 0) return SW_OK;
  SW_CUDA(cudaMemcpy(out_host, h->hist + SW_HIST_WORDS * (first - h->t_base),
                     (size_t)count * SW_HIST_WORDS * sizeof(int64_t), cudaMemcpyDeviceToHost),
          "histogram copy");
  return SW_OK;
}

int sw_labels(sw_lattice* h, int32_t* out, int32_t out_is_device) {
  if (!h || !out) return fail(SW_EINVAL, "NULL argument");
  const size_t N = (size_t)h->L * h->L;
  int32_t* dst = out;
  if (!out_is_device) {
    if (!h->label_buf) SW_CUDA(cudaMalloc(&h->label_buf, N * sizeof(int32_t)), "label buffer");
    dst = h->label_buf;
  }
  sw::SweepArgs a = args_of(h);
  int rc = run_clusters(h, a);
  if (rc != SW_OK) return rc;
  a.labels = dst;
  SW_CUDA(sw::launch_phase3(h->shape, a, true, h->stream), "phase 3 (labels) launch");
  if (out_is_device) return SW_OK;
  SW_CUDA(cudaMemcpyAsync(out, dst, N * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream), "labels copy");
  return sync_and_check(h);
}

int sw_spins(sw_lattice* h, int8_t* out, int32_t out_is_device) {
  if (!h || !out) return fail(SW_EINVAL, "NULL argument");
  const size_t N = (size_t)h->L * h->L;
  SW_CUDA(cudaMemcpyAsync(out, h->spins, N, out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          h->stream),
          "spins copy");
  if (out_is_device) return SW_OK;
  return sync_and_check(h);
}

namespace {

// After an asynchronous host set_state: if this call's check flagged the new
// spins, copy the previous state (now in the staging buffer) back and raise
// kErrBadSpin on the handle's error word unless an earlier error is still
// pending there (first writer wins, so nothing unreported is overwritten).
// Nothing else is done when the flag is clear, so the launch costs a few
// microseconds.
__global__ void restore_if_bad_kernel(int8_t* spins, const int8_t* previous, int64_t n, const int* check,
                                      int* err) {
  if (*reinterpret_cast<const volatile int*>(check) == 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(err, 0, sw::kErrBadSpin);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nv = n / 16;
  uint4* d = reinterpret_cast<uint4*>(spins);
  const uint4* s = reinterpret_cast<const uint4*>(previous);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) d[i] = s[i];
  for (int64_t i = 16 * nv + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) spins[i] = previous[i];
}

}  // namespace

int sw_set_state_async(sw_lattice* h, const int8_t* spins, uint32_t t) {
  if (!h || !spins) return fail(SW_EINVAL, "NULL argument");
  const size_t N = (size_t)h->L * h->L;
  if (!h->staging) SW_CUDA(cudaMalloc(&h->staging, N), "staging buffer");
  if (!h->check_flag) SW_CUDA(cudaMalloc(&h->check_flag, sizeof(int)), "check flag");
  // the check runs on a flag of its own: the handle's error word may still
  // hold an error that no synchronising call has reported yet
  SW_CUDA(cudaMemsetAsync(h->check_flag, 0, sizeof(int), h->stream), "check flag reset");
  SW_CUDA(cudaMemcpyAsync(h->staging, spins, N, cudaMemcpyHostToDevice, h->stream), "spins copy");
  SW_CUDA(sw::launch_check_spins(h->staging, (int64_t)N, h->check_flag, h->stream), "spin check launch");
  int8_t* previous = h->spins;
  h->spins = h->staging;
  h->staging = previous;
  restore_if_bad_kernel<<<4 * 152, 256, 0, h->stream>>>(h->spins, h->staging, (int64_t)N, h->check_flag,
                                                         h->tb.err);
  SW_CUDA(cudaGetLastError(), "restore launch");
  h->t = t;
  h->t_base = t;
  return SW_OK;
}

int sw_set_state(sw_lattice* h, const int8_t* spins, uint32_t t, int32_t in_is_device) {
  if (!h || !spins) return fail(SW_EINVAL, "NULL argument");
  const size_t N = (size_t)h->L * h->L;
  if (in_is_device) {
    SW_CUDA(cudaMemsetAsync(h->tb.err, 0, sizeof(int), h->stream), "error flag reset");
    SW_CUDA(cudaMemcpyAsync(h->spins, spins, N, cudaMemcpyDeviceToDevice, h->stream), "spins copy");
    SW_CUDA(sw::launch_check_spins(h->spins, (int64_t)N, h->tb.err, h->stream), "spin check launch");
  } else {
    if (!h->staging) SW_CUDA(cudaMalloc(&h->staging, N), "staging buffer");
    if (!h->check_flag) SW_CUDA(cudaMalloc(&h->check_flag, sizeof(int)), "check flag");
    SW_CUDA(cudaMemsetAsync(h->check_flag, 0, sizeof(int), h->stream), "check flag reset");
    SW_CUDA(cudaMemcpyAsync(h->staging, spins, N, cudaMemcpyHostToDevice, h->stream), "spins copy");
    SW_CUDA(sw::launch_check_spins(h->staging, (int64_t)N, h->check_flag, h->stream), "spin check launch");
    int bad = 0;
    SW_CUDA(cudaMemcpyAsync(&bad, h->check_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "check flag read");
    SW_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    if (bad) return fail(SW_EINVAL, "sw_set_state: spins contain values other than +1/-1");
    int8_t* old = h->spins;
    h->spins = h->staging;
    h->staging = old;
    SW_CUDA(cudaMemsetAsync(h->tb.err, 0, sizeof(int), h->stream), "error flag reset");
  }
  h->t = t;
  h->t_base = t;
  return SW_OK;
}

int sw_num_shapes(void) { return sw::kNumShapes; }

int sw_shape_info(int32_t shape, int32_t* tile_w, int32_t* tile_h, int32_t* strip_h, int32_t* threads) {
  if (shape < 0 || shape >= sw::kNumShapes) return fail(SW_EINVAL, "unknown tile shape %d", shape);
  const sw::TileShape ts = sw::shape_of(shape);
  if (tile_w) *tile_w = ts.tw();
  if (tile_h) *tile_h = ts.th;
  if (strip_h) *strip_h = ts.h;
  if (threads) *threads = ts.threads();
  return SW_OK;
}

int sw_tune_shape(int32_t log2_bucket, int32_t shape) {
  if (log2_bucket < 0 || log2_bucket >= kBuckets) return fail(SW_EINVAL, "bucket must be in [0, %d)", kBuckets);
  if (shape < -1 || shape >= sw::kNumShapes) return fail(SW_EINVAL, "unknown tile shape %d", shape);
  shape_for(2, true);  // initialise the table
  g_tuned[log2_bucket].store(shape);
  return SW_OK;
}

int sw_lattice_shape(sw_lattice* h, int32_t* shape) {
  if (!h || !shape) return fail(SW_EINVAL, "NULL argument");
  *shape = h->shape;
  return SW_OK;
}

int sw_timing(sw_lattice* h, int32_t enable) {
  if (!h) return fail(SW_EINVAL, "handle is NULL");
  if (enable) {
    SW_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    SW_CUDA(drain_marks(h), "timing events");
    for (int k = 0; k < SW_TIMING_PHASES; ++k) {
      h->phase_ms[k] = 0.0;
      h->phase_launches[k] = 0;
    }
  }
  h->timing_on = enable != 0;
  return SW_OK;
}

int sw_timing_read(sw_lattice* h, double* ms_out, int64_t* launches_out) {
  if (!h) return fail(SW_EINVAL, "handle is NULL");
  SW_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
  SW_CUDA(drain_marks(h), "timing events");
  for (int k = 0; k < SW_TIMING_PHASES; ++k) {
    if (ms_out) ms_out[k] = h->phase_ms[k];
    if (launches_out) launches_out[k] = h->phase_launches[k];
  }
  return SW_OK;
}

int sw_labels_equivalence(sw_lattice* h, int32_t* out, int32_t out_is_device, int32_t* iterations) {
  if (!h || !out) return fail(SW_EINVAL, "NULL argument");
  const size_t N = (size_t)h->L * h->L;
  if (!h->bond_buf) SW_CUDA(cudaMalloc(&h->bond_buf, N), "bond buffer");
  if (!h->ref_buf) SW_CUDA(cudaMalloc(&h->ref_buf, N * sizeof(int32_t)), "reference buffer");
  if (!h->le_flag) SW_CUDA(cudaMalloc(&h->le_flag, sizeof(int)), "iteration flag");
  int32_t* dst = out;
  if (!out_is_device) {
    if (!h->label_buf) SW_CUDA(cudaMalloc(&h->label_buf, N * sizeof(int32_t)), "label buffer");
    dst = h->label_buf;
  }
  sw::SweepArgs a = args_of(h);
  a.em = nullptr;
  a.hist = nullptr;
  a.csize = nullptr;
  SW_CUDA(sw::launch_phase1(h->shape, a, h->stream), "phase 1 launch");
  SW_CUDA(sw::launch_export_bonds(h->shape, a, h->bond_buf, h->stream), "bond export launch");
  int its = 0;
  SW_CUDA(sw::run_label_equivalence(h->bond_buf, h->L, dst, h->ref_buf, h->le_flag, h->tb.err, 1 << 20, &its,
                                    h->stream),
          "label equivalence");
  if (iterations) *iterations = its < 0 ? -its : its;
  if (its < 0) return fail(SW_ETIMEOUT, "label equivalence did not converge within its iteration cap");
  if (!out_is_device)
    SW_CUDA(cudaMemcpyAsync(out, dst, N * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream), "labels copy");
  return sync_and_check(h);
}

int sw_bonds(sw_lattice* h, uint8_t* out_host) {
  if (!h || !out_host) return fail(SW_EINVAL, "NULL argument");
  const size_t N = (size_t)h->L * h->L;
  if (!h->bond_buf) SW_CUDA(cudaMalloc(&h->bond_buf, N), "bond buffer");
  sw::SweepArgs a = args_of(h);
  int rc = run_clusters(h, a);
  if (rc != SW_OK) return rc;
  SW_CUDA(sw::launch_export_bonds(h->shape, a, h->bond_buf, h->stream), "bond export launch");
  SW_CUDA(cudaMemcpyAsync(out_host, h->bond_buf, N, cudaMemcpyDeviceToHost, h->stream), "bonds copy");
  return sync_and_check(h);
}

}  // extern "C"
