// sw_noalloc.cu -- sw_sweep_noalloc: the Swendsen-Wang sweep for callers
// that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: a host application or framework
// whose own allocator has already reserved the GPU's memory and hands out
// nothing else, a plugin host that forbids device allocation, or a loop on a
// latency-critical path where cudaMalloc's implicit device-wide
// synchronisation is not acceptable. For them this entry point runs the same
// three sweep kernels as sw_sweep, on spins, an E/M output and an error word
// that the caller owns, with the kernels' working buffers taken from one
// file-scope device array instead of from allocations. A lattice of side at
// most 181 needs no buffers at all: it is swept inside one CTA's shared
// memory (sw_small.cu).
//
// The array is a static __device__ object, so every GPU that loads the
// library holds it (kNoallocScratchBytes, under 4 MiB) until the process
// exits. Its name in host code is only a host-side stand-in for the device
// object; the device address is obtained once per device with
// cudaGetSymbolAddress and passed to the kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "sw.h"
#include "sw_internal.h"

namespace {

constexpr int kNoallocShape = 6;  // 128 x 64 tiles, 2-row strips, as sw_sweep uses for L > 64
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct ScratchLayout {
  size_t tbits, roots, bmask, rbits, nodes, bslot, bbits, nslots, total;
};

// Buffer sizes of the tile pipeline (as sw_create allocates them) for side L;
// `threads` counts row-words (one 32-bit word per row per word column).
constexpr ScratchLayout layout_for(int L) {
  constexpr int th = sw::shape_of(kNoallocShape).th;
  constexpr int tw = 32 * sw::shape_of(kNoallocShape).wpr;
  constexpr int threads = (tw / 32) * th;
  constexpr int slots = 2 * (tw + th);
  constexpr int border = 2 * th + 2 * tw;
  constexpr int bbits = 2 * (th / 32) + 2 * (tw / 32);
  const size_t ntiles = (size_t)((L + tw - 1) / tw) * (size_t)((L + th - 1) / th);
  ScratchLayout s{};
  s.tbits = 0;
  s.roots = s.tbits + align256(ntiles * 3 * threads * sizeof(uint32_t));
  s.bmask = s.roots + align256(ntiles * (size_t)tw * th * sizeof(uint16_t));
  s.rbits = s.bmask + align256(ntiles * threads * sizeof(uint32_t));
  s.nodes = s.rbits + align256(ntiles * threads * sizeof(uint32_t));
  s.bslot = s.nodes + align256(ntiles * slots * sizeof(uint64_t));
  s.bbits = s.bslot + align256(ntiles * border * sizeof(uint16_t));
  s.nslots = s.bbits + align256(ntiles * bbits * sizeof(uint32_t));
  s.total = s.nslots + align256(ntiles * sizeof(int32_t));
  return s;
}

constexpr size_t kNoallocScratchBytes = layout_for(SW_NOALLOC_MAX_L).total;

// The kernels' working buffers for every call on this device.
static __device__ __align__(256) unsigned char g_sweep_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sweep_scratch on the current device, looked up on the
// first call for that device.
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sweep_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

uint32_t threshold_for(double beta) {
  const double p = -expm1(-2.0 * beta);
  const double scaled = floor(ldexp(p, 32));
  if (scaled >= 4294967295.0) return 0xffffffffu;
  return (uint32_t)scaled;
}

}  // namespace

extern "C" int sw_sweep_noalloc(int8_t* spins, int32_t L, double beta, uint64_t seed, uint32_t t0, int32_t n,
                                int64_t* em, int32_t* err, void* stream) {
  if (!spins || !em || !err) return sw::record_error(SW_EINVAL, "sw_sweep_noalloc: NULL pointer argument");
  if (L < 2 || L > SW_NOALLOC_MAX_L)
    return sw::record_error(SW_EINVAL, "sw_sweep_noalloc: L must be in [2, SW_NOALLOC_MAX_L = 1024]");
  if (!(beta >= 0.0) || isinf(beta)) return sw::record_error(SW_EINVAL, "sw_sweep_noalloc: beta must be finite and >= 0");
  if (n < 0) return sw::record_error(SW_EINVAL, "sw_sweep_noalloc: n must be >= 0");
  cudaStream_t st0 = (cudaStream_t)stream;
  if (L <= sw::kSmallMaxL) {
    // the whole lattice fits one CTA's shared memory: no scratch at all
    sw::SmallArgs s{};
    s.L = L;
    s.thr = threshold_for(beta);
    s.rule = 0;
    s.t0 = t0;
    s.n = n;
    s.ks = sw::make_key_schedule(seed);
    s.spins = spins;
    s.em = em;
    s.err = err;
    cudaError_t e0 = cudaMemsetAsync(err, 0, sizeof(int32_t), st0);
    if (e0 == cudaSuccess) e0 = sw::launch_small(s, st0);
    if (e0 != cudaSuccess) return sw::record_error(SW_ECUDA, cudaGetErrorString(e0));
    return SW_OK;
  }
  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return sw::record_error(SW_ECUDA, cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)stream;
  const ScratchLayout lay = layout_for(L);
  const sw::TileShape ts = sw::shape_of(kNoallocShape);
  static_assert(layout_for(SW_NOALLOC_MAX_L).total < (4u << 20), "scratch must stay under 4 MiB");

  sw::SweepArgs a{};
  a.g.L = L;
  a.g.tiles_x = (L + ts.tw() - 1) / ts.tw();
  a.g.tiles_y = (L + ts.th - 1) / ts.th;
  a.g.aligned16 = (L % 16) == 0 && ((uintptr_t)spins % 16) == 0;
  a.thr = threshold_for(beta);
  a.ks = sw::make_key_schedule(seed);
  a.tb.tbits = reinterpret_cast<uint32_t*>(base + lay.tbits);
  a.tb.roots = reinterpret_cast<uint16_t*>(base + lay.roots);
  a.tb.bmask = reinterpret_cast<uint32_t*>(base + lay.bmask);
  a.tb.rbits = reinterpret_cast<uint32_t*>(base + lay.rbits);
  a.tb.nodes = reinterpret_cast<uint64_t*>(base + lay.nodes);
  a.tb.bslot = reinterpret_cast<uint16_t*>(base + lay.bslot);
  a.tb.bbits = reinterpret_cast<uint32_t*>(base + lay.bbits);
  a.tb.nslots = reinterpret_cast<int32_t*>(base + lay.nslots);
  a.tb.err = err;
  a.spins_in = spins;
  a.spins_out = spins;
  // Every scratch word a sweep reads is written earlier in the same sweep, so
  // only the caller's error word has to start at zero.
  e = cudaMemsetAsync(err, 0, sizeof(int32_t), st);
  for (int32_t k = 0; k < n && e == cudaSuccess; ++k) {
    a.t = t0 + (uint32_t)k;
    a.em = em + 2 * (size_t)k;
    e = sw::launch_phase1(kNoallocShape, a, st);
    if (e == cudaSuccess) e = sw::launch_phase2(kNoallocShape, a, st);
    if (e == cudaSuccess) e = sw::launch_phase3(kNoallocShape, a, false, st);
  }
  if (e != cudaSuccess) return sw::record_error(SW_ECUDA, cudaGetErrorString(e));
  return SW_OK;
}
