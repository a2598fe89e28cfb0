// sw_potts.cu -- Swendsen-Wang sweeps of the q-state Potts model (the
// paper's §6 generalisation), H = -sum over the 2N edges of
// delta(s_i, s_j), states 0..q-1 as int8.
//
// A sweep runs on the tiled path of the Ising sweep (tile shape
// kPottsShape, 128 x 64 sites):
//   phase 1  bonds and tile clusters: an edge bonds iff its two states are
//            equal and its word of the site pair's Philox block (C5) is
//            below thr, thr from p = 1 - exp(-beta); then the band-scan
//            tile labelling, border slots and global nodes of the Ising
//            phase 1 (the bond masks are all it looks at);
//   phase 2  the cross-tile merge, and the resolve pass that draws each
//            border cluster's new state floor(x0 q / 2^32), x0 from block
//            (root, t, 3, 0), root its smallest site (C9);
//   phase 3  inner clusters draw their state the same way, every site takes
//            its cluster's, and E = -(edges joining equal states),
//            M = (sites in state 0) are reduced in int64.
// For q = 2 and twice the Ising coupling this is the Ising sweep with the
// assignment rule (C6b), state 1 <-> spin -1.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <new>

#include "sw.h"
#include "sw_internal.h"

namespace {

__device__ __forceinline__ int8_t potts_state(uint32_t x, int q) {
  return (int8_t)(((uint64_t)x * (uint64_t)q) >> 32);
}

// C7 for Potts: site i starts in state floor(x0 q / 2^32), x0 the first word
// of block (i, 0, 2, 0) (hot), or in state 0 (cold).
__global__ void potts_init_kernel(int8_t* s, int64_t n, int q, sw::KeySchedule ks, int cold) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s[i] = cold ? (int8_t)0 : potts_state(sw::philox4x32_10(make_uint4((uint32_t)i, 0u, 2u, 0u), ks).x, q);
}

__global__ void potts_check_kernel(const int8_t* s, int64_t n, int q, int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (s[i] < 0 || s[i] >= q) atomicCAS(err, 0, sw::kErrBadSpin);
}

int grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152LL * 16) g = 152LL * 16;
  return (int)(g < 1 ? 1 : g);
}

thread_local char g_msg[256];

int pfail(int code, const char* what) { return sw::record_error(code, what); }

}  // namespace

struct sw_potts {
  int L = 0, q = 0;
  uint32_t thr = 0;
  sw::KeySchedule ks{};
  int64_t t = 0, t_base = 0, cap = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  sw::Geometry g{};
  sw::TileBuffers tb{};
  int8_t* s = nullptr;        // states [L][L]
  int8_t* staging = nullptr;  // sw_potts_set_state's checked copy
  int32_t* label_buf = nullptr;
  int64_t* em = nullptr;      // [cap][2]
};

namespace {

#define P_CUDA(call, what)                                                          \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      snprintf(g_msg, sizeof g_msg, "%s: %s", what, cudaGetErrorString(e_));        \
      return pfail(e_ == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA, g_msg); \
    }                                                                               \
  } while (0)

void free_potts(sw_potts* h) {
  void* ptrs[] = {h->s,         h->staging,   h->label_buf,  h->em,       h->tb.tbits, h->tb.roots,
                  h->tb.bmask,  h->tb.rbits,  h->tb.nodes,   h->tb.bslot, h->tb.bbits, h->tb.nslots,
                  h->tb.err,    h->tb.nval};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// Synchronise and turn the device error flag into a status.
int check_potts(sw_potts* h) {
  P_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
  int flag = 0;
  P_CUDA(cudaMemcpy(&flag, h->tb.err, sizeof(int), cudaMemcpyDeviceToHost), "error flag read");
  switch (flag) {
    case sw::kErrNone: return SW_OK;
    case sw::kErrUnionCap: return pfail(SW_ETIMEOUT, "a capped union-find loop gave up");
    case sw::kErrBadSpin:
      // the state was not replaced: report once
      P_CUDA(cudaMemset(h->tb.err, 0, sizeof(int)), "error flag reset");
      return pfail(SW_EINVAL, "a state outside 0..q-1 was given");
    case sw::kErrSlotOverflow: return pfail(SW_EDEVICE, "device: tile border slots overflowed");
    case sw::kErrCopyTimeout: return pfail(SW_ETIMEOUT, "device: a bulk copy into shared memory did not complete");
    default: return pfail(SW_EDEVICE, "device error flag set");
  }
}

int grow(sw_potts* h, int64_t need) {
  if (need <= h->cap) return SW_OK;
  int64_t ncap = h->cap ? h->cap : 1024;
  while (ncap < need) ncap *= 2;
  int64_t* em = nullptr;
  P_CUDA(cudaMalloc(&em, (size_t)ncap * 2 * sizeof(int64_t)), "trace growth");
  if (h->cap) {
    cudaError_t e = cudaMemcpyAsync(em, h->em, (size_t)h->cap * 2 * sizeof(int64_t), cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      cudaFree(em);
      P_CUDA(e, "trace growth");
    }
    cudaFree(h->em);
  }
  h->em = em;
  h->cap = ncap;
  return SW_OK;
}

uint32_t potts_thr(double beta) {
  const double p = -expm1(-beta);
  const double scaled = floor(ldexp(p, 32));
  if (scaled >= 4294967295.0) return 0xffffffffu;
  return (uint32_t)scaled;
}

sw::SweepArgs args_of(const sw_potts* h) {
  sw::SweepArgs a{};
  a.g = h->g;
  a.thr = h->thr;
  a.t = (uint32_t)h->t;
  a.rule = SW_RULE_ASSIGN;
  a.q = (uint32_t)h->q;
  a.ks = h->ks;
  a.tb = h->tb;
  a.spins_in = h->s;
  a.spins_out = h->s;
  return a;
}

// Phases 1-2 of the current states and counter: bonds, tile clusters, the
// merge and each border cluster's new state.
int clusters(sw_potts* h, const sw::SweepArgs& a) {
  P_CUDA(sw::launch_potts_phase1(a, h->stream), "Potts phase 1 launch");
  P_CUDA(sw::launch_phase2(sw::kPottsShape, a, h->stream), "Potts phase 2 launch");
  return SW_OK;
}

}  // namespace

extern "C" {

uint32_t sw_potts_threshold(double beta) {
  if (!(beta >= 0.0) || isinf(beta)) return 0u;
  return potts_thr(beta);
}

int sw_potts_create(int32_t L, int32_t q, double beta, uint64_t seed, int32_t init, void* stream, sw_potts** out) {
  if (!out) return pfail(SW_EINVAL, "out is NULL");
  *out = nullptr;
  if (L < 2 || (int64_t)L * L >= ((int64_t)1 << 31)) return pfail(SW_EINVAL, "L outside 2 <= L, L*L < 2^31");
  if (q < 2 || q > 127) return pfail(SW_EINVAL, "q must be in 2..127");
  if (!(beta >= 0.0) || isinf(beta)) return pfail(SW_EINVAL, "beta must be finite and >= 0");
  if (init != SW_INIT_HOT && init != SW_INIT_COLD) return pfail(SW_EINVAL, "init must be SW_INIT_HOT or SW_INIT_COLD");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return pfail(SW_ECUDA, "no CUDA device available (libsw has no CPU fallback)");
  }
  sw_potts* h = new (std::nothrow) sw_potts();
  if (!h) return pfail(SW_ENOMEM, "host allocation failed");
  h->L = L;
  h->q = q;
  h->thr = potts_thr(beta);
  h->ks = sw::make_key_schedule(seed);
  const sw::TileShape ts = sw::shape_of(sw::kPottsShape);
  h->g.L = L;
  h->g.tiles_x = (L + ts.tw() - 1) / ts.tw();
  h->g.tiles_y = (L + ts.th - 1) / ts.th;
  h->g.aligned16 = (L % 16) == 0;
  const size_t ntiles = (size_t)h->g.tiles_x * h->g.tiles_y;
  const size_t n = (size_t)L * L;
  cudaError_t e = cudaSuccess;
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    h->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaMalloc(&h->s, n);
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.tbits, ntiles * 3 * ts.row_words() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.roots, ntiles * ts.sites() * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.bmask, ntiles * ts.row_words() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.rbits, ntiles * ts.row_words() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.nodes, ntiles * ts.max_slots() * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.bslot, ntiles * ts.boundary_sites() * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.bbits, ntiles * ts.bbits_words() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.nslots, ntiles * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.nval, ntiles * ts.max_slots());
  if (e == cudaSuccess) e = cudaMalloc(&h->tb.err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->tb.err, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) {
    potts_init_kernel<<<grid_of((int64_t)n), 256, 0, h->stream>>>(h->s, (int64_t)n, q, h->ks, init == SW_INIT_COLD);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    snprintf(g_msg, sizeof g_msg, "sw_potts_create: %s", cudaGetErrorString(e));
    free_potts(h);
    delete h;
    return pfail(e == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA, g_msg);
  }
  const int rc = grow(h, 1024);
  if (rc != SW_OK) {
    free_potts(h);
    delete h;
    return rc;
  }
  *out = h;
  return SW_OK;
}

int sw_potts_sweep(sw_potts* h, int32_t n) {
  if (!h) return pfail(SW_EINVAL, "handle is NULL");
  if (n < 0) return pfail(SW_EINVAL, "n must be >= 0");
  int rc = grow(h, h->t - h->t_base + n);
  if (rc != SW_OK) return rc;
  for (int32_t k = 0; k < n; ++k) {
    sw::SweepArgs a = args_of(h);
    a.em = h->em + 2 * (h->t - h->t_base);  // zeroed by phase 1
    rc = clusters(h, a);
    if (rc != SW_OK) return rc;
    P_CUDA(sw::launch_potts_phase3(a, h->stream), "Potts phase 3 launch");
    h->t += 1;
  }
  return SW_OK;
}

int sw_potts_observables(sw_potts* h, int64_t first, int64_t count, int64_t* E_host, int64_t* M_host) {
  if (!h) return pfail(SW_EINVAL, "handle is NULL");
  if (count < 0 || first < h->t_base || first + count > h->t) return pfail(SW_EINVAL, "sweep range outside the trace");
  int rc = check_potts(h);
  if (rc != SW_OK) return rc;
  if (count == 0) return SW_OK;
  int64_t* buf = (int64_t*)malloc((size_t)count * 2 * sizeof(int64_t));
  if (!buf) return pfail(SW_ENOMEM, "host allocation failed");
  cudaError_t e = cudaMemcpy(buf, h->em + 2 * (first - h->t_base), (size_t)count * 2 * sizeof(int64_t),
                             cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    for (int64_t k = 0; k < count; ++k) {
      if (E_host) E_host[k] = buf[2 * k];
      if (M_host) M_host[k] = buf[2 * k + 1];
    }
  }
  free(buf);
  P_CUDA(e, "trace copy");
  return SW_OK;
}

int sw_potts_states(sw_potts* h, int8_t* out, int32_t out_is_device) {
  if (!h || !out) return pfail(SW_EINVAL, "NULL argument");
  const size_t n = (size_t)h->L * h->L;
  P_CUDA(cudaMemcpyAsync(out, h->s, n, out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream),
         "states copy");
  if (out_is_device) return SW_OK;
  return check_potts(h);
}

int sw_potts_set_state(sw_potts* h, const int8_t* states, uint32_t t, int32_t in_is_device) {
  if (!h || !states) return pfail(SW_EINVAL, "NULL argument");
  const size_t n = (size_t)h->L * h->L;
  int rc = check_potts(h);
  if (rc != SW_OK) return rc;
  if (!h->staging) P_CUDA(cudaMalloc(&h->staging, n), "staging buffer");
  // checked in the staging buffer before it replaces the state
  P_CUDA(cudaMemcpyAsync(h->staging, states, n, in_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         h->stream),
         "states copy");
  potts_check_kernel<<<grid_of((int64_t)n), 256, 0, h->stream>>>(h->staging, (int64_t)n, h->q, h->tb.err);
  P_CUDA(cudaGetLastError(), "state check launch");
  rc = check_potts(h);
  if (rc != SW_OK) return rc;
  P_CUDA(cudaMemcpyAsync(h->s, h->staging, n, cudaMemcpyDeviceToDevice, h->stream), "states copy");
  h->t = t;
  h->t_base = t;
  return SW_OK;
}

int sw_potts_labels(sw_potts* h, int32_t* out, int32_t out_is_device) {
  if (!h || !out) return pfail(SW_EINVAL, "NULL argument");
  const size_t n = (size_t)h->L * h->L;
  int32_t* dst = out;
  if (!out_is_device) {
    if (!h->label_buf) P_CUDA(cudaMalloc(&h->label_buf, n * sizeof(int32_t)), "label buffer");
    dst = h->label_buf;
  }
  sw::SweepArgs a = args_of(h);
  int rc = clusters(h, a);
  if (rc != SW_OK) return rc;
  a.labels = dst;
  P_CUDA(sw::launch_phase3(sw::kPottsShape, a, true, h->stream), "labels launch");
  if (out_is_device) return SW_OK;
  P_CUDA(cudaMemcpyAsync(out, dst, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream), "labels copy");
  return check_potts(h);
}

int sw_potts_get_sweep(sw_potts* h, uint32_t* t_out) {
  if (!h || !t_out) return pfail(SW_EINVAL, "NULL argument");
  *t_out = (uint32_t)h->t;
  return SW_OK;
}

int sw_potts_destroy(sw_potts* h) {
  if (!h) return SW_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_potts(h);
  delete h;
  return SW_OK;
}

}  // extern "C"
