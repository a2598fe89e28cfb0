// sw_potts.cu -- Swendsen-Wang sweeps of the q-state Potts model (the
// paper's §6 generalisation), H = -sum over the 2N edges of
// delta(s_i, s_j), states 0..q-1 as int8.
//
// One sweep is four site-parallel kernels over global memory:
//   bonds   a thread per Philox block (site pair, C5 counters): an edge bonds
//           iff its two states are equal and its word < thr, thr from
//           p = 1 - exp(-beta); every site starts as its own root;
//   unite   a thread per site unites the two ends of its east and south
//           bonds (lock-free union-find over int32 parents, the larger root
//           hung under the smaller with atomicMin, path halving), so every
//           root ends as its cluster's smallest site (C9);
//   roots   every site points at its root; each root draws its cluster's
//           new state floor(x0 q / 2^32) from block (root, t, 3, 0);
//   assign  every site takes its root's state; E = -(edges joining equal
//           states) and M = (sites in state 0) are reduced in int64.
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

constexpr int kPottsFindCap = 1 << 24;
constexpr int kPottsUnionCap = 1 << 16;

__device__ __forceinline__ int8_t potts_state(uint32_t x, int q) {
  return (int8_t)(((uint64_t)x * (uint64_t)q) >> 32);
}

__device__ __forceinline__ int pfind(int* par, int x, int* err) {
  for (int it = 0;; ++it) {
    const int p = __ldcg(par + x);
    if (p == x) return x;
    const int gp = __ldcg(par + p);
    if (gp == p) return p;
    if (it >= kPottsFindCap) {
      atomicCAS(err, 0, 1);
      return p;
    }
    atomicMin(par + x, gp);  // halving: x now points at an ancestor
    x = gp;
  }
}

__device__ void punite(int* par, int a, int b, int* err) {
  for (int it = 0; it < kPottsUnionCap; ++it) {
    a = pfind(par, a, err);
    b = pfind(par, b, err);
    if (a == b) return;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicMin(par + a, b);
    if (old == a) return;
    a = old;
  }
  atomicCAS(err, 0, 1);
}

__global__ void potts_init_kernel(int8_t* s, int64_t n, int q, sw::KeySchedule ks, int cold) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s[i] = cold ? (int8_t)0 : potts_state(sw::philox4x32_10(make_uint4((uint32_t)i, 0u, 2u, 0u), ks).x, q);
}

__global__ void potts_check_kernel(const int8_t* s, int64_t n, int q, int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (s[i] < 0 || s[i] >= q) atomicCAS(err, 0, 2);
}

__global__ void potts_bonds_kernel(const int8_t* s, uint8_t* bonds, int* par, int L, uint32_t thr, uint32_t t,
                                   sw::KeySchedule ks, int64_t* em) {
  const int64_t n = (int64_t)L * L;
  const int64_t npairs = (n + 1) / 2;
  if (blockIdx.x == 0 && threadIdx.x < 2) em[threadIdx.x] = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = sw::philox4x32_10(make_uint4((uint32_t)p, t, 0u, 0u), ks);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int64_t i = 2 * p + j;
      if (i >= n) break;
      const int y = (int)(i / L), x = (int)(i - (int64_t)y * L);
      const int8_t si = s[i];
      const int8_t se = s[(int64_t)y * L + (x + 1 == L ? 0 : x + 1)];
      const int8_t ss = s[(int64_t)(y + 1 == L ? 0 : y + 1) * L + x];
      const uint32_t ue = j ? w.z : w.x, us = j ? w.w : w.y;
      bonds[i] = (uint8_t)((si == se && ue < thr ? 1u : 0u) | (si == ss && us < thr ? 2u : 0u));
      par[i] = (int)i;
    }
  }
}

__global__ void potts_unite_kernel(const uint8_t* bonds, int* par, int L, int* err) {
  const int64_t n = (int64_t)L * L;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t b = bonds[i];
    if (!b) continue;
    const int y = (int)(i / L), x = (int)(i - (int64_t)y * L);
    if (b & 1u) punite(par, (int)i, (int)((int64_t)y * L + (x + 1 == L ? 0 : x + 1)), err);
    if (b & 2u) punite(par, (int)i, (int)((int64_t)(y + 1 == L ? 0 : y + 1) * L + x), err);
  }
}

__global__ void potts_roots_kernel(int* par, int8_t* val, int64_t n, int q, uint32_t t, sw::KeySchedule ks,
                                   int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)i, p = __ldcg(par + r);
    for (int it = 0; p != r; ++it) {
      if (it >= kPottsFindCap) {
        atomicCAS(err, 0, 1);
        break;
      }
      r = p;
      p = __ldcg(par + r);
    }
    par[i] = r;  // concurrent stores all write roots
    if (r == (int)i) val[i] = potts_state(sw::philox4x32_10(make_uint4((uint32_t)i, t, 3u, 0u), ks).x, q);
  }
}

__global__ void potts_assign_kernel(int8_t* s, const int* par, const int8_t* val, int L, int64_t* em) {
  const int64_t n = (int64_t)L * L;
  long long e = 0, m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / L), x = (int)(i - (int64_t)y * L);
    const int8_t v = val[par[i]];
    const int8_t ve = val[par[(int64_t)y * L + (x + 1 == L ? 0 : x + 1)]];
    const int8_t vs = val[par[(int64_t)(y + 1 == L ? 0 : y + 1) * L + x]];
    s[i] = v;
    e -= (v == ve) + (v == vs);
    m += v == 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    m += __shfl_xor_sync(0xffffffffu, m, o);
  }
  __shared__ long long red[2][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = e;
    red[1][warp] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long et = 0, mt = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      et += red[0][k];
      mt += red[1][k];
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(em), (unsigned long long)et);
    atomicAdd(reinterpret_cast<unsigned long long*>(em + 1), (unsigned long long)mt);
  }
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
  int8_t* s = nullptr;
  uint8_t* bonds = nullptr;
  int* par = nullptr;
  int8_t* val = nullptr;
  int64_t* em = nullptr;
  int* err = nullptr;
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
  void* ptrs[] = {h->s, h->bonds, h->par, h->val, h->em, h->err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

int check_potts(sw_potts* h) {
  P_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
  int flag = 0;
  P_CUDA(cudaMemcpy(&flag, h->err, sizeof(int), cudaMemcpyDeviceToHost), "error flag read");
  if (flag == 1) return pfail(SW_ETIMEOUT, "a capped union-find loop gave up");
  if (flag == 2) return pfail(SW_EINVAL, "a state outside 0..q-1 was given");
  if (flag != 0) return pfail(SW_EDEVICE, "device error flag set");
  return SW_OK;
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

// Bonds of the current states and counter, clusters to roots.
int clusters(sw_potts* h) {
  const int64_t n = (int64_t)h->L * h->L;
  const uint32_t t = (uint32_t)h->t;
  int64_t* em = h->em + 2 * (h->t - h->t_base);
  potts_bonds_kernel<<<grid_of((n + 1) / 2), 256, 0, h->stream>>>(h->s, h->bonds, h->par, h->L, h->thr, t, h->ks, em);
  potts_unite_kernel<<<grid_of(n), 256, 0, h->stream>>>(h->bonds, h->par, h->L, h->err);
  potts_roots_kernel<<<grid_of(n), 256, 0, h->stream>>>(h->par, h->val, n, h->q, t, h->ks, h->err);
  P_CUDA(cudaGetLastError(), "Potts sweep launch");
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
  const size_t n = (size_t)L * L;
  cudaError_t e = cudaSuccess;
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    h->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaMalloc(&h->s, n);
  if (e == cudaSuccess) e = cudaMalloc(&h->bonds, n);
  if (e == cudaSuccess) e = cudaMalloc(&h->par, n * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->val, n);
  if (e == cudaSuccess) e = cudaMalloc(&h->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
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
  const int64_t N = (int64_t)h->L * h->L;
  for (int32_t k = 0; k < n; ++k) {
    rc = clusters(h);
    if (rc != SW_OK) return rc;
    int64_t* em = h->em + 2 * (h->t - h->t_base);
    potts_assign_kernel<<<grid_of(N), 256, 0, h->stream>>>(h->s, h->par, h->val, h->L, em);
    P_CUDA(cudaGetLastError(), "Potts assign launch");
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
  // staged in the per-sweep value buffer and checked before it replaces the state
  P_CUDA(cudaMemcpyAsync(h->val, states, n, in_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         h->stream),
         "states copy");
  potts_check_kernel<<<grid_of((int64_t)n), 256, 0, h->stream>>>(h->val, (int64_t)n, h->q, h->err);
  P_CUDA(cudaGetLastError(), "state check launch");
  rc = check_potts(h);
  if (rc != SW_OK) {
    cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
    cudaStreamSynchronize(h->stream);
    return rc;
  }
  P_CUDA(cudaMemcpyAsync(h->s, h->val, n, cudaMemcpyDeviceToDevice, h->stream), "states copy");
  h->t = t;
  h->t_base = t;
  return SW_OK;
}

int sw_potts_labels(sw_potts* h, int32_t* out, int32_t out_is_device) {
  if (!h || !out) return pfail(SW_EINVAL, "NULL argument");
  int rc = grow(h, h->t - h->t_base + 1);  // the bonds kernel zeroes the next trace row
  if (rc != SW_OK) return rc;
  rc = clusters(h);
  if (rc != SW_OK) return rc;
  const size_t n = (size_t)h->L * h->L;
  P_CUDA(cudaMemcpyAsync(out, h->par, n * sizeof(int32_t),
                         out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream),
         "labels copy");
  if (out_is_device) return SW_OK;
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
