// sw_phi4.cu -- the multicluster update of the O(4) phi^4 theory in four
// dimensions (the paper's §3, Eqs. 2 and 3), conventions O1-O5 of
// include/sw.h.
//
// One update at counter t:
//   host      the direction r, uniform on the 3-sphere (O3), by rejection
//             from Philox blocks, computed on the host;
//   project   a thread per site: a_x = phi_x . r; every site starts as its
//             own root;
//   bonds     a thread per site draws the words of block (x, t, 4, 0) and
//             bonds its four forward edges (Eq. 2): none unless the two
//             projections have the same sign, else iff w < (1 - e^{-z}) 2^32
//             with z = 4 kappa a_x a_y; the exponential is this file's own
//             (range reduction and a Taylor polynomial with fused
//             multiply-adds), so the decisions are reproducible bit for bit;
//   unite     lock-free union-find over int32 parents (larger root under the
//             smaller with atomicMin), so roots are the clusters' smallest
//             sites;
//   roots     every site points at its root; each root draws its flip
//             (bit 31 of word 0 of block (root, t, 6, 0));
//   reflect   every site of a flipped cluster is reflected in the hyperplane
//             orthogonal to r (Eq. 3): phi <- phi - 2 (phi . r) r;
//   observe   E = sum over the 4N edges of phi_x . phi_{x+mu} and M = sum of
//             phi, reduced in binary64 (the summation order differs from a
//             serial sum, so these agree with one to rounding only).
// Every operation that feeds a bond decision or a new field value is an
// explicitly rounded intrinsic, so nothing is contracted differently from a
// serial restatement compiled without contraction.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cmath>
#include <new>

#include "sw.h"
#include "sw_internal.h"

namespace {

constexpr int kFindCap = 1 << 24;
constexpr int kUnionCap = 1 << 16;

struct Dir {
  double r[4];
};

// One site's field, binary64 x 4 (O1), 32-byte aligned.
struct __align__(32) F4 {
  double x, y, z, w;
};

// e^{-z} for 0 <= z <= 40 (0 beyond, where 1 - e^{-z} rounds to 1): z =
// n ln2 + r with a 32-bit head of ln2 (n * head exact) and its tail (Cody
// and Waite), e^{-r} by the Taylor series to degree 14 with fused
// multiply-adds (remainder below 2^-60 for |r| <= 0.35), then 2^-n.
__device__ double exp_neg(double z) {
  constexpr double kLn2Head = 0x1.62e42feep-1;
  constexpr double kLn2Tail = 0x1.a39ef35793c76p-33;
  constexpr double kInvLn2 = 0x1.71547652b82fep+0;
  constexpr double kInvFact[15] = {0x1p+0,
                                   0x1p+0,
                                   0x1p-1,
                                   0x1.5555555555555p-3,
                                   0x1.5555555555555p-5,
                                   0x1.1111111111111p-7,
                                   0x1.6c16c16c16c17p-10,
                                   0x1.a01a01a01a01ap-13,
                                   0x1.a01a01a01a01ap-16,
                                   0x1.71de3a556c734p-19,
                                   0x1.27e4fb7789f5cp-22,
                                   0x1.ae64567f544e4p-26,
                                   0x1.1eed8eff8d898p-29,
                                   0x1.6124613a86d09p-33,
                                   0x1.93974a8c07c9dp-37};
  if (z > 40.0) return 0.0;
  const double n = floor(__dadd_rn(__dmul_rn(z, kInvLn2), 0.5));
  const double r = __fma_rn(-n, kLn2Tail, __fma_rn(-n, kLn2Head, z));
  double p = kInvFact[14];
#pragma unroll
  for (int k = 13; k >= 0; --k) p = __fma_rn(p, -r, kInvFact[k]);
  return ldexp(p, -(int)n);
}

__device__ __forceinline__ double proj(const F4 f, const Dir& d) {
  return __fma_rn(f.w, d.r[3], __fma_rn(f.z, d.r[2], __fma_rn(f.y, d.r[1], __dmul_rn(f.x, d.r[0]))));
}

// The coordinates of site x = c0 + L c1 + L^2 c2 + L^3 c3 (O2); L^4 < 2^31,
// so 32-bit arithmetic holds every index.
struct Coords {
  uint32_t c[4];
};
__device__ __forceinline__ Coords coords_of(uint32_t x, uint32_t L) {
  Coords k;
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    const uint32_t q = x / L;
    k.c[mu] = x - q * L;
    x = q;
  }
  k.c[3] = x;
  return k;
}

// The forward neighbour of x in direction mu (periodic), stride = L^mu.
__device__ __forceinline__ uint32_t nb(uint32_t x, int mu, const Coords& k, uint32_t L, uint32_t stride) {
  return k.c[mu] == L - 1 ? x - (L - 1) * stride : x + stride;
}

// The bond decision of Eq. 2 for the edge (x, y): bonded iff q = a_x a_y > 0
// and w < (1 - e^{-z}) 2^32 with z = k4 q, all in binary64 with exp_neg.
// GB300 runs binary64 at a small fraction of its binary32 rate, so a
// binary32 estimate decides first, from the projections rounded to binary32
// (af, each within 2^-24 relative): with both |af| >= 2^-60 the binary64
// product is positive exactly when the signs agree, z in binary32 (three
// roundings of 2^-24 and two products) is within 5 * 2^-24 relative, so
// e^{-z} from expf (2 ulp) is within 40 * 5 * 2^-24 + 2^-22 of the binary64
// value for z <= 40, and (1 - e) 2^32 is then within 2^16 of the binary64
// threshold. A word more than 2^18 from the estimate takes the same decision
// as the binary64 test; the others (about 1e-4 of the edges), edges with a
// tiny projection and z near 40 take the binary64 test itself.
__device__ __forceinline__ bool bonded_exact(double ax, double ay, double k4, uint32_t w) {
  const double q = __dmul_rn(ax, ay);
  if (!(q > 0.0)) return false;
  const double e = exp_neg(__dmul_rn(k4, q));
  return __uint2double_rn(w) < __dmul_rn(__dsub_rn(1.0, e), 0x1p32);
}

__device__ __forceinline__ bool bonded(const double* a, uint32_t x, uint32_t y, float fx, float fy, float k4f,
                                       double k4, uint32_t w) {
  const float mx = fabsf(fx), my = fabsf(fy);
  if (mx >= 0x1p-60f && my >= 0x1p-60f) {
    if ((__float_as_uint(fx) ^ __float_as_uint(fy)) >> 31) return false;  // opposite signs: q < 0
    const float zf = __fmul_rn(__fmul_rn(k4f, mx), my);
    if (zf > 40.01f) return true;  // z > 40: e^{-z} is 0 in exp_neg, the threshold 2^32
    if (zf < 39.99f) {
      const float tf = __fmul_rn(__fsub_rn(1.0f, expf(-zf)), 0x1p32f);
      const float wf = (float)w;  // within 2^8 of w
      if (wf < tf - 0x1p18f) return true;
      if (wf > tf + 0x1p18f) return false;
    }
  }
  return bonded_exact(a[x], a[y], k4, w);
}

__device__ __forceinline__ double unit_interval(uint32_t w) {
  return __dsub_rn(__dmul_rn(__dadd_rn(__uint2double_rn(w), 0.5), 0x1p-31), 1.0);
}

__device__ int find_root(int* par, int x, int* err) {
  for (int it = 0;; ++it) {
    const int p = __ldcg(par + x);
    if (p == x) return x;
    const int gp = __ldcg(par + p);
    if (gp == p) return p;
    if (it >= kFindCap) {
      atomicCAS(err, 0, 1);
      return p;
    }
    atomicMin(par + x, gp);
    x = gp;
  }
}

__device__ void unite(int* par, int a, int b, int* err) {
  for (int it = 0; it < kUnionCap; ++it) {
    a = find_root(par, a, err);
    b = find_root(par, b, err);
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

#define GRID_LOOP(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void phi4_init_kernel(F4* phi, int64_t n, sw::KeySchedule ks, int cold) {
  GRID_LOOP(x, n) {
    if (cold) {
      phi[x] = F4{1.0, 0.0, 0.0, 0.0};
    } else {
      const uint4 w = sw::philox4x32_10(make_uint4((uint32_t)x, 0u, 7u, 0u), ks);
      phi[x] = F4{unit_interval(w.x), unit_interval(w.y), unit_interval(w.z), unit_interval(w.w)};
    }
  }
}

// The projections in binary64 and, for the bond kernel's first test, rounded
// to binary32.
__global__ void phi4_project_kernel(const F4* phi, double* a, float* af, int* par, int64_t n, Dir d) {
  GRID_LOOP(x, n) {
    const double v = proj(phi[x], d);
    a[x] = v;
    af[x] = __double2float_rn(v);
    par[x] = (int)x;
  }
}

__global__ void phi4_bonds_kernel(const double* a, const float* af, uint8_t* bonds, int L, int64_t n, double k4,
                                  uint32_t t, sw::KeySchedule ks) {
  const float k4f = __double2float_rn(k4);
  GRID_LOOP(i, n) {
    const uint32_t x = (uint32_t)i;
    const Coords k = coords_of(x, (uint32_t)L);
    const uint4 w4 = sw::philox4x32_10(make_uint4(x, t, 4u, 0u), ks);
    const uint32_t w[4] = {w4.x, w4.y, w4.z, w4.w};
    const float fx = af[x];
    uint8_t b = 0;
    uint32_t stride = 1;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const uint32_t y = nb(x, mu, k, (uint32_t)L, stride);
      if (bonded(a, x, y, fx, af[y], k4f, k4, w[mu])) b |= (uint8_t)(1u << mu);
      stride *= (uint32_t)L;
    }
    bonds[x] = b;
  }
}

__global__ void phi4_unite_kernel(const uint8_t* bonds, int* par, int L, int64_t n, int* err) {
  GRID_LOOP(i, n) {
    const uint32_t x = (uint32_t)i;
    const uint8_t b = bonds[x];
    if (!b) continue;
    const Coords k = coords_of(x, (uint32_t)L);
    uint32_t stride = 1;
    for (int mu = 0; mu < 4; ++mu) {
      if ((b >> mu) & 1u) unite(par, (int)x, (int)nb(x, mu, k, (uint32_t)L, stride), err);
      stride *= (uint32_t)L;
    }
  }
}

__global__ void phi4_roots_kernel(int* par, uint8_t* flip, int64_t n, uint32_t t, sw::KeySchedule ks, int* err) {
  GRID_LOOP(x, n) {
    int r = (int)x, p = __ldcg(par + r);
    for (int it = 0; p != r; ++it) {
      if (it >= kFindCap) {
        atomicCAS(err, 0, 1);
        break;
      }
      r = p;
      p = __ldcg(par + r);
    }
    par[x] = r;  // concurrent stores all write roots
    if (r == (int)x) flip[x] = (uint8_t)(sw::philox4x32_10(make_uint4((uint32_t)x, t, 6u, 0u), ks).x >> 31);
  }
}

__global__ void phi4_reflect_kernel(F4* phi, const double* a, const int* par, const uint8_t* flip, int64_t n,
                                    Dir d) {
  GRID_LOOP(x, n) {
    if (!flip[par[x]]) continue;
    const double m2a = __dmul_rn(-2.0, a[x]);
    F4 f = phi[x];
    f.x = __fma_rn(m2a, d.r[0], f.x);
    f.y = __fma_rn(m2a, d.r[1], f.y);
    f.z = __fma_rn(m2a, d.r[2], f.z);
    f.w = __fma_rn(m2a, d.r[3], f.w);
    phi[x] = f;
  }
}

__global__ void phi4_observe_kernel(const F4* phi, int L, int64_t n, double* out /* E, M0..M3 */) {
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  GRID_LOOP(i, n) {
    const uint32_t x = (uint32_t)i;
    const Coords k = coords_of(x, (uint32_t)L);
    const F4 f = phi[x];
    uint32_t stride = 1;
    for (int mu = 0; mu < 4; ++mu) {
      const F4 g = phi[nb(x, mu, k, (uint32_t)L, stride)];
      v[0] += f.x * g.x + f.y * g.y + f.z * g.z + f.w * g.w;
      stride *= (uint32_t)L;
    }
    v[1] += f.x;
    v[2] += f.y;
    v[3] += f.z;
    v[4] += f.w;
  }
  __shared__ double red[5][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[k][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
    atomicAdd(out + threadIdx.x, s);
  }
}

int grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152LL * 16) g = 152LL * 16;
  return (int)(g < 1 ? 1 : g);
}

thread_local char g_msg[256];

int ffail(int code, const char* what) { return sw::record_error(code, what); }

double unit_interval_host(uint32_t w) { return ((double)w + 0.5) * 0x1p-31 - 1.0; }

}  // namespace

struct sw_phi4 {
  int L = 0;
  int64_t n = 0;
  double kappa = 0.0;
  uint64_t seed = 0;
  sw::KeySchedule ks{};
  int64_t t = 0, t_base = 0, cap = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  F4* phi = nullptr;
  double* a = nullptr;
  float* af = nullptr;  // the projections rounded to binary32 (the bond kernel's first test)
  int* par = nullptr;
  uint8_t* bonds = nullptr;
  uint8_t* flip = nullptr;
  double* obs = nullptr;  // [cap][5]: E, M0..M3
  int* err = nullptr;
};

namespace {

#define F_CUDA(call, what)                                                          \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      snprintf(g_msg, sizeof g_msg, "%s: %s", what, cudaGetErrorString(e_));        \
      return ffail(e_ == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA, g_msg); \
    }                                                                               \
  } while (0)

void free_phi4(sw_phi4* h) {
  void* ptrs[] = {h->phi, h->a, h->af, h->par, h->bonds, h->flip, h->obs, h->err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

int check_phi4(sw_phi4* h) {
  F_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
  int flag = 0;
  F_CUDA(cudaMemcpy(&flag, h->err, sizeof(int), cudaMemcpyDeviceToHost), "error flag read");
  if (flag == 1) return ffail(SW_ETIMEOUT, "a capped union-find loop gave up");
  if (flag != 0) return ffail(SW_EDEVICE, "device error flag set");
  return SW_OK;
}

int grow(sw_phi4* h, int64_t need) {
  if (need <= h->cap) return SW_OK;
  int64_t ncap = h->cap ? h->cap : 1024;
  while (ncap < need) ncap *= 2;
  double* obs = nullptr;
  F_CUDA(cudaMalloc(&obs, (size_t)ncap * 5 * sizeof(double)), "trace growth");
  if (h->cap) {
    cudaError_t e = cudaMemcpyAsync(obs, h->obs, (size_t)h->cap * 5 * sizeof(double), cudaMemcpyDeviceToDevice,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      cudaFree(obs);
      F_CUDA(e, "trace growth");
    }
    cudaFree(h->obs);
  }
  h->obs = obs;
  h->cap = ncap;
  return SW_OK;
}

// O3 on the host: the first attempt k with 2^-20 < |v|^2 <= 1.
int direction(uint64_t seed, uint32_t t, double r[4]) {
  const sw::KeySchedule ks = sw::make_key_schedule(seed);
  for (uint32_t k = 0; k < 1000; ++k) {
    const uint4 w = sw::philox4x32_10(make_uint4(k, t, 5u, 0u), ks);
    const double v[4] = {unit_interval_host(w.x), unit_interval_host(w.y), unit_interval_host(w.z),
                         unit_interval_host(w.w)};
    const double s = std::fma(v[3], v[3], std::fma(v[2], v[2], std::fma(v[1], v[1], v[0] * v[0])));
    if (s <= 1.0 && s > 0x1p-20) {
      const double nrm = std::sqrt(s);
      for (int a = 0; a < 4; ++a) r[a] = v[a] / nrm;
      return 0;
    }
  }
  return -1;
}

// Direction, projections, bonds, clusters and flips of update t.
int clusters(sw_phi4* h, Dir& d) {
  if (direction(h->seed, (uint32_t)h->t, d.r) != 0) return ffail(SW_EDEVICE, "no direction found");
  const int g = grid_of(h->n);
  phi4_project_kernel<<<g, 256, 0, h->stream>>>(h->phi, h->a, h->af, h->par, h->n, d);
  phi4_bonds_kernel<<<g, 256, 0, h->stream>>>(h->a, h->af, h->bonds, h->L, h->n, 4.0 * h->kappa, (uint32_t)h->t,
                                              h->ks);
  phi4_unite_kernel<<<g, 256, 0, h->stream>>>(h->bonds, h->par, h->L, h->n, h->err);
  phi4_roots_kernel<<<g, 256, 0, h->stream>>>(h->par, h->flip, h->n, (uint32_t)h->t, h->ks, h->err);
  F_CUDA(cudaGetLastError(), "phi4 update launch");
  return SW_OK;
}

}  // namespace

extern "C" {

int sw_phi4_direction(uint64_t seed, uint32_t t, double* r_out) {
  if (!r_out) return ffail(SW_EINVAL, "NULL argument");
  if (direction(seed, t, r_out) != 0) return ffail(SW_EDEVICE, "no direction found");
  return SW_OK;
}

int sw_phi4_create(int32_t L, double kappa, uint64_t seed, int32_t init, void* stream, sw_phi4** out) {
  if (!out) return ffail(SW_EINVAL, "out is NULL");
  *out = nullptr;
  if (L < 2 || (int64_t)L * L * L * L >= ((int64_t)1 << 31)) return ffail(SW_EINVAL, "L outside 2 <= L, L^4 < 2^31");
  if (!(kappa >= 0.0) || std::isinf(kappa)) return ffail(SW_EINVAL, "kappa must be finite and >= 0");
  if (init != SW_INIT_HOT && init != SW_INIT_COLD) return ffail(SW_EINVAL, "init must be SW_INIT_HOT or SW_INIT_COLD");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return ffail(SW_ECUDA, "no CUDA device available (libsw has no CPU fallback)");
  }
  sw_phi4* h = new (std::nothrow) sw_phi4();
  if (!h) return ffail(SW_ENOMEM, "host allocation failed");
  h->L = L;
  h->n = (int64_t)L * L * L * L;
  h->kappa = kappa;
  h->seed = seed;
  h->ks = sw::make_key_schedule(seed);
  const size_t n = (size_t)h->n;
  cudaError_t e = cudaSuccess;
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    h->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaMalloc(&h->phi, n * sizeof(F4));
  if (e == cudaSuccess) e = cudaMalloc(&h->a, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->af, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->par, n * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->bonds, n);
  if (e == cudaSuccess) e = cudaMalloc(&h->flip, n);
  if (e == cudaSuccess) e = cudaMalloc(&h->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) {
    phi4_init_kernel<<<grid_of(h->n), 256, 0, h->stream>>>(h->phi, h->n, h->ks, init == SW_INIT_COLD);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    snprintf(g_msg, sizeof g_msg, "sw_phi4_create: %s", cudaGetErrorString(e));
    free_phi4(h);
    delete h;
    return ffail(e == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA, g_msg);
  }
  const int rc = grow(h, 1024);
  if (rc != SW_OK) {
    free_phi4(h);
    delete h;
    return rc;
  }
  *out = h;
  return SW_OK;
}

int sw_phi4_sweep(sw_phi4* h, int32_t n) {
  if (!h) return ffail(SW_EINVAL, "handle is NULL");
  if (n < 0) return ffail(SW_EINVAL, "n must be >= 0");
  int rc = grow(h, h->t - h->t_base + n);
  if (rc != SW_OK) return rc;
  const int g = grid_of(h->n);
  for (int32_t k = 0; k < n; ++k) {
    Dir d;
    rc = clusters(h, d);
    if (rc != SW_OK) return rc;
    double* o = h->obs + 5 * (h->t - h->t_base);
    F_CUDA(cudaMemsetAsync(o, 0, 5 * sizeof(double), h->stream), "trace row");
    phi4_reflect_kernel<<<g, 256, 0, h->stream>>>(h->phi, h->a, h->par, h->flip, h->n, d);
    phi4_observe_kernel<<<g, 256, 0, h->stream>>>(h->phi, h->L, h->n, o);
    F_CUDA(cudaGetLastError(), "phi4 reflect launch");
    h->t += 1;
  }
  return SW_OK;
}

int sw_phi4_observables(sw_phi4* h, int64_t first, int64_t count, double* E_host, double* M_host) {
  if (!h) return ffail(SW_EINVAL, "handle is NULL");
  if (count < 0 || first < h->t_base || first + count > h->t) return ffail(SW_EINVAL, "update range outside the trace");
  int rc = check_phi4(h);
  if (rc != SW_OK) return rc;
  if (count == 0) return SW_OK;
  double* buf = (double*)malloc((size_t)count * 5 * sizeof(double));
  if (!buf) return ffail(SW_ENOMEM, "host allocation failed");
  cudaError_t e = cudaMemcpy(buf, h->obs + 5 * (first - h->t_base), (size_t)count * 5 * sizeof(double),
                             cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    for (int64_t k = 0; k < count; ++k) {
      if (E_host) E_host[k] = buf[5 * k];
      if (M_host)
        for (int a = 0; a < 4; ++a) M_host[4 * k + a] = buf[5 * k + 1 + a];
    }
  }
  free(buf);
  F_CUDA(e, "trace copy");
  return SW_OK;
}

int sw_phi4_field(sw_phi4* h, double* out, int32_t out_is_device) {
  if (!h || !out) return ffail(SW_EINVAL, "NULL argument");
  F_CUDA(cudaMemcpyAsync(out, h->phi, (size_t)h->n * sizeof(F4),
                         out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream),
         "field copy");
  if (out_is_device) return SW_OK;
  return check_phi4(h);
}

int sw_phi4_set_field(sw_phi4* h, const double* in, uint32_t t, int32_t in_is_device) {
  if (!h || !in) return ffail(SW_EINVAL, "NULL argument");
  int rc = check_phi4(h);
  if (rc != SW_OK) return rc;
  F_CUDA(cudaMemcpyAsync(h->phi, in, (size_t)h->n * sizeof(F4),
                         in_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream),
         "field copy");
  rc = check_phi4(h);
  if (rc != SW_OK) return rc;
  h->t = t;
  h->t_base = t;
  return SW_OK;
}

int sw_phi4_labels(sw_phi4* h, int32_t* out, int32_t out_is_device) {
  if (!h || !out) return ffail(SW_EINVAL, "NULL argument");
  Dir d;
  int rc = clusters(h, d);
  if (rc != SW_OK) return rc;
  F_CUDA(cudaMemcpyAsync(out, h->par, (size_t)h->n * sizeof(int32_t),
                         out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream),
         "labels copy");
  if (out_is_device) return SW_OK;
  return check_phi4(h);
}

int sw_phi4_get_sweep(sw_phi4* h, uint32_t* t_out) {
  if (!h || !t_out) return ffail(SW_EINVAL, "NULL argument");
  *t_out = (uint32_t)h->t;
  return SW_OK;
}

int sw_phi4_destroy(sw_phi4* h) {
  if (!h) return SW_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_phi4(h);
  delete h;
  return SW_OK;
}

}  // extern "C"
