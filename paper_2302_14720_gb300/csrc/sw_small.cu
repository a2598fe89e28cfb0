// sw_small.cu -- whole sweeps of a small lattice (L <= kSmallMaxL) in one CTA.
//
// A lattice of at most 181 x 181 sites fits one CTA's shared memory whole:
// spins and bonds as bit masks, and a 16-bit union-find parent per site.
// One launch runs n sweeps back to back with block barriers between the
// steps, so a small lattice costs no cross-tile merge and no launch per
// phase. The steps and their results are those of the tiled path:
//   bonds (§2.1, C5)  a thread per Philox block (two consecutive sites);
//   clusters (§2.3)   the two ends of every bond are united, the larger root
//                     hung under the smaller, so every root is its
//                     cluster's smallest site (C9);
//   new spins (§2.4)  the flip bits of all site indices are filled from
//                     their blocks and each root reads its own (C6), or
//                     each root draws C6b's fresh spin; a warp per row
//                     word sets its 32 sites;
//   E and M (C10)     from the new bit masks, int64, one trace row per sweep.
// Spins are read at the start and written back after the last sweep.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sw_internal.h"
#include "sw_philox.cuh"

namespace sw {
namespace {

constexpr int kSmallThreads = 1024;
constexpr int kSmallUnionCap = 1 << 20;

// Replace the 16-bit entry at p by v if it is larger; returns the old entry.
__device__ __forceinline__ uint32_t small_atomic_min_u16(uint16_t* p, uint32_t v) {
  unsigned int* w = reinterpret_cast<unsigned int*>(reinterpret_cast<uintptr_t>(p) & ~uintptr_t(3));
  const int sh = (reinterpret_cast<uintptr_t>(p) & 2u) ? 16 : 0;
  unsigned int old = *reinterpret_cast<volatile unsigned int*>(w);
  for (;;) {
    const uint32_t cur = (old >> sh) & 0xFFFFu;
    if (cur <= v) return cur;
    const unsigned int nw = (old & ~(0xFFFFu << sh)) | (v << sh);
    const unsigned int seen = atomicCAS(w, old, nw);
    if (seen == old) return cur;
    old = seen;
  }
}

// Root of x while other threads may be uniting (path halving).
__device__ __forceinline__ int small_find(volatile uint16_t* par, int x) {
  for (;;) {
    const int p = par[x];
    if (p == x) return x;
    const int gp = par[p];
    if (gp == p) return p;
    par[x] = (uint16_t)gp;
    x = gp;
  }
}

__device__ void small_unite(uint16_t* par, int a, int b, int* err) {
  for (int it = 0; it < kSmallUnionCap; ++it) {
    a = small_find(par, a);
    b = small_find(par, b);
    if (a == b) return;
    if (a < b) {
      const int tmp = a;
      a = b;
      b = tmp;
    }
    const int old = (int)small_atomic_min_u16(&par[a], (uint32_t)b);
    if (old == a) return;
    a = old;
  }
  atomicCAS(err, 0, 1);
}

__device__ __forceinline__ uint32_t spin_bit(const uint32_t* s, int wpl, int y, int x) {
  return (s[y * wpl + (x >> 5)] >> (x & 31)) & 1u;
}

template <typename T>
__device__ __forceinline__ T small_warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kSmallThreads, 1) small_sweep_kernel(const SmallArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  constexpr int NT = kSmallThreads, NW = NT / 32;
  __shared__ long long s_red[2][NW];
  __shared__ uint16_t s_rootq[NW][64];  // roots waiting for their draw
  const int L = a.L, N = L * L, WPL = (L + 31) >> 5, RWN = L * WPL, DW = (N + 31) >> 5;
  uint32_t* s_spin = smem;       // [RWN] sign bits (1 = -1)
  uint32_t* s_e = s_spin + RWN;  // [RWN] east bonds
  uint32_t* s_s = s_e + RWN;     // [RWN] south bonds
  uint32_t* s_dec = s_s + RWN;   // [DW] decision bit of every root
  uint16_t* par = reinterpret_cast<uint16_t*>(s_dec + DW);  // [N]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int rw = warp; rw < RWN; rw += NW) {
    const int y = rw / WPL, x = (rw % WPL) * 32 + lane;
    const bool minus = x < L && a.spins[(size_t)y * L + x] < 0;
    const uint32_t m = __ballot_sync(0xffffffffu, minus);
    if (lane == 0) s_spin[rw] = m;
  }
  __syncthreads();

  for (int k = 0; k < a.n; ++k) {
    const uint32_t t = a.t0 + (uint32_t)k;
    for (int i = tid; i < RWN; i += NT) {
      s_e[i] = 0u;
      s_s[i] = 0u;
    }
    for (int i = tid; i < DW; i += NT) s_dec[i] = 0u;
    for (int i = tid; i < N; i += NT) par[i] = (uint16_t)i;
    __syncthreads();

    // ---- bonds (§2.1): block (p, t, 0, 0) serves sites 2p and 2p+1 (C5)
    for (int p = tid; 2 * p < N; p += NT) {
      const uint4 q = philox4x32_10(make_uint4((uint32_t)p, t, 0u, 0u), a.ks);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int i = 2 * p + j;
        if (i >= N) break;
        const int y = i / L, x = i - y * L;
        const int xe = x + 1 == L ? 0 : x + 1, ys = y + 1 == L ? 0 : y + 1;
        const uint32_t si = spin_bit(s_spin, WPL, y, x);
        const uint32_t we = j ? q.z : q.x, ws = j ? q.w : q.y;
        const uint32_t bit = 1u << (x & 31);
        if (si == spin_bit(s_spin, WPL, y, xe) && we < a.thr) atomicOr(&s_e[y * WPL + (x >> 5)], bit);
        if (si == spin_bit(s_spin, WPL, ys, x) && ws < a.thr) atomicOr(&s_s[y * WPL + (x >> 5)], bit);
      }
    }
    __syncthreads();

    // ---- clusters (§2.3)
    for (int i = tid; i < N; i += NT) {
      const int y = i / L, x = i - y * L;
      const int rw = y * WPL + (x >> 5);
      const uint32_t bit = 1u << (x & 31);
      if (s_e[rw] & bit) small_unite(par, i, y * L + (x + 1 == L ? 0 : x + 1), a.err);
      if (s_s[rw] & bit) small_unite(par, i, (y + 1 == L ? 0 : y + 1) * L + x, a.err);
    }
    __syncthreads();

    // ---- every site points at its root; roots draw their decision. Flip
    // rule (C6): word k of s_dec, the bits of site indices 32k .. 32k+31, is
    // word k & 3 of block k >> 2, so every word is filled from its block and
    // each root reads its own bit. Assignment rule (C6b): the roots are
    // queued per warp and drawn 32 at a time so that every lane draws.
    const bool flip_rule = a.rule == 0;
    if (flip_rule) {
      for (int b = tid; 4 * b < DW; b += NT) {
        const uint4 q4 = philox4x32_10(make_uint4((uint32_t)b, t, 1u, 0u), a.ks);
        s_dec[4 * b] = q4.x;
        if (4 * b + 1 < DW) s_dec[4 * b + 1] = q4.y;
        if (4 * b + 2 < DW) s_dec[4 * b + 2] = q4.z;
        if (4 * b + 3 < DW) s_dec[4 * b + 3] = q4.w;
      }
    }
    {
      uint16_t* q = s_rootq[warp];
      int qh = 0, qn = 0;  // the same in every lane of the warp
      for (int i0 = warp * 32; i0 < N; i0 += NT) {
        const int i = i0 + lane;
        bool isroot = false;
        if (i < N) {
          int r = i, p = par[r];
          while (p != r) {
            r = p;
            p = par[r];
          }
          par[i] = (uint16_t)r;  // concurrent stores all write roots
          isroot = r == i && !flip_rule;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, isroot);
        if (isroot) q[(qh + qn + __popc(m & ((1u << lane) - 1u))) & 63] = (uint16_t)i;
        qn += __popc(m);
        __syncwarp();
        if (qn >= 32) {
          const int x = q[(qh + lane) & 63];
          if (decision_bit((uint32_t)x, t, a.ks, a.rule)) atomicOr(&s_dec[x >> 5], 1u << (x & 31));
          qh += 32;
          qn -= 32;
          __syncwarp();
        }
      }
      if (lane < qn) {
        const int x = q[(qh + lane) & 63];
        if (decision_bit((uint32_t)x, t, a.ks, a.rule)) atomicOr(&s_dec[x >> 5], 1u << (x & 31));
      }
    }
    __syncthreads();

    // ---- new spins (§2.4): a warp per row word, a lane per site
    for (int rw = warp; rw < RWN; rw += NW) {
      const int y = rw / WPL, x = (rw % WPL) * 32 + lane;
      bool d = false;
      if (x < L) {
        const int r = par[y * L + x];
        d = (s_dec[r >> 5] >> (r & 31)) & 1u;
      }
      const uint32_t dm = __ballot_sync(0xffffffffu, d);
      if (lane == 0) s_spin[rw] = (a.rule ? 0u : s_spin[rw]) ^ dm;
    }
    __syncthreads();

    // ---- E and M of the new state (C10)
    long long e = 0, m = 0;
    for (int rw = tid; rw < RWN; rw += NT) {
      const int y = rw / WPL, w = rw % WPL;
      const int nb = min(32, L - 32 * w);
      const uint32_t vm = nb == 32 ? 0xffffffffu : ((1u << nb) - 1u);
      const uint32_t s = s_spin[rw];
      uint32_t sE;
      if (32 * w + nb == L) {  // last word of the row: its last site wraps to column 0
        sE = ((s >> 1) & (vm >> 1)) | ((s_spin[y * WPL] & 1u) << (nb - 1));
      } else {
        sE = (s >> 1) | ((s_spin[rw + 1] & 1u) << 31);
      }
      const uint32_t sS = s_spin[(y + 1 == L ? 0 : y + 1) * WPL + w];
      e += 2 * (__popc((s ^ sE) & vm) + __popc((s ^ sS) & vm)) - 2 * nb;
      m += nb - 2 * __popc(s & vm);
    }
    e = small_warp_sum(e);
    m = small_warp_sum(m);
    if (lane == 0) {
      s_red[0][warp] = e;
      s_red[1][warp] = m;
    }
    __syncthreads();
    if (tid == 0) {
      long long et = 0, mt = 0;
      for (int q = 0; q < NW; ++q) {
        et += s_red[0][q];
        mt += s_red[1][q];
      }
      a.em[2 * k] = et;
      a.em[2 * k + 1] = mt;
    }
    __syncthreads();
  }

  for (int rw = warp; rw < RWN; rw += NW) {
    const int y = rw / WPL, x = (rw % WPL) * 32 + lane;
    if (x < L) a.spins[(size_t)y * L + x] = ((s_spin[rw] >> lane) & 1u) ? (int8_t)-1 : (int8_t)1;
  }
}

size_t small_smem_bytes(int L) {
  const size_t N = (size_t)L * L, WPL = (size_t)(L + 31) / 32, RWN = (size_t)L * WPL, DW = (N + 31) / 32;
  return (3 * RWN + DW) * sizeof(uint32_t) + N * sizeof(uint16_t);
}

}  // namespace

cudaError_t launch_small(const SmallArgs& a, cudaStream_t st) {
  if (a.L < 2 || a.L > kSmallMaxL) return cudaErrorInvalidValue;
  if (a.n <= 0) return cudaSuccess;
  const size_t dyn = small_smem_bytes(kSmallMaxL);
  static bool attr_done = false;  // set once per process; the attribute is per function
  if (!attr_done) {
    const cudaError_t e =
        cudaFuncSetAttribute(small_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  small_sweep_kernel<<<1, kSmallThreads, small_smem_bytes(a.L), st>>>(a);
  return cudaGetLastError();
}

}  // namespace sw
