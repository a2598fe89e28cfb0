// sw_small.cu -- whole sweeps of a small lattice (L <= kSmallMaxL) in one CTA.
//
// A lattice of at most 181 x 181 sites fits one CTA's shared memory whole:
// spins and bonds as bit masks, and a 16-bit union-find parent per site.
// One launch runs n sweeps back to back with block barriers between the
// steps, so a small lattice costs no cross-tile merge and no launch per
// phase. The steps and their results are those of the tiled path:
//   bonds (§2.1, C5)  a warp per row word, a lane per site, the word's bond
//                     masks assembled by ballot;
//   clusters (§2.3)   union-find over runs (stretches of a row word joined
//                     by east bonds), a lane per bond that joins two runs;
//                     the larger root is hung under the smaller, so every
//                     root is its cluster's smallest site (C9);
//   new spins (§2.4)  the flip bits of all site indices are filled from
//                     their blocks and each root reads its own (C6), or
//                     each root draws C6b's fresh spin; a warp per row
//                     word sets its 32 sites from their runs' roots;
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

// Hang root a under b if a is still a root: one 16-bit compare-and-swap of
// par[a] from a to b. Returns the entry found (a on success).
__device__ __forceinline__ int small_link_root(uint16_t* par, int a, int b) {
  return (int)atomicCAS(reinterpret_cast<unsigned short*>(par + a), (unsigned short)a, (unsigned short)b);
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
    const int old = small_link_root(par, a, b);
    if (old == a) return;
    a = old;  // another thread linked a first: carry on from its new parent
  }
  atomicCAS(err, 0, 1);
}

// Highest run start at or below bit b of a word (R always has bit 0 set).
__device__ __forceinline__ int small_run_start(uint32_t R, int b) {
  return 31 - __clz(R & (0xffffffffu >> (31 - b)));
}

template <typename T>
__device__ __forceinline__ T small_warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The n sweeps of one lattice by the whole CTA (smem: small_smem_bytes(L)).
__device__ __forceinline__ void small_body(const SmallArgs& a, uint32_t* smem) {
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
  // lanes per row word for bonds and unions: as many as the threads allow
  // (a power of two, at most 32), each taking 32 / G consecutive columns
  int G = 1;
  while (G < 32 && 2 * G * RWN <= NT) G *= 2;
  const int PER = 32 / G, sub = lane % G;

  for (int rw = warp; rw < RWN; rw += NW) {
    const int y = rw / WPL, x = (rw % WPL) * 32 + lane;
    const bool minus = x < L && a.spins[(size_t)y * L + x] < 0;
    const uint32_t m = __ballot_sync(0xffffffffu, minus);
    if (lane == 0) s_spin[rw] = m;
  }
  __syncthreads();

  for (int k = 0; k < a.n; ++k) {
    const uint32_t t = a.t0 + (uint32_t)k;
    for (int i = tid; i < DW; i += NT) s_dec[i] = 0u;
    for (int i = tid; i < N; i += NT) par[i] = (uint16_t)i;

    // ---- bonds (§2.1): G lanes per row word, each drawing a stretch of
    // 32 / G sites (one block for the two sites of a pair when both lie in
    // its stretch, C5); the word's masks are or-reduced across the G lanes
    for (int rw0 = warp * (32 / G); rw0 < RWN; rw0 += NT / G) {
      const int rw = rw0 + lane / G;
      uint32_t eb = 0u, sb = 0u;
      int y = 0, w = 0, nb = 0;
      if (rw < RWN) {
        y = rw / WPL;
        w = rw % WPL;
        nb = min(32, L - 32 * w);
        const uint32_t i0 = (uint32_t)(y * L + 32 * w);
        const int b1 = min(nb, sub * PER + PER);
        for (int b = sub * PER; b < b1; ++b) {
          const uint32_t i = i0 + b;
          const uint4 q = philox4x32_10(make_uint4(i >> 1, t, 0u, 0u), a.ks);
          if ((i & 1u) == 0u && b + 1 < b1) {  // both sites of the pair
            eb |= ((uint32_t)(q.x < a.thr) << b) | ((uint32_t)(q.z < a.thr) << (b + 1));
            sb |= ((uint32_t)(q.y < a.thr) << b) | ((uint32_t)(q.w < a.thr) << (b + 1));
            ++b;
          } else {
            eb |= (uint32_t)(((i & 1u) ? q.z : q.x) < a.thr) << b;
            sb |= (uint32_t)(((i & 1u) ? q.w : q.y) < a.thr) << b;
          }
        }
      }
      for (int o = 1; o < G; o <<= 1) {
        eb |= __shfl_xor_sync(0xffffffffu, eb, o);
        sb |= __shfl_xor_sync(0xffffffffu, sb, o);
      }
      if (rw < RWN && sub == 0) {
        const uint32_t vm = nb == 32 ? 0xffffffffu : ((1u << nb) - 1u);
        const uint32_t sp = s_spin[rw];
        // east neighbours: the next site in the word; the word's last site
        // meets the next word's first, or column 0 of its row (periodic)
        const uint32_t nxt = w + 1 < WPL ? s_spin[rw + 1] : s_spin[y * WPL];
        const uint32_t sE = ((sp >> 1) & (vm >> 1)) | ((nxt & 1u) << (nb - 1));
        const uint32_t sS = s_spin[(y + 1 == L ? 0 : y + 1) * WPL + w];
        s_e[rw] = eb & ~(sp ^ sE) & vm;
        s_s[rw] = sb & ~(sp ^ sS) & vm;
      }
    }
    __syncthreads();

    // ---- clusters (§2.3) over runs: a run is a stretch of a row word
    // joined by east bonds inside the word, and its first site is its
    // union-find node. Unions join the runs that the bonds between words,
    // across the row's periodic wrap and between rows connect; the larger
    // node is hung under the smaller, so every root is its cluster's
    // smallest site (C9: a cluster's smallest site starts a run). G lanes
    // share a row word, each uniting the bonds of its 32 / G columns in turn.
    for (int rw = tid / G; rw < RWN; rw += NT / G) {
      const int y = rw / WPL, w = rw % WPL, nb = min(32, L - 32 * w);
      const uint32_t vm = nb == 32 ? 0xffffffffu : ((1u << nb) - 1u), lastb = 1u << (nb - 1);
      const uint32_t mine = (PER == 32 ? 0xffffffffu : ((1u << PER) - 1u)) << (sub * PER);
      const uint32_t e = s_e[rw], ein = e & ~lastb, R = ~(ein << 1) & vm;
      const int base = y * L + 32 * w;
      const int yn = y + 1 == L ? 0 : y + 1, rwn = yn * WPL + w, basen = yn * L + 32 * w;
      const uint32_t en = s_e[rwn] & ~lastb, Rn = ~(en << 1) & vm, d = s_s[rw];
      // a south bond is redundant when the one left of it joins the same two runs
      uint32_t need = d & ~((d & ein & en) << 1) & mine;
      while (need) {
        const int j = __ffs(need) - 1;
        need &= need - 1;
        small_unite(par, base + small_run_start(R, j), basen + small_run_start(Rn, j), a.err);
      }
      if ((e & lastb & mine) != 0u)
        small_unite(par, base + small_run_start(R, nb - 1), w + 1 < WPL ? base + nb : y * L, a.err);
    }
    __syncthreads();

    // ---- every run start points at its root; roots draw their decision. Flip
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
          const int y = i / L, x = i - y * L;
          const bool starts = (x & 31) == 0 || !((s_e[y * WPL + (x >> 5)] >> ((x & 31) - 1)) & 1u);
          if (starts) {
            int r = i, p = par[r];
            while (p != r) {
              r = p;
              p = par[r];
            }
            par[i] = (uint16_t)r;  // concurrent stores all write roots
            isroot = r == i && !flip_rule;
          }
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

    // ---- new spins (§2.4): a warp per row word, a lane per site, each site
    // taking the decision of its run's root
    for (int rw = warp; rw < RWN; rw += NW) {
      const int y = rw / WPL, w = rw % WPL, nb = min(32, L - 32 * w);
      bool d = false;
      if (lane < nb) {
        const uint32_t vm = nb == 32 ? 0xffffffffu : ((1u << nb) - 1u);
        const uint32_t R = ~((s_e[rw] & ~(1u << (nb - 1))) << 1) & vm;
        const int r = par[y * L + 32 * w + small_run_start(R, lane)];
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

__global__ void __launch_bounds__(kSmallThreads, 1) small_sweep_kernel(const SmallArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  small_body(a, smem);
}

// Batch replicas on the one-CTA path: CTA i runs replica small[i] for the
// sweeps of this chunk it has left (at most n), writes its trace rows and
// then advances its counter, trace row and sweeps left itself (the tiled
// schedule's counter advance skips these replicas).
__global__ void __launch_bounds__(kSmallThreads, 1)
    small_batch_kernel(const BatchArgs b, const int* small, int n) {
  extern __shared__ __align__(16) uint32_t smem[];
  ReplicaDesc* D = b.descs + small[blockIdx.x];
  if (!D->active || D->t_left <= 0) return;
  const int m = D->t_left < n ? (int)D->t_left : n;
  SmallArgs a;
  a.L = D->a.g.L;
  a.thr = D->a.thr;
  a.rule = D->a.rule;
  a.t0 = D->t;
  a.n = m;
  a.ks = D->a.ks;
  a.spins = D->a.spins_out;
  a.em = D->em_base + 2 * D->em_next;
  a.err = D->a.tb.err;
  small_body(a, smem);
  __syncthreads();
  if (threadIdx.x == 0) {
    D->t += (uint32_t)m;
    D->em_next += m;
    D->t_left -= m;
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

cudaError_t launch_small_batch(const BatchArgs& b, const int* small, int nsmall, int max_L, int n, cudaStream_t st) {
  if (nsmall <= 0 || n <= 0) return cudaSuccess;
  if (max_L < 2 || max_L > kSmallMaxL) return cudaErrorInvalidValue;
  static bool attr_done = false;
  if (!attr_done) {
    const cudaError_t e = cudaFuncSetAttribute(small_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)small_smem_bytes(kSmallMaxL));
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  small_batch_kernel<<<nsmall, kSmallThreads, small_smem_bytes(max_L), st>>>(b, small, n);
  return cudaGetLastError();
}

}  // namespace sw
