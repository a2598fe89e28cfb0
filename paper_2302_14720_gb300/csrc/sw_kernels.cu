// sw_kernels.cu -- the Swendsen-Wang sweep on sm_103a.
//
// One sweep (paper §2) runs as three kernels over square-ish tiles of
// TW = 32*WPR columns by TH rows; one thread owns one 32-site word of one
// tile row and keeps its sites as bit masks (bit k = site x0+32w+k).
//
//  phase 1 (bonds §2.1 + tile-local clusters §2.3)
//    - int8 spins -> sign bits; the tile's east halo column and south halo
//      row are read too, so every east/south bond of the tile can be drawn;
//    - Philox-4x32-10 block (site>>1, t, 0, 0) gives the east and south words
//      of two consecutive sites (C5); bond iff equal spins and word < thr;
//    - union-find in shared memory over word-local runs of east bonds: a run
//      is a maximal stretch of east-bonded sites inside one word, its start
//      is its node; south bonds and word-crossing east bonds unite runs
//      (atomicMin towards the smaller index, so each tile component's root
//      is its smallest site -- the "lowest value label" of §2.3);
//    - every tile component that touches the tile border gets a slot; slot
//      nodes are initialised in a global 64-bit union-find whose entries are
//      (key << 32 | parent node), key = smallest global site index of the
//      tile component, so comparing entries compares keys;
//    - stores the spin/east/south bit masks (12 bytes per 32 sites), the
//      slot of each border site, the out-going border bonds and the halo
//      spins (a few hundred bytes per tile).
//  phase 2 (clusters across tiles, §2.3; device-side, no host round trip
//    as in §5's maintenance kernel)
//    - one thread per bonded tile-border edge (including the periodic wrap)
//      unites the two slot nodes with 64-bit atomicMin; consecutive edges
//      joining the same two slots are skipped.
//  phase 3 (new spins §2.4 + E/M, or canonical labels)
//    - rebuilds the tile-local union-find from the stored bit masks, takes
//      each border component's global root (its key is the cluster's
//      canonical label, C9) and each inner component's own root;
//    - one Philox block (root, t, 1, 0) per root decides the flip (C6); the
//      flip mask of a word is built from its runs with a prefix xor;
//    - writes the new int8 spins, and reduces E and M (C10) in int64 using
//      the new spins of the halo sites (their old spins from phase 1 and
//      their clusters' flips);
//    - optionally accumulates cluster sizes (C11), inner clusters in the
//      tile and border clusters at their global root node (phase 4 bins
//      those).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sw_internal.h"

namespace sw {
namespace {

constexpr int kUnionCap = 1 << 20;        // retries of one shared-memory union
constexpr int kGlobalUnionCap = 1 << 16;  // retries of one global union
constexpr int kGlobalFindCap = 1 << 20;   // steps of one global find
constexpr int kFlagClaim = 0x40000000;

// Highest run start at or below bit b (R always has bit 0 set for valid b).
__device__ __forceinline__ int run_start(uint32_t R, int b) {
  return 31 - __clz(R & (0xffffffffu >> (31 - b)));
}

// Four int8 spins (+1 = 0x01, -1 = 0xFF) -> four sign bits.
__device__ __forceinline__ uint32_t sign_bits4(uint32_t w) {
  return ((w & 0x80808080u) * 0x00204081u) >> 28;
}
// Four sign bits -> four int8 spins.
__device__ __forceinline__ uint32_t spin_bytes4(uint32_t nib) {
  const uint32_t spread = (nib * 0x00204081u) & 0x01010101u;
  return 0x01010101u | (spread * 0xFEu);
}

__device__ __forceinline__ uint32_t load_spin_bits(const int8_t* p, int nb, bool vec) {
  if (vec && nb == 32) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
    const uint4 u = __ldg(q), v = __ldg(q + 1);
    return sign_bits4(u.x) | (sign_bits4(u.y) << 4) | (sign_bits4(u.z) << 8) | (sign_bits4(u.w) << 12) |
           (sign_bits4(v.x) << 16) | (sign_bits4(v.y) << 20) | (sign_bits4(v.z) << 24) |
           (sign_bits4(v.w) << 28);
  }
  uint32_t bits = 0;
  for (int k = 0; k < nb; ++k) bits |= (uint32_t)(p[k] < 0) << k;
  return bits;
}

__device__ __forceinline__ void store_spin_bits(int8_t* p, uint32_t bits, int nb, bool vec) {
  if (vec && nb == 32) {
    uint4 u, v;
    u.x = spin_bytes4(bits & 0xFu);
    u.y = spin_bytes4((bits >> 4) & 0xFu);
    u.z = spin_bytes4((bits >> 8) & 0xFu);
    u.w = spin_bytes4((bits >> 12) & 0xFu);
    v.x = spin_bytes4((bits >> 16) & 0xFu);
    v.y = spin_bytes4((bits >> 20) & 0xFu);
    v.z = spin_bytes4((bits >> 24) & 0xFu);
    v.w = spin_bytes4(bits >> 28);
    uint4* q = reinterpret_cast<uint4*>(p);
    q[0] = u;
    q[1] = v;
    return;
  }
  for (int k = 0; k < nb; ++k) p[k] = ((bits >> k) & 1u) ? (int8_t)-1 : (int8_t)1;
}

// ------------------------------------------------ shared-memory union-find

__device__ __forceinline__ int find_local(const volatile int* par, int x) {
  int p = par[x];
  while (p != x) {
    x = p;
    p = par[x];
  }
  return x;
}

// Entries only ever decrease (par[x] <= x), so finds terminate; a failed
// atomicMin means another thread linked `a` first, and the loop carries on
// with a's new parent. The cap only guards against corrupted memory.
__device__ void unite_local(int* par, int a, int b, int* err) {
  for (int it = 0; it < kUnionCap; ++it) {
    a = find_local(par, a);
    b = find_local(par, b);
    if (a == b) return;
    if (a < b) {
      const int tmp = a;
      a = b;
      b = tmp;
    }
    const int old = atomicMin(&par[a], b);
    if (old == a) return;
    a = old;
  }
  atomicCAS(err, 0, kErrUnionCap);
}

// ------------------------------------------------------- global union-find

__device__ __forceinline__ uint64_t ld_node(const uint64_t* p) {
  return (uint64_t)__ldcg(reinterpret_cast<const unsigned long long*>(p));
}

// Root entry (key << 32 | root) of node x, halving the path on the way.
// Entries point at strictly smaller keys, so the walk ends; the cap only
// guards against corrupted memory and raises the error flag.
__device__ uint64_t find_global(uint64_t* nodes, uint32_t x, int* err) {
  uint64_t v = ld_node(nodes + x);
  for (int it = 0; (uint32_t)v != x; ++it) {
    if (it >= kGlobalFindCap) {
      atomicCAS(err, 0, kErrUnionCap);
      break;
    }
    const uint32_t p = (uint32_t)v;
    const uint64_t vp = ld_node(nodes + p);
    if ((uint32_t)vp == p) return vp;
    atomicMin(reinterpret_cast<unsigned long long*>(nodes + x), (unsigned long long)vp);
    x = (uint32_t)vp;
    v = ld_node(nodes + x);
  }
  return v;
}

__device__ void unite_global(uint64_t* nodes, uint32_t a, uint32_t b, int* err) {
  for (int it = 0; it < kGlobalUnionCap; ++it) {
    uint64_t va = find_global(nodes, a, err);
    uint64_t vb = find_global(nodes, b, err);
    if (va == vb) return;
    if (va < vb) {
      const uint64_t tmp = va;
      va = vb;
      vb = tmp;
    }
    // hang the root with the larger key under the one with the smaller key
    const unsigned long long old =
        atomicMin(reinterpret_cast<unsigned long long*>(nodes + (uint32_t)va), (unsigned long long)vb);
    if (old == va) return;
    a = (uint32_t)old;
    b = (uint32_t)vb;
  }
  atomicCAS(err, 0, kErrUnionCap);
}

// ----------------------------------------------------------- tile helpers

template <int WPR, int TH>
struct Tile {
  static constexpr int TW = 32 * WPR;
  static constexpr int NT = WPR * TH;
  static constexpr int NB = 2 * TH + 2 * TW;        // border sites: left, right, top, bottom
  static constexpr int MS = 2 * (TW + TH);          // slots per tile
  static constexpr int BBW = 2 * (TH / 32) + 2 * (TW / 32);
  static constexpr int OFF_EOUT = 0, OFF_SOUT = TH / 32, OFF_HE = TH / 32 + TW / 32,
                       OFF_HS = 2 * (TH / 32) + TW / 32;
  static_assert(TH % 32 == 0, "TH must be a multiple of 32");
  static_assert(TW <= NT && TH <= NT, "halo passes need one thread per halo site");
  static_assert(BBW <= NT, "tile bits are written by one thread each");
};

struct TilePos {
  int tile, tx, ty, x0, y0, ncols, nrows;
};

template <int TW, int TH>
__device__ __forceinline__ TilePos tile_pos(const Geometry& g, int tile) {
  TilePos p;
  p.tile = tile;
  p.tx = tile % g.tiles_x;
  p.ty = tile / g.tiles_x;
  p.x0 = p.tx * TW;
  p.y0 = p.ty * TH;
  p.ncols = min(TW, g.L - p.x0);
  p.nrows = min(TH, g.L - p.y0);
  return p;
}

// Site of border position j (left col, right col, top row, bottom row), or
// false when j lies beyond a ragged tile edge.
template <int TW, int TH>
__device__ __forceinline__ bool border_site(const TilePos& p, int j, int& y, int& x) {
  if (j < TH) { y = j; x = 0; return y < p.nrows; }
  if (j < 2 * TH) { y = j - TH; x = p.ncols - 1; return y < p.nrows; }
  if (j < 2 * TH + TW) { y = 0; x = j - 2 * TH; return x < p.ncols; }
  y = p.nrows - 1;
  x = j - 2 * TH - TW;
  return x < p.ncols;
}

// Tile-local union-find over word-local runs. e_int / d_int exclude bonds
// leaving the tile. s_eint holds e_int of every row-word of the tile.
template <int WPR, int TH>
__device__ __forceinline__ void tile_unions(int* par, uint32_t R, uint32_t e_int, uint32_t d_int,
                                            uint32_t vmask, int ry, int w, int nrows,
                                            const uint32_t (*s_eint)[WPR], int lbase, int* err) {
  constexpr int TW = 32 * WPR;
  if ((e_int >> 31) & 1u) unite_local(par, lbase + run_start(R, 31), lbase + 32, err);
  if (d_int && ry + 1 < nrows) {
    const uint32_t eb = s_eint[ry + 1][w];
    const uint32_t Rb = ~(eb << 1) & vmask;
    // an S bond at b is redundant when b-1 has one too and b-1,b share a run in both rows
    uint32_t need = d_int & ~((d_int & e_int & eb) << 1);
    while (need) {
      const int b = __ffs(need) - 1;
      need &= need - 1;
      unite_local(par, lbase + run_start(R, b), lbase + TW + run_start(Rb, b), err);
    }
  }
}

__device__ __forceinline__ void compress_runs(int* par, uint32_t R, int lbase) {
  while (R) {
    const int b = __ffs(R) - 1;
    R &= R - 1;
    par[lbase + b] = find_local(par, lbase + b);
  }
}

__device__ __forceinline__ void init_parents(int* par, int lbase) {
  int4* p4 = reinterpret_cast<int4*>(par + lbase);
#pragma unroll
  for (int k = 0; k < 8; ++k) p4[k] = make_int4(lbase + 4 * k, lbase + 4 * k + 1, lbase + 4 * k + 2, lbase + 4 * k + 3);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int log2_floor(uint32_t v) { return 31 - __clz(v); }

// ================================================================ phase 1

template <int WPR, int TH>
__global__ void __launch_bounds__(WPR * TH) phase1_kernel(const SweepArgs a) {
  using T = Tile<WPR, TH>;
  constexpr int TW = T::TW, NT = T::NT, NB = T::NB, MS = T::MS, BBW = T::BBW;
  __shared__ __align__(16) int par[TH * TW];
  __shared__ uint32_t s_spin[TH][WPR];
  __shared__ uint32_t s_eint[TH][WPR];
  __shared__ uint32_t s_bb[BBW];
  __shared__ int s_broot[NB];
  __shared__ int s_nslots;

  const Geometry& g = a.g;
  const int L = g.L;
  const TilePos P = tile_pos<TW, TH>(g, blockIdx.x);
  const int tid = threadIdx.x, ry = tid / WPR, w = tid % WPR;
  uint32_t* eout = s_bb + T::OFF_EOUT;
  uint32_t* sout = s_bb + T::OFF_SOUT;
  uint32_t* hE = s_bb + T::OFF_HE;
  uint32_t* hS = s_bb + T::OFF_HS;

  if (tid < BBW) s_bb[tid] = 0u;
  if (tid == 0) s_nslots = 0;

  // ---- spins of my word
  const int nb = max(0, min(32, P.ncols - 32 * w));
  const bool rowv = ry < P.nrows;
  const uint32_t vmask = (!rowv || nb == 0) ? 0u : (nb == 32 ? 0xffffffffu : ((1u << nb) - 1u));
  uint32_t s = 0;
  if (vmask) s = load_spin_bits(a.spins_in + (size_t)(P.y0 + ry) * L + P.x0 + 32 * w, nb, g.aligned16);
  s_spin[ry][w] = s;
  __syncthreads();

  // ---- east halo column and south halo row (periodic wrap)
  const int xe = (P.x0 + P.ncols) % L;
  const int ys = (P.y0 + P.nrows) % L;
  if (tid < TH) {
    const bool bit = tid < P.nrows && a.spins_in[(size_t)(P.y0 + tid) * L + xe] < 0;
    const uint32_t m = __ballot_sync(0xffffffffu, bit);
    if ((tid & 31) == 0) hE[tid >> 5] = m;
  }
  if (tid < WPR) {
    const int nbw = max(0, min(32, P.ncols - 32 * tid));
    hS[tid] = nbw ? load_spin_bits(a.spins_in + (size_t)ys * L + P.x0 + 32 * tid, nbw, g.aligned16) : 0u;
  }
  __syncthreads();

  // ---- bonds (§2.1)
  const bool lastword = nb > 0 && 32 * (w + 1) >= P.ncols;  // holds the tile's last column
  const int pl = P.ncols - 1 - 32 * w;                       // that column's bit
  uint32_t sE;
  if (lastword) {
    const uint32_t hb = (hE[ry >> 5] >> (ry & 31)) & 1u;
    sE = ((s >> 1) & ((1u << pl) - 1u)) | (hb << pl);
  } else {
    sE = (s >> 1) | ((w + 1 < WPR) ? (s_spin[ry][w + 1] << 31) : 0u);
  }
  const uint32_t sS = (ry + 1 < P.nrows) ? s_spin[ry + 1][w] : hS[w];
  const uint32_t eqE = ~(s ^ sE) & vmask, eqS = ~(s ^ sS) & vmask;

  uint32_t rE = 0, rS = 0;
  if (vmask) {
    const uint32_t i0 = (uint32_t)(P.y0 + ry) * (uint32_t)L + (uint32_t)(P.x0 + 32 * w);
    if ((L & 1) == 0) {
      // even L: sites i0+b, i0+b+1 (b even) share Philox block (i0+b)/2
#pragma unroll 4
      for (int b = 0; b < 32; b += 2) {
        if (b < nb) {
          const uint4 r = philox4x32_10(make_uint4((i0 + b) >> 1, a.t, 0u, 0u), a.ks);
          rE |= ((uint32_t)(r.x < a.thr) << b) | ((uint32_t)(r.z < a.thr) << (b + 1));
          rS |= ((uint32_t)(r.y < a.thr) << b) | ((uint32_t)(r.w < a.thr) << (b + 1));
        }
      }
    } else {
      for (int b = 0; b < nb; ++b) {
        const uint32_t i = i0 + b;
        const uint4 r = philox4x32_10(make_uint4(i >> 1, a.t, 0u, 0u), a.ks);
        const uint32_t we = (i & 1u) ? r.z : r.x, ws = (i & 1u) ? r.w : r.y;
        rE |= (uint32_t)(we < a.thr) << b;
        rS |= (uint32_t)(ws < a.thr) << b;
      }
    }
  }
  const uint32_t e = eqE & rE, d = eqS & rS;
  const uint32_t e_int = lastword ? (e & ~(1u << pl)) : e;
  const uint32_t d_int = (ry + 1 < P.nrows) ? d : 0u;
  s_eint[ry][w] = e_int;
  if (lastword && ((e >> pl) & 1u)) atomicOr(&eout[ry >> 5], 1u << (ry & 31));
  if (rowv && ry == P.nrows - 1) sout[w] = d;
  {
    uint32_t* tb = a.tb.tbits + (size_t)P.tile * 3 * NT;
    tb[tid] = s;
    tb[NT + tid] = e;
    tb[2 * NT + tid] = d;
  }

  // ---- tile-local clusters (§2.3)
  const int lbase = ry * TW + 32 * w;
  init_parents(par, lbase);
  __syncthreads();
  const uint32_t R = ~(e_int << 1) & vmask;
  tile_unions<WPR, TH>(par, R, e_int, d_int, vmask, ry, w, P.nrows, s_eint, lbase, a.tb.err);
  __syncthreads();
  compress_runs(par, R, lbase);
  __syncthreads();

  // ---- border components -> slots and global nodes
  for (int j = tid; j < NB; j += NT) {
    int y, x, r = -1;
    if (border_site<TW, TH>(P, j, y, x)) {
      const int rs = run_start(~(s_eint[y][x >> 5] << 1), x & 31);
      r = par[y * TW + (x & ~31) + rs];
    }
    s_broot[j] = r;
  }
  __syncthreads();
  for (int j = tid; j < NB; j += NT) {
    const int r = s_broot[j];
    if (r >= 0 && atomicCAS(&par[r], r, kFlagClaim) == r) {
      const int slot = atomicAdd(&s_nslots, 1);
      par[r] = kFlagClaim | slot;
      const uint32_t node = (uint32_t)P.tile * MS + (uint32_t)slot;
      const uint32_t key = (uint32_t)(P.y0 + r / TW) * (uint32_t)L + (uint32_t)(P.x0 + r % TW);
      a.tb.nodes[node] = ((uint64_t)key << 32) | node;
      if (a.csize) a.csize[node] = 0u;
    }
  }
  __syncthreads();
  uint16_t* bs = a.tb.bslot + (size_t)P.tile * NB;
  for (int j = tid; j < NB; j += NT) {
    const int r = s_broot[j];
    bs[j] = r >= 0 ? (uint16_t)(par[r] & ~kFlagClaim) : (uint16_t)0xFFFFu;
  }
  if (tid < BBW) a.tb.bbits[(size_t)P.tile * BBW + tid] = s_bb[tid];
  if (tid == 0) {
    if (s_nslots > MS) atomicCAS(a.tb.err, 0, kErrSlotOverflow);
    a.tb.nslots[P.tile] = s_nslots;
  }
  if (P.tile == 0) {
    if (a.em && tid < 2) a.em[tid] = 0;
    if (a.hist && tid < 34) a.hist[tid] = 0;
  }
}

// ================================================================ phase 2

template <int WPR, int TH>
__global__ void phase2_kernel(const SweepArgs a) {
  using T = Tile<WPR, TH>;
  constexpr int TW = T::TW, NB = T::NB, MS = T::MS, BBW = T::BBW;
  const Geometry& g = a.g;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)g.tiles_x * g.tiles_y * (TH + TW);
  if (idx >= total) return;
  const int tile = (int)(idx / (TH + TW));
  const int k = (int)(idx % (TH + TW));
  const TilePos P = tile_pos<TW, TH>(g, tile);
  const uint32_t* bb = a.tb.bbits + (size_t)tile * BBW;
  const uint16_t* bs = a.tb.bslot + (size_t)tile * NB;
  if (k < TH) {
    const int y = k;
    if (y >= P.nrows) return;
    const uint32_t* eo = bb + T::OFF_EOUT;
    if (!((eo[y >> 5] >> (y & 31)) & 1u)) return;
    const int tileE = P.ty * g.tiles_x + (P.tx + 1) % g.tiles_x;
    const uint16_t* bsE = a.tb.bslot + (size_t)tileE * NB;
    const uint16_t sa = bs[TH + y], sb = bsE[y];
    if (y > 0 && ((eo[(y - 1) >> 5] >> ((y - 1) & 31)) & 1u) && bs[TH + y - 1] == sa && bsE[y - 1] == sb) return;
    unite_global(a.tb.nodes, (uint32_t)tile * MS + sa, (uint32_t)tileE * MS + sb, a.tb.err);
  } else {
    const int x = k - TH;
    if (x >= P.ncols) return;
    const uint32_t* so = bb + T::OFF_SOUT;
    if (!((so[x >> 5] >> (x & 31)) & 1u)) return;
    const int tileS = ((P.ty + 1) % g.tiles_y) * g.tiles_x + P.tx;
    const uint16_t* bsS = a.tb.bslot + (size_t)tileS * NB;
    const uint16_t sa = bs[2 * TH + TW + x], sb = bsS[2 * TH + x];
    if (x > 0 && ((so[(x - 1) >> 5] >> ((x - 1) & 31)) & 1u) && bs[2 * TH + TW + x - 1] == sa &&
        bsS[2 * TH + x - 1] == sb)
      return;
    unite_global(a.tb.nodes, (uint32_t)tile * MS + sa, (uint32_t)tileS * MS + sb, a.tb.err);
  }
}

// ================================================================ phase 3

// MODE 0: flips + E/M; 1: flips + E/M + cluster sizes; 2: canonical labels.
template <int WPR, int TH, int MODE>
__global__ void __launch_bounds__(WPR * TH) phase3_kernel(const SweepArgs a) {
  using T = Tile<WPR, TH>;
  constexpr int TW = T::TW, NT = T::NT, NB = T::NB, MS = T::MS, BBW = T::BBW;
  constexpr bool HIST = MODE == 1, LABELS = MODE == 2;
  __shared__ __align__(16) int par[TH * TW];
  __shared__ uint32_t s_eint[TH][WPR];
  __shared__ uint32_t s_snew[TH][WPR];
  __shared__ uint32_t s_iflip[NT];       // flip bit of inner roots, one word per thread
  __shared__ int s_broot[NB];
  __shared__ int s_slotval[MS];          // flip bit (flip modes) or canonical label (labels mode)
  __shared__ uint32_t s_slotroot[HIST ? MS : 1];
  __shared__ uint32_t s_hEnew[TH / 32], s_hSnew[TW / 32];
  __shared__ long long s_red[2][NT / 32];
  __shared__ unsigned long long s_hist[HIST ? 34 : 1];
  extern __shared__ __align__(16) int s_size[];  // HIST: [TH * TW]

  const Geometry& g = a.g;
  const int L = g.L;
  const TilePos P = tile_pos<TW, TH>(g, blockIdx.x);
  const int tid = threadIdx.x, ry = tid / WPR, w = tid % WPR;

  const uint32_t* tb = a.tb.tbits + (size_t)P.tile * 3 * NT;
  const uint32_t s = tb[tid], e = tb[NT + tid], d = tb[2 * NT + tid];
  const int nb = max(0, min(32, P.ncols - 32 * w));
  const bool rowv = ry < P.nrows;
  const uint32_t vmask = (!rowv || nb == 0) ? 0u : (nb == 32 ? 0xffffffffu : ((1u << nb) - 1u));
  const bool lastword = nb > 0 && 32 * (w + 1) >= P.ncols;
  const int pl = P.ncols - 1 - 32 * w;
  const uint32_t e_int = lastword ? (e & ~(1u << pl)) : e;
  const uint32_t d_int = (ry + 1 < P.nrows) ? d : 0u;
  s_eint[ry][w] = e_int;
  const int lbase = ry * TW + 32 * w;
  init_parents(par, lbase);
  if (HIST) {
    int4* z = reinterpret_cast<int4*>(s_size + lbase);
#pragma unroll
    for (int k = 0; k < 8; ++k) z[k] = make_int4(0, 0, 0, 0);
    if (tid < 34) s_hist[tid] = 0ull;
  }
  __syncthreads();
  const uint32_t R = ~(e_int << 1) & vmask;
  tile_unions<WPR, TH>(par, R, e_int, d_int, vmask, ry, w, P.nrows, s_eint, lbase, a.tb.err);
  __syncthreads();
  compress_runs(par, R, lbase);

  // ---- global roots of this tile's slots
  const int nsl = a.tb.nslots[P.tile];
  for (int j = tid; j < nsl; j += NT) {
    const uint64_t v = find_global(a.tb.nodes, (uint32_t)P.tile * MS + j, a.tb.err);
    const uint32_t key = (uint32_t)(v >> 32);
    s_slotval[j] = LABELS ? (int)key : (int)flip_bit(key, a.t, a.ks);
    if (HIST) s_slotroot[j] = (uint32_t)v;
  }
  __syncthreads();
  for (int j = tid; j < NB; j += NT) {
    int y, x, r = -1;
    if (border_site<TW, TH>(P, j, y, x)) {
      const int rs = run_start(~(s_eint[y][x >> 5] << 1), x & 31);
      r = par[y * TW + (x & ~31) + rs];
    }
    s_broot[j] = r;
  }
  __syncthreads();
  // border roots: par[r] = -1 - slot
  const uint16_t* bs = a.tb.bslot + (size_t)P.tile * NB;
  for (int j = tid; j < NB; j += NT) {
    const int r = s_broot[j];
    if (r >= 0) par[r] = -1 - (int)bs[j];
  }
  __syncthreads();
  // inner roots of my word: their flip bits (one Philox block per root)
  if (!LABELS) {
    uint32_t fl = 0, RR = R;
    while (RR) {
      const int b = __ffs(RR) - 1;
      RR &= RR - 1;
      const int l = lbase + b;
      if (par[l] == l) {
        const uint32_t key = (uint32_t)(P.y0 + ry) * (uint32_t)L + (uint32_t)(P.x0 + 32 * w + b);
        fl |= flip_bit(key, a.t, a.ks) << b;
      }
    }
    s_iflip[tid] = fl;
    __syncthreads();
  }

  // ---- per run: root and its decision
  uint32_t tmask = 0, fprev = 0;
  {
    uint32_t RR = R;
    while (RR) {
      const int b = __ffs(RR) - 1;
      RR &= RR - 1;
      const int l = lbase + b;
      int r = l, p = par[l];
      if (p >= 0 && p != l) {
        r = p;
        p = par[r];
      }
      // p < 0: border root with slot -1-p; p == r: inner root r
      if (LABELS) {
        const int nxt = RR ? (__ffs(RR) - 1) : nb;
        const int key = p < 0 ? s_slotval[-1 - p]
                              : (int)((uint32_t)(P.y0 + r / TW) * (uint32_t)L + (uint32_t)(P.x0 + r % TW));
        int32_t* out = a.labels + (size_t)(P.y0 + ry) * L + P.x0 + 32 * w;
        for (int x = b; x < nxt; ++x) out[x] = key;
      } else {
        const uint32_t f = p < 0 ? (uint32_t)s_slotval[-1 - p] : ((s_iflip[r >> 5] >> (r & 31)) & 1u);
        tmask |= (f ^ fprev) << b;
        fprev = f;
        if (HIST) {
          const int nxt = RR ? (__ffs(RR) - 1) : nb;
          atomicAdd(&s_size[r], nxt - b);
        }
      }
    }
  }
  if (LABELS) return;

  // prefix xor turns "decision changes at this run start" into per-site flips
  tmask ^= tmask << 1;
  tmask ^= tmask << 2;
  tmask ^= tmask << 4;
  tmask ^= tmask << 8;
  tmask ^= tmask << 16;
  const uint32_t snew = s ^ (tmask & vmask);
  if (vmask) store_spin_bits(a.spins_out + (size_t)(P.y0 + ry) * L + P.x0 + 32 * w, snew, nb, g.aligned16);
  s_snew[ry][w] = snew;

  // ---- new spins of the halo sites: old spin (phase 1) xor their cluster's flip
  const uint32_t* bbits = a.tb.bbits + (size_t)P.tile * BBW;
  if (tid < TH) {
    bool bit = false;
    if (tid < P.nrows) {
      const int tileE = P.ty * g.tiles_x + (P.tx + 1) % g.tiles_x;
      const uint16_t slot = a.tb.bslot[(size_t)tileE * NB + tid];
      const uint64_t v = find_global(a.tb.nodes, (uint32_t)tileE * MS + slot, a.tb.err);
      const uint32_t old = (bbits[T::OFF_HE + (tid >> 5)] >> (tid & 31)) & 1u;
      bit = (old ^ flip_bit((uint32_t)(v >> 32), a.t, a.ks)) != 0u;
    }
    const uint32_t m = __ballot_sync(0xffffffffu, bit);
    if ((tid & 31) == 0) s_hEnew[tid >> 5] = m;
  }
  if (tid < TW) {
    bool bit = false;
    if (tid < P.ncols) {
      const int tileS = ((P.ty + 1) % g.tiles_y) * g.tiles_x + P.tx;
      const uint16_t slot = a.tb.bslot[(size_t)tileS * NB + 2 * TH + tid];
      const uint64_t v = find_global(a.tb.nodes, (uint32_t)tileS * MS + slot, a.tb.err);
      const uint32_t old = (bbits[T::OFF_HS + (tid >> 5)] >> (tid & 31)) & 1u;
      bit = (old ^ flip_bit((uint32_t)(v >> 32), a.t, a.ks)) != 0u;
    }
    const uint32_t m = __ballot_sync(0xffffffffu, bit);
    if ((tid & 31) == 0) s_hSnew[tid >> 5] = m;
  }
  __syncthreads();

  // ---- E and M of the new state (C10)
  uint32_t sEn;
  if (lastword) {
    const uint32_t hb = (s_hEnew[ry >> 5] >> (ry & 31)) & 1u;
    sEn = ((snew >> 1) & ((1u << pl) - 1u)) | (hb << pl);
  } else {
    sEn = (snew >> 1) | ((w + 1 < WPR) ? (s_snew[ry][w + 1] << 31) : 0u);
  }
  const uint32_t sSn = (ry + 1 < P.nrows) ? s_snew[ry + 1][w] : s_hSnew[w];
  const int nv = __popc(vmask);
  const int unequal = __popc((snew ^ sEn) & vmask) + __popc((snew ^ sSn) & vmask);
  long long eloc = 2LL * unequal - 2LL * nv;
  long long mloc = (long long)nv - 2LL * __popc(snew & vmask);
  eloc = warp_sum(eloc);
  mloc = warp_sum(mloc);
  if ((tid & 31) == 0) {
    s_red[0][tid >> 5] = eloc;
    s_red[1][tid >> 5] = mloc;
  }

  if (HIST) {
    // sizes are complete after this barrier: bin inner clusters here, send
    // border pieces to their global root
    __syncthreads();
    uint32_t RR = R;
    while (RR) {
      const int b = __ffs(RR) - 1;
      RR &= RR - 1;
      const int l = lbase + b;
      const int p = par[l];
      if (p == l) {
        const uint32_t sz = (uint32_t)s_size[l];
        atomicAdd(&s_hist[0], 1ull);
        atomicAdd(&s_hist[1], (unsigned long long)sz * sz);
        atomicAdd(&s_hist[2 + log2_floor(sz)], 1ull);
      } else if (p < 0) {
        atomicAdd(&a.csize[s_slotroot[-1 - p]], (uint32_t)s_size[l]);
      }
    }
  }
  __syncthreads();
  if (tid < 32) {
    long long ev = 0, mv = 0;
    for (int k = tid; k < NT / 32; k += 32) {
      ev += s_red[0][k];
      mv += s_red[1][k];
    }
    ev = warp_sum(ev);
    mv = warp_sum(mv);
    if (tid == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(a.em), (unsigned long long)ev);
      atomicAdd(reinterpret_cast<unsigned long long*>(a.em + 1), (unsigned long long)mv);
    }
  }
  if (HIST && tid < 34 && s_hist[tid]) atomicAdd(reinterpret_cast<unsigned long long*>(a.hist + tid), s_hist[tid]);
}

// ================================================================ phase 4

template <int WPR, int TH>
__global__ void phase4_kernel(const SweepArgs a) {
  using T = Tile<WPR, TH>;
  constexpr int MS = T::MS;
  __shared__ unsigned long long s_hist[34];
  if (threadIdx.x < 34) s_hist[threadIdx.x] = 0ull;
  __syncthreads();
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)a.g.tiles_x * a.g.tiles_y * MS;
  if (n < total) {
    const int tile = (int)(n / MS), slot = (int)(n % MS);
    if (slot < a.tb.nslots[tile]) {
      const uint64_t v = ld_node(a.tb.nodes + n);
      if ((uint32_t)v == (uint32_t)n) {
        const uint32_t sz = a.csize[n];
        atomicAdd(&s_hist[0], 1ull);
        atomicAdd(&s_hist[1], (unsigned long long)sz * sz);
        atomicAdd(&s_hist[2 + log2_floor(sz)], 1ull);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 34 && s_hist[threadIdx.x])
    atomicAdd(reinterpret_cast<unsigned long long*>(a.hist + threadIdx.x), s_hist[threadIdx.x]);
}

// ================================================================ helpers

__global__ void init_kernel(int8_t* spins, long long n, KeySchedule ks, int cold) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int8_t v = 1;
    if (!cold) v = (philox4x32_10(make_uint4((uint32_t)i, 0u, 2u, 0u), ks).x >> 31) ? (int8_t)-1 : (int8_t)1;
    spins[i] = v;
  }
}

__global__ void check_spins_kernel(const int8_t* spins, long long n, int* err) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int8_t v = spins[i];
    if (v != 1 && v != -1) atomicCAS(err, 0, kErrBadSpin);
  }
}

template <int WPR, int TH>
__global__ void export_bonds_kernel(const SweepArgs a, uint8_t* out) {
  constexpr int TW = 32 * WPR, NT = WPR * TH;
  const int L = a.g.L;
  const long long n = (long long)L * L;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / L), x = (int)(i % L);
    const int tile = (y / TH) * a.g.tiles_x + x / TW;
    const int ry = y % TH, xx = x % TW;
    const int t = ry * WPR + (xx >> 5), b = xx & 31;
    const uint32_t* tb = a.tb.tbits + (size_t)tile * 3 * NT;
    out[i] = (uint8_t)(((tb[NT + t] >> b) & 1u) | (((tb[2 * NT + t] >> b) & 1u) << 1));
  }
}

int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g > 152LL * 64) g = 152LL * 64;
  return (int)(g < 1 ? 1 : g);
}

template <int WPR, int TH>
cudaError_t launch_all(int which, const SweepArgs& a, int mode, uint8_t* out, cudaStream_t st) {
  using T = Tile<WPR, TH>;
  const int ntiles = a.g.tiles_x * a.g.tiles_y;
  switch (which) {
    case 1:
      phase1_kernel<WPR, TH><<<ntiles, T::NT, 0, st>>>(a);
      break;
    case 2: {
      const long long total = (long long)ntiles * (TH + T::TW);
      phase2_kernel<WPR, TH><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a);
      break;
    }
    case 3:
      if (mode == 0) {
        phase3_kernel<WPR, TH, 0><<<ntiles, T::NT, 0, st>>>(a);
      } else if (mode == 1) {
        const size_t dyn = (size_t)TH * T::TW * sizeof(int);
        static bool attr_done = false;
        if (!attr_done) {
          cudaError_t e = cudaFuncSetAttribute(phase3_kernel<WPR, TH, 1>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
          if (e != cudaSuccess) return e;
          attr_done = true;
        }
        phase3_kernel<WPR, TH, 1><<<ntiles, T::NT, dyn, st>>>(a);
      } else {
        phase3_kernel<WPR, TH, 2><<<ntiles, T::NT, 0, st>>>(a);
      }
      break;
    case 4: {
      const long long total = (long long)ntiles * T::MS;
      phase4_kernel<WPR, TH><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a);
      break;
    }
    case 5:
      export_bonds_kernel<WPR, TH><<<grid_for((long long)a.g.L * a.g.L, 256), 256, 0, st>>>(a, out);
      break;
  }
  return cudaGetLastError();
}

cudaError_t dispatch(int shape, int which, const SweepArgs& a, int mode, uint8_t* out, cudaStream_t st) {
  switch (shape) {
    case 0: return launch_all<4, 64>(which, a, mode, out, st);
    case 1: return launch_all<4, 32>(which, a, mode, out, st);
    case 2: return launch_all<2, 64>(which, a, mode, out, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_init(int8_t* spins, int L, uint64_t seed, int cold, cudaStream_t st) {
  const long long n = (long long)L * L;
  init_kernel<<<grid_for(n, 256), 256, 0, st>>>(spins, n, make_key_schedule(seed), cold);
  return cudaGetLastError();
}

cudaError_t launch_check_spins(const int8_t* spins, int64_t n, int* err, cudaStream_t st) {
  check_spins_kernel<<<grid_for(n, 256), 256, 0, st>>>(spins, n, err);
  return cudaGetLastError();
}

cudaError_t launch_phase1(int shape, const SweepArgs& a, cudaStream_t st) { return dispatch(shape, 1, a, 0, nullptr, st); }
cudaError_t launch_phase2(int shape, const SweepArgs& a, cudaStream_t st) { return dispatch(shape, 2, a, 0, nullptr, st); }
cudaError_t launch_phase3(int shape, const SweepArgs& a, bool labels_mode, cudaStream_t st) {
  return dispatch(shape, 3, a, labels_mode ? 2 : (a.hist && a.csize ? 1 : 0), nullptr, st);
}
cudaError_t launch_phase4(int shape, const SweepArgs& a, cudaStream_t st) { return dispatch(shape, 4, a, 0, nullptr, st); }
cudaError_t launch_export_bonds(int shape, const SweepArgs& a, uint8_t* out, cudaStream_t st) {
  return dispatch(shape, 5, a, 0, out, st);
}

}  // namespace sw
