// sw_kernels.cu -- the Swendsen-Wang sweep on sm_103a.
//
// One sweep (paper §2) runs as three phases (four launches) over tiles of TW = 32*WPR
// columns by TH rows. Sites are handled as bit masks, 32 per 32-bit word
// (bit k = site x0+32w+k). Phase 1 runs one warp per 32-column band of the
// tile; phase 3 runs one thread per word column of an H-row strip.
//
//  phase 1 (bonds §2.1 + tile-local clusters §2.3)
//    - int8 spins -> sign bits; the tile's east halo column and south halo
//      row are read too, so every east/south bond of the tile can be drawn;
//    - Philox-4x32-10 block (site>>1, t, 0, 0) gives the east and south words
//      of two consecutive sites (C5); bond iff equal spins and word < thr;
//    - clusters: a Hoshen-Kopelman scan down each 32-column band of the tile,
//      one warp per band and one lane per column. Runs (maximal stretches of
//      east bonds inside one row word) take the label of the run above them
//      that they are bonded to, or their first site as a new label; four bit
//      masks per row word (row_masks) say which column passes the label down
//      and which bonds join a second run above, whose labels are then united
//      (lock-free 16-bit union-find, the larger root under the smaller). Bands
//      are joined across their east bonds, and every new label is pointed at
//      its root, the smallest site of the tile component -- the "lowest value
//      label" of §2.3;
//    - every tile component that touches the tile border gets a slot; slot
//      nodes are initialised in a global 64-bit union-find whose entries are
//      (key << 32 | parent node), key = smallest global site index of the
//      tile component, so comparing entries compares keys;
//    - stores the spin/east/south bit masks (12 bytes per 32 sites), the
//      label of every site (16 bits), the slot of each border site, the
//      out-going border bonds and the halo spins (a few hundred bytes per
//      tile).
//  phase 2 (clusters across tiles, §2.3; device-side, no host round trip
//    as in §5's maintenance kernel)
//    - one thread per bonded tile-border edge (including the periodic wrap)
//      unites the two slot nodes with 64-bit atomicMin; consecutive edges
//      joining the same two slots are skipped.
//  phase 3 (new spins §2.4 + E/M, or canonical labels)
//    - receives the labels of the tile by one bulk copy (a run's root is
//      its label's entry), takes each border
//      component's decision from its global root (its key is the cluster's
//      canonical label, C9) and each inner component's from its own root;
//    - under the flip rule (C6) the bits of a row word's 32 site indices
//      come from one Philox block, so all inner roots of the word are
//      decided by one draw; the flip mask of a word is built from its runs
//      with a prefix xor;
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
constexpr long long kBulkWaitCycles = 1LL << 31;  // ~1 s at the SM clock: limit of a bulk-copy wait

// Four int8 spins (+1 = 0x01, -1 = 0xFF) -> four sign bits.
__device__ __forceinline__ uint32_t sign_bits4(uint32_t w) {
  return ((w & 0x80808080u) * 0x00204081u) >> 28;
}
// Four sign bits -> four int8 spins.
__device__ __forceinline__ uint32_t spin_bytes4(uint32_t nib) {
  const uint32_t spread = (nib * 0x00204081u) & 0x01010101u;
  return 0x01010101u | (spread * 0xFEu);
}

// Spins are loaded past L1 (ld.cg): other CTAs of the fused batch kernel
// write them earlier in the same launch, and L1 is not kept coherent.
__device__ __forceinline__ uint32_t load_spin_bits(const int8_t* p, int nb, bool vec) {
  if (vec && nb == 32) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
    const uint4 u = __ldcg(q), v = __ldcg(q + 1);
    return sign_bits4(u.x) | (sign_bits4(u.y) << 4) | (sign_bits4(u.z) << 8) | (sign_bits4(u.w) << 12) |
           (sign_bits4(v.x) << 16) | (sign_bits4(v.y) << 20) | (sign_bits4(v.z) << 24) |
           (sign_bits4(v.w) << 28);
  }
  uint32_t bits = 0;
  for (int k = 0; k < nb; ++k) bits |= (uint32_t)(__ldcg(p + k) < 0) << k;
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

// §6 (q-state Potts): bit b of eqE / eqS is set iff site x0 + b of `row`
// has the same state as its east neighbour (column x0 + b + 1 mod L) / as
// the site below it (`rowS`, the next row mod L); nb valid columns. A whole
// 16-byte aligned word compares four states per instruction.
__device__ __forceinline__ void potts_equal_bits(const int8_t* row, const int8_t* rowS, int x0, int nb, int L,
                                                 bool vec, uint32_t& eqE, uint32_t& eqS) {
  if (vec && nb == 32) {
    const uint4 a0 = *reinterpret_cast<const uint4*>(row + x0), a1 = *reinterpret_cast<const uint4*>(row + x0 + 16);
    const uint4 b0 = *reinterpret_cast<const uint4*>(rowS + x0), b1 = *reinterpret_cast<const uint4*>(rowS + x0 + 16);
    const uint32_t A[9] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w,
                           (uint32_t)(uint8_t)row[x0 + 32 == L ? 0 : x0 + 32]};
    const uint32_t B[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
    uint32_t e = 0u, d = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      // the four east neighbours of word k's states: bytes 1-3 of word k, byte 0 of word k + 1
      e |= sign_bits4(__vcmpeq4(A[k], __funnelshift_r(A[k], A[k + 1], 8))) << (4 * k);
      d |= sign_bits4(__vcmpeq4(A[k], B[k])) << (4 * k);
    }
    eqE = e;
    eqS = d;
    return;
  }
  uint32_t e = 0u, d = 0u;
  for (int b = 0; b < nb; ++b) {
    const int x = x0 + b;
    const int8_t v = row[x];
    e |= (uint32_t)(v == row[x + 1 == L ? 0 : x + 1]) << b;
    d |= (uint32_t)(v == rowS[x]) << b;
  }
  eqE = e;
  eqS = d;
}

// ------------------------------------------------ shared-memory union-find
// Parents are 16-bit local site indices (par[x] <= x; roots point to
// themselves).

// Hang root a under b if a is still a root: one 16-bit compare-and-swap of
// par[a] from a to b. Returns the entry found (a on success).
__device__ __forceinline__ int link_root_u16(uint16_t* par, int a, int b) {
  return (int)atomicCAS(reinterpret_cast<unsigned short*>(par + a), (unsigned short)a, (unsigned short)b);
}


// Lock-free unions of one warp, one pair per lane (lanes with active ==
// false take part without a pair). Every lane runs the same loop, one step
// per trip: while a lane's two nodes are not both roots, each moves to its
// grandparent (path halving, plain 16-bit stores of ancestors); at two
// distinct roots the larger is hung under the smaller by a 16-bit
// compare-and-swap, and a failed link (another lane linked that root first)
// carries on from the root's new parent. The trip condition is decided for
// the whole warp (__any_sync), so the lanes stay together and a trip costs one
// pass of the warp, however the lanes' paths differ. The cap only guards
// against corrupted memory. Every lane of the warp must call this.
__device__ void unite_warp(uint16_t* par, int a, int b, bool active, int* err) {
  bool done = !active;
  for (int it = 0; __any_sync(0xffffffffu, !done); ++it) {
    if (it >= kUnionCap) {
      if (!done) atomicCAS(err, 0, kErrUnionCap);
      break;
    }
    if (done) continue;
    const int pa = par[a], pb = par[b];
    if (pa == a && pb == b) {
      if (a == b) {
        done = true;
      } else {
        const int hi = max(a, b), lo = min(a, b);
        const int old = link_root_u16(par, hi, lo);
        done = old == hi;
        a = old;  // on failure: the linked root's new parent
        b = lo;
      }
    } else {
      if (pa != a) {
        const int ga = par[pa];
        if (ga != pa) par[a] = (uint16_t)ga;
        a = ga;
      }
      if (pb != b) {
        const int gb = par[pb];
        if (gb != pb) par[b] = (uint16_t)gb;
        b = gb;
      }
    }
  }
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

// Root entries of nodes a and b: the walks of find_global, advanced in step
// so that the two chains of dependent loads are in flight together.
__device__ void find_global2(uint64_t* nodes, uint32_t a, uint32_t b, uint64_t& va, uint64_t& vb, int* err) {
  va = ld_node(nodes + a);
  vb = ld_node(nodes + b);
  for (int it = 0;; ++it) {
    const bool ra = (uint32_t)va == a, rb = (uint32_t)vb == b;
    if (ra && rb) return;
    if (it >= kGlobalFindCap) {
      atomicCAS(err, 0, kErrUnionCap);
      return;
    }
    const uint32_t pa = (uint32_t)va, pb = (uint32_t)vb;
    const uint64_t wa = ra ? va : ld_node(nodes + pa);  // the parents' entries
    const uint64_t wb = rb ? vb : ld_node(nodes + pb);
    const bool ha = !ra && (uint32_t)wa != pa, hb = !rb && (uint32_t)wb != pb;  // parent not a root: halve
    if (ha) atomicMin(reinterpret_cast<unsigned long long*>(nodes + a), (unsigned long long)wa);
    if (hb) atomicMin(reinterpret_cast<unsigned long long*>(nodes + b), (unsigned long long)wb);
    if (!ra) a = ha ? (uint32_t)wa : pa;
    if (!rb) b = hb ? (uint32_t)wb : pb;
    va = ha ? ld_node(nodes + a) : wa;  // the grandparents' entries, or the roots'
    vb = hb ? ld_node(nodes + b) : wb;
  }
}

__device__ void unite_global(uint64_t* nodes, uint32_t a, uint32_t b, int* err) {
  for (int it = 0; it < kGlobalUnionCap; ++it) {
    uint64_t va, vb;
    find_global2(nodes, a, b, va, vb, err);
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

template <int WPR, int TH, int H>
struct Tile {
  static constexpr int TW = 32 * WPR;
  static constexpr int NS = TH / H;                 // strips per tile
  static constexpr int NT = WPR * NS;               // threads per tile
  static constexpr int RW = WPR * TH;               // row-words per tile
  static constexpr int NB = 2 * TH + 2 * TW;        // border sites: left, right, top, bottom
  static constexpr int MS = 2 * (TW + TH);          // slots per tile
  static constexpr int BBW = 2 * (TH / 32) + 2 * (TW / 32);
  static constexpr int OFF_EOUT = 0, OFF_SOUT = TH / 32, OFF_HE = TH / 32 + TW / 32,
                       OFF_HS = 2 * (TH / 32) + TW / 32;
  static_assert(TH % 32 == 0 && TH % H == 0, "TH must be a multiple of 32 and of H");
  static_assert(NT % 32 == 0, "whole warps per tile");
  static_assert(TW * TH <= 32768, "16-bit parents with a mark bit");
  static_assert(MS < 32768, "slots fit below the mark bit");
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

// Valid bits of word w in a tile with ncols valid columns. Every shift in
// these kernels keeps its count inside [0, 31]: an out-of-range shift is
// undefined behaviour, and the optimiser has been seen to act on it even
// behind a guarding conditional.
__device__ __forceinline__ uint32_t word_mask(int ncols, int w) {
  const int nb = max(0, min(32, ncols - 32 * w));
  return nb == 0 ? 0u : (0xffffffffu >> (32 - nb));
}

// Bit of the tile's last valid column inside word w (0 if w does not hold it).
__device__ __forceinline__ uint32_t last_column_bit(int ncols, int w) {
  const int pl = ncols - 1 - 32 * w;
  return (pl >= 0 && pl < 32) ? (1u << (pl & 31)) : 0u;
}

// ------------------------------------------------- row masks of the band scan
//
// Phase 1 labels a tile by a Hoshen-Kopelman scan down each 32-column band:
// the rows are visited top to bottom, every run (a maximal stretch of east
// bonds inside one row word) takes the label of the run above it that it is
// bonded to, or a new label (its first site) when it has no bond upwards,
// and a run bonded to several runs above that carry different labels makes
// those labels equivalent (a union). What each run of a row needs -- which of
// its columns passes the label down, which columns join a further run above
// -- follows from four bit masks of the row, computed for all runs of a word
// at once.

// Bits j of D whose interval (previous bit of D below j, j] holds a bit of X
// (for the lowest bit of D the interval starts at bit 0). One addition scans
// all intervals: a bit of X outside D starts a carry that runs up through the
// bits outside D and stops on the next bit of D.
__device__ __forceinline__ uint32_t carry_hit(uint32_t X, uint32_t D) {
  const uint32_t nd = ~D;
  return ((nd + (X & nd)) & D) | (X & D);
}

// Masks of row word B given the row word A above it in the same band. eB, eA:
// east bonds inside the tile (bit 31 = bond into the next word, not part of a
// run here); vB, vA: valid columns; D: south bonds from A into B.
//   R: run starts of B;
//   F: the first column of each run of B with a bond upwards -- the run takes
//      the label of the site above that column;
//   S: F, plus the start of every run with no bond upwards (a new label);
//   M: the other bonds upwards that reach a run of A different from the one
//      reached by the previous bond of the same run of B -- each asks for a
//      union of that run's label with the label of the run of B.
struct RowMasks {
  uint32_t R, S, F, M;
};
__device__ __forceinline__ RowMasks row_masks(uint32_t eB, uint32_t vB, uint32_t eA, uint32_t vA, uint32_t D) {
  const uint32_t RB = ~(eB << 1) & vB;
  const uint32_t RA = ~(eA << 1) & vA;
  const uint32_t F = carry_hit(RB, D);
  const uint32_t M = carry_hit(RA, D) & ~F;
  // runs of B that hold a bit of D: the same scan on the reversed word, where
  // a run's start is the top of its interval
  const uint32_t withD = __brev(carry_hit(__brev(D), __brev(RB)));
  RowMasks m;
  m.R = RB;
  m.F = F;
  m.M = M;
  m.S = F | (RB & ~withD);
  return m;
}

// Sum of v over the lanes below this one.
__device__ __forceinline__ int warp_exclusive_sum(int v, int lane) {
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  return incl - v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int log2_floor(uint32_t v) { return 31 - __clz(v); }

// --------------------------------------------- bulk copies into shared memory

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Called by one thread: start a copy of `bytes` from global memory at src to
// shared memory at dst on the copy engine (cp.async.bulk; both addresses
// 16-byte aligned, bytes a multiple of 16), its completion counted on the
// mbarrier `bar` (initialised here for one arrival plus the transaction
// bytes). Other threads may wait on `bar` only after a block barrier.
__device__ __forceinline__ void bulk_load_start(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Wait until the copy counted on `bar` has landed; false after about a
// second without completion.
__device__ __forceinline__ bool bulk_load_wait(unsigned long long* bar) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar))
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kBulkWaitCycles) return false;
  }
}

// Exclusive prefix sums of popc(mask[i]), i < RW, into pre[i]; returns the
// total. Words are split into contiguous chunks of C per thread. Called by
// every thread of the block (contains barriers).
template <int RW, int NT>
__device__ __forceinline__ int block_popc_prefix(const uint32_t* mask, uint32_t* pre, uint32_t* s_wsum) {
  constexpr int C = (RW + NT - 1) / NT;
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t loc[C];
  uint32_t sum = 0;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int i = tid * C + c;
    loc[c] = sum;
    sum += i < RW ? (uint32_t)__popc(mask[i]) : 0u;
  }
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t v = lane < NW ? s_wsum[lane] : 0u;
    uint32_t in2 = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, in2, o);
      if (lane >= o) in2 += t;
    }
    __syncwarp();
    if (lane < NW) s_wsum[lane] = in2 - v;
    if (lane == 31) s_wsum[32] = in2;
  }
  __syncthreads();
  const uint32_t base = s_wsum[warp] + incl - sum;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int i = tid * C + c;
    if (i < RW) pre[i] = base + loc[c];
  }
  const int total = (int)s_wsum[32];
  __syncthreads();
  return total;
}

// Slot of border root r: its rank among the marked roots in index order.
__device__ __forceinline__ int slot_of(const uint32_t* bmask, const uint32_t* pre, int r) {
  return (int)(pre[r >> 5] + (uint32_t)__popc(bmask[r >> 5] & ((1u << (r & 31)) - 1u)));
}

// The sweep arguments of a tile: the kernel parameter for one lattice (tile
// T), or the replica descriptor of batch tile T. k: sweeps past the
// descriptor's counter (the fused batch kernel runs several sweeps in one
// launch; a replica takes part in sweep k only while k < its sweeps left).
template <bool BATCH>
__device__ __forceinline__ bool cta_args(const SweepArgs& a0, const BatchArgs& b, int T, int k, SweepArgs& A,
                                         int& tile) {
  if (!BATCH) {
    A = a0;
    tile = T;
    return true;
  }
  const int r = b.tile_rep[T];
  if (r < 0) return false;  // a spare tile of the launch bucket
  const ReplicaDesc* D = b.descs + r;
  A = D->a;
  A.t = D->t + (uint32_t)k;
  A.em = D->em_base + 2 * (D->em_next + k);
  tile = T - D->tile0;
  return D->active != 0 && D->t_left > k;
}

// ================================================================ phase 1

// The bond draws (C5) of the row word of sites i0 .. i0 + nb - 1 in sweep t:
// bit b of .x (.y) is set iff the east (south) word of site i0 + b is below
// thr. Site i takes words x0 (east) and x1 (south) of block (i >> 1, t, 0, 0)
// when i is even, x2 and x3 when it is odd.
__device__ __forceinline__ uint2 bond_draws(uint32_t i0, int nb, int L, uint32_t t, uint32_t thr,
                                            const KeySchedule& ks) {
  uint32_t rE = 0u, rS = 0u;
  if ((L & 1) == 0) {
    // even L: sites i0+b, i0+b+1 (b even) share Philox block (i0+b)/2
    if (nb == 32) {
      // a whole word: each comparison is the carry of one subtraction, added
      // into the mask as its new lowest bit (a set carry: q >= thr, no bond),
      // so site 0 ends at bit 31; one bit reversal and a complement at the
      // end. Fewer integer-pipe operations than a compare and a select each.
#pragma unroll 4
      for (int b = 0; b < 32; b += 2) {
        const uint4 q = philox4x32_10(make_uint4((i0 + b) >> 1, t, 0u, 0u), ks);
        asm("{\n\t.reg .u32 d;\n\t"
            "sub.cc.u32 d, %2, %6;\n\taddc.u32 %0, %0, %0;\n\t"
            "sub.cc.u32 d, %4, %6;\n\taddc.u32 %0, %0, %0;\n\t"
            "sub.cc.u32 d, %3, %6;\n\taddc.u32 %1, %1, %1;\n\t"
            "sub.cc.u32 d, %5, %6;\n\taddc.u32 %1, %1, %1;\n\t}"
            : "+r"(rE), "+r"(rS)
            : "r"(q.x), "r"(q.y), "r"(q.z), "r"(q.w), "r"(thr));
      }
      rE = __brev(~rE);
      rS = __brev(~rS);
    } else {
#pragma unroll 4
      for (int b = 0; b < 32; b += 2) {
        if (b < nb) {
          const uint4 q = philox4x32_10(make_uint4((i0 + b) >> 1, t, 0u, 0u), ks);
          rE |= ((uint32_t)(q.x < thr) << b) | ((uint32_t)(q.z < thr) << (b + 1));
          rS |= ((uint32_t)(q.y < thr) << b) | ((uint32_t)(q.w < thr) << (b + 1));
        }
      }
    }
  } else {
    for (int b = 0; b < nb; ++b) {
      const uint32_t i = i0 + b;
      const uint4 q = philox4x32_10(make_uint4(i >> 1, t, 0u, 0u), ks);
      const uint32_t we = (i & 1u) ? q.z : q.x, ws = (i & 1u) ? q.w : q.y;
      rE |= (uint32_t)(we < thr) << b;
      rS |= (uint32_t)(ws < thr) << b;
    }
  }
  return make_uint2(rE, rS);
}

// Phase 1 runs one warp per 32-column band and asks for 1280 resident
// threads an SM (at most 51 registers a thread; ten CTAs of 128 threads also
// fit their shared memory).
// Phase 3 runs strips of H rows; with two-row strips it asks for 1280
// resident threads an SM as well. Taller strips would spill under that bound
// and keep the compiler's choice.
template <int NT, int H>
constexpr int strip_min_blocks() {
  return H == 2 ? 1280 / NT : 1;
}

template <int NT>
constexpr int band_min_blocks() {
  return 1280 / NT > 0 ? 1280 / NT : 1;
}

// One CTA per tile, one warp per 32-column band (word column) of it.
//  1. spins -> sign bits, halo, bonds (§2.1): row words handed out so that
//     consecutive threads read consecutive 32-site words of a row;
//  2. row masks (row_masks) of every row of the band, one lane per row;
//  3. the scan (§2.3): the warp walks the band's rows top to bottom, lane l
//     holding column l; per row each lane finds its run's start and the
//     column that names the run (S), and reads the label from that column's
//     lane: the label of the site above it (F) or that site's own index (a
//     new label). Labels are tile-local site indices, so the smaller of two
//     equivalent labels is the smaller site. Every site's label is stored in
//     par[]; a new label's entry (par[x] = x) is a union-find root;
//  4. the unions: each bond of M (its two sites carry the labels to unite)
//     and each east bond across a band border, by a lock-free union run by
//     all lanes of a warp together (unite_warp: the larger root hung under
//     the smaller); then every new label is pointed at its root, so that
//     par[par[x]] is the root of site x, the component's smallest site -- the
//     "lowest value label" of §2.3;
//  5. border components get slots and global nodes, as the cross-tile merge
//     (phase 2) needs them; par, the masks and the tables go to global memory.
// Shared memory of phase 1 for one tile.
template <int WPR, int TH, int H>
struct P1Shared {
  using T = Tile<WPR, TH, H>;
  alignas(16) uint16_t par[TH * T::TW];  // label of every site; a label's entry is its union-find parent
  // spin bits and south bonds of the row words; once the row masks are
  // built, the warps' union work lists; after the unions, sd[0] holds the
  // border-root marks and sd[1] the border sites' roots (int16)
  alignas(16) uint32_t sd[2][TH][WPR];
  union {
    uint32_t eint[TH][WPR];  // east bonds inside the tile (to the cross-band unions)
    uint32_t pre[T::RW];     // then the prefix counts of the border-root marks
  };
  uint32_t bb[T::BBW];
  uint32_t wsum[33];
  // the border sites' roots live in sd[1] where they fit (TH >= 64), else here
  static constexpr bool kOwnBroot = T::NB * sizeof(int16_t) > sizeof(uint32_t) * TH * WPR;
  int16_t broot_own[kOwnBroot ? T::NB : 1];
  __device__ int16_t* broot() { return kOwnBroot ? broot_own : reinterpret_cast<int16_t*>(&sd[1][0][0]); }
};

// SPINS_GIVEN: the caller has put the spin words in S.sd[0] and the halo's
// spins in S.bb (east column, south row), as phase 3 of the previous sweep
// leaves them (phase31_kernel); the spins are not read from global memory.
// POTTS: spins_in holds q-state Potts states (§6); an edge may bond iff its
// two states are equal, and no spin words or halo spins are kept.
template <int WPR, int TH, int H, bool BATCH, bool SPINS_GIVEN = false, bool POTTS = false>
__device__ __forceinline__ void phase1_body(P1Shared<WPR, TH, H>& S, const SweepArgs& a0, const BatchArgs& bat,
                                            int T, int k) {
  using Tl = Tile<WPR, TH, H>;
  constexpr int TW = Tl::TW, NB = Tl::NB, MS = Tl::MS, BBW = Tl::BBW, RW = Tl::RW;
  constexpr int NT = 32 * WPR;  // threads of phase 1
  constexpr int RPL = TH / 32;  // rows per lane
  static_assert(TH % 32 == 0, "whole warps of rows");
  uint16_t* const par = S.par;
  uint32_t(&s_sd)[2][TH][WPR] = S.sd;
  uint32_t(&s_eint)[TH][WPR] = S.eint;
  uint32_t* const s_bb = S.bb;
  int16_t* const s_broot = S.broot();  // written after the unions
  uint32_t* const s_pre = S.pre;
  uint32_t* const s_wsum = S.wsum;
  uint32_t(*const s_spin)[WPR] = s_sd[0];
  uint32_t(*const s_dint)[WPR] = s_sd[1];
  uint32_t* const s_bmask = &s_sd[0][0][0];  // border roots (RW words), after the unions
  constexpr int kListCap = 4 * TH;           // entries of a warp's work list: fills s_sd
  static_assert(WPR * kListCap * sizeof(uint16_t) == sizeof(s_sd), "work lists fill s_sd");

  SweepArgs a;
  int tile;
  if (!cta_args<BATCH>(a0, bat, T, k, a, tile)) return;
  const Geometry& g = a.g;
  const int L = g.L;
  const TilePos P = tile_pos<TW, TH>(g, tile);
  const int tid = threadIdx.x, lane = tid & 31, warp0 = tid & ~31;
  uint32_t* eout = s_bb + Tl::OFF_EOUT;
  uint32_t* sout = s_bb + Tl::OFF_SOUT;
  uint32_t* hE = s_bb + Tl::OFF_HE;
  uint32_t* hS = s_bb + Tl::OFF_HS;

  if (SPINS_GIVEN || POTTS) {
    // out-going bond bits; the halo is given (or, for Potts, not kept)
    for (int i = tid; i < (POTTS ? BBW : Tl::OFF_HE); i += NT) s_bb[i] = 0u;
    __syncthreads();
  } else {
    for (int i = tid; i < BBW; i += NT) s_bb[i] = 0u;

    // ---- spins: thread tid takes row words tid, tid + NT, ... (row-major)
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      const int rw = tid + NT * i, y = rw / WPR, w = rw % WPR;
      const int nbw = max(0, min(32, P.ncols - 32 * w));
      uint32_t sb = 0u;
      if (y < P.nrows && nbw)
        sb = load_spin_bits(a.spins_in + (size_t)(P.y0 + y) * L + P.x0 + 32 * w, nbw, g.aligned16);
      s_spin[y][w] = sb;
    }
    __syncthreads();

    // ---- east halo column and south halo row (periodic wrap)
    const int xe = (P.x0 + P.ncols) % L;
    const int ys = (P.y0 + P.nrows) % L;
    for (int b0 = warp0; b0 < TH; b0 += NT) {
      const int y = b0 + lane;
      const bool bit = y < P.nrows && __ldcg(a.spins_in + (size_t)(P.y0 + y) * L + xe) < 0;
      const uint32_t m = __ballot_sync(0xffffffffu, bit);
      if (lane == 0) hE[b0 >> 5] = m;
    }
    for (int ww = tid; ww < WPR; ww += NT) {
      const int nbw = max(0, min(32, P.ncols - 32 * ww));
      hS[ww] = nbw ? load_spin_bits(a.spins_in + (size_t)ys * L + P.x0 + 32 * ww, nbw, g.aligned16) : 0u;
    }
    __syncthreads();
  }

  // ---- bonds (§2.1), same row words as the spins
  uint32_t* tb = a.tb.tbits + (size_t)P.tile * 3 * RW;
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    const int rw = tid + NT * i, y = rw / WPR, w = rw % WPR;
    const int nb = max(0, min(32, P.ncols - 32 * w));
    const uint32_t vmask = y < P.nrows ? word_mask(P.ncols, w) : 0u;
    const uint32_t lbit = last_column_bit(P.ncols, w);  // nonzero iff this word holds the tile's last column
    uint32_t s = 0u, eqE = 0u, eqS = 0u;
    if (POTTS) {
      if (vmask) {
        const int yg = P.y0 + y;
        potts_equal_bits(a.spins_in + (size_t)yg * L, a.spins_in + (size_t)(yg + 1 == L ? 0 : yg + 1) * L,
                         P.x0 + 32 * w, nb, L, g.aligned16, eqE, eqS);
        eqE &= vmask;
        eqS &= vmask;
      }
    } else {
      s = s_spin[y][w];
      uint32_t sE;
      if (lbit) {
        const uint32_t hb = (hE[y >> 5] >> (y & 31)) & 1u;
        sE = ((s >> 1) & (lbit - 1u)) | (hb ? lbit : 0u);
      } else {
        sE = (s >> 1) | ((w + 1 < WPR) ? (s_spin[y][w + 1] << 31) : 0u);
      }
      const uint32_t sS = (y + 1 < P.nrows) ? s_spin[y + 1][w] : hS[w];
      eqE = ~(s ^ sE) & vmask;
      eqS = ~(s ^ sS) & vmask;
    }
    uint32_t rE = 0, rS = 0;
    if (vmask) {
      if (a.draws_in) {
        const uint2 d = __ldcs(a.draws_in + (size_t)P.tile * RW + rw);
        rE = d.x;
        rS = d.y;
      } else {
        const uint2 d = bond_draws((uint32_t)(P.y0 + y) * (uint32_t)L + (uint32_t)(P.x0 + 32 * w), nb, L, a.t,
                                   a.thr, a.ks);
        rE = d.x;
        rS = d.y;
      }
    }
    const uint32_t e = eqE & rE, d = eqS & rS;
    s_eint[y][w] = e & ~lbit;
    s_dint[y][w] = (y + 1 < P.nrows) ? d : 0u;
    if (vmask && (e & lbit)) atomicOr(&eout[y >> 5], 1u << (y & 31));
    if (vmask && y == P.nrows - 1) sout[w] = d;
    tb[rw] = s;
    tb[RW + rw] = e;
    tb[2 * RW + rw] = d;
  }
  __syncthreads();

  // ---- row masks of my band: warp w = word column w, lane l holds rows l + 32 j
  const int w = tid >> 5;
  const uint32_t wmask = word_mask(P.ncols, w);
  uint32_t mR[RPL], mS[RPL], mF[RPL], mM[RPL];
#pragma unroll
  for (int j = 0; j < RPL; ++j) {
    const int y = lane + 32 * j;
    mR[j] = mS[j] = mF[j] = mM[j] = 0u;
    if (y < P.nrows && wmask) {
      const uint32_t eA = y > 0 ? s_eint[y - 1][w] : 0u, D = y > 0 ? s_dint[y - 1][w] : 0u;
      const RowMasks m = row_masks(s_eint[y][w], wmask, eA, y > 0 ? wmask : 0u, D);
      mR[j] = m.R;
      mS[j] = m.S;
      mF[j] = m.F;
      mM[j] = m.M;
    }
  }

  // ---- the scan (§2.3) down my band, lane = column: label propagation only;
  // the unions that M asks for are done afterwards from the stored labels
  if (wmask) {  // the same in every lane of the warp
    const uint32_t le = 0xffffffffu >> (31 - lane);  // bits 0..lane
    uint32_t lab = 0u;                                // label of my column's site in the row above
    int own = 32 * w + lane;                          // my column's site in the current row
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
      const int rows = min(32, P.nrows - 32 * j);
#pragma unroll 4
      for (int yy = 0; yy < rows; ++yy) {
        const uint32_t R = __shfl_sync(0xffffffffu, mR[j], yy);
        const uint32_t S = __shfl_sync(0xffffffffu, mS[j], yy);
        const uint32_t F = __shfl_sync(0xffffffffu, mF[j], yy);
        const int s = 31 - __clz(R & le);                   // start of my run (bit 0 is always a start)
        const int src = __ffs(S & (0xffffffffu << s)) - 1;  // the column that names my run
        const uint32_t v = ((F >> lane) & 1u) ? lab : (uint32_t)own;
        lab = __shfl_sync(0xffffffffu, v, src);
        par[own] = (uint16_t)lab;
        own += TW;
      }
    }
  }
  __syncthreads();

  // ---- unions inside the band: every bond of M (the site above and the
  // site below it carry labels of two runs that M says may differ). The
  // warp lists its bonds in shared memory (in rounds of kListCap) and works
  // through the list with one state machine per lane: a lane takes the next
  // entry as soon as its union is done, and each warp-wide trip moves every
  // busy lane one step (both nodes a halving step up, or at two distinct roots
  // the larger hung under the smaller). Only this warp touches its band's
  // labels here, so a link is a plain store checked after __syncwarp: when
  // two lanes hang the same root in one trip, one store stands and the other
  // lane goes on from the root's new parent.
  {
    uint16_t* list = reinterpret_cast<uint16_t*>(&s_sd[0][0][0]) + w * kListCap;
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < RPL; ++j) cnt += __popc(mM[j]);
    const int first = warp_exclusive_sum(cnt, lane);
    const int total = __shfl_sync(0xffffffffu, first + cnt, 31);
    for (int r0 = 0; r0 < total; r0 += kListCap) {  // the same rounds in every lane
      int idx = first;
#pragma unroll
      for (int j = 0; j < RPL; ++j) {
        for (uint32_t m = mM[j]; m; m &= m - 1, ++idx)
          if (idx >= r0 && idx < r0 + kListCap)
            list[idx - r0] = (uint16_t)((lane + 32 * j) * TW + 32 * w + __ffs(m) - 1);
      }
      __syncwarp();
      const int n = min(kListCap, total - r0);
      int k = lane, xa = 0, xb = 0;
      bool busy = false;
      for (int it = 0;; ++it) {
        if (!busy && k < n) {
          xb = list[k];  // a site bonded to the site above it
          xa = xb - TW;
          k += 32;
          busy = true;
        }
        if (!__any_sync(0xffffffffu, busy)) break;
        if (it >= kUnionCap) {
          if (busy) atomicCAS(a.tb.err, 0, kErrUnionCap);
          break;
        }
        int hi = -1, lo = 0;
        if (busy) {
          const int pa = par[xa], pb = par[xb];
          if (pa == xa && pb == xb) {
            if (xa == xb) {
              busy = false;
            } else {
              hi = max(xa, xb);
              lo = min(xa, xb);
              par[hi] = (uint16_t)lo;
            }
          } else {
            if (pa != xa) {
              const int ga = par[pa];
              if (ga != pa) par[xa] = (uint16_t)ga;
              xa = ga;
            }
            if (pb != xb) {
              const int gb = par[pb];
              if (gb != pb) par[xb] = (uint16_t)gb;
              xb = gb;
            }
          }
        }
        __syncwarp();
        if (hi >= 0) {
          const int now = par[hi];
          busy = now != lo;
          xa = now;
          xb = lo;
        }
      }
      __syncwarp();  // the list is rewritten by the next round
    }
  }
  __syncthreads();

  for (int i = tid; i < RW; i += NT) s_bmask[i] = 0u;  // the work lists are done with
  // (the next writes to s_bmask follow the barriers below)

  // ---- east bonds across band borders: two warps' labels, so the links are
  // compare-and-swaps (unite_warp)
  {
    uint32_t cross = 0u;  // bit j: row lane + 32 j has an east bond into the next band
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
      const int y = lane + 32 * j;
      if (w + 1 < WPR && y < P.nrows && (s_eint[y][w] >> 31)) cross |= 1u << j;
    }
    while (__any_sync(0xffffffffu, cross != 0u)) {
      int xa = 0;
      const bool have = cross != 0u;
      if (have) {
        xa = (lane + 32 * (__ffs(cross) - 1)) * TW + 32 * w + 31;  // last column of my word
        cross &= cross - 1;
      }
      unite_warp(par, xa, xa + 1, have, a.tb.err);
    }
  }
  __syncthreads();

  // ---- every new label is pointed at its root, and the roots are marked
  // for phase 3; par[par[x]] is then the root of site x. The trees are
  // shallow: three parents are read straight away and the walk goes on only
  // in the rare case that the third is not a root yet.
  {
    uint32_t* rb = a.tb.rbits + (size_t)P.tile * RW;
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
      const int y = lane + 32 * j, base = y * TW + 32 * w;
      uint32_t roots = 0u;
      for (uint32_t m = mS[j] & ~mF[j]; m; m &= m - 1) {
        const int b = __ffs(m) - 1, x = base + b;
        int r = par[x];
        if (r == x) {
          roots |= 1u << b;
        } else {
          r = par[par[r]];
          for (int p = par[r]; p != r; p = par[r]) r = p;
          par[x] = (uint16_t)r;
        }
      }
      rb[y * WPR + w] = roots;
    }
  }
  __syncthreads();

  // ---- border components -> slots (rank of the root in index order) and global nodes
  for (int j0 = 0; j0 < NB; j0 += NT) {  // the same trips in every lane (a warp-wide walk)
    const int j = j0 + tid;
    int y = 0, x = 0, r = 0;  // a lane without a border site walks from site 0, a root
    const bool ok = j < NB && border_site<TW, TH>(P, j, y, x);
    if (ok) r = par[y * TW + x];
    int p = par[r];
    while (__any_sync(0xffffffffu, p != r)) {
      if (p != r) {
        r = p;
        p = par[r];
      }
    }
    if (ok) atomicOr(&s_bmask[r >> 5], 1u << (r & 31));
    if (j < NB) s_broot[j] = ok ? (int16_t)r : (int16_t)-1;
  }
  __syncthreads();
  const int nsl = block_popc_prefix<RW, NT>(s_bmask, s_pre, s_wsum);
  {
    constexpr int C = (RW + NT - 1) / NT;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int i = tid * C + c;
      if (i >= RW) break;
      uint32_t m = s_bmask[i];
      uint32_t slot = s_pre[i];
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int r = i * 32 + b;
        const uint32_t node = (uint32_t)P.tile * MS + slot;
        const uint32_t key = (uint32_t)(P.y0 + r / TW) * (uint32_t)L + (uint32_t)(P.x0 + r % TW);
        a.tb.nodes[node] = ((uint64_t)key << 32) | node;
        if (a.csize) a.csize[node] = 0u;
        ++slot;
      }
    }
  }
  uint16_t* bs = a.tb.bslot + (size_t)P.tile * NB;
  for (int j = tid; j < NB; j += NT) {
    const int r = s_broot[j];
    bs[j] = r >= 0 ? (uint16_t)slot_of(s_bmask, s_pre, r) : (uint16_t)0xFFFFu;
  }
  // labels and border marks for phase 3
  {
    const uint4* src = reinterpret_cast<const uint4*>(par);
    uint4* dst = reinterpret_cast<uint4*>(a.tb.roots + (size_t)P.tile * (TW * TH));
    for (int i = tid; i < TW * TH / 8; i += NT) dst[i] = src[i];
    uint32_t* bm = a.tb.bmask + (size_t)P.tile * RW;
    for (int i = tid; i < RW; i += NT) bm[i] = s_bmask[i];
  }
  for (int i = tid; i < BBW; i += NT) a.tb.bbits[(size_t)P.tile * BBW + i] = s_bb[i];
  if (tid == 0) {
    if (nsl > MS) atomicCAS(a.tb.err, 0, kErrSlotOverflow);
    a.tb.nslots[P.tile] = nsl;
  }
  if (P.tile == 0) {
    if (a.em && tid < 2) a.em[tid] = 0;
    for (int i = tid; a.hist && i < 34; i += NT) a.hist[i] = 0;
  }
}

// The stand-alone phase 1 asks for eleven CTAs an SM (at most 40 registers a
// thread, 8 bytes spilled; its 19.6 KB of shared memory fit eleven times):
// 1.1 % faster than ten at L = 8192.
template <int NT>
constexpr int phase1_min_blocks() {
  return 1408 / NT > 0 ? 1408 / NT : 1;
}

template <int WPR, int TH, int H, bool BATCH>
__global__ void __launch_bounds__(32 * WPR, phase1_min_blocks<32 * WPR>())
    phase1_kernel(const SweepArgs a0, const BatchArgs bat) {
  __shared__ P1Shared<WPR, TH, H> S;
  phase1_body<WPR, TH, H, BATCH>(S, a0, bat, blockIdx.x, 0);
}

// ================================================================ phase 2

// Out-going border edge e of a tile (e < TH: the east edge of row e; else
// the south edge of column e - TH): true, with the two slot nodes to unite,
// iff the edge is bonded and does not repeat the previous edge's slot pair.
template <int WPR, int TH, int H>
__device__ __forceinline__ bool border_union(const SweepArgs& a, const TilePos& P, int tile, int e, uint32_t& na,
                                             uint32_t& nb) {
  using Tl = Tile<WPR, TH, H>;
  constexpr int TW = Tl::TW, NB = Tl::NB, MS = Tl::MS, BBW = Tl::BBW;
  const Geometry& g = a.g;
  const uint32_t* bb = a.tb.bbits + (size_t)tile * BBW;
  const uint16_t* bs = a.tb.bslot + (size_t)tile * NB;
  int i, off_out, off_a, off_b, nbr;
  if (e < TH) {
    i = e;
    if (i >= P.nrows) return false;
    off_out = Tl::OFF_EOUT;
    off_a = TH;  // my right column
    off_b = 0;   // the east tile's left column
    nbr = P.ty * g.tiles_x + (P.tx + 1) % g.tiles_x;
  } else {
    i = e - TH;
    if (i >= P.ncols) return false;
    off_out = Tl::OFF_SOUT;
    off_a = 2 * TH + TW;  // my bottom row
    off_b = 2 * TH;       // the south tile's top row
    nbr = ((P.ty + 1) % g.tiles_y) * g.tiles_x + P.tx;
  }
  const uint32_t* out = bb + off_out;
  if (!((out[i >> 5] >> (i & 31)) & 1u)) return false;
  const uint16_t* bsN = a.tb.bslot + (size_t)nbr * NB;
  const uint16_t sa = __ldcg(bs + off_a + i), sb = __ldcg(bsN + off_b + i);
  if (sa >= __ldcg(a.tb.nslots + tile) || sb >= __ldcg(a.tb.nslots + nbr)) {
    atomicCAS(a.tb.err, 0, kErrSlotOverflow);
    return false;
  }
  if (i > 0 && ((out[(i - 1) >> 5] >> ((i - 1) & 31)) & 1u) && __ldcg(bs + off_a + i - 1) == sa &&
      __ldcg(bsN + off_b + i - 1) == sb)
    return false;
  na = (uint32_t)tile * MS + sa;
  nb = (uint32_t)nbr * MS + sb;
  return true;
}

// Per tile, every out-going border edge: TH east edges (rows) then TW south
// edges (columns), one edge per thread at a time.
template <int WPR, int TH, int H, bool BATCH>
__device__ __forceinline__ void phase2_body(const SweepArgs& a0, const BatchArgs& bat, int T, int k) {
  using Tl = Tile<WPR, TH, H>;
  SweepArgs a;
  int tile;
  if (!cta_args<BATCH>(a0, bat, T, k, a, tile)) return;
  const TilePos P = tile_pos<Tl::TW, TH>(a.g, tile);
  for (int e = threadIdx.x; e < TH + Tl::TW; e += blockDim.x) {
    uint32_t na, nb;
    if (border_union<WPR, TH, H>(a, P, tile, e, na, nb)) unite_global(a.tb.nodes, na, nb, a.tb.err);
  }
}

// ------------------------------------------------ bond draws of the next sweep
//
// The bond draws of sweep t + 1 (C5) depend on the seed, the counter and the
// site, not on the spins, so they are taken during the cross-tile merge of
// sweep t: the merge's walks are chains of dependent L2 loads that leave the
// SMs' integer multiply pipes idle, and the Philox rounds are bound by
// those. kDrawWarps extra warps of every phase 2 and resolve CTA draw a share
// of their tile's row words (the first draw_split in phase 2, the rest in
// resolve) into a.draws_out; phase 1 of sweep t + 1 reads them.
constexpr int kDrawWarps = 2;
template <int RW>
constexpr int draw_split() {
  return RW - RW / 4;
}

template <int WPR, int TH, int H>
__device__ __forceinline__ void draw_next_bonds(const SweepArgs& a, int tile, int d, int rw0, int rw1) {
  using Tl = Tile<WPR, TH, H>;
  constexpr int RW = Tl::RW;
  const TilePos P = tile_pos<Tl::TW, TH>(a.g, tile);
  const int L = a.g.L;
  for (int rw = rw0 + d; rw < rw1; rw += 32 * kDrawWarps) {
    const int y = rw / WPR, w = rw % WPR;
    const int nb = max(0, min(32, P.ncols - 32 * w));
    if (y < P.nrows && nb > 0)
      __stcs(a.draws_out + (size_t)tile * RW + rw,
             bond_draws((uint32_t)(P.y0 + y) * (uint32_t)L + (uint32_t)(P.x0 + 32 * w), nb, L, a.t + 1u, a.thr, a.ks));
  }
}

// With a.draws_out the block has kDrawWarps more warps than edges (TH + TW
// threads); they draw the first draw_split row words of the tile.
template <int WPR, int TH, int H, bool BATCH>
__global__ void phase2_kernel(const SweepArgs a0, const BatchArgs bat) {
  using Tl = Tile<WPR, TH, H>;
  if (!BATCH && a0.draws_out && threadIdx.x >= TH + Tl::TW) {
    draw_next_bonds<WPR, TH, H>(a0, blockIdx.x, threadIdx.x - (TH + Tl::TW), 0, draw_split<Tl::RW>());
    return;
  }
  phase2_body<WPR, TH, H, BATCH>(a0, bat, blockIdx.x, 0);
}

// ------------------------------------------------------------- resolve

// Runs after every union of the sweep is done. Each slot node of the tile
// is rewritten to name its component's root directly, together with the
// root's key (the component's minimum site, C9) and the decision drawn
// for it (C6, or §2.4's assignment): bits 0-31 root node, 32-62 root key,
// 63 decision; for the Potts model the new state goes to nval. Keys are site
// indices below 2^31, so bit 63 is free. Walks only read; a thread writes
// only its own node, and the parent field it leaves (the root) is an
// ancestor, so walks of other threads that meet a rewritten node still end
// at the same root. Phase 3 then reads a slot's decision in one load.
// Slot node x, whose walk ended at root node `root` with entry v: the root's
// key and the decision drawn for it (for the Potts model, its new state into
// nval).
__device__ __forceinline__ void resolve_write(const SweepArgs& a, uint32_t x, uint32_t root, uint64_t v) {
  const uint32_t key = (uint32_t)(v >> 32) & 0x7fffffffu;
  uint32_t f = 0u;
  if (a.q)
    a.tb.nval[x] = (uint8_t)potts_new_state(key, a.t, a.ks, a.q);  // §6: the decision is a state
  else
    f = decision_bit(key, a.t, a.ks, a.rule);
  a.tb.nodes[x] = ((uint64_t)(key | (f << 31)) << 32) | root;
}

// nthr: the threads that walk slots (the first nthr of the block).
template <int WPR, int TH, int H, bool BATCH>
__device__ __forceinline__ void resolve_body(const SweepArgs& a0, const BatchArgs& bat, int T, int k, int nthr) {
  constexpr int MS = Tile<WPR, TH, H>::MS;
  SweepArgs a;
  int tile;
  if (!cta_args<BATCH>(a0, bat, T, k, a, tile)) return;
  const int nsl = min(a.tb.nslots[tile], MS);
  for (int j = threadIdx.x; j < nsl; j += nthr) {
    const uint32_t x = (uint32_t)tile * MS + j;
    uint32_t cur = x;
    uint64_t v = ld_node(a.tb.nodes + cur);
    for (int it = 0; (uint32_t)v != cur; ++it) {
      if (it >= kGlobalFindCap) {
        atomicCAS(a.tb.err, 0, kErrUnionCap);
        break;
      }
      cur = (uint32_t)v;
      v = ld_node(a.tb.nodes + cur);
    }
    resolve_write(a, x, cur, v);
  }
}

// Slot walks by the first kResolveThreads threads; with a.draws_out,
// kDrawWarps more warps draw the tile's row words from draw_split on.
constexpr int kResolveThreads = 128;
template <int WPR, int TH, int H, bool BATCH>
__global__ void resolve_kernel(const SweepArgs a0, const BatchArgs bat) {
  using Tl = Tile<WPR, TH, H>;
  if (threadIdx.x >= kResolveThreads) {
    if (!BATCH && a0.draws_out)
      draw_next_bonds<WPR, TH, H>(a0, blockIdx.x, threadIdx.x - kResolveThreads, draw_split<Tl::RW>(), Tl::RW);
    return;
  }
  resolve_body<WPR, TH, H, BATCH>(a0, bat, blockIdx.x, 0, kResolveThreads);
}

// ================================================================ phase 3

// MODE 0: flips + E/M; 1: flips + E/M + cluster sizes; 2: canonical labels.
// Shared memory of phase 3 for one tile.
template <int WPR, int TH, int H, int MODE>
struct P3Shared {
  using T = Tile<WPR, TH, H>;
  static constexpr bool HIST = MODE == 1, LABELS = MODE == 2;
  alignas(16) uint16_t par[TH * T::TW];  // labels from phase 1: par[par[x]] is the tile root of x
  uint32_t bmask[T::RW];                 // border roots
  uint32_t pre[T::RW];
  uint32_t wsum[33];
  uint32_t flip[T::RW];                  // decision bit of every root (flip, or new sign)
  uint32_t snew[TH][WPR];
  int slotkey[LABELS ? T::MS : 1];       // labels mode: canonical label of every slot
  uint32_t slotdec[(T::MS + 31) / 32];   // flip modes: decision bit of every slot
  uint32_t slotroot[HIST ? T::MS : 1];
  uint32_t hEnew[TH / 32], hSnew[T::TW / 32];
  long long red[2][T::NT / 32];
  unsigned long long hist[HIST ? 34 : 1];
  unsigned long long roots_bar;          // completion of the labels tile's bulk copy into par
};

// Returns false when the labels' bulk copy did not land (the CTA's shared
// memory may still be written by it: the caller must not reuse it).
template <int WPR, int TH, int H, int MODE, bool BATCH>
__device__ __forceinline__ bool phase3_body(P3Shared<WPR, TH, H, MODE>& S, uint32_t* s_size, const SweepArgs& a0,
                                            const BatchArgs& bat, int T, int ksweep) {
  using Tl = Tile<WPR, TH, H>;
  constexpr int TW = Tl::TW, NT = Tl::NT, NB = Tl::NB, MS = Tl::MS, BBW = Tl::BBW, RW = Tl::RW;
  constexpr bool HIST = MODE == 1, LABELS = MODE == 2;
  uint16_t* const par = S.par;
  uint32_t* const s_bmask = S.bmask;
  uint32_t* const s_pre = S.pre;
  uint32_t* const s_wsum = S.wsum;
  uint32_t* const s_flip = S.flip;
  uint32_t(&s_snew)[TH][WPR] = S.snew;
  int* const s_slotkey = S.slotkey;
  uint32_t* const s_slotdec = S.slotdec;
  uint32_t* const s_slotroot = S.slotroot;
  uint32_t* const s_hEnew = S.hEnew;
  uint32_t* const s_hSnew = S.hSnew;
  long long(&s_red)[2][NT / 32] = S.red;
  unsigned long long* const s_hist = S.hist;
  unsigned long long& s_roots_bar = S.roots_bar;

  SweepArgs a;
  int tile;
  if (!cta_args<BATCH>(a0, bat, T, ksweep, a, tile)) return true;
  const Geometry& g = a.g;
  const int L = g.L;
  const TilePos P = tile_pos<TW, TH>(g, tile);
  const int tid = threadIdx.x, w = tid % WPR, k = tid / WPR, y0r = k * H;
  const int lane = tid & 31, warp0 = tid & ~31;
  const int nv = max(0, min(H, P.nrows - y0r));
  const int nb = max(0, min(32, P.ncols - 32 * w));
  const uint32_t wmask = word_mask(P.ncols, w);
  const uint32_t lbit = last_column_bit(P.ncols, w);
  const bool lastword = lbit != 0u;

  const uint32_t* tb = a.tb.tbits + (size_t)P.tile * 3 * RW;
  const uint16_t* groots = a.tb.roots + (size_t)P.tile * (TW * TH);
  const uint32_t* gbm = a.tb.bmask + (size_t)P.tile * RW;
  // the tile roots (every tile's block is 16-byte aligned) travel on the
  // copy engine while the decisions are drawn; the first parent read waits
  if (tid == 0) bulk_load_start(par, groots, TW * TH * sizeof(uint16_t), &s_roots_bar);
  // the global loads that only read phase 1's output go out together here
  // (spin and east masks, border-root and root masks, the slot count), so
  // that no later stage waits on a DRAM round trip of its own
  const uint32_t* grb = a.tb.rbits + (size_t)P.tile * RW;
  const int nsl = a.tb.nslots[P.tile];
  uint32_t s[H], e_int[H], rbw[H];
#pragma unroll
  for (int r = 0; r < H; ++r) {
    const int y = y0r + r, rw = y * WPR + w, base = y * TW + 32 * w;
    s[r] = tb[rw];
    e_int[r] = tb[RW + rw] & ~lbit;
    rbw[r] = LABELS ? 0u : grb[rw];
    s_bmask[rw] = gbm[rw];
    if (HIST) {  // the 32 sizes of this row word: 16 words of two 16-bit counters
      int4* z = reinterpret_cast<int4*>(s_size + base / 2);
#pragma unroll
      for (int q = 0; q < 4; ++q) z[q] = make_int4(0, 0, 0, 0);
    }
  }
  if (HIST)
    for (int i = tid; i < 34; i += NT) s_hist[i] = 0ull;
  for (int i = tid; i < (MS + 31) / 32; i += NT) s_slotdec[i] = 0u;
  __syncthreads();
  if (block_popc_prefix<RW, NT>(s_bmask, s_pre, s_wsum) != nsl && tid == 0) atomicCAS(a.tb.err, 0, kErrSlotOverflow);

  // ---- this tile's slots: root key and flip, as the resolve pass left them
  for (int j = tid; j < nsl; j += NT) {
    const uint64_t v = ld_node(a.tb.nodes + (uint32_t)P.tile * MS + j);
    if (LABELS) s_slotkey[j] = (int)((uint32_t)(v >> 32) & 0x7fffffffu);
    else if (v >> 63) atomicOr(&s_slotdec[j >> 5], 1u << (j & 31));
    if (HIST) s_slotroot[j] = (uint32_t)v;
  }
  if (!LABELS) {
    // ---- new spins of the halo sites: old spin (phase 1) xor their cluster's
    // flip; the two dependent loads (slot, then node) overlap the labels copy
    const uint32_t* bbits = a.tb.bbits + (size_t)P.tile * BBW;
    for (int b0 = warp0; b0 < TH; b0 += NT) {
      const int y = b0 + lane;
      bool bit = false;
      if (y < P.nrows) {
        const int tileE = P.ty * g.tiles_x + (P.tx + 1) % g.tiles_x;
        uint16_t slot = __ldcg(a.tb.bslot + (size_t)tileE * NB + y);
        if (slot >= MS) {
          atomicCAS(a.tb.err, 0, kErrSlotOverflow);
          slot = 0;
        }
        const uint64_t v = ld_node(a.tb.nodes + (uint32_t)tileE * MS + slot);
        const uint32_t old = (bbits[Tl::OFF_HE + (y >> 5)] >> (y & 31)) & 1u;
        bit = ((a.rule ? 0u : old) ^ (uint32_t)(v >> 63)) != 0u;
      }
      const uint32_t m = __ballot_sync(0xffffffffu, bit);
      if (lane == 0) s_hEnew[b0 >> 5] = m;
    }
    for (int b0 = warp0; b0 < TW; b0 += NT) {
      const int x = b0 + lane;
      bool bit = false;
      if (x < P.ncols) {
        const int tileS = ((P.ty + 1) % g.tiles_y) * g.tiles_x + P.tx;
        uint16_t slot = __ldcg(a.tb.bslot + (size_t)tileS * NB + 2 * TH + x);
        if (slot >= MS) {
          atomicCAS(a.tb.err, 0, kErrSlotOverflow);
          slot = 0;
        }
        const uint64_t v = ld_node(a.tb.nodes + (uint32_t)tileS * MS + slot);
        const uint32_t old = (bbits[Tl::OFF_HS + (x >> 5)] >> (x & 31)) & 1u;
        bit = ((a.rule ? 0u : old) ^ (uint32_t)(v >> 63)) != 0u;
      }
      const uint32_t m = __ballot_sync(0xffffffffu, bit);
      if (lane == 0) s_hSnew[b0 >> 5] = m;
    }
  }
  __syncthreads();

  // ---- decision bit of every root of my strip: border roots from their slot,
  // the others drawn here (phase 1 marked the roots). Under the flip rule
  // (C6) one Philox block holds the bits of 128 consecutive site indices, so
  // a row word's inner roots take their bits from one draw. Under the
  // assignment rule each root draws its own block: the lanes of a warp walk
  // their inner roots in step and queue them (in s_snew, free until the new
  // spins); the queue is drawn 64 roots at a time, two draws per lane.
  if (!LABELS) {
    const int warp = tid >> 5;
    constexpr int QC = 128;  // queue entries per warp
    static_assert((NT / 32) * QC <= 2 * TH * WPR, "root queues fit in s_snew");
    uint16_t* q = reinterpret_cast<uint16_t*>(&s_snew[0][0]) + warp * QC;
    int qh = 0, qn = 0;  // the same in every lane of the warp
    auto draw = [&](int x) {
      const uint32_t key = (uint32_t)(P.y0 + x / TW) * (uint32_t)L + (uint32_t)(P.x0 + x % TW);
      return decision_bit(key, a.t, a.ks, a.rule);
    };
#pragma unroll
    for (int r = 0; r < H; ++r) s_flip[(y0r + r) * WPR + w] = 0u;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const int y = y0r + r, base = y * TW + 32 * w, rw = y * WPR + w;
      const uint32_t bm = s_bmask[rw];
      uint32_t inner = r < nv ? rbw[r] & ~bm : 0u;
      uint32_t fl = 0, B = r < nv ? bm : 0u;
      while (B) {
        const int b = __ffs(B) - 1;
        B &= B - 1;
        const int sl = slot_of(s_bmask, s_pre, base + b);
        fl |= (sl < nsl ? (s_slotdec[sl >> 5] >> (sl & 31)) & 1u : 0u) << b;
      }
      if (!a.rule && inner) {
        fl |= flip_bits32((uint32_t)(P.y0 + y) * (uint32_t)L + (uint32_t)(P.x0 + 32 * w), a.t, a.ks) & inner;
        inner = 0u;
      }
      if (fl) atomicOr(&s_flip[rw], fl);
      while (__any_sync(0xffffffffu, inner != 0u)) {
        const bool have = inner != 0u;
        int x = 0;
        if (have) {
          x = base + __ffs(inner) - 1;
          inner &= inner - 1;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, have);
        if (have) q[(qh + qn + __popc(m & ((1u << lane) - 1u))) & (QC - 1)] = (uint16_t)x;
        qn += __popc(m);
        __syncwarp();
        if (qn >= 64) {
          const int x0 = q[(qh + lane) & (QC - 1)], x1 = q[(qh + 32 + lane) & (QC - 1)];
          const uint32_t f0 = draw(x0), f1 = draw(x1);
          if (f0) atomicOr(&s_flip[x0 >> 5], 1u << (x0 & 31));
          if (f1) atomicOr(&s_flip[x1 >> 5], 1u << (x1 & 31));
          qh += 64;
          qn -= 64;
          __syncwarp();
        }
      }
    }
    for (int k2 = lane; k2 < qn; k2 += 32) {
      const int x = q[(qh + k2) & (QC - 1)];
      if (draw(x)) atomicOr(&s_flip[x >> 5], 1u << (x & 31));
    }
    __syncthreads();
  }

  {
    const bool landed = bulk_load_wait(&s_roots_bar);
    if (!landed) atomicCAS(a.tb.err, 0, kErrCopyTimeout);
    if (__syncthreads_or(!landed)) {
      if (!landed) bulk_load_wait(&s_roots_bar);  // once more before the CTA's shared memory is released
      return false;
    }
    // every thread has passed the wait: the barrier's word may be reused
    // (the fused batch kernel overlays it with other data)
    if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&s_roots_bar)) : "memory");
  }

  // ---- per run: its root's decision; new spins of my strip. A row of labels
  // is 256 bytes, so the rows all start in bank 0, and every row word has a
  // run start at its column 0: walked in column order, the 32 lanes' first
  // label loads would meet in two banks. The flip modes walk each word's run
  // starts cyclically from a lane-dependent column instead (8 strips x 4
  // words of a warp -> 32 different banks for the first load), record each
  // run's decision at its start, and spread the decisions over the runs
  // afterwards with a segmented prefix OR.
  const int rot = ((k & 7) << 2) | ((w >> 1 & 1) << 1);
  // HIST: a lane adds up the lengths of consecutive runs of one root and
  // sends the sum when the root changes (a tile's runs mostly belong to few
  // clusters near order, which made per-run shared atomics serialise)
  int acc_rt = -1;
  uint32_t acc_len = 0u;
  uint32_t snew[H];
#pragma unroll
  for (int r = 0; r < H; ++r) {
    snew[r] = s[r];
    if (r >= nv || !wmask) continue;
    const int y = y0r + r, base = y * TW + 32 * w;
    const uint32_t Rall = ~(e_int[r] << 1) & wmask;  // run starts
    if (LABELS) {
      uint32_t R = Rall;
      while (R) {
        const int b = __ffs(R) - 1;
        R &= R - 1;
        const int rt = par[par[base + b]];  // the run's label, then the label's root
        const int nxt = R ? (__ffs(R) - 1) : nb;
        int key;
        if ((s_bmask[rt >> 5] >> (rt & 31)) & 1u) {
          const int sl = slot_of(s_bmask, s_pre, rt);
          key = sl < nsl ? s_slotkey[sl] : 0;
        } else {
          key = (int)((uint32_t)(P.y0 + rt / TW) * (uint32_t)L + (uint32_t)(P.x0 + rt % TW));
        }
        int32_t* out = a.labels + (size_t)(P.y0 + y) * L + P.x0 + 32 * w;
        for (int x = b; x < nxt; ++x) out[x] = key;
      }
    } else {
      uint32_t Rr = __funnelshift_r(Rall, Rall, rot);  // bit i: run start at column (i + rot) mod 32
      uint32_t D = 0u;                                // decision of each run, at its start
      while (Rr) {
        const int b = (__ffs(Rr) - 1 + rot) & 31;
        Rr &= Rr - 1;
        const int rt = par[par[base + b]];  // the run's label, then the label's root
        D |= ((s_flip[rt >> 5] >> (rt & 31)) & 1u) << b;
        if (HIST) {
          const uint32_t above = Rall & ~((2u << b) - 1u);  // run starts after b (b = 31: none)
          const uint32_t len = (uint32_t)((above ? __ffs(above) - 1 : nb) - b);
          if (rt == acc_rt) {
            acc_len += len;
          } else {
            if (acc_rt >= 0) atomicAdd(&s_size[acc_rt >> 1], acc_len << ((acc_rt & 1) << 4));
            acc_rt = rt;
            acc_len = len;
          }
        }
      }
      // segmented prefix OR: a site takes the decision of its run's start
      uint32_t G = ~Rall;  // sites that continue the run of the site before them
      D |= (D << 1) & G;
      G &= G << 1;
      D |= (D << 2) & G;
      G &= G << 2;
      D |= (D << 4) & G;
      G &= G << 4;
      D |= (D << 8) & G;
      G &= G << 8;
      D |= (D << 16) & G;
      snew[r] = (a.rule ? 0u : s[r]) ^ (D & wmask);
      store_spin_bits(a.spins_out + (size_t)(P.y0 + y) * L + P.x0 + 32 * w, snew[r], nb, g.aligned16);
    }
  }
  if (LABELS) return true;
  if (HIST) {  // the lanes' last sums: one atomic per root and warp
    __syncwarp();
    const uint32_t peers = __match_any_sync(0xffffffffu, acc_rt);
    const uint32_t sum = __reduce_add_sync(peers, acc_len);
    if (acc_rt >= 0 && lane == __ffs(peers) - 1) atomicAdd(&s_size[acc_rt >> 1], sum << ((acc_rt & 1) << 4));
  }
#pragma unroll
  for (int r = 0; r < H; ++r) s_snew[y0r + r][w] = snew[r];

  __syncthreads();

  // ---- E and M of the new state (C10)
  int eloc = 0, mloc = 0;
#pragma unroll
  for (int r = 0; r < H; ++r) {
    if (r >= nv || !wmask) continue;
    const int y = y0r + r;
    uint32_t sEn;
    if (lastword) {
      const uint32_t hb = (s_hEnew[y >> 5] >> (y & 31)) & 1u;
      sEn = ((snew[r] >> 1) & (lbit - 1u)) | (hb ? lbit : 0u);
    } else {
      sEn = (snew[r] >> 1) | ((w + 1 < WPR) ? (s_snew[y][w + 1] << 31) : 0u);
    }
    const uint32_t sSn = (y + 1 < P.nrows) ? (r + 1 < H ? snew[r + 1] : s_snew[y + 1][w]) : s_hSnew[w];
    const int nvb = __popc(wmask);
    const int unequal = __popc((snew[r] ^ sEn) & wmask) + __popc((snew[r] ^ sSn) & wmask);
    eloc += 2 * unequal - 2 * nvb;
    mloc += nvb - 2 * __popc(snew[r] & wmask);
  }
  long long ev = warp_sum((long long)eloc), mv = warp_sum((long long)mloc);
  if (lane == 0) {
    s_red[0][tid >> 5] = ev;
    s_red[1][tid >> 5] = mv;
  }

  if (HIST) {
    // sizes are complete after this barrier: bin the inner clusters (the
    // tile roots phase 1 marked, less the border roots), send border pieces
    // to their global root. Counts, sums of squares (at most 8192^2 a tile)
    // and bins 0-7 (8-bit fields: at most 64 roots a thread) add up in
    // registers and once per warp into the shared histogram.
    __syncthreads();
    uint32_t cnt = 0u, sq = 0u, bins03 = 0u, bins47 = 0u;
#pragma unroll
    for (int r = 0; r < H; ++r) {
      if (r >= nv || !wmask) continue;
      const int base = (y0r + r) * TW + 32 * w, rw = (y0r + r) * WPR + w;
      const uint32_t bm = s_bmask[rw];
      for (uint32_t m = rbw[r]; m; m &= m - 1) {
        const int b = __ffs(m) - 1, l = base + b;
        const uint32_t sz = (s_size[l >> 1] >> ((l & 1) << 4)) & 0xffffu;
        if ((bm >> b) & 1u) {
          const int sl = slot_of(s_bmask, s_pre, l);
          if (sl < nsl) atomicAdd(&a.csize[s_slotroot[sl]], sz);
        } else {
          const int bin = log2_floor(sz);
          cnt += 1u;
          sq += sz * sz;
          if (bin < 4) bins03 += 1u << (8 * bin);
          else if (bin < 8) bins47 += 1u << (8 * (bin - 4));
          else atomicAdd(&s_hist[2 + bin], 1ull);
        }
      }
    }
    __syncwarp();
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    sq = __reduce_add_sync(0xffffffffu, sq);
    uint32_t bsum[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      bsum[q] = __reduce_add_sync(0xffffffffu, (bins03 >> (8 * q)) & 0xffu);
      bsum[4 + q] = __reduce_add_sync(0xffffffffu, (bins47 >> (8 * q)) & 0xffu);
    }
    if (lane == 0) {
      if (cnt) atomicAdd(&s_hist[0], (unsigned long long)cnt);
      if (sq) atomicAdd(&s_hist[1], (unsigned long long)sq);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (bsum[q]) atomicAdd(&s_hist[2 + q], (unsigned long long)bsum[q]);
    }
  }
  __syncthreads();
  if (tid < 32) {
    long long e2 = 0, m2 = 0;
    for (int q = tid; q < NT / 32; q += 32) {
      e2 += s_red[0][q];
      m2 += s_red[1][q];
    }
    e2 = warp_sum(e2);
    m2 = warp_sum(m2);
    if (tid == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(a.em), (unsigned long long)e2);
      atomicAdd(reinterpret_cast<unsigned long long*>(a.em + 1), (unsigned long long)m2);
    }
  }
  if (HIST)
    for (int i = tid; i < 34; i += NT)
      if (s_hist[i]) atomicAdd(reinterpret_cast<unsigned long long*>(a.hist + i), s_hist[i]);
  return true;
}

template <int WPR, int TH, int H, int MODE, bool BATCH>
__global__ void __launch_bounds__(WPR * (TH / H), strip_min_blocks<WPR * (TH / H), H>())
    phase3_kernel(const SweepArgs a0, const BatchArgs bat) {
  __shared__ P3Shared<WPR, TH, H, MODE> S;
  extern __shared__ __align__(16) uint32_t s_size[];  // HIST: [TH * TW / 2], two 16-bit sizes a word
  phase3_body<WPR, TH, H, MODE, BATCH>(S, s_size, a0, bat, blockIdx.x, 0);
}

// ================================================================ phase 4

template <int WPR, int TH, int H>
__global__ void phase4_kernel(const SweepArgs a) {
  using T = Tile<WPR, TH, H>;
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

// ================================================================ batch

__global__ void batch_advance_kernel(const BatchArgs b) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= b.nrep) return;
  ReplicaDesc* D = b.descs + r;
  if (!D->active || D->small || D->t_left <= 0) return;
  D->t += 1;
  D->em_next += 1;
  D->t_left -= 1;
}

// ========================================================== fused batch kernel

constexpr long long kBarrierWaitCycles = 1LL << 31;  // ~1 s at the SM clock: limit of a grid-barrier wait

// Grid-wide barrier of the fused batch kernel. Every thread fences its
// global writes, then one thread per CTA arrives (an atomic add on the
// count); the last to arrive resets the count and opens the next
// generation, the others wait for it. Every CTA of the launch must be
// resident, which the cooperative launch guarantees (or it fails). The wait
// is bounded (about a second): then the CTA raises kErrBarrierTimeout and
// the function returns false, and the caller returns.
__device__ bool grid_sync(GridBarrier* gb, int* err) {
  __shared__ int s_ok;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = &gb->gen;
    const unsigned int gen = *vgen;
    __threadfence();
    if (atomicAdd(&gb->count, 1u) + 1u == gridDim.x) {
      gb->count = 0u;
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (clock64() - t0 > kBarrierWaitCycles) {
          atomicCAS(err, 0, kErrBarrierTimeout);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int WPR, int TH, int H>
union FusedShared {
  P1Shared<WPR, TH, H> p1;
  P3Shared<WPR, TH, H, 0> p3;
};

// nsweeps whole sweeps of every replica with tiles, in one launch: the
// phases of a sweep run over all batch tiles (CTA c takes tiles c, c + grid,
// ...), separated by grid barriers, since a phase reads what the previous
// one wrote for neighbouring tiles. Replica r takes part in sweep k while
// k < its sweeps left (cta_args). At the end CTA 0 advances every replica's
// counter and trace row by the sweeps it ran. The phases are the same code
// as the separate launches (the *_body functions), so the results are too.
template <int WPR, int TH, int H>
__global__ void __launch_bounds__(32 * WPR, band_min_blocks<32 * WPR>())
    batch_fused_kernel(const BatchArgs b, int nsweeps, int ntiles) {
  static_assert(Tile<WPR, TH, H>::NT == 32 * WPR, "phases 1 and 3 run the same block");
  __shared__ FusedShared<WPR, TH, H> U;
  const SweepArgs none{};
  for (int k = 0; k < nsweeps; ++k) {
    for (int T = blockIdx.x; T < ntiles; T += gridDim.x) {
      phase1_body<WPR, TH, H, true>(U.p1, none, b, T, k);
      __syncthreads();  // the next tile reuses the shared memory
    }
    if (!grid_sync(b.gbar, b.err)) return;
    for (int T = blockIdx.x; T < ntiles; T += gridDim.x) phase2_body<WPR, TH, H, true>(none, b, T, k);
    if (!grid_sync(b.gbar, b.err)) return;
    for (int T = blockIdx.x; T < ntiles; T += gridDim.x) resolve_body<WPR, TH, H, true>(none, b, T, k, blockDim.x);
    if (!grid_sync(b.gbar, b.err)) return;
    for (int T = blockIdx.x; T < ntiles; T += gridDim.x) {
      const bool ok = phase3_body<WPR, TH, H, 0, true>(U.p3, nullptr, none, b, T, k);
      __syncthreads();
      if (!ok) return;  // a bulk copy may still write this CTA's shared memory
    }
    if (!grid_sync(b.gbar, b.err)) return;
  }
  if (blockIdx.x == 0) {
    for (int r = threadIdx.x; r < b.nrep; r += blockDim.x) {
      ReplicaDesc* D = b.descs + r;
      if (!D->active || D->small || D->t_left <= 0) continue;
      const int64_t m = D->t_left < nsweeps ? D->t_left : nsweeps;
      D->t += (uint32_t)m;
      D->em_next += m;
      D->t_left -= m;
    }
  }
}

// Phase 3 of sweep t and phase 1 of sweep t + 1 of one tile, in one CTA.
// Phase 3 leaves the tile's new spin words and its halo sites' new spins in
// shared memory, and these are the first things phase 1 of the next sweep
// reads, so they are handed over there instead of through global memory (the
// int8 spins are still written: the state stays in HBM). a3 and a1 are the
// two sweeps' arguments; they name different border-slot, slot-count and
// node tables (by sweep parity), because other tiles' phase 3 of sweep t
// still reads this tile's tables of sweep t while this CTA writes those of
// sweep t + 1. Every other table a tile writes is read by that tile alone.
template <int WPR, int TH, int H>
__global__ void __launch_bounds__(32 * WPR, band_min_blocks<32 * WPR>())
    phase31_kernel(const SweepArgs a3, const SweepArgs a1) {
  using Tl = Tile<WPR, TH, H>;
  constexpr int NT = 32 * WPR, RPL = TH / 32, NHE = TH / 32, NH = TH / 32 + Tl::TW / 32;
  static_assert(Tl::NT == NT, "phases 1 and 3 run the same block");
  __shared__ FusedShared<WPR, TH, H> U;
  const int tid = threadIdx.x;
  if (!phase3_body<WPR, TH, H, 0, false>(U.p3, nullptr, a3, BatchArgs{}, blockIdx.x, 0)) return;
  uint32_t words[RPL], halo = 0u;
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    const int rw = tid + NT * i;
    words[i] = U.p3.snew[rw / WPR][rw % WPR];
  }
  if (tid < NHE) halo = U.p3.hEnew[tid];
  else if (tid < NH) halo = U.p3.hSnew[tid - NHE];
  __syncthreads();  // the two sweeps' shared memory overlaps
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    const int rw = tid + NT * i;
    U.p1.sd[0][rw / WPR][rw % WPR] = words[i];
  }
  if (tid < NHE) U.p1.bb[Tl::OFF_HE + tid] = halo;
  else if (tid < NH) U.p1.bb[Tl::OFF_HS + tid - NHE] = halo;
  __syncthreads();
  phase1_body<WPR, TH, H, false, true>(U.p1, a1, BatchArgs{}, blockIdx.x, 0);
}

template <int WPR, int TH, int H>
cudaError_t launch_fused_shape(const BatchArgs& b, int ntiles, int nsweeps, cudaStream_t st) {
  auto kern = batch_fused_kernel<WPR, TH, H>;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * WPR, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  int grid = per_sm * nsm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(32 * WPR);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, b, nsweeps, ntiles);
}

// ================================================================ Potts (§6)

// Phase 1 of a q-state Potts sweep: the Ising phase 1 with the bond masks of
// equal states (phase1_body's POTTS form).
template <int WPR, int TH, int H>
__global__ void __launch_bounds__(32 * WPR, band_min_blocks<32 * WPR>())
    potts_phase1_kernel(const SweepArgs a) {
  __shared__ P1Shared<WPR, TH, H> S;
  phase1_body<WPR, TH, H, false, false, true>(S, a, BatchArgs{}, blockIdx.x, 0);
}

constexpr int kPottsP3Threads = 256;  // threads per tile of the Potts phase 3

template <int WPR, int TH, int H, int NT>
struct PottsP3Shared {
  using T = Tile<WPR, TH, H>;
  alignas(16) uint16_t par[TH * T::TW];  // labels from phase 1: par[par[x]] is the tile root of x
  alignas(16) uint8_t val[TH * T::TW];   // new state of every tile root (indexed by its site)
  alignas(16) uint8_t snew[TH][T::TW];   // new states of the tile
  alignas(16) uint8_t hS[T::TW];         // new states of the south halo row
  uint8_t hE[TH];                        // new states of the east halo column
  uint8_t slotval[T::MS];                // new state of every slot's cluster (from resolve)
  alignas(16) uint32_t bmask[T::RW];     // border roots
  uint32_t pre[T::RW];
  uint32_t wsum[33];
  long long red[2][NT / 32];
};

// Phase 3 of a q-state Potts sweep for one tile (§6): every cluster takes the
// state drawn for its root (a border cluster the one resolve left in its slot,
// an inner one drawn here from its root's key), every site its cluster's, and
// E = -(edges joining equal states), M = (sites in state 0) of the new
// configuration are summed in int64.
template <int WPR, int TH, int H>
__global__ void __launch_bounds__(kPottsP3Threads) potts_phase3_kernel(const SweepArgs a) {
  using Tl = Tile<WPR, TH, H>;
  constexpr int TW = Tl::TW, NT = kPottsP3Threads, NB = Tl::NB, MS = Tl::MS, RW = Tl::RW;
  constexpr int G = TW / 4;  // four-site groups per row
  static_assert(RW % NT == 0, "whole rounds of row words");
  __shared__ PottsP3Shared<WPR, TH, H, NT> S;
  const Geometry& g = a.g;
  const int L = g.L;
  const TilePos P = tile_pos<TW, TH>(g, blockIdx.x);
  const int tid = threadIdx.x, lane = tid & 31;

  {
    const uint4* src = reinterpret_cast<const uint4*>(a.tb.roots + (size_t)P.tile * (TW * TH));
    uint4* dst = reinterpret_cast<uint4*>(S.par);
    for (int i = tid; i < TW * TH / 8; i += NT) dst[i] = src[i];
    const uint32_t* gbm = a.tb.bmask + (size_t)P.tile * RW;
    for (int i = tid; i < RW; i += NT) S.bmask[i] = gbm[i];
  }
  __syncthreads();
  const int nsl = a.tb.nslots[P.tile];
  if (block_popc_prefix<RW, NT>(S.bmask, S.pre, S.wsum) != nsl && tid == 0) atomicCAS(a.tb.err, 0, kErrSlotOverflow);
  for (int j = tid; j < nsl && j < MS; j += NT) S.slotval[j] = a.tb.nval[(size_t)P.tile * MS + j];
  // the halo's new states: its sites are border sites of the neighbour tiles,
  // so their clusters have slots there
  const int tileE = P.ty * g.tiles_x + (P.tx + 1) % g.tiles_x;
  const int tileS = ((P.ty + 1) % g.tiles_y) * g.tiles_x + P.tx;
  for (int y = tid; y < P.nrows; y += NT) {
    uint16_t slot = a.tb.bslot[(size_t)tileE * NB + y];
    if (slot >= MS) {
      atomicCAS(a.tb.err, 0, kErrSlotOverflow);
      slot = 0;
    }
    S.hE[y] = a.tb.nval[(size_t)tileE * MS + slot];
  }
  for (int x = tid; x < P.ncols; x += NT) {
    uint16_t slot = a.tb.bslot[(size_t)tileS * NB + 2 * TH + x];
    if (slot >= MS) {
      atomicCAS(a.tb.err, 0, kErrSlotOverflow);
      slot = 0;
    }
    S.hS[x] = a.tb.nval[(size_t)tileS * MS + slot];
  }
  __syncthreads();

  // ---- the new state of every tile root (phase 1 marked them): a border
  // root's from its slot; the inner roots of a warp's row words are listed
  // (a prefix sum places each lane's roots; the list lives in S.snew, free
  // until the new states) and drawn 32 at a time, every lane with a root
  {
    constexpr int QW = TH * TW / 2 / (NT / 32);  // list entries per warp
    const uint32_t* grb = a.tb.rbits + (size_t)P.tile * RW;
    uint16_t* list = reinterpret_cast<uint16_t*>(&S.snew[0][0]) + (tid >> 5) * QW;
#pragma unroll
    for (int it = 0; it < RW / NT; ++it) {
      const int rw = tid + NT * it;  // tile-local sites rw * 32 + b (row-major, TW = 32 WPR)
      const uint32_t roots = rw / WPR < P.nrows ? grb[rw] : 0u;
      const uint32_t bm = S.bmask[rw];
      for (uint32_t m = roots & bm; m; m &= m - 1) {
        const int x = rw * 32 + __ffs(m) - 1;
        const int sl = slot_of(S.bmask, S.pre, x);
        S.val[x] = sl < nsl ? S.slotval[sl] : (uint8_t)0;
      }
      const uint32_t inner = roots & ~bm;
      const int cnt = __popc(inner);
      const int first = warp_exclusive_sum(cnt, lane);
      const int total = __shfl_sync(0xffffffffu, first + cnt, 31);
      for (int r0 = 0; r0 < total; r0 += QW) {  // one round unless most sites are roots
        int idx = first;
        for (uint32_t m = inner; m; m &= m - 1, ++idx)
          if (idx >= r0 && idx < r0 + QW) list[idx - r0] = (uint16_t)(rw * 32 + __ffs(m) - 1);
        __syncwarp();
        const int n = min(QW, total - r0);
        for (int k = lane; k < n; k += 32) {
          const int x = list[k];
          const uint32_t key = (uint32_t)(P.y0 + x / TW) * (uint32_t)L + (uint32_t)(P.x0 + x % TW);
          S.val[x] = (uint8_t)potts_new_state(key, a.t, a.ks, a.q);
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();

  // ---- every site takes its root's state, four sites per thread and step
  for (int i = tid; i < TH * G; i += NT) {
    const int y = i / G, x = 4 * (i % G);
    if (y >= P.nrows || x >= P.ncols) continue;
    const int base = y * TW + x;
    uint32_t word = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (x + k < P.ncols) word |= (uint32_t)S.val[S.par[S.par[base + k]]] << (8 * k);
    *reinterpret_cast<uint32_t*>(&S.snew[y][x]) = word;
    int8_t* out = a.spins_out + (size_t)(P.y0 + y) * L + P.x0 + x;
    if (g.aligned16 && x + 4 <= P.ncols) {
      *reinterpret_cast<uint32_t*>(out) = word;
    } else {
      for (int k = 0; k < 4 && x + k < P.ncols; ++k) out[k] = (int8_t)(word >> (8 * k));
    }
  }
  __syncthreads();

  // ---- E and M of the new states: east and south edge of every site
  long long e = 0, m = 0;
  for (int i = tid; i < TH * G; i += NT) {
    const int y = i / G, x = 4 * (i % G);
    if (y >= P.nrows || x >= P.ncols) continue;
    const uint32_t cur = *reinterpret_cast<const uint32_t*>(&S.snew[y][x]);
    if (x + 4 < P.ncols) {
      const uint32_t nxt = *reinterpret_cast<const uint32_t*>(&S.snew[y][x + 4]);
      const uint32_t south = y + 1 < P.nrows ? *reinterpret_cast<const uint32_t*>(&S.snew[y + 1][x])
                                             : *reinterpret_cast<const uint32_t*>(&S.hS[x]);
      e -= (__popc(__vcmpeq4(cur, __funnelshift_r(cur, nxt, 8))) + __popc(__vcmpeq4(cur, south))) >> 3;
      m += __popc(__vcmpeq4(cur, 0u)) >> 3;
    } else {
      for (int k = 0; k < 4 && x + k < P.ncols; ++k) {
        const uint32_t v = (cur >> (8 * k)) & 0xffu;
        const uint32_t ve = x + k + 1 < P.ncols ? S.snew[y][x + k + 1] : S.hE[y];
        const uint32_t vs = y + 1 < P.nrows ? S.snew[y + 1][x + k] : S.hS[x + k];
        e -= (v == ve) + (v == vs);
        m += v == 0u;
      }
    }
  }
  e = warp_sum(e);
  m = warp_sum(m);
  if (lane == 0) {
    S.red[0][tid >> 5] = e;
    S.red[1][tid >> 5] = m;
  }
  __syncthreads();
  if (tid == 0) {
    long long et = 0, mt = 0;
    for (int k = 0; k < NT / 32; ++k) {
      et += S.red[0][k];
      mt += S.red[1][k];
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(a.em), (unsigned long long)et);
    atomicAdd(reinterpret_cast<unsigned long long*>(a.em + 1), (unsigned long long)mt);
  }
}

// ================================================================ helpers

__global__ void init_kernel(int8_t* spins, long long n, KeySchedule ks, int cold) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int8_t v = 1;
    if (!cold) v = (philox4x32_10(make_uint4((uint32_t)i, 0u, 2u, 0u), ks).x >> 31) ? (int8_t)-1 : (int8_t)1;
    spins[i] = v;
  }
}

// Every spin must be +1 (0x01) or -1 (0xFF). 16 bytes per thread step,
// four at a time with byte-wise compares; the buffer is the library's own
// (16-byte aligned), the ragged tail goes byte by byte.
// Every byte must be +1 or -1. A streaming read: each thread keeps four
// independent 16-byte loads in flight per trip, so that a grid of whole SMs
// reaches the HBM rate.
__global__ void check_spins_kernel(const int8_t* spins, long long n, int* err) {
  const long long stride = (long long)gridDim.x * blockDim.x, i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nv = n / 16;
  const uint4* p = reinterpret_cast<const uint4*>(spins);
  auto ok4 = [](uint32_t w) { return (__vcmpeq4(w, 0x01010101u) | __vcmpeq4(w, 0xFFFFFFFFu)) == 0xFFFFFFFFu; };
  bool bad = false;
  for (long long i = i0; i < nv; i += 4 * stride) {
    uint4 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = i + k * stride < nv ? p[i + k * stride] : make_uint4(~0u, ~0u, ~0u, ~0u);
#pragma unroll
    for (int k = 0; k < 4; ++k) bad |= !(ok4(v[k].x) && ok4(v[k].y) && ok4(v[k].z) && ok4(v[k].w));
  }
  for (long long i = 16 * nv + i0; i < n; i += stride) bad |= spins[i] != 1 && spins[i] != -1;
  if (bad) atomicCAS(err, 0, kErrBadSpin);
}

template <int WPR, int TH, int H>
__global__ void export_bonds_kernel(const SweepArgs a, uint8_t* out) {
  constexpr int TW = 32 * WPR, RW = WPR * TH;
  const int L = a.g.L;
  const long long n = (long long)L * L;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / L), x = (int)(i % L);
    const int tile = (y / TH) * a.g.tiles_x + x / TW;
    const int ry = y % TH, xx = x % TW;
    const int rw = ry * WPR + (xx >> 5), b = xx & 31;
    const uint32_t* tb = a.tb.tbits + (size_t)tile * 3 * RW;
    out[i] = (uint8_t)(((tb[RW + rw] >> b) & 1u) | (((tb[2 * RW + rw] >> b) & 1u) << 1));
  }
}

int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g > 152LL * 64) g = 152LL * 64;
  return (int)(g < 1 ? 1 : g);
}

template <int WPR, int TH, int H, int PL>
cudaError_t launch_all(int which, const SweepArgs& a, int mode, uint8_t* out, cudaStream_t st,
                       const BatchArgs* batch, int batch_tiles) {
  using T = Tile<WPR, TH, H>;
  const int ntiles = batch ? batch_tiles : a.g.tiles_x * a.g.tiles_y;
  switch (which) {
    case 1:
      phase1_kernel<WPR, TH, H, false><<<ntiles, 32 * WPR, 0, st>>>(a, BatchArgs{});
      break;
    case 2:
      {
        const int xd = a.draws_out ? 32 * kDrawWarps : 0;  // the warps that draw the next sweep's bonds
        phase2_kernel<WPR, TH, H, false><<<ntiles, TH + T::TW + xd, 0, st>>>(a, BatchArgs{});
        resolve_kernel<WPR, TH, H, false><<<ntiles, kResolveThreads + xd, 0, st>>>(a, BatchArgs{});
      }
      break;
    case 3:
      if (mode == 0) {
        phase3_kernel<WPR, TH, H, 0, false><<<ntiles, T::NT, 0, st>>>(a, BatchArgs{});
      } else if (mode == 1) {
        const size_t dyn = (size_t)TH * T::TW * sizeof(uint16_t);
        static bool attr_done = false;
        if (!attr_done) {
          cudaError_t e = cudaFuncSetAttribute(phase3_kernel<WPR, TH, H, 1, false>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
          if (e != cudaSuccess) return e;
          attr_done = true;
        }
        phase3_kernel<WPR, TH, H, 1, false><<<ntiles, T::NT, dyn, st>>>(a, BatchArgs{});
      } else {
        phase3_kernel<WPR, TH, H, 2, false><<<ntiles, T::NT, 0, st>>>(a, BatchArgs{});
      }
      break;
    case 11:
      phase1_kernel<WPR, TH, H, true><<<ntiles, 32 * WPR, 0, st>>>(a, *batch);
      break;
    case 12:
      phase2_kernel<WPR, TH, H, true><<<ntiles, TH + T::TW, 0, st>>>(a, *batch);
      resolve_kernel<WPR, TH, H, true><<<ntiles, kResolveThreads, 0, st>>>(a, *batch);
      break;
    case 13:
      phase3_kernel<WPR, TH, H, 0, true><<<ntiles, T::NT, 0, st>>>(a, *batch);
      break;
    case 4: {
      const long long total = (long long)ntiles * T::MS;
      phase4_kernel<WPR, TH, H><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a);
      break;
    }
    case 5:
      export_bonds_kernel<WPR, TH, H><<<grid_for((long long)a.g.L * a.g.L, 256), 256, 0, st>>>(a, out);
      break;
  }
  return cudaGetLastError();
}

template <int V>
cudaError_t launch_shape(int which, const SweepArgs& a, int mode, uint8_t* out, cudaStream_t st,
                         const BatchArgs* batch, int batch_tiles) {
  constexpr TileShape ts = shape_of(V);
  return launch_all<ts.wpr, ts.th, ts.h, ts.pl>(which, a, mode, out, st, batch, batch_tiles);
}

cudaError_t dispatch(int shape, int which, const SweepArgs& a, int mode, uint8_t* out, cudaStream_t st,
                     const BatchArgs* batch = nullptr, int batch_tiles = 0) {
  switch (shape) {
    case 0: return launch_shape<0>(which, a, mode, out, st, batch, batch_tiles);
    case 1: return launch_shape<1>(which, a, mode, out, st, batch, batch_tiles);
    case 2: return launch_shape<2>(which, a, mode, out, st, batch, batch_tiles);
    case 3: return launch_shape<3>(which, a, mode, out, st, batch, batch_tiles);
    case 4: return launch_shape<4>(which, a, mode, out, st, batch, batch_tiles);
    case 5: return launch_shape<5>(which, a, mode, out, st, batch, batch_tiles);
    case 6: return launch_shape<6>(which, a, mode, out, st, batch, batch_tiles);
    case 7: return launch_shape<7>(which, a, mode, out, st, batch, batch_tiles);
    case 8: return launch_shape<8>(which, a, mode, out, st, batch, batch_tiles);
    case 9: return launch_shape<9>(which, a, mode, out, st, batch, batch_tiles);
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
  check_spins_kernel<<<grid_for(n, 256 * 4) < 152 * 8 ? grid_for(n, 256 * 4) : 152 * 8, 256, 0, st>>>(spins, n, err);
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

cudaError_t launch_potts_phase1(const SweepArgs& a, cudaStream_t st) {
  constexpr TileShape ts = shape_of(kPottsShape);
  potts_phase1_kernel<ts.wpr, ts.th, ts.h><<<a.g.tiles_x * a.g.tiles_y, 32 * ts.wpr, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_potts_phase3(const SweepArgs& a, cudaStream_t st) {
  constexpr TileShape ts = shape_of(kPottsShape);
  potts_phase3_kernel<ts.wpr, ts.th, ts.h><<<a.g.tiles_x * a.g.tiles_y, kPottsP3Threads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_batch_phase(int shape, int which, const BatchArgs& b, int ntiles, cudaStream_t st) {
  if (which < 1 || which > 3) return cudaErrorInvalidValue;
  if (ntiles <= 0) return cudaSuccess;
  return dispatch(shape, 10 + which, SweepArgs{}, 0, nullptr, st, &b, ntiles);
}

cudaError_t launch_batch_advance(const BatchArgs& b, cudaStream_t st) {
  if (b.nrep <= 0) return cudaSuccess;
  batch_advance_kernel<<<(b.nrep + 127) / 128, 128, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_phase31(int shape, const SweepArgs& a3, const SweepArgs& a1, cudaStream_t st) {
  const int ntiles = a3.g.tiles_x * a3.g.tiles_y;
  switch (shape) {
    case 4:
      phase31_kernel<shape_of(4).wpr, shape_of(4).th, shape_of(4).h><<<ntiles, 32 * shape_of(4).wpr, 0, st>>>(a3, a1);
      return cudaGetLastError();
    case 6:
      phase31_kernel<shape_of(6).wpr, shape_of(6).th, shape_of(6).h><<<ntiles, 32 * shape_of(6).wpr, 0, st>>>(a3, a1);
      return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

bool batch_fused_supported(int shape) {
  if (shape < 0 || shape >= kNumShapes) return false;
  const TileShape ts = shape_of(shape);
  return ts.th == 32 * ts.h;
}

cudaError_t launch_batch_fused(int shape, const BatchArgs& b, int ntiles, int nsweeps, cudaStream_t st) {
  if (ntiles <= 0 || nsweeps <= 0) return cudaSuccess;
  switch (shape) {
    case 4: return launch_fused_shape<shape_of(4).wpr, shape_of(4).th, shape_of(4).h>(b, ntiles, nsweeps, st);
    case 6: return launch_fused_shape<shape_of(6).wpr, shape_of(6).th, shape_of(6).h>(b, ntiles, nsweeps, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sw
