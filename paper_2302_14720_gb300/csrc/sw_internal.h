// sw_internal.h -- interface between the C ABI layer (sw_api.cu) and the
// sweep kernels (sw_kernels.cu). Not installed; not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sw_philox.cuh"

namespace sw {

// Device error flag values (first writer wins).
enum DeviceError : int {
  kErrNone = 0,
  kErrUnionCap = 1,     // a union-find retry loop hit its iteration cap
  kErrBadSpin = 2,      // sw_set_state from device memory saw a value other than +1/-1
  kErrSlotOverflow = 3, // more boundary components than slots (cannot happen; checked)
  kErrCopyTimeout = 4,  // a bulk copy into shared memory did not land within its time limit
  kErrBarrierTimeout = 5,  // a grid barrier of the fused batch kernel did not open within its time limit
};

// A tile shape: TW = 32*WPR columns by TH rows. Phase 1 runs one warp per
// 32-column band (32 * WPR threads); in phase 3 each thread owns one 32-site
// word column of an H-row strip of the tile (WPR * TH/H threads per tile).
// Tiles are laid over the L x L lattice from the origin; the last tile
// column and row may be ragged.
struct TileShape {
  int wpr;  // 32-bit words per tile row
  int th;   // rows per tile
  int h;    // rows per thread strip
  int pl;   // rounds of pairwise strip merging done without atomics
  int tw() const { return 32 * wpr; }
  int row_words() const { return wpr * th; }
  int sites() const { return tw() * th; }
  int threads() const { return wpr * (th / h); }
  int max_slots() const { return 2 * (tw() + th); }     // boundary sites bound the slots
  int boundary_sites() const { return 2 * th + 2 * tw(); }
  int bbits_words() const { return 2 * (th / 32) + 2 * (tw() / 32); }
};

// Shapes compiled into the library; index = variant id.
constexpr int kNumShapes = 10;
__host__ __device__ constexpr TileShape shape_of(int v) {
  return v == 0   ? TileShape{4, 64, 4, 0}
         : v == 1 ? TileShape{4, 64, 8, 0}
         : v == 2 ? TileShape{2, 64, 4, 0}
         : v == 3 ? TileShape{8, 64, 4, 0}
         : v == 4 ? TileShape{4, 128, 4, 0}
         : v == 5 ? TileShape{8, 64, 8, 0}
         : v == 6 ? TileShape{4, 64, 2, 0}
         : v == 7 ? TileShape{4, 32, 2, 0}
         : v == 8 ? TileShape{8, 32, 2, 0}
                  : TileShape{16, 32, 2, 0};
}

// Per-lattice device buffers of the tile pipeline.
struct TileBuffers {
  uint32_t* tbits;   // [ntiles][3][row_words]: spin bits, east-bond bits, south-bond bits per row-word
  uint16_t* roots;   // [ntiles][sites]: tile-local label of every site; a label's entry is its root (phase 1 -> phase 3)
  uint32_t* bmask;   // [ntiles][row_words]: bit set at every tile root that touches the tile border
  uint32_t* rbits;   // [ntiles][row_words]: bit set at every tile root
  uint64_t* nodes;   // [ntiles * max_slots]: global union-find, (key << 32) | parent node
  uint16_t* bslot;   // [ntiles][boundary_sites]: slot of each boundary site (left, right, top, bottom)
  uint32_t* bbits;   // [ntiles][bbits_words]: E-out bonds, S-out bonds, east halo spins, south halo spins
  int32_t* nslots;   // [ntiles]
  int* err;          // device error flag
  uint8_t* nval;     // Potts only, [ntiles * max_slots]: new state of each slot's cluster (resolve -> phase 3)
};

struct Geometry {
  int L;
  int tiles_x, tiles_y;
  int aligned16;  // rows start on 16-byte boundaries (L % 16 == 0)
};

struct SweepArgs {
  Geometry g;
  uint32_t thr;        // bond threshold (C3)
  uint32_t t;          // sweep counter (C5, C6)
  uint32_t rule;       // new spins: 0 flip each cluster with probability 1/2 (C6), 1 assign a fresh spin (§2.4)
  uint32_t q;          // 0: Ising spins +-1; q >= 2: Potts states 0..q-1 in spins_in / spins_out (§6)
  KeySchedule ks;      // Philox key schedule of the seed (C4)
  TileBuffers tb;
  const int8_t* spins_in;
  int8_t* spins_out;   // flip mode: new spins (may alias spins_in)
  int64_t* em;         // flip mode: E, M accumulators of this sweep (zeroed by phase 1)
  int64_t* hist;       // flip mode: SW_HIST_WORDS accumulators or nullptr
  uint32_t* csize;     // flip mode with hist: per-node cluster size accumulators [nodes]
  int32_t* labels;     // labels mode: int32 [L][L] output
  // The C5 draws of a sweep depend on the seed, the counter and the site,
  // not on the spins, so they can be taken ahead of time: per row word of a
  // tile ([ntiles][row_words]) the mask of east and of south words below thr.
  const uint2* draws_in;  // phase 1: the draws of sweep t, or nullptr (phase 1 draws them)
  uint2* draws_out;       // phase 2 + resolve: where to leave the draws of sweep t + 1, or nullptr
};

inline int ntiles_of(const Geometry& g) { return g.tiles_x * g.tiles_y; }

// One replica of a batch, resident on the device. `a` holds its geometry,
// threshold, key schedule, buffers and spins; the sweep counter and the
// trace position advance on the device, so one captured launch sequence can
// be replayed for any number of sweeps.
struct ReplicaDesc {
  SweepArgs a;
  int tile0;          // first tile of this replica in the batch's tile numbering
  int active;         // 0: slot free (its tiles are not launched)
  uint32_t t;         // counter of the next sweep (C8)
  int64_t t_left;     // sweeps still to run (the replica idles at 0)
  int64_t* em_base;   // E/M trace [cap][2]
  int64_t em_next;    // trace row of the next sweep
  int small;          // 1: runs on the one-CTA path (small_batch_kernel advances it)
};

// Arrival count and generation of the fused batch kernel's grid barrier.
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};

struct BatchArgs {
  ReplicaDesc* descs;
  const int* tile_rep;  // batch tile -> replica index
  int nrep;
  int* err;             // the batch's device error flag (fused kernel)
  GridBarrier* gbar;    // the fused kernel's grid barrier (zeroed before each launch)
};

// Set the thread's last error message (sw_last_error) and return code.
int record_error(int code, const char* msg);

// Tile shape for a lattice of side L: SW_TILE_SHAPE override, else the
// tuned entry of L's size bucket, else the built-in default.
int default_shape(int L);

// Launchers (sw_kernels.cu). Each returns cudaGetLastError() of its launches.
cudaError_t launch_init(int8_t* spins, int L, uint64_t seed, int cold, cudaStream_t st);
cudaError_t launch_check_spins(const int8_t* spins, int64_t n, int* err, cudaStream_t st);
// Phase 1: bonds + tile-local labelling + boundary slot tables (one CTA per tile).
cudaError_t launch_phase1(int shape, const SweepArgs& a, cudaStream_t st);
// Phase 2: union of tile components across bonded tile-boundary edges.
cudaError_t launch_phase2(int shape, const SweepArgs& a, cudaStream_t st);
// Phase 3: canonical roots, flips, new spins, E/M (+ statistics), or labels.
cudaError_t launch_phase3(int shape, const SweepArgs& a, bool labels_mode, cudaStream_t st);
// Phase 4 (statistics only): log2 histogram of cluster sizes held at global roots.
cudaError_t launch_phase4(int shape, const SweepArgs& a, cudaStream_t st);
// Batch: phase 1, 2 or 3 (which = 1..3) over `ntiles` tiles of all replicas.
cudaError_t launch_batch_phase(int shape, int which, const BatchArgs& b, int ntiles, cudaStream_t st);
// Batch: advance every active replica's sweep counter and trace row by one.
cudaError_t launch_batch_advance(const BatchArgs& b, cudaStream_t st);
// Batch, fused schedule: one cooperative launch runs nsweeps whole sweeps of
// every replica with tiles (all four phases, grid barriers between them) and
// advances the replicas' counters itself. Only shapes whose phases 1 and 3
// take the same block (TH == 32 H) have it: batch_fused_supported.
bool batch_fused_supported(int shape);
// Phase 3 of sweep t (a3) and phase 1 of sweep t + 1 (a1) in one launch, the
// new spins handed over in shared memory (flip or assignment rule, no
// statistics). Same shapes as batch_fused_supported.
cudaError_t launch_phase31(int shape, const SweepArgs& a3, const SweepArgs& a1, cudaStream_t st);
cudaError_t launch_batch_fused(int shape, const BatchArgs& b, int ntiles, int nsweeps, cudaStream_t st);

// Whole sweeps of one small lattice in one CTA (sw_small.cu). 181^2 < 2^15,
// so 16-bit parents index every site.
constexpr int kSmallMaxL = 181;
// sw_sweep takes the one-CTA path up to this side; from about L = 160 on the
// tiled path is as fast on GB300 (62 us per sweep either way at L = 160).
constexpr int kSmallSweepMaxL = 144;
struct SmallArgs {
  int L;
  uint32_t thr;    // C3
  uint32_t rule;   // 0 flip (C6), 1 assign (C6b)
  uint32_t t0;     // counter of the first sweep
  int n;           // sweeps to run
  KeySchedule ks;  // C4
  int8_t* spins;   // int8 [L][L], read at the start and written at the end
  int64_t* em;     // [n][2] E, M after each sweep
  int* err;        // device error flag
};
cudaError_t launch_small(const SmallArgs& a, cudaStream_t st);
// Batch: the replicas listed in small[0..nsmall) (sides <= max_L <=
// kSmallMaxL) run up to n sweeps each on the one-CTA path, one CTA per
// replica, and advance their own counters.
cudaError_t launch_small_batch(const BatchArgs& b, const int* small, int nsmall, int max_L, int n, cudaStream_t st);

// The paper's label-equivalence iteration (§2.3) over exported bonds
// (uint8 per site, bit 0 east, bit 1 south); comparator only (sw_equiv.cu).
// iterations: count run, negated if max_iter was reached first.
cudaError_t run_label_equivalence(const uint8_t* bonds, int L, int32_t* lab, int32_t* ref, int* d_changed, int* err,
                                  int max_iter, int* iterations, cudaStream_t st);
// Debug: expand the stored bond bits into uint8 [L][L] (bit0 east, bit1 south).
cudaError_t launch_export_bonds(int shape, const SweepArgs& a, uint8_t* out, cudaStream_t st);

// q-state Potts sweeps (§6) on the 128x64 tile shape: phase 1 bonds equal
// states, phase 2 (launch_phase2) is the Ising one with resolve drawing each
// border cluster's new state into tb.nval, and phase 3 assigns the states and
// sums E, M. Labels come from launch_phase3's labels mode. a.q >= 2.
constexpr int kPottsShape = 6;
cudaError_t launch_potts_phase1(const SweepArgs& a, cudaStream_t st);
cudaError_t launch_potts_phase3(const SweepArgs& a, cudaStream_t st);

}  // namespace sw
