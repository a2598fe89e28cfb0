/*
 * sw.h -- C ABI of libsw: Swendsen-Wang dynamics of the 2D Ising model on a
 * periodic square lattice, run on one GB300 (sm_103a).
 *
 * A sweep is the three computing steps of the paper's §2 (Swendsen-Wang
 * Algorithm): bond formation (§2.1), cluster formation (§2.3) and assignment
 * of new spins (§2.4), followed by the energy and magnetisation measurement
 * that closes §2 (H = -sum_<ij> s_i s_j, M = sum_i s_i). The erasure steps
 * (§2.2, §2.5) need no code: new spins overwrite the old ones and bonds are
 * transient.
 *
 * ---------------------------------------------------------------------------
 * Conventions (the paper fixes none of these; every result below is integer
 * and fully determined by them, so two implementations agree bit for bit)
 * ---------------------------------------------------------------------------
 *  C1  Lattice L x L, periodic. site = y*L + x. The east neighbour of (y,x) is
 *      (y,(x+1)%L), the south neighbour ((y+1)%L,x). Each site owns its east
 *      and south edge (§2.1 and Fig. 2: a site checks the neighbours to its
 *      east and south), so there are 2N edges, N = L*L. For L = 2 the two
 *      edges between a pair of sites are distinct edges.
 *  C2  Bond probability p = 1 - exp(-2*beta*J), J = 1. (§2.1 prints
 *      1 - exp(-1/k_B T); with H = -sum s_i s_j from §2 the Swendsen-Wang rule
 *      is 1 - exp(-2 beta), and only that reading puts the transition the
 *      paper reports in §4 (k_B T ~ 2.25) at the Onsager point 2.269.)
 *  C3  Threshold, computed once on the host in binary64:
 *        thr = (uint32) min(floor(ldexp(-expm1(-2*beta), 32)), 0xFFFFFFFF).
 *      A like-spin pair bonds iff its Philox word u satisfies u < thr
 *      (strict). beta must be finite and >= 0. The beta used is the literal
 *      value passed in.
 *  C4  Generator: Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw,
 *      "Parallel random numbers: as easy as 1, 2, 3", SC'11). Key
 *      (k0,k1) = (seed & 0xffffffff, seed >> 32); counter (c0,c1,c2,c3);
 *      output words x0..x3.
 *  C5  Bond draws of sweep t: counter (site>>1, t, 0, 0); site i takes word
 *      x[2*(i&1) + dir], dir 0 = east, 1 = south. One Philox block serves two
 *      consecutive sites and both directions.
 *  C6  Cluster flip of sweep t: one output bit per site index. Block
 *      (b, t, 1, 0) serves the indices 128b .. 128b+127 in order: index i
 *      takes bit (i & 31) of word x[(i >> 5) & 3] of block (i >> 7, t, 1, 0).
 *      The cluster whose canonical label (C9) is root flips iff the bit of
 *      index root is 1; then every site of it takes s <- -s. (The paper's
 *      §2.4 assigns each cluster a fresh random spin; with monochrome
 *      clusters both rules give the same distribution.)
 *  C6b Assignment rule (optional, sw_set_rule / sw_batch_set_rule, §2.4 as
 *      printed): counter (root, t, 3, 0), word x0; every site of the
 *      cluster takes s = (x0>>31) ? -1 : +1, whatever its old spin.
 *  C7  Hot start: counter (site, 0, 2, 0), word x0; s = (x0>>31) ? -1 : +1.
 *      Cold start: every spin +1.
 *  C8  Sweep counter t starts at 0 at creation and grows by one per sweep,
 *      across calls: sw_sweep(h,a); sw_sweep(h,b) == sw_sweep(h,a+b).
 *  C9  Labels: label[i] = the smallest site index in the bond-connected
 *      cluster of i (the "lowest value label" of §2.3). The cluster's root
 *      is that site. int32, so L*L < 2^31 (L <= 46340); L >= 2.
 *  C10 Observables after each sweep, int64: E = -sum_i s_i (s_E(i) + s_S(i))
 *      over the 2N edges, M = sum_i s_i (§2 divides M by N; the caller
 *      divides).
 *  C11 Cluster statistics (optional, per sweep): n_clusters, sum_C |C|^2,
 *      and 32 log2 bins, bin k = number of clusters with 2^k <= |C| < 2^(k+1).
 *
 * ---------------------------------------------------------------------------
 * General rules
 * ---------------------------------------------------------------------------
 *  - Every call returns SW_OK (0) or a negative status below; after a
 *    failure sw_last_error() gives a message (thread-local).
 *  - The library owns all device memory of a handle. Host buffers passed in
 *    belong to the caller and are only read or written during the call.
 *  - A device pointer passed with *_is_device = 1 must be device memory of
 *    the handle's device; the call orders itself on the handle's stream.
 *  - Work runs asynchronously on the handle's stream; calls that return data
 *    to the host (sw_observables, sw_histograms, host-buffer forms of
 *    sw_labels/sw_spins/sw_bonds) synchronise that stream and check the
 *    device error flag (SW_EDEVICE / SW_ETIMEOUT).
 *  - There is no CPU fallback: without a usable GPU, sw_create returns
 *    SW_ECUDA.
 */
#ifndef SW_H
#define SW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SW_OK        0
#define SW_EINVAL   (-1)  /* bad argument: L<2, L*L >= 2^31, beta not finite or < 0, n < 0, range */
#define SW_ENOMEM   (-2)  /* device or host allocation failed */
#define SW_ECUDA    (-3)  /* a CUDA runtime call failed (includes: no GPU) */
#define SW_EDEVICE  (-4)  /* a kernel raised the device error flag (an internal bound was exceeded) */
#define SW_ETIMEOUT (-5)  /* a capped device-side wait or retry loop gave up */

#define SW_INIT_HOT  0
#define SW_INIT_COLD 1

#define SW_RULE_FLIP   0  /* C6: each cluster flips with probability 1/2 (default) */
#define SW_RULE_ASSIGN 1  /* C6b: each cluster gets a fresh spin (§2.4 as printed) */

/* int64 words per sweep written by sw_histograms: n_clusters, sum |C|^2, 32 bins (C11). */
#define SW_HIST_WORDS 34

typedef struct sw_lattice sw_lattice;

/* Bond threshold of C3 for inverse temperature beta (§2.1 bond probability,
 * read as p = 1 - exp(-2 beta)). Returns 0 for beta = 0 and 0xFFFFFFFF once p
 * rounds to 1. For beta < 0, NaN or inf it returns 0 and sets the last error;
 * sw_create rejects such beta with SW_EINVAL. Pure host function. */
uint32_t sw_threshold(double beta);

/* Create a lattice of side L at inverse temperature beta.
 *  L      : 2 <= L <= 46340.
 *  beta   : finite, >= 0.
 *  seed   : Philox key (C4).
 *  init   : SW_INIT_HOT (C7) or SW_INIT_COLD (all +1).
 *  stream : a cudaStream_t of the current device, or NULL for a stream the
 *           library creates and owns. All work of the handle runs on it.
 *  out    : receives the handle. The handle owns its device memory (int8
 *           spins [L][L] row-major, tile records, per-sweep trace) until
 *           sw_destroy.
 * The sweep counter starts at 0 (C8). The initial state is not part of the
 * trace. Errors: SW_EINVAL, SW_ENOMEM, SW_ECUDA. */
int sw_create(int32_t L, double beta, uint64_t seed, int32_t init, void* stream,
              sw_lattice** out);

/* Release every resource of h (synchronises its stream first). NULL is a no-op. */
int sw_destroy(sw_lattice* h);

/* Run n >= 0 sweeps (§2: bonds §2.1, clusters §2.3, new spins §2.4, then
 * the E/M measurement) asynchronously on the handle's stream; sweeps use
 * counters t, t+1, ..., t+n-1 and the counter ends at t+n (C8). After each
 * sweep E and M (C10), and the C11 statistics if enabled, are appended to
 * the device-side trace. Errors: SW_EINVAL (n < 0), SW_ENOMEM (trace
 * growth), SW_ECUDA. Device-side failures are reported by the next call that
 * synchronises. A lattice with L <= 144 and statistics off runs all n
 * sweeps in one CTA-sized launch (the whole lattice in shared memory)
 * unless the environment variable SW_TILE_SHAPE was set at sw_create, which
 * keeps it on the tiled path; the results are the same. Between the sweeps
 * of one call the bond draws of the next sweep (C5: they depend on the
 * seed, the counter and the site, not on the spins) are taken during the
 * current sweep's cross-tile merge; a later call whose first counter is the
 * one they were drawn for reads them too (0.25 byte per site of the
 * handle's memory). */
int sw_sweep(sw_lattice* h, int32_t n);

/* Current sweep counter t (the counter the next sweep will use). */
int sw_get_sweep(sw_lattice* h, uint32_t* t_out);

/* Copy E and M (C10) of sweeps [first, first+count) to the host arrays
 * E_host[count], M_host[count] (either may be NULL). Sweep indices are
 * absolute counters; the trace holds the sweeps run since sw_create or the
 * last sw_set_state, so first must be >= that start and first+count <= the
 * current counter, else SW_EINVAL. Synchronises; checks the error flag. */
int sw_observables(sw_lattice* h, int64_t first, int64_t count,
                   int64_t* E_host, int64_t* M_host);

/* Enable (1) or disable (0) the per-sweep C11 cluster statistics for the
 * sweeps that follow. Sweeps run while disabled read back as zeros. */
int sw_histogram(sw_lattice* h, int32_t enable);

/* New-spin rule of the sweeps that follow: SW_RULE_FLIP (C6, the default)
 * or SW_RULE_ASSIGN (C6b, §2.4). Any other value: SW_EINVAL. */
int sw_set_rule(sw_lattice* h, int32_t rule);

/* Copy the C11 statistics of sweeps [first, first+count) to
 * out_host[count][SW_HIST_WORDS] (int64, row per sweep). Same range rules
 * and synchronisation as sw_observables. */
int sw_histograms(sw_lattice* h, int64_t first, int64_t count, int64_t* out_host);

/* Canonical cluster labels (C9, §2.3) of the bond graph that the NEXT sweep
 * (counter t) draws from the current spins; the state is not changed.
 * out: int32 [L][L]; host memory if out_is_device == 0 (then the call
 * synchronises), else device memory of the handle's device (asynchronous
 * on the handle's stream). */
int sw_labels(sw_lattice* h, int32_t* out, int32_t out_is_device);

/* The same labels as sw_labels, computed by the paper's label-equivalence
 * iteration (§2.3: labels start as site indices; each site proposes the
 * smallest bonded neighbour label as its label's reference; references are
 * collapsed and every site relabelled; repeat until no proposal) instead of
 * the tile union-find. A comparator for measurements, not used by the
 * sweep. *iterations (may be NULL) receives the number of iterations run.
 * Synchronises once per iteration. SW_ETIMEOUT if 2^20 iterations do not
 * converge. */
int sw_labels_equivalence(sw_lattice* h, int32_t* out, int32_t out_is_device, int32_t* iterations);

/* Current spins, int8 [L][L] row-major, values +1/-1. Host or device out as
 * for sw_labels. */
int sw_spins(sw_lattice* h, int8_t* out, int32_t out_is_device);

/* Replace the state: spins int8 [L][L] and the sweep counter t. Every
 * value must be +1 or -1. Host input is copied to a device staging buffer
 * and checked there before it replaces the state: the call synchronises and
 * returns SW_EINVAL, leaving the state untouched, if a value is invalid.
 * Device input is copied and checked asynchronously; a bad value is
 * reported as SW_EINVAL by the next synchronising call. Clears the trace
 * (its start becomes t) and any device error still pending from earlier
 * calls. Used to resume a run from a checkpoint. */
int sw_set_state(sw_lattice* h, const int8_t* spins, uint32_t t, int32_t in_is_device);

/* sw_set_state from host memory without waiting: the copy into the staging
 * buffer, its check and the exchange of buffers are queued on the handle's
 * stream and the call returns at once, so a host loop can queue the next
 * state while the GPU still sweeps. spins_host (int8 [L][L]) must stay
 * unchanged until the stream has copied it (pinned memory makes the copy
 * asynchronous; pageable memory is copied before the call returns). A value
 * other than +1/-1 is reported as SW_EINVAL by the next synchronising call,
 * and the spins are then those from before this call (a kernel copies them
 * back); the counter is t and the trace starts at t either way. The call
 * never clears an error that is still pending from earlier work, so queuing
 * a valid state after an invalid one still ends in SW_EINVAL; a reported
 * SW_EINVAL of this kind is cleared by the report. */
int sw_set_state_async(sw_lattice* h, const int8_t* spins_host, uint32_t t);

/* Debug export of the bonds that the NEXT sweep (counter t) draws from the
 * current spins (§2.1): out_host uint8 [L][L], bit0 = east bond,
 * bit1 = south bond. Synchronises. The state is not changed. */
int sw_bonds(sw_lattice* h, uint8_t* out_host);

/* Per-phase device timing of the sweeps that follow: with enable = 1 every
 * phase launch of sw_sweep is bracketed by CUDA events on the handle's
 * stream (accumulators cleared); enable = 0 stops recording. Phases:
 * 0 = bonds + tile-local clusters, 1 = cross-tile merge, 2 = flips + E/M,
 * 3 = cluster statistics, 4 = flips + E/M of a sweep together with the bonds
 * and tile-local clusters of the next sweep of the same call (one launch,
 * on the 128x64 and 128x128 tile shapes with statistics off; a call's last
 * sweep runs phase 2 alone). Not part of the paper: measurement support. */
#define SW_TIMING_PHASES 5
int sw_timing(sw_lattice* h, int32_t enable);

/* Synchronise, then report for each of the SW_TIMING_PHASES phases the
 * summed device time in milliseconds (ms_out[SW_TIMING_PHASES]) and the
 * number of kernel launches (launches_out[SW_TIMING_PHASES]) recorded since
 * sw_timing(h, 1). Either pointer may be NULL. */
int sw_timing_read(sw_lattice* h, double* ms_out, int64_t* launches_out);

/* ---------------------------------------------------------------------------
 * Batched form: many independent lattices (replicas) of any sides and
 * temperatures advanced together. The paper runs one lattice at a time; this
 * applies its sweep (§2) to every replica at once, each replica following
 * exactly the chain it would follow alone (same conventions C1-C10, keyed by
 * its own seed and counter), so results are bit-identical to sw_sweep.
 * Every phase of a sweep is one launch over the tiles of all replicas, or a
 * whole n-sweep chunk is one persistent launch (sw_batch_set_schedule); the
 * n-sweep sequence is captured as a CUDA graph and replayed while the
 * membership and n stay the same. Replicas may be added and removed between
 * sw_batch_sweep calls (continuous batching).
 * --------------------------------------------------------------------------- */
typedef struct sw_batch sw_batch;

/* Create a batch with n >= 0 replicas (side L[i], beta[i], seed[i], init[i]
 * or SW_INIT_HOT when init is NULL). shape: a compiled tile shape index or
 * -1 for the default. stream: as for sw_create. The batch owns all device
 * memory of its replicas. Errors: SW_EINVAL, SW_ENOMEM, SW_ECUDA. */
int sw_batch_create(int32_t n, const int32_t* L, const double* beta, const uint64_t* seed,
                    const int32_t* init, int32_t shape, void* stream, sw_batch** out);

/* Add one replica; *slot_out receives its slot (stable until removed; freed
 * slots are reused). Its sweep counter starts at 0. */
int sw_batch_add(sw_batch* b, int32_t L, double beta, uint64_t seed, int32_t init, int32_t* slot_out);

/* Remove the replica in `slot` (synchronises the stream, frees its memory). */
int sw_batch_remove(sw_batch* b, int32_t slot);

/* Advance every replica by n >= 0 sweeps, asynchronously on the batch's
 * stream. Errors: SW_EINVAL, SW_ENOMEM (trace growth), SW_ECUDA. */
int sw_batch_sweep(sw_batch* b, int32_t n);

/* Let the replica in `slot` run only sweeps_left more sweeps (from its
 * current counter); later sw_batch_sweep calls leave it idle once they are
 * done, so it stops exactly at its target while the others go on. A
 * negative value removes the limit. */
int sw_batch_set_limit(sw_batch* b, int32_t slot, int64_t sweeps_left);

/* New-spin rule (SW_RULE_FLIP or SW_RULE_ASSIGN) of the replica in `slot`
 * for the sweeps that follow. */
int sw_batch_set_rule(sw_batch* b, int32_t slot, int32_t rule);

/* How sw_batch_sweep runs the sweeps (the results are the same bits either
 * way; §2's sweep applied to every replica):
 *   SW_SCHEDULE_PHASES (default): per sweep, one launch per phase over the
 *     tiles of all replicas (phases 1, 2 + resolve, 3) and a counter
 *     advance; the n-sweep sequence is one captured CUDA graph;
 *   SW_SCHEDULE_FUSED: one persistent cooperative launch runs all n sweeps
 *     (CTAs stay resident and take tiles in turn; the phases are separated
 *     by grid barriers whose waits are bounded, a stuck barrier ending in
 *     SW_ETIMEOUT from the next synchronising call), captured as a CUDA
 *     graph with the barrier's reset (or launched directly where the
 *     cooperative launch cannot be captured).
 * The fused schedule needs a tile shape whose phases 1 and 3 run the same
 * block (64-row tiles of 2-row strips, 128-row tiles of 4-row strips):
 * SW_EINVAL otherwise. Synchronises the stream when the schedule changes. */
#define SW_SCHEDULE_PHASES 0
#define SW_SCHEDULE_FUSED 1
int sw_batch_set_schedule(sw_batch* b, int32_t schedule);

/* Replicas of side L <= max_L run on the one-CTA path (a whole lattice in
 * one CTA's shared memory, all sweeps of a chunk in one block, as sw_sweep
 * does for small lattices): one CTA per such replica, launched before the
 * tiled work of each chunk; the others stay on the tiles. 0 (the default)
 * puts every replica on the tiles. The results are the same bits either
 * way; the choice only moves time (the one-CTA path holds a whole SM for a
 * small lattice, the tiles share SMs between replicas). max_L must be 0 or
 * 2..181, else SW_EINVAL. Synchronises the stream when it changes. */
int sw_batch_set_small(sw_batch* b, int32_t max_L);

/* Sweep counter of the replica in `slot`. */
int sw_batch_get_sweep(sw_batch* b, int32_t slot, uint32_t* t_out);

/* E and M of the replica's sweeps [first, first+count) (absolute counters,
 * since its creation), as sw_observables. Synchronises; checks the error
 * flag. */
int sw_batch_observables(sw_batch* b, int32_t slot, int64_t first, int64_t count,
                         int64_t* E_host, int64_t* M_host);

/* Current spins of the replica, int8 [L][L], host (synchronises) or device. */
int sw_batch_spins(sw_batch* b, int32_t slot, int8_t* out, int32_t out_is_device);

/* Number of active replicas, their total sites and the device bytes they
 * hold (any pointer may be NULL). */
int sw_batch_info(sw_batch* b, int32_t* n_active, int64_t* sites, int64_t* device_bytes);

/* Device bytes that sw_batch_add of a replica of side L, run for `sweeps`
 * sweeps under a limit, makes this batch hold (spins, tile buffers and E/M
 * trace, as requested from the allocator): the figure a server admits
 * requests against its memory budget by. */
int sw_batch_footprint(sw_batch* b, int32_t L, int64_t sweeps, int64_t* bytes);

/* Release the batch and all its replicas. NULL is a no-op. */
int sw_batch_destroy(sw_batch* b);

/* ---------------------------------------------------------------------------
 * q-state Potts model (the paper's §6 generalisation of the sweep)
 * ---------------------------------------------------------------------------
 *  P1  States int8 in 0..q-1, 2 <= q <= 127; lattice and edges as C1.
 *      H = -sum over the 2N edges of delta(s_i, s_j).
 *  P2  Equal neighbours bond with probability p = 1 - exp(-beta); threshold
 *      thr = (uint32) min(floor(ldexp(-expm1(-beta), 32)), 0xFFFFFFFF); the
 *      bond draws are C5's, with "equal states" for "equal spins".
 *  P3  Labels C9. New states: the cluster rooted at r takes
 *      floor(x0 * q / 2^32), x0 = word 0 of Philox block (r, t, 3, 0).
 *  P4  Hot start: floor(x0 * q / 2^32), x0 = word 0 of block (i, 0, 2, 0);
 *      cold start: every state 0.
 *  P5  Observables after each sweep, int64: E = -(number of edges joining
 *      equal states), M = number of sites in state 0.
 *  For q = 2 and beta = 2 beta_Ising this is the Ising sweep with the
 *  assignment rule (C6b), state 1 <-> spin -1. The sweep runs site-parallel
 *  kernels over global memory (a union-find over int32 parents). Rules of
 *  the Ising handle (ownership, streams, statuses) apply.
 * --------------------------------------------------------------------------- */
typedef struct sw_potts sw_potts;

/* Threshold P2 for beta; 0 for an invalid beta. */
uint32_t sw_potts_threshold(double beta);

/* New Potts lattice: SW_EINVAL for L outside [2, 46340], q outside 2..127,
 * a bad beta or init; SW_ECUDA without a GPU. */
int sw_potts_create(int32_t L, int32_t q, double beta, uint64_t seed, int32_t init, void* stream,
                    sw_potts** out);

/* n >= 0 sweeps with counters t .. t+n-1 (C8); E and M (P5) appended to the trace. */
int sw_potts_sweep(sw_potts* h, int32_t n);

/* E and M of sweeps [first, first+count) (absolute counters, as sw_observables). */
int sw_potts_observables(sw_potts* h, int64_t first, int64_t count, int64_t* E_host, int64_t* M_host);

/* Current states, int8 [L][L], host (synchronises) or device. */
int sw_potts_states(sw_potts* h, int8_t* out, int32_t out_is_device);

/* Replace the states (host or device int8 [L][L]) and set the counter to t;
 * the trace restarts at t. A state outside 0..q-1: SW_EINVAL, state kept. */
int sw_potts_set_state(sw_potts* h, const int8_t* states, uint32_t t, int32_t in_is_device);

/* Canonical labels (C9) of the bonds the next sweep draws; the states and
 * the counter are not changed. */
int sw_potts_labels(sw_potts* h, int32_t* out, int32_t out_is_device);

/* Counter of the next sweep. */
int sw_potts_get_sweep(sw_potts* h, uint32_t* t_out);

/* Release the lattice (synchronises its stream). NULL is a no-op. */
int sw_potts_destroy(sw_potts* h);

/* ---------------------------------------------------------------------------
 * O(4) phi^4 theory in four dimensions: the multicluster update (§3, Eqs. 2
 * and 3)
 * ---------------------------------------------------------------------------
 *  O1  Lattice L^4, periodic, site x = x0 + L (x1 + L (x2 + L x3)); each
 *      site owns its 4 edges to x + e_mu. Field phi_x in R^4, binary64,
 *      stored [N][4].
 *  O2  Hot start: component a of phi_x = (w_a + 0.5) 2^-31 - 1, w_a the
 *      words of Philox block (x, 0, 7, 0); cold start phi_x = (1, 0, 0, 0).
 *  O3  Direction r of update t, uniform on the unit 3-sphere: attempts
 *      k = 0, 1, ...: v_a = (w_a + 0.5) 2^-31 - 1 from block (k, t, 5, 0),
 *      s = fma(v3, v3, fma(v2, v2, fma(v1, v1, v0 * v0))); the first attempt
 *      with 2^-20 < s <= 1 gives r_a = v_a / sqrt(s).
 *  O4  Projection a_x = fma(phi3, r3, fma(phi2, r2, fma(phi1, r1, phi0 *
 *      r0))). Edge (x, mu), y = x + e_mu, bonds iff q = a_x a_y > 0 and
 *      (double) w_mu < (1 - e) 2^32 with e = e^{-(4 kappa) q} (Eq. 2), w_mu =
 *      word mu of block (x, t, 4, 0). e is computed by the library's own
 *      exponential (Cody-Waite reduction with a 32-bit head of ln 2, Taylor
 *      series to degree 14 with fused multiply-adds, 0 for arguments above
 *      40), so the decisions are reproducible bit for bit.
 *  O5  Clusters: labels C9. The cluster rooted at r is flipped iff bit 31 of
 *      word 0 of block (r, t, 6, 0); a flipped site's component a becomes
 *      fma(-2 a_x, r_a, phi_a) (Eq. 3: reflection in the hyperplane
 *      orthogonal to r).
 *  Observables per update, binary64: E = sum over the 4N edges of
 *  phi_x . phi_{x+mu}, M = sum_x phi_x (4 components). They are reduced in
 *  parallel, so they match a serial sum to rounding, not bit for bit; the
 *  field itself is bit-exact.
 * --------------------------------------------------------------------------- */
typedef struct sw_phi4 sw_phi4;

/* Direction O3 of update t. r_out: 4 doubles. */
int sw_phi4_direction(uint64_t seed, uint32_t t, double* r_out);

/* New field on an L^4 torus (2 <= L, L^4 < 2^31), hopping coupling kappa
 * (finite, >= 0), start O2. */
int sw_phi4_create(int32_t L, double kappa, uint64_t seed, int32_t init, void* stream, sw_phi4** out);

/* n >= 0 multicluster updates with counters t .. t+n-1. */
int sw_phi4_sweep(sw_phi4* h, int32_t n);

/* E_host[count] and M_host[count][4] of updates [first, first+count). */
int sw_phi4_observables(sw_phi4* h, int64_t first, int64_t count, double* E_host, double* M_host);

/* The field, double [N][4], host (synchronises) or device. */
int sw_phi4_field(sw_phi4* h, double* out, int32_t out_is_device);

/* Replace the field (host or device double [N][4]) and set the counter to t. */
int sw_phi4_set_field(sw_phi4* h, const double* in, uint32_t t, int32_t in_is_device);

/* Labels C9 of the bonds the next update draws; the field is not changed. */
int sw_phi4_labels(sw_phi4* h, int32_t* out, int32_t out_is_device);

/* Counter of the next update. */
int sw_phi4_get_sweep(sw_phi4* h, uint32_t* t_out);

/* Release the field (synchronises its stream). NULL is a no-op. */
int sw_phi4_destroy(sw_phi4* h);

/* Largest side accepted by sw_sweep_noalloc. */
#define SW_NOALLOC_MAX_L 1024

/* Allocation-free sweep. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- a host framework
 * whose allocator has already reserved the GPU's memory, a plugin host that
 * forbids device allocation, or a latency-critical loop that cannot accept
 * cudaMalloc's implicit device-wide synchronisation. It runs the same sweep
 * as sw_sweep (same conventions C1-C10, bit-identical results) without a
 * handle and without allocating anything.
 *  spins  : device int8 [L][L] (+1/-1), the state; read and updated in place.
 *  L      : 2 <= L <= SW_NOALLOC_MAX_L, else SW_EINVAL.
 *  beta   : finite, >= 0 (C2, C3).
 *  seed   : Philox key (C4).
 *  t0, n  : sweeps use counters t0 .. t0+n-1 (C8); n >= 0.
 *  em     : device int64 [n][2], output: E and M after each sweep (C10).
 *  err    : device int32 [1], output: set to 0 by the call, then to a
 *           nonzero code if a capped device retry loop gave up.
 *  stream : cudaStream_t for all work (NULL = the legacy default stream).
 * For L <= 181 the whole lattice is swept inside one CTA's shared memory
 * and nothing else is used. For larger L the kernels' working buffers live
 * in one file-scope __device__ array of
 * under 4 MiB that every GPU loading the library holds until exit. The first
 * call on a device looks up that array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and its contents persist between calls, so calls
 * that overlap on the GPU (other streams, other host threads) race and
 * corrupt each other's results: serialise them. Work is asynchronous on the
 * stream; argument errors return SW_EINVAL before anything is enqueued,
 * launch failures SW_ECUDA. Calls no cudaMalloc/cudaFree. */
int sw_sweep_noalloc(int8_t* spins, int32_t L, double beta, uint64_t seed, uint32_t t0, int32_t n,
                     int64_t* em, int32_t* err, void* stream);

/* ---------------------------------------------------------------------------
 * Tile shapes (measurement and tuning support; the paper fixes 32-wide tiles,
 * §5). A sweep runs over tiles of tile_w x tile_h sites, each thread scanning
 * a strip of strip_h rows of one 32-site word column.
 * --------------------------------------------------------------------------- */

/* Number of tile shapes compiled into the library (indices 0 .. n-1). */
int sw_num_shapes(void);

/* Geometry of a compiled tile shape (any output pointer may be NULL). */
int sw_shape_info(int32_t shape, int32_t* tile_w, int32_t* tile_h, int32_t* strip_h, int32_t* threads);

/* Process-wide preference: lattices whose side L has ceil(log2 L) ==
 * log2_bucket (0..16) use `shape` from now on in sw_create, and batches
 * created with shape -1 use the entry of their largest L; shape -1 restores
 * the built-in default (64x64 tiles up to L = 64; then for a lattice 128x32
 * tiles up to L = 1024 and 128x64 above, for a batch 128x64). Results never
 * depend on the shape. */
int sw_tune_shape(int32_t log2_bucket, int32_t shape);

/* The tile shape index a lattice was created with (its tiled path; sides up
 * to 144 run whole sweeps in one CTA unless SW_TILE_SHAPE is set). */
int sw_lattice_shape(sw_lattice* h, int32_t* shape);

/* Message of the last failed call on this thread ("" if none). */
const char* sw_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SW_H */
