/*
 * sw_oracle.c -- serial CPU oracle for Swendsen-Wang dynamics of the 2D
 * Ising model (Protzman & Giedt, "GPU Acceleration of Swendson-Wang
 * Dynamics", §2).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * statement of what one sweep computes. Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it. It shares no code,
 * header, table or constant generator with the CUDA library; the
 * conventions it follows (lattice indexing, threshold, Philox keying, flip
 * rule, labels, observables) are restated here from their definitions.
 *
 * One sweep at counter t, exactly in the order of §2:
 *   1. bonds (§2.1): for every site i and direction d in {east, south},
 *      bond iff s_i == s_j and the Philox word assigned to (i, d) is below
 *      the threshold thr = floor(2^32 * (1 - exp(-2 beta)));
 *   2. spins are not erased explicitly (§2.2);
 *   3. clusters (§2.3): breadth-first search over the bond graph, sources
 *      taken in increasing site order, so every site receives the smallest
 *      site index of its cluster (the "lowest value label");
 *   4. new spins (§2.4): cluster with root r flips iff the Philox bit drawn
 *      for index r in sweep t is set (one block per 128 indices);
 *   5. bonds are dropped (§2.5);
 *   then E = -sum over the 2N edges of s_i s_j and M = sum s_i (end of §2).
 *
 * Philox-4x32-10 follows Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): ten rounds of the 4-word Philox
 * S-box (two 32x32->64 multiplications, the high halves xored with the other
 * two words and the round key, the words permuted), with the key bumped by
 * the Weyl increments between rounds.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Philox */

/* Multipliers and Weyl key increments of Philox-4x32 (Salmon et al. 2011). */
#define PHILOX_MUL_A 0xD2511F53u
#define PHILOX_MUL_B 0xCD9E8D57u
#define PHILOX_WEYL_A 0x9E3779B9u /* golden ratio */
#define PHILOX_WEYL_B 0xBB67AE85u /* sqrt(3) - 1 */

void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod_a = (uint64_t)PHILOX_MUL_A * x0;
        uint64_t prod_b = (uint64_t)PHILOX_MUL_B * x2;
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t y0 = hi_b ^ x1 ^ k0;
        uint32_t y1 = lo_b;
        uint32_t y2 = hi_a ^ x3 ^ k1;
        uint32_t y3 = lo_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_WEYL_A;
        k1 += PHILOX_WEYL_B;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void philox_seeded(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    oracle_philox(ctr, key, out);
}

/* ------------------------------------------------------------- threshold */

/* thr = floor(2^32 * (1 - exp(-2 beta))), capped at 2^32 - 1; 0 for invalid
 * beta (the caller rejects it). Bond probability of §2.1 read as
 * 1 - exp(-2 beta J) with J = 1. */
uint32_t oracle_threshold(double beta) {
    if (!(beta >= 0.0) || isinf(beta)) return 0u;
    double p = -expm1(-2.0 * beta);
    double scaled = floor(ldexp(p, 32));
    if (scaled >= 4294967295.0) return 0xffffffffu;
    return (uint32_t)scaled;
}

/* ---------------------------------------------------------- initial state */

/* Hot start: site i takes -1 iff the top bit of word x0 of Philox block
 * (i, 0, 2, 0) is set. Cold start: all +1. (Fig. 1 starts from random
 * spins; the generator is this library's convention.) */
void oracle_init(int L, uint64_t seed, int cold, int8_t* s) {
    int64_t N = (int64_t)L * L;
    for (int64_t i = 0; i < N; ++i) {
        if (cold) { s[i] = 1; continue; }
        uint32_t w[4];
        philox_seeded(seed, (uint32_t)i, 0u, 2u, 0u, w);
        s[i] = (w[0] >> 31) ? (int8_t)-1 : (int8_t)1;
    }
}

/* ------------------------------------------------------------------ bonds */

/* §2.1: each site tests its east and south neighbour. bonds[i] bit0 = east
 * bond of i, bit1 = south bond of i. Word for (i, dir) is word
 * 2*(i&1)+dir of Philox block (i>>1, t, 0, 0). */
void oracle_bonds(int L, uint64_t seed, uint32_t t, uint32_t thr, const int8_t* s, uint8_t* bonds) {
    for (int y = 0; y < L; ++y) {
        for (int x = 0; x < L; ++x) {
            int64_t i = (int64_t)y * L + x;
            int64_t east = (int64_t)y * L + (x + 1) % L;
            int64_t south = (int64_t)((y + 1) % L) * L + x;
            uint32_t w[4];
            philox_seeded(seed, (uint32_t)(i >> 1), t, 0u, 0u, w);
            uint32_t u_east = w[2 * (i & 1) + 0];
            uint32_t u_south = w[2 * (i & 1) + 1];
            uint8_t b = 0;
            if (s[i] == s[east] && u_east < thr) b |= 1u;
            if (s[i] == s[south] && u_south < thr) b |= 2u;
            bonds[i] = b;
        }
    }
}

/* ----------------------------------------------------------------- labels */

/* §2.3: every site gets the lowest site index of its bond-connected
 * cluster. Breadth-first search with sources in increasing index order:
 * the first unvisited site met is the minimum of its cluster. queue must
 * hold N entries. Returns the number of clusters. */
int64_t oracle_labels(int L, const uint8_t* bonds, int32_t* label, int32_t* queue) {
    int64_t N = (int64_t)L * L;
    for (int64_t i = 0; i < N; ++i) label[i] = -1;
    int64_t n_clusters = 0;
    for (int64_t src = 0; src < N; ++src) {
        if (label[src] >= 0) continue;
        ++n_clusters;
        int64_t head = 0, tail = 0;
        label[src] = (int32_t)src;
        queue[tail++] = (int32_t)src;
        while (head < tail) {
            int64_t i = queue[head++];
            int y = (int)(i / L), x = (int)(i % L);
            int64_t nb[4];
            int has[4];
            /* east: own bond bit0 */
            nb[0] = (int64_t)y * L + (x + 1) % L;             has[0] = bonds[i] & 1u;
            /* south: own bond bit1 */
            nb[1] = (int64_t)((y + 1) % L) * L + x;           has[1] = (bonds[i] >> 1) & 1u;
            /* west: the east bond of the west neighbour */
            nb[2] = (int64_t)y * L + (x + L - 1) % L;         has[2] = bonds[nb[2]] & 1u;
            /* north: the south bond of the north neighbour */
            nb[3] = (int64_t)((y + L - 1) % L) * L + x;       has[3] = (bonds[nb[3]] >> 1) & 1u;
            for (int k = 0; k < 4; ++k) {
                if (has[k] && label[nb[k]] < 0) {
                    label[nb[k]] = (int32_t)src;
                    queue[tail++] = (int32_t)nb[k];
                }
            }
        }
    }
    return n_clusters;
}

/* ------------------------------------------------------------------- flip */

/* §2.4 with the flip reading: Philox block (b, t, 1, 0) holds one bit for
 * each of the site indices 128b .. 128b+127, words x0..x3 in order, bit 0
 * first; the cluster rooted at r flips iff the bit of index r is set. */
void oracle_flip(int L, uint64_t seed, uint32_t t, const int32_t* label, int8_t* s) {
    int64_t N = (int64_t)L * L;
    for (int64_t i = 0; i < N; ++i) {
        uint32_t r = (uint32_t)label[i];
        uint32_t w[4];
        philox_seeded(seed, r / 128u, t, 1u, 0u, w);
        uint32_t bit = (w[(r % 128u) / 32u] >> (r % 32u)) & 1u;
        if (bit) s[i] = (int8_t)(-s[i]);
    }
}

/* Apply an explicit flip decision per cluster: flip_of_root[r] (0/1) is read
 * at the root r = label[i]. Used by exact transition-matrix tests, which
 * enumerate every flip pattern instead of drawing it. */
void oracle_apply_flips(int L, const int32_t* label, const uint8_t* flip_of_root, int8_t* s) {
    int64_t N = (int64_t)L * L;
    for (int64_t i = 0; i < N; ++i)
        if (flip_of_root[label[i]]) s[i] = (int8_t)(-s[i]);
}

/* §2.4 as the paper prints it (the assignment reading): every cluster gets
 * a fresh spin, -1 iff the top bit of word x0 of Philox block (r, t, 3, 0)
 * is set, r = the cluster's root; the old spins are not read. */
void oracle_assign(int L, uint64_t seed, uint32_t t, const int32_t* label, int8_t* s) {
    int64_t N = (int64_t)L * L;
    for (int64_t i = 0; i < N; ++i) {
        uint32_t w[4];
        philox_seeded(seed, (uint32_t)label[i], t, 3u, 0u, w);
        s[i] = (w[0] >> 31) ? (int8_t)-1 : (int8_t)1;
    }
}

/* Apply an explicit new spin per cluster: minus_of_root[r] (0/1, 1 = -1) is
 * read at the root r = label[i]. Used by exact transition-matrix tests. */
void oracle_apply_assign(int L, const int32_t* label, const uint8_t* minus_of_root, int8_t* s) {
    int64_t N = (int64_t)L * L;
    for (int64_t i = 0; i < N; ++i) s[i] = minus_of_root[label[i]] ? (int8_t)-1 : (int8_t)1;
}

/* ------------------------------------------------------------ observables */

/* End of §2: H = -sum over nearest-neighbour pairs of s_i s_j (each of the
 * 2N edges once) and M = sum s_i (unnormalised). */
void oracle_observe(int L, const int8_t* s, int64_t* E, int64_t* M) {
    int64_t e = 0, m = 0;
    for (int y = 0; y < L; ++y) {
        for (int x = 0; x < L; ++x) {
            int64_t i = (int64_t)y * L + x;
            int64_t east = (int64_t)y * L + (x + 1) % L;
            int64_t south = (int64_t)((y + 1) % L) * L + x;
            e -= (int64_t)s[i] * s[east];
            e -= (int64_t)s[i] * s[south];
            m += s[i];
        }
    }
    *E = e;
    *M = m;
}

/* Cluster statistics of a labelling: hist[0] = number of clusters,
 * hist[1] = sum of squared sizes, hist[2+k] = clusters with
 * 2^k <= size < 2^(k+1), k = 0..31. count must hold N entries. */
void oracle_histogram(int L, const int32_t* label, int64_t* hist, int64_t* count) {
    int64_t N = (int64_t)L * L;
    memset(hist, 0, 34 * sizeof(int64_t));
    for (int64_t i = 0; i < N; ++i) count[i] = 0;
    for (int64_t i = 0; i < N; ++i) count[label[i]] += 1;
    for (int64_t r = 0; r < N; ++r) {
        if (label[r] != r) continue;
        int64_t size = count[r];
        int k = 0;
        while ((size >> (k + 1)) != 0) ++k;
        hist[0] += 1;
        hist[1] += size * size;
        hist[2 + k] += 1;
    }
}

/* -------------------------------------------------------------- the chain */

/* Run n sweeps with counters t0 .. t0+n-1 from the state s (updated in
 * place). E_out/M_out[n] receive the observables after each sweep;
 * hist_out (nullable) receives 34 words per sweep. rule 0 flips clusters
 * (oracle_flip), rule 1 assigns them fresh spins (oracle_assign). Returns
 * 0, or -1 on allocation failure. */
int oracle_run(int L, double beta, uint64_t seed, uint32_t t0, int n, int8_t* s,
               int64_t* E_out, int64_t* M_out, int64_t* hist_out, int rule) {
    int64_t N = (int64_t)L * L;
    uint32_t thr = oracle_threshold(beta);
    uint8_t* bonds = (uint8_t*)malloc((size_t)N);
    int32_t* label = (int32_t*)malloc((size_t)N * sizeof(int32_t));
    int32_t* queue = (int32_t*)malloc((size_t)N * sizeof(int32_t));
    int64_t* count = hist_out ? (int64_t*)malloc((size_t)N * sizeof(int64_t)) : NULL;
    if (!bonds || !label || !queue || (hist_out && !count)) {
        free(bonds); free(label); free(queue); free(count);
        return -1;
    }
    for (int k = 0; k < n; ++k) {
        uint32_t t = t0 + (uint32_t)k;
        oracle_bonds(L, seed, t, thr, s, bonds);
        oracle_labels(L, bonds, label, queue);
        if (rule == 1) oracle_assign(L, seed, t, label, s);
        else oracle_flip(L, seed, t, label, s);
        oracle_observe(L, s, &E_out[k], &M_out[k]);
        if (hist_out) oracle_histogram(L, label, hist_out + 34 * (int64_t)k, count);
    }
    free(bonds); free(label); free(queue); free(count);
    return 0;
}

/* ======================================================= q-state Potts */
/* The paper's §6 generalisation to the q-state Potts model, H = -sum over
 * the 2N edges of delta(s_i, s_j), states 0..q-1 stored as int8. The SW
 * rule bonds equal neighbours with probability 1 - exp(-beta); the bond
 * draws (C5), BFS labels (C9) and oracle_bonds/oracle_labels are those of
 * the Ising sweep; each cluster is assigned a new state uniform in q. For
 * q = 2 and beta_Potts = 2 beta this chain is the Ising chain with the
 * assignment rule, state 1 <-> spin -1. */

/* thr = floor(2^32 * (1 - exp(-beta))), capped at 2^32 - 1. */
uint32_t oracle_potts_threshold(double beta) {
    if (!(beta >= 0.0) || isinf(beta)) return 0u;
    double p = -expm1(-beta);
    double scaled = floor(ldexp(p, 32));
    if (scaled >= 4294967295.0) return 0xffffffffu;
    return (uint32_t)scaled;
}

/* A uniform state in 0..q-1 from a 32-bit word: floor(x * q / 2^32). */
static int8_t potts_state(uint32_t x, int q) {
    return (int8_t)(((uint64_t)x * (uint64_t)q) >> 32);
}

/* Hot start: state from word x0 of block (i, 0, 2, 0); cold start: all 0. */
void oracle_potts_init(int L, int q, uint64_t seed, int cold, int8_t* s) {
    int64_t N = (int64_t)L * L;
    for (int64_t i = 0; i < N; ++i) {
        if (cold) { s[i] = 0; continue; }
        uint32_t w[4];
        philox_seeded(seed, (uint32_t)i, 0u, 2u, 0u, w);
        s[i] = potts_state(w[0], q);
    }
}

/* New states: the cluster rooted at r takes the state from word x0 of
 * block (r, t, 3, 0). */
void oracle_potts_assign(int L, int q, uint64_t seed, uint32_t t, const int32_t* label, int8_t* s) {
    int64_t N = (int64_t)L * L;
    for (int64_t i = 0; i < N; ++i) {
        uint32_t w[4];
        philox_seeded(seed, (uint32_t)label[i], t, 3u, 0u, w);
        s[i] = potts_state(w[0], q);
    }
}

/* Explicit new state per cluster, read at the root (exact-kernel tests). */
void oracle_potts_apply(int L, const int32_t* label, const uint8_t* state_of_root, int8_t* s) {
    int64_t N = (int64_t)L * L;
    for (int64_t i = 0; i < N; ++i) s[i] = (int8_t)state_of_root[label[i]];
}

/* E = -(number of edges joining equal states), M = number of sites in state 0. */
void oracle_potts_observe(int L, const int8_t* s, int64_t* E, int64_t* M) {
    int64_t e = 0, m = 0;
    for (int y = 0; y < L; ++y) {
        for (int x = 0; x < L; ++x) {
            int64_t i = (int64_t)y * L + x;
            if (s[i] == s[(int64_t)y * L + (x + 1) % L]) e -= 1;
            if (s[i] == s[(int64_t)((y + 1) % L) * L + x]) e -= 1;
            if (s[i] == 0) m += 1;
        }
    }
    *E = e;
    *M = m;
}

int oracle_potts_run(int L, int q, double beta, uint64_t seed, uint32_t t0, int n, int8_t* s,
                     int64_t* E_out, int64_t* M_out) {
    int64_t N = (int64_t)L * L;
    uint32_t thr = oracle_potts_threshold(beta);
    uint8_t* bonds = (uint8_t*)malloc((size_t)N);
    int32_t* label = (int32_t*)malloc((size_t)N * sizeof(int32_t));
    int32_t* queue = (int32_t*)malloc((size_t)N * sizeof(int32_t));
    if (!bonds || !label || !queue) {
        free(bonds); free(label); free(queue);
        return -1;
    }
    for (int k = 0; k < n; ++k) {
        uint32_t t = t0 + (uint32_t)k;
        oracle_bonds(L, seed, t, thr, s, bonds);
        oracle_labels(L, bonds, label, queue);
        oracle_potts_assign(L, q, seed, t, label, s);
        oracle_potts_observe(L, s, &E_out[k], &M_out[k]);
    }
    free(bonds); free(label); free(queue);
    return 0;
}
