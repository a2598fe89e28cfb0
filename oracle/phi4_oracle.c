/*
 * phi4_oracle.c -- serial CPU oracle for the multicluster update of the O(4)
 * phi^4 theory in four dimensions (the paper's §3, Eqs. 2 and 3).
 *
 * TEST INFRASTRUCTURE ONLY, like sw_oracle.c: the tests, the smoke check and
 * the benchmark's CPU leg load it; the library never does.
 *
 * One update at counter t, in the paper's order:
 *   1. a random direction r, uniform on the unit 3-sphere (O3);
 *   2. every edge (x, x+mu) bonds with probability
 *        p = 1 - exp(min(0, -4 kappa (phi_x . r)(phi_{x+mu} . r)))    (Eq. 2)
 *      -- only edges whose two projections have the same sign can bond;
 *   3. clusters of the bond graph, each labelled by its smallest site;
 *   4. every cluster is flipped with probability 1/2, a flip reflecting the
 *      field of its sites in the hyperplane orthogonal to r:
 *        phi_x <- phi_x - 2 (phi_x . r) r                              (Eq. 3)
 *   5. observables: E = sum over the 4N edges of phi_x . phi_{x+mu} and the
 *      four components of M = sum_x phi_x.
 * Floating point decides the bonds, so every step that feeds a decision is
 * specified operation by operation (explicit fused multiply-adds; the file
 * is compiled in ISO C mode, which contracts nothing else), and the
 * exponential is this file's own (exp_neg below), so the library can take
 * the same decisions bit for bit.
 *
 * Conventions (the paper fixes none of them):
 *  O1 lattice L^4, periodic, site x = x0 + L (x1 + L (x2 + L x3)); each site
 *     owns its 4 edges to x + e_mu; field phi_x in R^4, binary64 [N][4].
 *  O2 hot start: component a of phi_x = (w_a + 0.5) 2^-31 - 1 from the
 *     words w_a of Philox block (x, 0, 7, 0); cold start phi_x = (1, 0, 0, 0).
 *  O3 direction of update t: attempts k = 0, 1, ...: v_a = (w_a + 0.5)
 *     2^-31 - 1 from block (k, t, 5, 0); s = fma(v3, v3, fma(v2, v2,
 *     fma(v1, v1, v0 v0))); the first attempt with 2^-20 < s <= 1 gives
 *     r_a = v_a / sqrt(s).
 *  O4 projection a_x = fma(phi3, r3, fma(phi2, r2, fma(phi1, r1, phi0 r0))).
 *     Edge (x, mu) with y = x + e_mu: q = a_x a_y; no bond if q <= 0; else
 *     z = (4 kappa) q, e = exp_neg(z), bond iff (double) w_mu < (1 - e) 2^32,
 *     w_mu = word mu of Philox block (x, t, 4, 0).
 *  O5 flip of the cluster rooted at r: bit 31 of word 0 of block (r, t, 6, 0);
 *     component a of a flipped site becomes fma(-2 a_x, r_a, phi_a).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

static void block(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    oracle_philox(ctr, key, out);
}

static double unit_interval(uint32_t w) { return ((double)w + 0.5) * 0x1p-31 - 1.0; }

/* e^{-z} for z >= 0, from the mathematics: z = n ln2 + r with n the nearest
 * integer to z / ln2 and ln2 split into a 32-bit head (n * head is exact) and
 * a tail (Cody and Waite's reduction); e^{-r}, |r| <= 0.35, from its Taylor
 * series to degree 14 (the remainder is below 2^-60) by Horner's rule with
 * fused multiply-adds; then the exact scaling by 2^-n. Above z = 40 it
 * returns 0: there e^{-z} < 2^-57 and 1 - e^{-z} rounds to 1 either way, so
 * no bond decision depends on the value, and subnormal scalings never occur. */
double phi4_exp_neg(double z) {
    static const double ln2_head = 0x1.62e42feep-1;
    static const double ln2_tail = 0x1.a39ef35793c76p-33;
    static const double inv_ln2 = 0x1.71547652b82fep+0;
    static const double c[15] = {
        0x1p+0, 0x1p+0, 0x1p-1, 0x1.5555555555555p-3, 0x1.5555555555555p-5, 0x1.1111111111111p-7,
        0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19,
        0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26, 0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33,
        0x1.93974a8c07c9dp-37};
    if (!(z >= 0.0)) return NAN;
    if (z > 40.0) return 0.0;
    const double n = floor(z * inv_ln2 + 0.5);
    const double r = fma(-n, ln2_tail, fma(-n, ln2_head, z));
    double p = c[14];
    for (int k = 13; k >= 0; --k) p = fma(p, -r, c[k]);
    return ldexp(p, -(int)n);
}

int phi4_direction(uint64_t seed, uint32_t t, double r[4]) {
    for (uint32_t k = 0; k < 1000; ++k) {
        uint32_t w[4];
        block(seed, k, t, 5u, 0u, w);
        double v[4];
        for (int a = 0; a < 4; ++a) v[a] = unit_interval(w[a]);
        const double s = fma(v[3], v[3], fma(v[2], v[2], fma(v[1], v[1], v[0] * v[0])));
        if (s <= 1.0 && s > 0x1p-20) {
            const double n = sqrt(s);
            for (int a = 0; a < 4; ++a) r[a] = v[a] / n;
            return 0;
        }
    }
    return -1;
}

void phi4_init(int L, uint64_t seed, int cold, double* phi) {
    const int64_t N = (int64_t)L * L * L * L;
    for (int64_t x = 0; x < N; ++x) {
        if (cold) {
            phi[4 * x] = 1.0;
            phi[4 * x + 1] = phi[4 * x + 2] = phi[4 * x + 3] = 0.0;
            continue;
        }
        uint32_t w[4];
        block(seed, (uint32_t)x, 0u, 7u, 0u, w);
        for (int a = 0; a < 4; ++a) phi[4 * x + a] = unit_interval(w[a]);
    }
}

static double proj(const double* f, const double r[4]) {
    return fma(f[3], r[3], fma(f[2], r[2], fma(f[1], r[1], f[0] * r[0])));
}

/* Neighbour of x in direction mu (+1 step, periodic). */
static int64_t nb(int L, int64_t x, int mu) {
    int64_t stride = 1;
    for (int m = 0; m < mu; ++m) stride *= L;
    const int64_t c = (x / stride) % L;
    return c == L - 1 ? x - (int64_t)(L - 1) * stride : x + stride;
}

/* Bonds of update t (O4): bit mu of bonds[x] = edge (x, x + e_mu). */
void phi4_bonds(int L, double kappa, uint64_t seed, uint32_t t, const double* phi, const double r[4],
                uint8_t* bonds) {
    const int64_t N = (int64_t)L * L * L * L;
    const double k4 = 4.0 * kappa;
    for (int64_t x = 0; x < N; ++x) {
        uint32_t w[4];
        block(seed, (uint32_t)x, t, 4u, 0u, w);
        const double ax = proj(phi + 4 * x, r);
        uint8_t b = 0;
        for (int mu = 0; mu < 4; ++mu) {
            const double ay = proj(phi + 4 * nb(L, x, mu), r);
            const double q = ax * ay;
            if (!(q > 0.0)) continue;
            const double e = phi4_exp_neg(k4 * q);
            if ((double)w[mu] < (1.0 - e) * 0x1p32) b |= (uint8_t)(1u << mu);
        }
        bonds[x] = b;
    }
}

/* Clusters by breadth-first search, sources in increasing index order, so
 * every site gets its cluster's smallest index. queue holds N entries. */
int64_t phi4_labels(int L, const uint8_t* bonds, int32_t* label, int32_t* queue) {
    const int64_t N = (int64_t)L * L * L * L;
    for (int64_t x = 0; x < N; ++x) label[x] = -1;
    int64_t nc = 0;
    for (int64_t src = 0; src < N; ++src) {
        if (label[src] >= 0) continue;
        ++nc;
        int64_t head = 0, tail = 0;
        label[src] = (int32_t)src;
        queue[tail++] = (int32_t)src;
        while (head < tail) {
            const int64_t x = queue[head++];
            for (int mu = 0; mu < 4; ++mu) {
                /* forward edge owned by x */
                const int64_t y = nb(L, x, mu);
                if ((bonds[x] >> mu) & 1u && label[y] < 0) {
                    label[y] = (int32_t)src;
                    queue[tail++] = (int32_t)y;
                }
                /* backward edge owned by the neighbour x - e_mu */
                int64_t stride = 1;
                for (int m = 0; m < mu; ++m) stride *= L;
                const int64_t c = (x / stride) % L;
                const int64_t z = c == 0 ? x + (int64_t)(L - 1) * stride : x - stride;
                if ((bonds[z] >> mu) & 1u && label[z] < 0) {
                    label[z] = (int32_t)src;
                    queue[tail++] = (int32_t)z;
                }
            }
        }
    }
    return nc;
}

/* Flips (O5): every cluster rooted at r is reflected iff bit 31 of word 0 of
 * block (r, t, 6, 0) is set. */
void phi4_reflect(int L, uint64_t seed, uint32_t t, const int32_t* label, const double r[4], double* phi) {
    const int64_t N = (int64_t)L * L * L * L;
    for (int64_t x = 0; x < N; ++x) {
        uint32_t w[4];
        block(seed, (uint32_t)label[x], t, 6u, 0u, w);
        if (!(w[0] >> 31)) continue;
        const double m2a = -2.0 * proj(phi + 4 * x, r);
        for (int a = 0; a < 4; ++a) phi[4 * x + a] = fma(m2a, r[a], phi[4 * x + a]);
    }
}

/* E = sum over the 4N edges of phi_x . phi_{x+mu}; M[a] = sum_x phi_x[a]. */
void phi4_observe(int L, const double* phi, double* E, double* M) {
    const int64_t N = (int64_t)L * L * L * L;
    double e = 0.0, m[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t x = 0; x < N; ++x) {
        for (int mu = 0; mu < 4; ++mu) {
            const double* f = phi + 4 * x;
            const double* g = phi + 4 * nb(L, x, mu);
            e += f[0] * g[0] + f[1] * g[1] + f[2] * g[2] + f[3] * g[3];
        }
        for (int a = 0; a < 4; ++a) m[a] += phi[4 * x + a];
    }
    *E = e;
    for (int a = 0; a < 4; ++a) M[a] = m[a];
}

/* n updates with counters t0 .. t0+n-1; E_out[n], M_out[n][4]. 0, or -1 on
 * allocation failure, -2 if no direction was found. */
int phi4_run(int L, double kappa, uint64_t seed, uint32_t t0, int n, double* phi, double* E_out, double* M_out) {
    const int64_t N = (int64_t)L * L * L * L;
    uint8_t* bonds = (uint8_t*)malloc((size_t)N);
    int32_t* label = (int32_t*)malloc((size_t)N * sizeof(int32_t));
    int32_t* queue = (int32_t*)malloc((size_t)N * sizeof(int32_t));
    if (!bonds || !label || !queue) {
        free(bonds); free(label); free(queue);
        return -1;
    }
    int rc = 0;
    for (int k = 0; k < n; ++k) {
        const uint32_t t = t0 + (uint32_t)k;
        double r[4];
        if (phi4_direction(seed, t, r) != 0) { rc = -2; break; }
        phi4_bonds(L, kappa, seed, t, phi, r, bonds);
        phi4_labels(L, bonds, label, queue);
        phi4_reflect(L, seed, t, label, r, phi);
        phi4_observe(L, phi, &E_out[k], &M_out[4 * k]);
    }
    free(bonds); free(label); free(queue);
    return rc;
}
