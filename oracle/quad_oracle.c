/*
 * Plain single-threaded CPU oracle of the quadripartite Metropolis sweep of
 * the Ising model on two lattices with a four-site unit cell (arXiv 2402.06415,
 * Results "optimising the partition", Fig. 5b/5d, Supplementary Fig. S4a-c):
 * every site of a unit cell belongs to a different one of four sublattices, no
 * two sites of one sublattice interact, so a sweep updates sublattice 0, 1, 2,
 * then 3, each as one parallel step.  TEST INFRASTRUCTURE: loaded only by the
 * tests, the smoke check and the benchmark's CPU baseline.
 *
 * Lattices (Lc x Lc periodic unit cells, 4 Lc^2 sites; spins stored as
 * s[q][Y][X], int8 +-1):
 *   SQUARE (0): the square lattice of side L = 2 Lc, site (x, y) = (2X + i,
 *     2Y + j), sublattice q = i + 2j.  Coupling J1 on the four nearest
 *     neighbours (x +- 1, y), (x, y +- 1); J2 on the four next-nearest
 *     (x +- 1, y +- 1).  J2 = 0 is the plain square lattice (Fig. S4a),
 *     J2 != 0 the NN + NNN model (Fig. S4b).
 *   SQOCT (1): the square-octagon (4.8.8) lattice (Fig. S4c): each cell is a
 *     square of sites A (q 0), B (1), C (2), D (3) joined A-B-C-D-A by J1 bonds;
 *     octagon bonds J2 join B(X, Y)-D(X+1, Y) and A(X, Y)-C(X, Y+1).  Every site
 *     has two J1 and one J2 neighbour.
 *
 * H = -(1/2) sum_i sum_{n in nbr(i)} J_{in} s_i s_n (each bond once; neighbour
 * lists keep multiplicity on the smallest tori).  A site with a1 antiparallel
 * J1 neighbours out of z1 and a2 antiparallel J2 neighbours out of z2 has
 * dE = 2 J1 (z1 - 2 a1) + 2 J2 (z2 - 2 a2) for its flip; Metropolis: flip iff
 * dE <= 0 or u < T(a1, a2) = floor(exp(-beta dE) 2^32) (the paper's step 2-3
 * with the integer thresholds of the square-lattice path).
 *
 * Random numbers: Philox4x32-10 keyed by the seed.  Word group g = Y Wq +
 * (X >> 5), Wq = ceil(Lc / 32), lane X & 31.  Start: s = +1 iff bit lane of
 * word 0 of Philox(g, 0, r, QUAD_INIT << 16 | q << 8).  Sweep t, sublattice q:
 * plane P_{4b+k} = word k of Philox(g, t, r, QUAD_MET << 16 | q << 8 | b),
 * b = 0..7, and u = sum_k bit_lane(P_k) 2^(31-k).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

enum { QUAD_TAG_INIT = 12, QUAD_TAG_MET = 13 };
enum { QUAD_SQUARE = 0, QUAD_SQOCT = 1 };

static void quad_block(uint64_t seed, uint32_t g, uint32_t t, uint32_t r, uint32_t w3, uint32_t o[4])
{
    uint32_t ctr[4] = {g, t, r, w3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, o);
}

static int wrap(int v, int n) { return ((v % n) + n) % n; }

typedef struct { int q, X, Y, type; } nbr_t;

/* Neighbour list of site (q, X, Y); returns its length. */
int orc_quad_neighbours(int lattice, int Lc, int q, int X, int Y, int out[32])
{
    nbr_t nb[8];
    int n = 0;
    if (lattice == QUAD_SQUARE) {
        int L = 2 * Lc;
        int x = 2 * X + (q & 1), y = 2 * Y + (q >> 1);
        static const int d[8][3] = {{1, 0, 1}, {-1, 0, 1}, {0, 1, 1}, {0, -1, 1},
                                    {1, 1, 2}, {1, -1, 2}, {-1, 1, 2}, {-1, -1, 2}};
        for (int k = 0; k < 8; ++k) {
            int xn = wrap(x + d[k][0], L), yn = wrap(y + d[k][1], L);
            nb[n].q = (xn & 1) + 2 * (yn & 1);
            nb[n].X = xn >> 1;
            nb[n].Y = yn >> 1;
            nb[n].type = d[k][2];
            ++n;
        }
    } else {
        /* A = 0, B = 1, C = 2, D = 3 around the square; octagon bonds B-D(+x), A-C(+y) */
        static const int ring_next[4] = {1, 2, 3, 0}, ring_prev[4] = {3, 0, 1, 2};
        nb[n].q = ring_next[q]; nb[n].X = X; nb[n].Y = Y; nb[n].type = 1; ++n;
        nb[n].q = ring_prev[q]; nb[n].X = X; nb[n].Y = Y; nb[n].type = 1; ++n;
        switch (q) {
        case 0: nb[n].q = 2; nb[n].X = X; nb[n].Y = wrap(Y + 1, Lc); break;
        case 1: nb[n].q = 3; nb[n].X = wrap(X + 1, Lc); nb[n].Y = Y; break;
        case 2: nb[n].q = 0; nb[n].X = X; nb[n].Y = wrap(Y - 1, Lc); break;
        default: nb[n].q = 1; nb[n].X = wrap(X - 1, Lc); nb[n].Y = Y; break;
        }
        nb[n].type = 2;
        ++n;
    }
    for (int k = 0; k < n; ++k) {
        out[4 * k] = nb[k].q;
        out[4 * k + 1] = nb[k].X;
        out[4 * k + 2] = nb[k].Y;
        out[4 * k + 3] = nb[k].type;
    }
    return n;
}

static int8_t at(const int8_t *s, int Lc, int q, int X, int Y)
{
    return s[((size_t)q * Lc + (size_t)Y) * Lc + (size_t)X];
}

/* (z1, z2): how many J1 and J2 neighbours a site has. */
void orc_quad_coordination(int lattice, int *z1, int *z2)
{
    *z1 = lattice == QUAD_SQUARE ? 4 : 2;
    *z2 = lattice == QUAD_SQUARE ? 4 : 1;
}

/* Threshold of class (a1, a2); *always = 1 when dE <= 0 (the flip is certain). */
uint32_t orc_quad_threshold(int lattice, double beta, double J1, double J2, int a1, int a2,
                            int *always)
{
    int z1, z2;
    orc_quad_coordination(lattice, &z1, &z2);
    double dE = 2.0 * J1 * (double)(z1 - 2 * a1) + 2.0 * J2 * (double)(z2 - 2 * a2);
    if (dE <= 0.0) {
        *always = 1;
        return 0xffffffffu;
    }
    *always = 0;
    double t = floor(exp(-beta * dE) * 4294967296.0);
    if (t >= 4294967295.0) return 0xffffffffu;
    return (uint32_t)t;
}

static int words_per_row(int Lc) { return (Lc + 31) / 32; }

void orc_quad_init(int Lc, uint64_t seed, uint32_t r, int8_t *s)
{
    int Wq = words_per_row(Lc);
    for (int q = 0; q < 4; ++q)
        for (int Y = 0; Y < Lc; ++Y)
            for (int X = 0; X < Lc; ++X) {
                uint32_t o[4];
                quad_block(seed, (uint32_t)(Y * Wq + (X >> 5)), 0, r,
                           (uint32_t)(QUAD_TAG_INIT << 16) | (uint32_t)(q << 8), o);
                s[((size_t)q * Lc + Y) * Lc + X] = ((o[0] >> (X & 31)) & 1u) ? 1 : -1;
            }
}

/* The uniform of site (q, X, Y) at sweep t. */
uint32_t orc_quad_uniform(int Lc, uint64_t seed, uint32_t r, uint32_t t, int q, int X, int Y)
{
    uint32_t g = (uint32_t)(Y * words_per_row(Lc) + (X >> 5));
    uint32_t u = 0;
    for (int b = 0; b < 8; ++b) {
        uint32_t o[4];
        quad_block(seed, g, t, r, (uint32_t)(QUAD_TAG_MET << 16) | (uint32_t)(q << 8) | (uint32_t)b, o);
        for (int k = 0; k < 4; ++k) u |= ((o[k] >> (X & 31)) & 1u) << (31 - (4 * b + k));
    }
    return u;
}

/* Antiparallel J1 and J2 neighbours of a site. */
void orc_quad_anti(int lattice, int Lc, const int8_t *s, int q, int X, int Y, int *a1, int *a2)
{
    int nb[32];
    int n = orc_quad_neighbours(lattice, Lc, q, X, Y, nb);
    int8_t me = at(s, Lc, q, X, Y);
    *a1 = *a2 = 0;
    for (int k = 0; k < n; ++k) {
        if (at(s, Lc, nb[4 * k], nb[4 * k + 1], nb[4 * k + 2]) == me) continue;
        if (nb[4 * k + 3] == 1) ++*a1; else ++*a2;
    }
}

/* B1 = sum over J1 bonds of s s', B2 likewise for J2, M = sum s (each bond once:
 * half the sum over every site's neighbour list). */
void orc_quad_observables(int lattice, int Lc, const int8_t *s, int64_t *B1, int64_t *B2, int64_t *M)
{
    int64_t b1 = 0, b2 = 0, m = 0;
    for (int q = 0; q < 4; ++q)
        for (int Y = 0; Y < Lc; ++Y)
            for (int X = 0; X < Lc; ++X) {
                int nb[32];
                int n = orc_quad_neighbours(lattice, Lc, q, X, Y, nb);
                int8_t me = at(s, Lc, q, X, Y);
                m += me;
                for (int k = 0; k < n; ++k) {
                    int v = me * at(s, Lc, nb[4 * k], nb[4 * k + 1], nb[4 * k + 2]);
                    if (nb[4 * k + 3] == 1) b1 += v; else b2 += v;
                }
            }
    *B1 = b1 / 2;
    *B2 = b2 / 2;
    *M = m;
}

/* One quarter sweep: every site of sublattice q gets one Metropolis trial. */
void orc_quad_quarter(int lattice, int Lc, double beta, double J1, double J2, uint64_t seed,
                      uint32_t r, uint32_t t, int q, int8_t *s)
{
    int z1, z2;
    orc_quad_coordination(lattice, &z1, &z2);
    uint32_t T[5][5];
    int always[5][5];
    for (int a1 = 0; a1 <= z1; ++a1)
        for (int a2 = 0; a2 <= z2; ++a2)
            T[a1][a2] = orc_quad_threshold(lattice, beta, J1, J2, a1, a2, &always[a1][a2]);
    for (int Y = 0; Y < Lc; ++Y)
        for (int X = 0; X < Lc; ++X) {
            int a1, a2;
            orc_quad_anti(lattice, Lc, s, q, X, Y, &a1, &a2);
            int flip = always[a1][a2];
            if (!flip) flip = orc_quad_uniform(Lc, seed, r, t, q, X, Y) < T[a1][a2];
            if (flip) s[((size_t)q * Lc + Y) * Lc + X] = (int8_t)-s[((size_t)q * Lc + Y) * Lc + X];
        }
}

/* n sweeps with counters t0 .. t0+n-1 (sublattices 0, 1, 2, 3); after sweep t,
 * (B1, B2, M) is appended iff (t + 1) % measure_every == 0.  Returns the
 * number of records, or -1 on bad arguments. */
int orc_quad_sweep(int lattice, int Lc, double beta, double J1, double J2, uint64_t seed,
                   uint32_t r, uint32_t t0, int n, int measure_every, int8_t *s, int64_t *B1,
                   int64_t *B2, int64_t *M)
{
    if (Lc < 2 || n < 0 || measure_every < 1 || (lattice != QUAD_SQUARE && lattice != QUAD_SQOCT))
        return -1;
    int rec = 0;
    for (int k = 0; k < n; ++k) {
        uint32_t t = t0 + (uint32_t)k;
        for (int q = 0; q < 4; ++q) orc_quad_quarter(lattice, Lc, beta, J1, J2, seed, r, t, q, s);
        if ((t + 1) % (uint32_t)measure_every == 0) {
            orc_quad_observables(lattice, Lc, s, &B1[rec], &B2[rec], &M[rec]);
            ++rec;
        }
    }
    return rec;
}
