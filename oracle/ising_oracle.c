/*
 * Plain, slow, single-threaded CPU oracle for the checkerboard Metropolis
 * sweep of the 2D square-lattice Ising model (J = 1, h = 0, periodic).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package entry's smoke check and
 * the benchmark's CPU-baseline / reference arm may load this library.  The
 * product path (the CUDA library) never links, loads or calls it, and it
 * shares no source with it: the Philox generator, the counter map, the
 * thresholds and the sweep below are written out again here, from their
 * definitions, so that a mistake on either side shows up as a mismatch.
 *
 * What it follows (arXiv 2402.06415):
 *   - Results A and Fig. 2: the square lattice is bipartite, so all sites of
 *     one sublattice are updated independently, then the other sublattice.
 *   - Supplementary "Detail of the MC calculation": per site (1) draw a
 *     uniform decision number p, (2) compute the local energy change and the
 *     acceptance P(dE) = exp(-beta dE), (3) update iff p < P (strict).
 *     The same supplementary section keeps the random numbers at full width
 *     and the Metropolis probability at full precision; here p is a full
 *     32-bit integer and P is the integer threshold floor(exp(-beta dE) 2^32),
 *     so "p < P" is an exact integer comparison.
 *   - The paper uses the XY model; the integer Ising restatement has local
 *     change dE = 2 s_x sum_n s_n in {-8,-4,0,4,8} (the Ising analogue of
 *     Eq. S1), so only dE = 4 and dE = 8 need a random test.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11) replaces the paper's per-site LCG, keyed
 * by the seed and addressed by (group, sweep, replica, tag|colour|block).
 *
 * Counter map (the reading this project fixes; both sides implement it):
 *   key      = (lo32(seed), hi32(seed))
 *   counter  = (g, t, r, tag << 16 | c << 8 | b)
 *   g        = y * Wc + (j >> 5), the 32-site group of colour-c sites
 *              j in [32w, 32w+32) of row y; Wc = ceil((L/2)/32)
 *   j        = x >> 1, the index of site (x, y) among the L/2 colour-c
 *              sites of row y, colour c = (x + y) & 1
 *   i        = j & 31, the site's lane inside its group
 *   INIT:  s(x,y) = +1 iff bit i of word 0 of Philox(g, 0, r, INIT<<16|c<<8)
 *   MET:   32 plane words P_0..P_31 per (group, sweep); P_{4b+q} is word q of
 *          Philox(g, t, r, MET<<16|c<<8|b), b = 0..7.  The site's uniform is
 *          u_i = sum_k bit_i(P_k) << (31 - k), i.e. plane 0 is the most
 *          significant bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_TAG_INIT = 1, ORC_TAG_MET = 2, ORC_TAG_PT = 3 };

/* ---------------------------------------------------------------------- */
/* Philox4x32-10 (SC'11, Sec. 4): 10 rounds of the 4-word S-box with two   */
/* 32x32->64 multiplies, key bumped by the Weyl constants between rounds.  */
/* ---------------------------------------------------------------------- */
static const uint32_t ORC_M0 = 0xD2511F53u;
static const uint32_t ORC_M1 = 0xCD9E8D57u;
static const uint32_t ORC_W0 = 0x9E3779B9u;
static const uint32_t ORC_W1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_W0;
            k1 += ORC_W1;
        }
        uint64_t p0 = (uint64_t)ORC_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)ORC_M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void orc_block(uint64_t seed, uint32_t g, uint32_t t, uint32_t r,
                      uint32_t tag, uint32_t c, uint32_t b, uint32_t out[4])
{
    uint32_t ctr[4] = {g, t, r, (tag << 16) | (c << 8) | b};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Words (32-site groups) per colour row. */
int orc_words_per_row(int L) { return (L / 2 + 31) / 32; }

/* ---------------------------------------------------------------------- */
/* Step 2 of the supplementary recipe: P(dE) = exp(-beta dE), here as an   */
/* integer threshold on a 32-bit uniform.  dE in {4, 8}.                   */
/* ---------------------------------------------------------------------- */
uint32_t orc_threshold(double beta, int dE)
{
    double p = exp(-beta * (double)dE);
    double t = floor(p * 4294967296.0);
    if (t >= 4294967295.0) return 0xffffffffu; /* beta -> 0 limit */
    if (t <= 0.0) return 0u;
    return (uint32_t)t;
}

/* Step 3: flip iff p < P(dE); dE <= 0 always flips.  n_anti = number of
 * antiparallel neighbours, dE = 8 - 4 n_anti. */
int orc_decide(int n_anti, uint32_t u, uint32_t thr4, uint32_t thr8)
{
    if (n_anti >= 2) return 1;
    if (n_anti == 1) return u < thr4;
    return u < thr8;
}

/* The 32 plane words of one group for one sweep (Metropolis tag). */
void orc_met_planes(uint64_t seed, uint32_t r, uint32_t t, int c, uint32_t g, uint32_t P[32])
{
    for (uint32_t b = 0; b < 8; ++b) {
        uint32_t o[4];
        orc_block(seed, g, t, r, ORC_TAG_MET, (uint32_t)c, b, o);
        for (int q = 0; q < 4; ++q) P[4 * b + q] = o[q];
    }
}

/* Site uniform from its group's planes: plane k gives bit (31 - k). */
uint32_t orc_assemble_u(const uint32_t P[32], int lane)
{
    uint32_t u = 0;
    for (int k = 0; k < 32; ++k) u |= ((P[k] >> lane) & 1u) << (31 - k);
    return u;
}

/* The uniform of site (x, y) at sweep t (slow: recomputes its group). */
uint32_t orc_site_uniform(int L, uint64_t seed, uint32_t r, uint32_t t, int x, int y)
{
    int c = (x + y) & 1;
    int j = x >> 1;
    uint32_t g = (uint32_t)y * (uint32_t)orc_words_per_row(L) + (uint32_t)(j >> 5);
    uint32_t P[32];
    orc_met_planes(seed, r, t, c, g, P);
    return orc_assemble_u(P, j & 31);
}

static int8_t site(const int8_t *s, int L, int x, int y)
{
    x = (x % L + L) % L;
    y = (y % L + L) % L;
    return s[(size_t)y * L + x];
}

/* Number of the 4 periodic nearest neighbours antiparallel to s(x, y). */
int orc_n_anti(int L, const int8_t *s, int x, int y)
{
    int8_t v = site(s, L, x, y);
    int n = 0;
    n += site(s, L, x + 1, y) != v;
    n += site(s, L, x - 1, y) != v;
    n += site(s, L, x, y + 1) != v;
    n += site(s, L, x, y - 1) != v;
    return n;
}

/* E = -sum_{x,y} s(x,y) [s(x+1,y) + s(x,y+1)]  (2 L^2 bonds), M = sum s. */
void orc_energy_mag(int L, const int8_t *s, int64_t *E, int64_t *M)
{
    int64_t e = 0, m = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int v = site(s, L, x, y);
            e -= v * (site(s, L, x + 1, y) + site(s, L, x, y + 1));
            m += v;
        }
    *E = e;
    *M = m;
}

/* Seeded random start: independent +-1, one Philox bit per site. */
void orc_init(int L, uint64_t seed, uint32_t r, int8_t *s)
{
    int Wc = orc_words_per_row(L);
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int c = (x + y) & 1;
            int j = x >> 1;
            uint32_t g = (uint32_t)y * (uint32_t)Wc + (uint32_t)(j >> 5);
            uint32_t o[4];
            orc_block(seed, g, 0, r, ORC_TAG_INIT, (uint32_t)c, 0, o);
            s[(size_t)y * L + x] = ((o[0] >> (j & 31)) & 1u) ? 1 : -1;
        }
}

/* One half sweep: every colour-c site gets one Metropolis trial with the
 * uniforms of sweep t.  Sites of one colour have no neighbour of the same
 * colour, so updating them in place in any order gives the same result. */
void orc_half_sweep(int L, uint32_t thr4, uint32_t thr8, uint64_t seed, uint32_t r,
                    uint32_t t, int c, int8_t *s)
{
    int Wc = orc_words_per_row(L);
    int half = L / 2;
    for (int y = 0; y < L; ++y)
        for (int w = 0; w < Wc; ++w) {
            uint32_t P[32];
            orc_met_planes(seed, r, t, c, (uint32_t)(y * Wc + w), P);
            for (int lane = 0; lane < 32; ++lane) {
                int j = 32 * w + lane;
                if (j >= half) break;
                int x = 2 * j + ((y + c) & 1);
                int n = orc_n_anti(L, s, x, y);
                uint32_t u = orc_assemble_u(P, lane);
                if (orc_decide(n, u, thr4, thr8)) s[(size_t)y * L + x] = (int8_t)-s[(size_t)y * L + x];
            }
        }
}

/* n_sweeps full sweeps (colour 0 then colour 1) with sweep counters
 * t0 .. t0+n_sweeps-1.  After sweep t, (E, M) is appended to the outputs iff
 * (t + 1) % measure_every == 0.  Returns the number of records written, or
 * -1 on bad arguments. */
int orc_sweep(int L, double beta, uint64_t seed, uint32_t r, uint32_t t0, int n_sweeps,
              int measure_every, int8_t *s, int64_t *E_out, int64_t *M_out)
{
    if (L < 2 || (L & 1) || n_sweeps < 0 || measure_every < 1) return -1;
    uint32_t thr4 = orc_threshold(beta, 4);
    uint32_t thr8 = orc_threshold(beta, 8);
    int rec = 0;
    for (int k = 0; k < n_sweeps; ++k) {
        uint32_t t = t0 + (uint32_t)k;
        orc_half_sweep(L, thr4, thr8, seed, r, t, 0, s);
        orc_half_sweep(L, thr4, thr8, seed, r, t, 1, s);
        if (((uint64_t)t + 1) % (uint64_t)measure_every == 0) {
            if (E_out && M_out) orc_energy_mag(L, s, &E_out[rec], &M_out[rec]);
            ++rec;
        }
    }
    return rec;
}

/* Exact number of 32-bit uniforms u with orc_decide(n_anti, u, ...) == 1,
 * found by bisection on the decision itself (it is monotone in u).  Used by
 * the detailed-balance tests to get the kernel's exact flip probability
 * count / 2^32 from the code the sweep runs. */
uint64_t orc_accept_count(int n_anti, uint32_t thr4, uint32_t thr8)
{
    if (!orc_decide(n_anti, 0u, thr4, thr8)) return 0;
    if (orc_decide(n_anti, 0xffffffffu, thr4, thr8)) return 4294967296ull;
    uint64_t lo = 0, hi = 0xffffffffull; /* decide(lo) = 1, decide(hi) = 0 */
    while (hi - lo > 1) {
        uint64_t mid = (lo + hi) / 2;
        if (orc_decide(n_anti, (uint32_t)mid, thr4, thr8)) lo = mid; else hi = mid;
    }
    return hi;
}

/* n_anti for every site of a stack of n configurations (L x L each), the same
 * count the sweep uses; out is n * L * L ints. */
void orc_n_anti_all(int L, int n, const int8_t *s, int32_t *out)
{
    for (int k = 0; k < n; ++k) {
        const int8_t *sk = s + (size_t)k * L * L;
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x)
                out[(size_t)k * L * L + (size_t)y * L + x] = orc_n_anti(L, sk, x, y);
    }
}

/* ---------------------------------------------------------------------- */
/* Parallel tempering (replica exchange) between adjacent temperatures of  */
/* one ladder.  Not in the paper (its MC runs one chain per lattice); the  */
/* textbook exchange rule: the configurations at slots a and a+1 swap with */
/* probability min(1, exp[(beta_a - beta_{a+1}) (E_a - E_{a+1})]).  Here   */
/* the swap is accepted iff u < floor(min(1, exp(d)) 2^32), u = word 0 of  */
/* Philox(a, n_step, ladder, PT<<16).  Step n_step pairs slots             */
/* (a, a+1) with a = n_step & 1, (n_step & 1) + 2, ...                     */
/* perm[a] = replica index at slot a; E[i] = energy of replica i.          */
/* ---------------------------------------------------------------------- */
void orc_pt_step(int n_beta, const double *betas, uint64_t seed, uint32_t ladder,
                 uint32_t n_step, const int64_t *E, int32_t *perm, int64_t *accepts,
                 int64_t *attempts)
{
    for (int a = (int)(n_step & 1u); a + 1 < n_beta; a += 2) {
        int32_t ra = perm[a], rb = perm[a + 1];
        double d = (betas[a] - betas[a + 1]) * (double)(E[ra] - E[rb]);
        uint64_t thr;
        if (d >= 0.0) {
            thr = 4294967296ull;
        } else {
            double t = floor(exp(d) * 4294967296.0);
            thr = t <= 0.0 ? 0ull : (uint64_t)t;
        }
        uint32_t o[4];
        orc_block(seed, (uint32_t)a, n_step, ladder, ORC_TAG_PT, 0, 0, o);
        if (attempts) attempts[a] += 1;
        if ((uint64_t)o[0] < thr) {
            perm[a] = rb;
            perm[a + 1] = ra;
            if (accepts) accepts[a] += 1;
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Swendsen-Wang cluster update (Swendsen & Wang, PRL 58, 86 (1987)); the  */
/* paper names cluster updates as the next step beyond its single-site MC. */
/* One step: every bond between equal spins is activated with probability  */
/* p = 1 - exp(-2 beta), i.e. iff u < floor(p 2^32), u = word (b & 3) of    */
/* Philox(b >> 2, step, r, SW_BOND << 16) for bond b = 2 (y L + x) + dir    */
/* (dir 0: to x+1, 1: to y+1); clusters = connected components of active   */
/* bonds; each cluster flips iff bit 31 of word (m & 3) of                  */
/* Philox(m >> 2, step, r, SW_FLIP << 16), m = its smallest site index.     */
/* ---------------------------------------------------------------------- */
enum { ORC_TAG_SW_BOND = 10, ORC_TAG_SW_FLIP = 11 };

uint32_t orc_sw_threshold(double beta)
{
    double p = 1.0 - exp(-2.0 * beta);
    double t = floor(p * 4294967296.0);
    if (t >= 4294967295.0) return 0xffffffffu;
    if (t <= 0.0) return 0u;
    return (uint32_t)t;
}

static uint32_t sw_find(uint32_t *parent, uint32_t a)
{
    while (parent[a] != a) a = parent[a];
    return a;
}

/* One SW step in place; parent is scratch of L*L entries.  Returns the
 * number of clusters. */
long long orc_sw_step(int L, double beta, uint64_t seed, uint32_t r, uint32_t step, int8_t *s,
                      uint32_t *parent)
{
    const uint32_t N = (uint32_t)L * (uint32_t)L;
    const uint32_t thr = orc_sw_threshold(beta);
    for (uint32_t i = 0; i < N; ++i) parent[i] = i;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x)
            for (int dir = 0; dir < 2; ++dir) {
                int xn = dir == 0 ? (x + 1) % L : x, yn = dir == 0 ? y : (y + 1) % L;
                uint32_t a = (uint32_t)(y * L + x), b = (uint32_t)(yn * L + xn);
                if (s[a] != s[b]) continue;
                uint32_t bond = 2 * a + (uint32_t)dir, o[4];
                orc_block(seed, bond >> 2, step, r, ORC_TAG_SW_BOND, 0, 0, o);
                if (o[bond & 3] >= thr) continue;
                uint32_t ra = sw_find(parent, a), rb = sw_find(parent, b);
                if (ra == rb) continue;
                if (ra < rb) parent[rb] = ra; else parent[ra] = rb;  /* root = smallest index */
            }
    long long clusters = 0;
    for (uint32_t i = 0; i < N; ++i) {
        uint32_t m = sw_find(parent, i);
        if (m == i) ++clusters;
        uint32_t o[4];
        orc_block(seed, m >> 2, step, r, ORC_TAG_SW_FLIP, 0, 0, o);
        if (o[m & 3] >> 31) s[i] = (int8_t)-s[i];
    }
    return clusters;
}

/* ---------------------------------------------------------------------- */
/* Wolff single-cluster update (Wolff, PRL 62, 361 (1989)), the other      */
/* cluster method next to Swendsen-Wang.  Step n: the seed site is          */
/* m = floor(u N / 2^32), u = word 0 of Philox(0, n, r, WOLFF_SEED << 16);   */
/* a bond b = 2 (y L + x) + dir between equal spins is active iff           */
/* u < floor((1 - exp(-2 beta)) 2^32), u = word (b & 3) of                  */
/* Philox(b >> 2, n, r, WOLFF_BOND << 16); the cluster of active bonds       */
/* containing the seed flips.  The cluster is a connected component, so it  */
/* does not depend on the order in which it is grown.                       */
/* ---------------------------------------------------------------------- */
enum { ORC_TAG_WOLFF_SEED = 16, ORC_TAG_WOLFF_BOND = 17 };

static int wolff_bond_active(uint64_t seed, uint32_t r, uint32_t step, uint32_t thr, uint32_t bond)
{
    uint32_t o[4];
    orc_block(seed, bond >> 2, step, r, ORC_TAG_WOLFF_BOND, 0, 0, o);
    return o[bond & 3] < thr;
}

uint32_t orc_wolff_seed_site(int L, uint64_t seed, uint32_t r, uint32_t step)
{
    uint32_t o[4];
    orc_block(seed, 0, step, r, ORC_TAG_WOLFF_SEED, 0, 0, o);
    return (uint32_t)(((uint64_t)o[0] * (uint64_t)((uint32_t)L * (uint32_t)L)) >> 32);
}

/* One Wolff step in place; stack and mark are scratch of L*L entries.
 * Returns the cluster size. */
long long orc_wolff_step(int L, double beta, uint64_t seed, uint32_t r, uint32_t step, int8_t *s,
                         uint32_t *stack, uint8_t *mark)
{
    const uint32_t N = (uint32_t)L * (uint32_t)L;
    const uint32_t thr = orc_sw_threshold(beta);
    memset(mark, 0, N);
    uint32_t m = orc_wolff_seed_site(L, seed, r, step);
    long long top = 0, size = 0;
    const int8_t s0 = s[m];
    stack[top++] = m;
    mark[m] = 1;
    while (top > 0) {
        uint32_t a = stack[--top];
        ++size;
        int x = (int)(a % (uint32_t)L), y = (int)(a / (uint32_t)L);
        /* the four bonds of site a: its own (to x+1, to y+1) and those of its
         * left and lower neighbours (from x-1, from y-1) */
        int xs[4] = {(x + 1) % L, x, (x + L - 1) % L, x};
        int ys[4] = {y, (y + 1) % L, y, (y + L - 1) % L};
        uint32_t bonds[4];
        bonds[0] = 2 * a;
        bonds[1] = 2 * a + 1;
        bonds[2] = 2 * (uint32_t)(y * L + xs[2]);
        bonds[3] = 2 * (uint32_t)(ys[3] * L + x) + 1;
        for (int k = 0; k < 4; ++k) {
            uint32_t b = (uint32_t)(ys[k] * L + xs[k]);
            if (mark[b] || s[b] != s0) continue;
            if (!wolff_bond_active(seed, r, step, thr, bonds[k])) continue;
            mark[b] = 1;
            stack[top++] = b;
        }
    }
    for (uint32_t i = 0; i < N; ++i)
        if (mark[i]) s[i] = (int8_t)-s[i];
    return size;
}
