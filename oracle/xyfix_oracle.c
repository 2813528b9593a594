/*
 * Plain single-threaded CPU oracle of the fixed-point XY sweep used for the
 * operand-precision study (arXiv 2402.06415, Supplementary "Operand bit width
 * optimization trial", Tab. S3): the spin angles are held as fixed-point
 * numbers with F fractional bits (the paper's (m, n) types with m - n = F:
 * (32,16), (24,12), (16,8) give F = 16, 12, 8; every integer part used here
 * needs at most 4 bits), the random numbers keep their full 32-bit width.
 * TEST INFRASTRUCTURE: loaded only by the tests, the smoke check and the
 * benchmark's CPU baseline.
 *
 * Reading of the fixed-point arithmetic (every quantity a signed integer
 * scaled by 2^-F, rounding to nearest, ties up, after each product):
 *   angle grid   theta_k = k 2^-F, k in [0, K), K = round(2 pi 2^F);
 *   tables       C[k] = floor(cos(theta_k) 2^F + 1/2), S[k] likewise for sin;
 *   local field  hx = sum_d C[k_d], hy = sum_d S[k_d] (exact integer sums);
 *   move         k' = floor(u1 K / 2^32) (u1 a full 32-bit word);
 *   energy       dE = -round(((C[k'] - C[k]) hx + (S[k'] - S[k]) hy) / 2^F)
 *                (the sign-corrected Eq. S1 in local-field form);
 *   acceptance   dE <= 0, or u2 < A[dE] = floor(exp(-beta dE 2^-F) 2^32)
 *                (u2 a full 32-bit word, A a table over dE in [1, 9 2^F));
 *                with qp = 1 the probability itself is held in the same
 *                fixed-point type first, truncated to F fractional bits:
 *                A[dE] = floor(exp(-beta dE 2^-F) 2^F) 2^(32-F) (clamped to
 *                2^32 - 1), the reading in which every operand of the update
 *                has the angle's type.
 * Sublattice (x + y) even first, then odd.  Random words: start k =
 * floor(w K / 2^32), w = word (n & 3) of Philox(n >> 2, 0, r, XYFIX_INIT << 16),
 * n = y L + x; sweep t, colour c: block Philox(j >> 1, t, r, XYFIX_MET << 16 |
 * c << 8), j = y (L/2) + (x >> 1), words 2 (j & 1) and 2 (j & 1) + 1 are u1, u2.
 * Records: E2 = sum over bonds of (C C' + S S') (scale 2^-2F; the energy is
 * -E2 2^-2F), Mx = sum C, My = sum S (scale 2^-F).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

enum { XYFIX_TAG_INIT = 15, XYFIX_TAG_MET = 14 };

static void fx_block(uint64_t seed, uint32_t a, uint32_t t, uint32_t r, uint32_t w3, uint32_t o[4])
{
    uint32_t ctr[4] = {a, t, r, w3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, o);
}

/* Number of grid angles for F fractional bits. */
int32_t orc_xyfix_K(int F)
{
    return (int32_t)floor(2.0 * 3.14159265358979323846 * ldexp(1.0, F) + 0.5);
}

/* Table entry k: cos and sin of k 2^-F, rounded to F fractional bits. */
void orc_xyfix_trig(int F, int32_t k, int32_t *c, int32_t *s)
{
    double a = ldexp((double)k, -F);
    double sc = ldexp(1.0, F);
    *c = (int32_t)floor(cos(a) * sc + 0.5);
    *s = (int32_t)floor(sin(a) * sc + 0.5);
}

/* Acceptance threshold for dE = e 2^-F > 0. */
uint32_t orc_xyfix_accept(int F, double beta, int32_t e, int qp)
{
    double dE = ldexp((double)e, -F);
    double t;
    if (qp)
        t = ldexp(floor(ldexp(exp(-beta * dE), F)), 32 - F);
    else
        t = floor(exp(-beta * dE) * 4294967296.0);
    if (t >= 4294967295.0) return 0xffffffffu;
    return (uint32_t)t;
}

/* Fixed-point energy change of moving a site from k to k2 in the local field
 * (hx, hy) (integers at scale 2^-F); result at scale 2^-F. */
int64_t orc_xyfix_dE(int F, int32_t k, int32_t k2, int64_t hx, int64_t hy)
{
    int32_t c, s, c2, s2;
    orc_xyfix_trig(F, k, &c, &s);
    orc_xyfix_trig(F, k2, &c2, &s2);
    int64_t p = (int64_t)(c2 - c) * hx + (int64_t)(s2 - s) * hy;  /* scale 2^-2F */
    int64_t r = (p + ((int64_t)1 << (F - 1))) >> F;                 /* nearest, ties up */
    return -r;
}

static int32_t at(const int32_t *k, int L, int x, int y)
{
    x = (x % L + L) % L;
    y = (y % L + L) % L;
    return k[(size_t)y * L + x];
}

void orc_xyfix_init(int L, int F, uint64_t seed, uint32_t r, int32_t *k)
{
    uint32_t K = (uint32_t)orc_xyfix_K(F);
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            uint32_t n = (uint32_t)(y * L + x), o[4];
            fx_block(seed, n >> 2, 0, r, (uint32_t)XYFIX_TAG_INIT << 16, o);
            k[(size_t)y * L + x] = (int32_t)(((uint64_t)o[n & 3] * K) >> 32);
        }
}

/* One sweep t in place; returns the number of accepted moves. */
int64_t orc_xyfix_sweep(int L, int F, int qp, double beta, uint64_t seed, uint32_t r, uint32_t t,
                        int32_t *k)
{
    uint32_t K = (uint32_t)orc_xyfix_K(F);
    int64_t acc = 0;
    for (int c = 0; c < 2; ++c)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                if (((x + y) & 1) != c) continue;
                int64_t hx = 0, hy = 0;
                const int dx[4] = {1, -1, 0, 0}, dy[4] = {0, 0, 1, -1};
                for (int d = 0; d < 4; ++d) {
                    int32_t cn, sn;
                    orc_xyfix_trig(F, at(k, L, x + dx[d], y + dy[d]), &cn, &sn);
                    hx += cn;
                    hy += sn;
                }
                uint32_t j = (uint32_t)(y * (L / 2) + (x >> 1)), o[4];
                fx_block(seed, j >> 1, t, r, ((uint32_t)XYFIX_TAG_MET << 16) | ((uint32_t)c << 8), o);
                uint32_t u1 = o[2 * (j & 1)], u2 = o[2 * (j & 1) + 1];
                int32_t k2 = (int32_t)(((uint64_t)u1 * K) >> 32);
                int32_t kold = k[(size_t)y * L + x];
                int64_t dE = orc_xyfix_dE(F, kold, k2, hx, hy);
                int ok = dE <= 0;
                if (!ok) ok = u2 < orc_xyfix_accept(F, beta, (int32_t)dE, qp);
                if (ok) {
                    k[(size_t)y * L + x] = k2;
                    ++acc;
                }
            }
    return acc;
}

void orc_xyfix_observables(int L, int F, const int32_t *k, int64_t *E2, int64_t *Mx, int64_t *My)
{
    int64_t e = 0, mx = 0, my = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int32_t c, s, c1, s1, c2, s2;
            orc_xyfix_trig(F, at(k, L, x, y), &c, &s);
            orc_xyfix_trig(F, at(k, L, x + 1, y), &c1, &s1);
            orc_xyfix_trig(F, at(k, L, x, y + 1), &c2, &s2);
            e += (int64_t)c * c1 + (int64_t)s * s1 + (int64_t)c * c2 + (int64_t)s * s2;
            mx += c;
            my += s;
        }
    *E2 = e;
    *Mx = mx;
    *My = my;
}
