/*
 * Plain single-threaded CPU oracle of the checkerboard Metropolis sweep of
 * the 2D XY model (arXiv 2402.06415, Eq. 1 and Supplementary "Detail of the MC
 * calculation for the XY model").  TEST INFRASTRUCTURE: loaded only by the
 * tests, the smoke check and the benchmark's CPU baseline.
 *
 * H = -sum_bonds cos(theta_x - theta_x+d) on the periodic L x L lattice.  Each
 * spin is kept as its unit vector u = (cos theta, sin theta).  Per site
 * (paper's three steps): (1) draw theta' uniform in [0, 2 pi) and p uniform in
 * [0, 1); (2) dE = -sum_d [cos(theta' - theta_d) - cos(theta - theta_d)]
 * (Eq. S1 with the sign of its second term corrected), written here in the
 * equivalent local-field form dE = -(u' - u) . h with h = sum_d u_d, and
 * P(dE) = exp(-beta dE); (3) update iff p < P.  Sublattice (x + y) even first,
 * then odd (Results A, Fig. 2).
 *
 * Arithmetic in the working precision (double or float); cos/sin/exp are this
 * file's own (Cody-Waite range reduction, Taylor polynomials evaluated by
 * Horner steps with explicit fused multiply-adds), so that a GPU implementation
 * following the same published recipe gets the same bits.
 *
 * Random numbers: Philox4x32-10 keyed by the seed (ising_oracle.c).  Site
 * n = y L + x; colour-compact index k = y (L/2) + (x >> 1).
 *   start:  theta = 2 pi * (w >> 8) 2^-24, w = word (n & 3) of
 *           Philox(n >> 2, 0, r, XY_INIT << 16)
 *   sweep t, colour c:  block Philox(k >> 1, t, r, XY_MET << 16 | c << 8);
 *           words 2 (k & 1) and 2 (k & 1) + 1 give theta' and p (top 24 bits).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

enum { XY_TAG_INIT = 8, XY_TAG_MET = 9 };

static void xy_block(uint64_t seed, uint32_t a, uint32_t t, uint32_t r, uint32_t w3, uint32_t o[4])
{
    uint32_t ctr[4] = {a, t, r, w3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, o);
}

/* ---------------- double precision ---------------- */
static const double D_PIO2_HI = 1.5707963267948966;     /* pi/2 rounded */
static const double D_PIO2_LO = 6.123233995736766e-17;  /* pi/2 - D_PIO2_HI */
static const double D_TWO_OVER_PI = 0.6366197723675814;
static const double D_LN2_HI = 0.6931471805599453;
static const double D_LN2_LO = 2.3190468138462996e-17;
static const double D_INV_LN2 = 1.4426950408889634;
static const double D_TWO_PI = 6.283185307179586;

/* cos and sin of r, |r| <= pi/4: Taylor series through r^16 / r^17 */
static void d_sincos_small(double r, double *s, double *c)
{
    double z = r * r;
    double pc = 1.0 / 20922789888000.0;              /* 1/16! */
    pc = fma(pc, z, -1.0 / 87178291200.0);           /* 1/14! */
    pc = fma(pc, z, 1.0 / 479001600.0);              /* 1/12! */
    pc = fma(pc, z, -1.0 / 3628800.0);
    pc = fma(pc, z, 1.0 / 40320.0);
    pc = fma(pc, z, -1.0 / 720.0);
    pc = fma(pc, z, 1.0 / 24.0);
    pc = fma(pc, z, -0.5);
    pc = fma(pc, z, 1.0);
    double ps = 1.0 / 355687428096000.0;             /* 1/17! */
    ps = fma(ps, z, -1.0 / 1307674368000.0);         /* 1/15! */
    ps = fma(ps, z, 1.0 / 6227020800.0);             /* 1/13! */
    ps = fma(ps, z, -1.0 / 39916800.0);
    ps = fma(ps, z, 1.0 / 362880.0);
    ps = fma(ps, z, -1.0 / 5040.0);
    ps = fma(ps, z, 1.0 / 120.0);
    ps = fma(ps, z, -1.0 / 6.0);
    ps = fma(ps, z, 1.0);
    *c = pc;
    *s = ps * r;
}

void orc_xy_sincos_d(double x, double *s, double *c)
{
    double k = rint(x * D_TWO_OVER_PI);
    double r = fma(-k, D_PIO2_HI, x);
    r = fma(-k, D_PIO2_LO, r);
    double ss, cc;
    d_sincos_small(r, &ss, &cc);
    int q = ((int)k) & 3;
    if (q == 0) { *s = ss; *c = cc; }
    else if (q == 1) { *s = cc; *c = -ss; }
    else if (q == 2) { *s = -ss; *c = -cc; }
    else { *s = -cc; *c = ss; }
}

double orc_xy_exp_d(double x)
{
    if (x < -700.0) return 0.0;
    double k = rint(x * D_INV_LN2);
    double r = fma(-k, D_LN2_HI, x);
    r = fma(-k, D_LN2_LO, r);
    double p = 1.0 / 6227020800.0;                   /* 1/13! */
    p = fma(p, r, 1.0 / 479001600.0);
    p = fma(p, r, 1.0 / 39916800.0);
    p = fma(p, r, 1.0 / 3628800.0);
    p = fma(p, r, 1.0 / 362880.0);
    p = fma(p, r, 1.0 / 40320.0);
    p = fma(p, r, 1.0 / 5040.0);
    p = fma(p, r, 1.0 / 720.0);
    p = fma(p, r, 1.0 / 120.0);
    p = fma(p, r, 1.0 / 24.0);
    p = fma(p, r, 1.0 / 6.0);
    p = fma(p, r, 0.5);
    p = fma(p, r, 1.0);
    p = fma(p, r, 1.0);
    return ldexp(p, (int)k);
}

/* ---------------- single precision ---------------- */
static const float F_PIO2_HI = 1.57079637f;
static const float F_PIO2_LO = -4.37113883e-08f;
static const float F_TWO_OVER_PI = 0.636619747f;
static const float F_LN2_HI = 0.693147182f;
static const float F_LN2_LO = -1.90465421e-09f;
static const float F_INV_LN2 = 1.44269502f;
static const float F_TWO_PI = 6.28318548f;

static void f_sincos_small(float r, float *s, float *c)
{
    float z = r * r;
    float pc = 1.0f / 40320.0f;
    pc = fmaf(pc, z, -1.0f / 720.0f);
    pc = fmaf(pc, z, 1.0f / 24.0f);
    pc = fmaf(pc, z, -0.5f);
    pc = fmaf(pc, z, 1.0f);
    float ps = 1.0f / 362880.0f;
    ps = fmaf(ps, z, -1.0f / 5040.0f);
    ps = fmaf(ps, z, 1.0f / 120.0f);
    ps = fmaf(ps, z, -1.0f / 6.0f);
    ps = fmaf(ps, z, 1.0f);
    *c = pc;
    *s = ps * r;
}

void orc_xy_sincos_f(float x, float *s, float *c)
{
    float k = rintf(x * F_TWO_OVER_PI);
    float r = fmaf(-k, F_PIO2_HI, x);
    r = fmaf(-k, F_PIO2_LO, r);
    float ss, cc;
    f_sincos_small(r, &ss, &cc);
    int q = ((int)k) & 3;
    if (q == 0) { *s = ss; *c = cc; }
    else if (q == 1) { *s = cc; *c = -ss; }
    else if (q == 2) { *s = -ss; *c = -cc; }
    else { *s = -cc; *c = ss; }
}

float orc_xy_exp_f(float x)
{
    if (x < -87.0f) return 0.0f;
    float k = rintf(x * F_INV_LN2);
    float r = fmaf(-k, F_LN2_HI, x);
    r = fmaf(-k, F_LN2_LO, r);
    float p = 1.0f / 40320.0f;
    p = fmaf(p, r, 1.0f / 5040.0f);
    p = fmaf(p, r, 1.0f / 720.0f);
    p = fmaf(p, r, 1.0f / 120.0f);
    p = fmaf(p, r, 1.0f / 24.0f);
    p = fmaf(p, r, 1.0f / 6.0f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    return ldexpf(p, (int)k);
}

/* ---------------- lattice (u stored as [L][L][2]) ---------------- */
#define XY_AT(u, L, x, y) ((u) + 2 * ((size_t)((((y) % (L)) + (L)) % (L)) * (L) + (size_t)((((x) % (L)) + (L)) % (L))))

void orc_xy_init_d(int L, uint64_t seed, uint32_t r, double *u)
{
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            uint32_t n = (uint32_t)(y * L + x), o[4];
            xy_block(seed, n >> 2, 0, r, XY_TAG_INIT << 16, o);
            double th = D_TWO_PI * ((double)(o[n & 3] >> 8) * (1.0 / 16777216.0));
            orc_xy_sincos_d(th, &XY_AT(u, L, x, y)[1], &XY_AT(u, L, x, y)[0]);
        }
}

void orc_xy_init_f(int L, uint64_t seed, uint32_t r, float *u)
{
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            uint32_t n = (uint32_t)(y * L + x), o[4];
            xy_block(seed, n >> 2, 0, r, XY_TAG_INIT << 16, o);
            float th = F_TWO_PI * ((float)(o[n & 3] >> 8) * (1.0f / 16777216.0f));
            orc_xy_sincos_f(th, &XY_AT(u, L, x, y)[1], &XY_AT(u, L, x, y)[0]);
        }
}

/* One full sweep (colour 0 then 1) at sweep index t; returns accepted count. */
long long orc_xy_sweep_d(int L, double beta, uint64_t seed, uint32_t r, uint32_t t, double *u)
{
    long long acc = 0;
    for (int c = 0; c < 2; ++c)
        for (int y = 0; y < L; ++y)
            for (int x = (y + c) & 1; x < L; x += 2) {
                uint32_t k = (uint32_t)(y * (L / 2) + (x >> 1)), o[4];
                xy_block(seed, k >> 1, t, r, (XY_TAG_MET << 16) | ((uint32_t)c << 8), o);
                uint32_t w1 = o[2 * (k & 1)], w2 = o[2 * (k & 1) + 1];
                double th = D_TWO_PI * ((double)(w1 >> 8) * (1.0 / 16777216.0));
                double p = (double)(w2 >> 8) * (1.0 / 16777216.0);
                const double *a = XY_AT(u, L, x + 1, y), *b = XY_AT(u, L, x - 1, y);
                const double *d = XY_AT(u, L, x, y + 1), *e = XY_AT(u, L, x, y - 1);
                double hx = a[0] + b[0];
                hx = hx + d[0];
                hx = hx + e[0];
                double hy = a[1] + b[1];
                hy = hy + d[1];
                hy = hy + e[1];
                double sn, cs;
                orc_xy_sincos_d(th, &sn, &cs);
                double *me = XY_AT(u, L, x, y);
                double dE = -(fma(cs - me[0], hx, (sn - me[1]) * hy));
                if (dE <= 0.0 || p < orc_xy_exp_d(-beta * dE)) {
                    me[0] = cs;
                    me[1] = sn;
                    ++acc;
                }
            }
    return acc;
}

long long orc_xy_sweep_f(int L, float beta, uint64_t seed, uint32_t r, uint32_t t, float *u)
{
    long long acc = 0;
    for (int c = 0; c < 2; ++c)
        for (int y = 0; y < L; ++y)
            for (int x = (y + c) & 1; x < L; x += 2) {
                uint32_t k = (uint32_t)(y * (L / 2) + (x >> 1)), o[4];
                xy_block(seed, k >> 1, t, r, (XY_TAG_MET << 16) | ((uint32_t)c << 8), o);
                uint32_t w1 = o[2 * (k & 1)], w2 = o[2 * (k & 1) + 1];
                float th = F_TWO_PI * ((float)(w1 >> 8) * (1.0f / 16777216.0f));
                float p = (float)(w2 >> 8) * (1.0f / 16777216.0f);
                const float *a = XY_AT(u, L, x + 1, y), *b = XY_AT(u, L, x - 1, y);
                const float *d = XY_AT(u, L, x, y + 1), *e = XY_AT(u, L, x, y - 1);
                float hx = a[0] + b[0];
                hx = hx + d[0];
                hx = hx + e[0];
                float hy = a[1] + b[1];
                hy = hy + d[1];
                hy = hy + e[1];
                float sn, cs;
                orc_xy_sincos_f(th, &sn, &cs);
                float *me = XY_AT(u, L, x, y);
                float dE = -(fmaf(cs - me[0], hx, (sn - me[1]) * hy));
                if (dE <= 0.0f || p < orc_xy_exp_f(-beta * dE)) {
                    me[0] = cs;
                    me[1] = sn;
                    ++acc;
                }
            }
    return acc;
}

/* E = -sum_x u_x . (u_{x+e1} + u_{x+e2}) and M = sum u, in double. */
void orc_xy_observables_d(int L, const double *u, double *E, double *Mx, double *My)
{
    double e = 0, mx = 0, my = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            const double *a = XY_AT(u, L, x, y), *b = XY_AT(u, L, x + 1, y), *d = XY_AT(u, L, x, y + 1);
            e -= a[0] * (b[0] + d[0]) + a[1] * (b[1] + d[1]);
            mx += a[0];
            my += a[1];
        }
    *E = e; *Mx = mx; *My = my;
}

void orc_xy_observables_f(int L, const float *u, double *E, double *Mx, double *My)
{
    double e = 0, mx = 0, my = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            const float *a = XY_AT(u, L, x, y), *b = XY_AT(u, L, x + 1, y), *d = XY_AT(u, L, x, y + 1);
            e -= (double)a[0] * ((double)b[0] + d[0]) + (double)a[1] * ((double)b[1] + d[1]);
            mx += a[0];
            my += a[1];
        }
    *E = e; *Mx = mx; *My = my;
}
