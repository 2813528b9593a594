/*
 * Multi-core timing build of the oracle's checkerboard sweep.
 *
 * TEST INFRASTRUCTURE, timing only.  It runs the same per-site steps as
 * orc_half_sweep in ising_oracle.c (same counter map, same thresholds, same
 * strict test), with the rows of one colour spread over OpenMP threads, the
 * way the paper times its CPU code with several threads (Supplementary,
 * Tab. S1: one OpenMP thread per row block of a sublattice).  Sites of one
 * colour have no neighbour of that colour and every uniform is a function of
 * (seed, sweep, site) alone, so the result equals the single-threaded sweep
 * bit for bit whatever the thread count; parity claims still rest on the
 * single-threaded oracle (a test checks the two agree).
 *
 * Compiled into liboracle.so with -fopenmp when the compiler supports it;
 * without it the pragmas are ignored and orc_omp_threads() reports 1.
 */
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* from ising_oracle.c */
int orc_words_per_row(int L);
uint32_t orc_threshold(double beta, int dE);
int orc_decide(int n_anti, uint32_t u, uint32_t thr4, uint32_t thr8);
void orc_met_planes(uint64_t seed, uint32_t r, uint32_t t, int c, uint32_t g, uint32_t P[32]);
uint32_t orc_assemble_u(const uint32_t P[32], int lane);
int orc_n_anti(int L, const int8_t *s, int x, int y);
void orc_energy_mag(int L, const int8_t *s, int64_t *E, int64_t *M);

/* Threads one parallel region of the sweep below uses. */
int orc_omp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void half_sweep_omp(int L, uint32_t thr4, uint32_t thr8, uint64_t seed, uint32_t r,
                           uint32_t t, int c, int8_t *s)
{
    int Wc = orc_words_per_row(L);
    int half = L / 2;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
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

/* Same contract as orc_sweep (records after sweep t iff (t + 1) % measure_every
 * == 0; returns the number of records, -1 on bad arguments). */
int orc_sweep_omp(int L, double beta, uint64_t seed, uint32_t r, uint32_t t0, int n_sweeps,
                  int measure_every, int8_t *s, int64_t *E_out, int64_t *M_out)
{
    if (L < 2 || (L & 1) || n_sweeps < 0 || measure_every < 1) return -1;
    uint32_t thr4 = orc_threshold(beta, 4);
    uint32_t thr8 = orc_threshold(beta, 8);
    int rec = 0;
    for (int k = 0; k < n_sweeps; ++k) {
        uint32_t t = t0 + (uint32_t)k;
        half_sweep_omp(L, thr4, thr8, seed, r, t, 0, s);
        half_sweep_omp(L, thr4, thr8, seed, r, t, 1, s);
        if (((uint64_t)t + 1) % (uint64_t)measure_every == 0) {
            if (E_out && M_out) orc_energy_mag(L, s, &E_out[rec], &M_out[rec]);
            ++rec;
        }
    }
    return rec;
}
