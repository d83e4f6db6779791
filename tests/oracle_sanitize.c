/*
 * oracle_sanitize.c -- drives every entry point of oracle/rad_oracle.c on small
 * inputs, for a build with AddressSanitizer and UndefinedBehaviorSanitizer
 * (test infrastructure: tests/test_oracle_sanitizers.py compiles and runs it).
 *
 * Every buffer is a heap allocation of exactly the size the oracle's interface
 * states, so a read or write past any of them is reported.  The cases cover
 * trajectories that cross the periodic box (unwrapping), empty and one-sample
 * windows, zero particles / directions / frequencies, a particle mask, both
 * summation modes, one and several OpenMP threads, and rejected arguments.
 * Besides memory safety it checks a few exact facts: uniform motion radiates
 * exactly nothing, a single particle's coherent and incoherent spectra agree,
 * spectra are non-negative and finite, and the thread count changes nothing
 * beyond summation order.  Prints "ok" and exits 0 when everything holds.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int rado_samples(int64_t n_calls, int64_t N, const double *x, const double *u, double dt,
                 double box_L, double *r, double *beta, double *bdot);
void rado_field(const double n[3], const double b[3], const double bd[3], double V[3]);
void rado_amplitude(int64_t N, int64_t j, int64_t m0, int64_t m1, const double *r,
                    const double *beta, const double *bdot, double dt, double q,
                    const double n[3], int32_t nf, const double *omega, double *A_re,
                    double *A_im);
int rado_spectrum(int64_t N, int64_t n_samp, const double *r, const double *beta,
                  const double *bdot, const double *charge, const unsigned char *include,
                  double dt, int32_t D, const double *dirs, int32_t nf, const double *omega,
                  int64_t s0, int64_t s1, int32_t coherent, double *S_out);
int rado_num_threads(void);
void rado_set_num_threads(int n);

static int failures = 0;
#define CHECK(cond, ...)                          \
    do {                                          \
        if (!(cond)) {                            \
            fprintf(stderr, "FAILED: " __VA_ARGS__); \
            fprintf(stderr, "\n");                \
            ++failures;                           \
        }                                         \
    } while (0)

/* 64-bit linear congruential generator (Knuth's MMIX constants) -> [0, 1) */
static uint64_t lcg_state = 0x1234567ull;
static double uniform01(void)
{
    lcg_state = lcg_state * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(lcg_state >> 11) * (1.0 / 9007199254740992.0);
}

static double *alloc_d(size_t n)
{
    double *p = (double *)malloc((n ? n : 1) * sizeof(double));
    if (!p) {
        fprintf(stderr, "out of memory\n");
        exit(2);
    }
    return p;
}

/* x, u: [n_calls][3][N]; particles drift through a box of side L (wrapped
 * back into [0, L)) while their momenta rotate, so positions cross the box. */
static void make_trajectory(int64_t n_calls, int64_t N, double dt, double L, int uniform,
                            double *x, double *u)
{
    for (int64_t j = 0; j < N; ++j) {
        double pos[3], mom[3];
        for (int c = 0; c < 3; ++c) {
            pos[c] = L * uniform01();
            mom[c] = 6.0 * uniform01() - 3.0;
        }
        const double w = uniform ? 0.0 : 0.5 + uniform01();   /* rotation rate about z */
        for (int64_t s = 0; s < n_calls; ++s) {
            for (int c = 0; c < 3; ++c) {
                double xc = fmod(pos[c], L);
                if (xc < 0.0) xc += L;
                x[(s * 3 + c) * N + j] = xc;
                u[(s * 3 + c) * N + j] = mom[c];
            }
            /* next half-step momentum: rotate about z by w dt */
            const double cw = cos(w * dt), sw = sin(w * dt);
            const double ux = mom[0] * cw - mom[1] * sw, uy = mom[0] * sw + mom[1] * cw;
            mom[0] = ux;
            mom[1] = uy;
            const double g = sqrt(1.0 + mom[0] * mom[0] + mom[1] * mom[1] + mom[2] * mom[2]);
            for (int c = 0; c < 3; ++c) pos[c] += dt * mom[c] / g;
        }
    }
}

static void run_case(int64_t n_calls, int64_t N, int32_t D, int32_t nf, int uniform)
{
    const double dt = 0.05, L = 0.7;
    const int64_t n_samp = n_calls - 1;
    double *x = alloc_d((size_t)(n_calls * 3 * N));
    double *u = alloc_d((size_t)(n_calls * 3 * N));
    double *r = alloc_d((size_t)(n_samp * 3 * N));
    double *beta = alloc_d((size_t)(n_samp * 3 * N));
    double *bdot = alloc_d((size_t)(n_samp * 3 * N));
    double *charge = alloc_d((size_t)N);
    unsigned char *include = (unsigned char *)malloc((size_t)(N ? N : 1));
    double *dirs = alloc_d((size_t)(3 * D));
    double *omega = alloc_d((size_t)nf);
    double *S1 = alloc_d((size_t)(D * nf));
    double *S2 = alloc_d((size_t)(D * nf));
    make_trajectory(n_calls, N, dt, L, uniform, x, u);
    for (int64_t j = 0; j < N; ++j) {
        charge[j] = (j % 3 == 0) ? 1.0 : -1.0;
        include[j] = (unsigned char)(j % 4 != 1);
    }
    for (int32_t d = 0; d < D; ++d) {
        const double th = 0.4 + 0.9 * d, ph = 0.3 * d;
        dirs[3 * d] = sin(th) * cos(ph);
        dirs[3 * d + 1] = sin(th) * sin(ph);
        dirs[3 * d + 2] = cos(th);
    }
    for (int32_t k = 0; k < nf; ++k) omega[k] = 0.1 * pow(1.37, k);

    CHECK(rado_samples(n_calls, N, x, u, dt, L, r, beta, bdot) == 0, "samples");
    const int64_t win[4][2] = {{0, n_samp}, {n_samp / 3, n_samp / 3 + 1}, {n_samp / 2, n_samp / 2},
                               {n_samp - 1, n_samp}};
    for (int w = 0; w < 4; ++w) {
        for (int coh = 0; coh < 2; ++coh) {
            for (int masked = 0; masked < 2; ++masked) {
                const unsigned char *inc = masked ? include : NULL;
                rado_set_num_threads(1);
                CHECK(rado_spectrum(N, n_samp, r, beta, bdot, charge, inc, dt, D, dirs, nf, omega,
                                    win[w][0], win[w][1], coh, S1) == 0, "spectrum");
                rado_set_num_threads(3);
                CHECK(rado_spectrum(N, n_samp, r, beta, bdot, charge, inc, dt, D, dirs, nf, omega,
                                    win[w][0], win[w][1], coh, S2) == 0, "spectrum (3 threads)");
                double smax = 0.0;
                for (int64_t i = 0; i < (int64_t)D * nf; ++i) {
                    CHECK(isfinite(S1[i]) && S1[i] >= 0.0, "finite non-negative S");
                    if (S1[i] > smax) smax = S1[i];
                }
                for (int64_t i = 0; i < (int64_t)D * nf; ++i)
                    CHECK(fabs(S1[i] - S2[i]) <= 1e-12 * smax, "thread count changed S[%lld]",
                          (long long)i);
                if (uniform) {
                    for (int64_t i = 0; i < (int64_t)D * nf; ++i)
                        CHECK(S1[i] == 0.0, "uniform motion radiates exactly nothing");
                }
            }
        }
    }
    /* one particle: coherent and incoherent spectra agree */
    if (N >= 1 && D >= 1 && nf >= 1) {
        unsigned char *only0 = (unsigned char *)calloc((size_t)N, 1);
        only0[0] = 1;
        rado_spectrum(N, n_samp, r, beta, bdot, charge, only0, dt, D, dirs, nf, omega, 0, n_samp,
                      0, S1);
        rado_spectrum(N, n_samp, r, beta, bdot, charge, only0, dt, D, dirs, nf, omega, 0, n_samp,
                      1, S2);
        for (int64_t i = 0; i < (int64_t)D * nf; ++i)
            CHECK(fabs(S1[i] - S2[i]) <= 1e-12 * (fabs(S1[i]) + 1e-300),
                  "one particle: coherent == incoherent");
        free(only0);
        /* the amplitude and field entry points on their own */
        double *Are = alloc_d((size_t)(3 * nf)), *Aim = alloc_d((size_t)(3 * nf));
        rado_amplitude(N, N - 1, 0, n_samp, r, beta, bdot, dt, charge[N - 1], dirs, nf, omega,
                       Are, Aim);
        for (int64_t i = 0; i < 3 * (int64_t)nf; ++i)
            CHECK(isfinite(Are[i]) && isfinite(Aim[i]), "finite amplitude");
        double V[3];
        rado_field(dirs, beta, bdot, V);
        CHECK(isfinite(V[0]) && isfinite(V[1]) && isfinite(V[2]), "finite field");
        free(Are);
        free(Aim);
    }
    /* rejected arguments leave the output alone past its zeroing */
    CHECK(rado_spectrum(N, n_samp, r, beta, bdot, charge, NULL, dt, D, dirs, nf, omega, 0,
                        n_samp + 1, 0, S1) == -1, "window past the samples is rejected");
    CHECK(rado_spectrum(N, n_samp, r, beta, bdot, charge, NULL, dt, D, dirs, nf, omega, 3, 2, 0,
                        S1) == -1, "reversed window is rejected");
    CHECK(rado_samples(1, N, x, u, dt, L, r, beta, bdot) == -1, "one call is rejected");
    CHECK(rado_samples(n_calls, N, x, u, 0.0, L, r, beta, bdot) == -1, "dt = 0 is rejected");

    free(x); free(u); free(r); free(beta); free(bdot); free(charge); free(include);
    free(dirs); free(omega); free(S1); free(S2);
}

int main(void)
{
    const int threads = rado_num_threads();
    run_case(41, 13, 3, 17, 0);     /* several particles, box crossings */
    run_case(41, 5, 2, 9, 1);       /* uniform motion */
    run_case(2, 1, 1, 1, 0);        /* the smallest valid problem: one sample */
    run_case(9, 0, 2, 4, 0);        /* no particles */
    run_case(9, 4, 0, 4, 0);        /* no directions */
    run_case(9, 4, 2, 0, 0);        /* no frequencies */
    rado_set_num_threads(threads);
    if (failures) {
        fprintf(stderr, "%d check(s) failed\n", failures);
        return 1;
    }
    printf("ok\n");
    return 0;
}
