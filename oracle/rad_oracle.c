/*
 * rad_oracle.c -- plain FP64 CPU oracle for the in-situ radiation spectrum.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The product path
 * (the CUDA library) never links, imports or calls it, and it shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (Frederiksen et al., "Radiation Spectral Synthesis of
 * Relativistic Filamentation", Sec. 2.2, the discretised P_omega integral, and
 * the Lienard-Wiechert far-field expression it cites from Rybicki & Lightman /
 * Jackson, Classical Electrodynamics eq. 14.67 with the positive-frequency
 * normalisation):
 *
 *   d^2W/(dw dOmega) = 1/(4 pi^2 c) | sum_j  A_j(n, w) |^2        (coherent)
 *                    = 1/(4 pi^2 c)   sum_j |A_j(n, w)|^2         (incoherent)
 *
 *   A_j(n, w) = sum_{m = s0}^{s1 - 1}  q_j V_{j,n,m} exp(i w phi_{j,n,m}) dt
 *   V         = n x ((n - beta) x betadot) / (1 - n.beta)^2
 *   phi       = t_m - n . r_m / c,      t_m = m dt,   c = 1.
 *
 * Readings of points the paper leaves open (it is silent or garbled on each):
 *   - E_ret of Sec. 2.2 is the Jackson retarded-time integrand V above, and the
 *     garbled phase is phi' = t' - n.r(t')/c.
 *   - the proportionality constant is q^2/(4 pi^2 c) with q inside A.
 *   - leapfrog time-centring: call s delivers x_s and u_{s-1/2}; sample m uses
 *     r_m = unwrapped x_m, beta_m = ubar/sqrt(1+ubar^2) with
 *     ubar = (u_{m-1/2} + u_{m+1/2})/2, and
 *     betadot_m = (beta_{m+1/2} - beta_{m-1/2})/dt; so sample m needs calls m
 *     and m+1.
 *   - the time integral is a rectangle rule (every sample has weight dt).
 *   - positions in a periodic box of side L are unwrapped by minimum image:
 *     r_m = x_m + L n_m with the integer image count n_0 = 0,
 *     n_m = n_{m-1} - nearest_integer((x_m - x_{m-1}) / L), i.e. the
 *     position plus whole box lengths (one rounding, not a running sum).
 *
 * Precision: FP64 throughout, libm sin/cos; build without fast-math and with
 * -ffp-contract=off so that the arithmetic is exactly what is written.
 *
 * Parity status: every function here is pinned by a CPU test against closed
 * forms (uniform motion, prescribed-dipole geometric sums, discrete Parseval,
 * synchrotron, Lienard sphere integral) or invariants; see the tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* small vector helpers, written out                                         */
/* ------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void cross3(const double a[3], const double b[3], double out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* Whole box lengths in a displacement d (periodic box of side L; L <= 0: none). */
static double image_jump(double d, double L)
{
    return L > 0.0 ? nearbyint(d / L) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Step 1: trajectory samples from the leapfrog states the PIC hands over.   */
/* Sec. 2.2 integrates over the particle history; the sampling and centring  */
/* are the readings listed in the header.                                    */
/*                                                                           */
/*   x, u     : [n_calls][3][N]  (call s: x_s and u_{s-1/2}, SoA per call)   */
/*   r, beta, bdot : [n_calls-1][3][N]  (sample m = 0 .. n_calls-2)          */
/* Returns 0, or -1 on bad sizes.                                            */
/* ------------------------------------------------------------------------ */
int rado_samples(int64_t n_calls, int64_t N, const double *x, const double *u,
                 double dt, double box_L, double *r, double *beta, double *bdot)
{
    if (n_calls < 2 || N < 0 || !(dt > 0.0)) return -1;
    const int64_t n_samp = n_calls - 1;
    for (int64_t j = 0; j < N; ++j) {
        double img[3] = {0.0, 0.0, 0.0};   /* image count n_m */
        double pos[3];
        for (int64_t m = 0; m < n_samp; ++m) {
            /* unwrapped position r_m = x_m + L n_m */
            for (int c = 0; c < 3; ++c) {
                const double xm = x[(m * 3 + c) * N + j];
                if (m > 0) img[c] -= image_jump(xm - x[((m - 1) * 3 + c) * N + j], box_L);
                pos[c] = box_L > 0.0 ? xm + box_L * img[c] : xm;
            }
            double um[3], up[3], ubar[3], bm[3], bp[3];
            for (int c = 0; c < 3; ++c) {
                um[c] = u[(m * 3 + c) * N + j];         /* u_{m-1/2}: call m   */
                up[c] = u[((m + 1) * 3 + c) * N + j];   /* u_{m+1/2}: call m+1 */
                ubar[c] = 0.5 * (um[c] + up[c]);
            }
            double gm = sqrt(1.0 + dot3(um, um));
            double gp = sqrt(1.0 + dot3(up, up));
            double gbar = sqrt(1.0 + dot3(ubar, ubar));
            for (int c = 0; c < 3; ++c) {
                bm[c] = um[c] / gm;
                bp[c] = up[c] / gp;
                r[(m * 3 + c) * N + j] = pos[c];
                beta[(m * 3 + c) * N + j] = ubar[c] / gbar;
                bdot[(m * 3 + c) * N + j] = (bp[c] - bm[c]) / dt;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Step 2: the Lienard-Wiechert far-field integrand (Jackson 14.67 form the  */
/* paper's E_ret stands for):  V = n x ((n - beta) x betadot) / (1-n.beta)^2 */
/* ------------------------------------------------------------------------ */
void rado_field(const double n[3], const double b[3], const double bd[3], double V[3])
{
    double nmb[3] = {n[0] - b[0], n[1] - b[1], n[2] - b[2]};
    double inner[3], outer[3];
    cross3(nmb, bd, inner);
    cross3(n, inner, outer);
    double kappa = 1.0 - dot3(n, b);
    double k2 = kappa * kappa;
    V[0] = outer[0] / k2;
    V[1] = outer[1] / k2;
    V[2] = outer[2] / k2;
}

/* ------------------------------------------------------------------------ */
/* Step 3: one particle's vector amplitude over samples [m0, m1) (Sec. 2.2): */
/*   A(w) = sum_m q V_m exp(i w (m dt - n.r_m)) dt,   for nf frequencies.    */
/* Sample arrays are [n_samp][3][N] indexed by the absolute sample m.        */
/* A_re, A_im: [nf][3].                                                      */
/* ------------------------------------------------------------------------ */
void rado_amplitude(int64_t N, int64_t j, int64_t m0, int64_t m1,
                    const double *r, const double *beta, const double *bdot,
                    double dt, double q, const double n[3],
                    int32_t nf, const double *omega, double *A_re, double *A_im)
{
    for (int32_t k = 0; k < nf; ++k)
        for (int c = 0; c < 3; ++c) A_re[k * 3 + c] = A_im[k * 3 + c] = 0.0;
    for (int64_t m = m0; m < m1; ++m) {
        double rm[3], bm[3], bdm[3], V[3];
        for (int c = 0; c < 3; ++c) {
            rm[c] = r[(m * 3 + c) * N + j];
            bm[c] = beta[(m * 3 + c) * N + j];
            bdm[c] = bdot[(m * 3 + c) * N + j];
        }
        rado_field(n, bm, bdm, V);
        double t = (double)m * dt;
        double phi = t - dot3(n, rm);
        for (int32_t k = 0; k < nf; ++k) {
            double th = omega[k] * phi;
            double cs = cos(th), sn = sin(th);
            for (int c = 0; c < 3; ++c) {
                double a = q * V[c] * dt;
                A_re[k * 3 + c] += a * cs;
                A_im[k * 3 + c] += a * sn;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Step 4: the spectrum of one window [s0, s1) for D directions and nf       */
/* frequencies (Sec. 2.2: coherent |sum_j A_j|^2 or incoherent              */
/* sum_j |A_j|^2, times 1/(4 pi^2 c)).                                       */
/*   charge[N]: q_j;  include[N] (may be NULL): 0 excludes a particle.       */
/*   S_out: [D][nf].                                                         */
/* Returns 0, or -1 on bad arguments.                                        */
/* ------------------------------------------------------------------------ */
int rado_spectrum(int64_t N, int64_t n_samp, const double *r, const double *beta,
                  const double *bdot, const double *charge, const unsigned char *include,
                  double dt, int32_t D, const double *dirs, int32_t nf, const double *omega,
                  int64_t s0, int64_t s1, int32_t coherent, double *S_out)
{
    if (s0 < 0 || s1 < s0 || s1 > n_samp || D < 0 || nf < 0 || N < 0) return -1;
    const double pref = 1.0 / (4.0 * PI * PI); /* c = 1 */
    const int64_t n_pairs = (int64_t)D * N;
    const int64_t out_len = (int64_t)D * nf;
    for (int64_t i = 0; i < out_len; ++i) S_out[i] = 0.0;
    if (out_len == 0) return 0;

    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    /* per-thread partial sums: incoherent |A_j|^2 per (d, k), or coherent sum_j A_j */
    const int64_t per_thread = coherent ? out_len * 6 : out_len;
    double *part = (double *)calloc((size_t)(per_thread * nthreads), sizeof(double));
    if (!part) return -1;

#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = part + (int64_t)tid * per_thread;
        double *Are = (double *)malloc(sizeof(double) * (size_t)(nf > 0 ? nf : 1) * 3);
        double *Aim = (double *)malloc(sizeof(double) * (size_t)(nf > 0 ? nf : 1) * 3);
#pragma omp for schedule(static)
        for (int64_t p = 0; p < n_pairs; ++p) {
            int32_t d = (int32_t)(p / N);
            int64_t j = p % N;
            if (include && !include[j]) continue;
            rado_amplitude(N, j, s0, s1, r, beta, bdot, dt, charge[j], dirs + 3 * d, nf,
                           omega, Are, Aim);
            for (int32_t k = 0; k < nf; ++k) {
                if (coherent) {
                    for (int c = 0; c < 3; ++c) {
                        mine[((int64_t)d * nf + k) * 6 + 2 * c] += Are[k * 3 + c];
                        mine[((int64_t)d * nf + k) * 6 + 2 * c + 1] += Aim[k * 3 + c];
                    }
                } else {
                    double p2 = 0.0;
                    for (int c = 0; c < 3; ++c)
                        p2 += Are[k * 3 + c] * Are[k * 3 + c] + Aim[k * 3 + c] * Aim[k * 3 + c];
                    mine[(int64_t)d * nf + k] += p2;
                }
            }
        }
        free(Are);
        free(Aim);
    }

    if (coherent) {
        for (int64_t i = 0; i < out_len; ++i) {
            double s2 = 0.0;
            for (int c = 0; c < 6; ++c) {
                double acc = 0.0;
                for (int t = 0; t < nthreads; ++t) acc += part[(int64_t)t * per_thread + i * 6 + c];
                s2 += acc * acc;
            }
            S_out[i] = pref * s2;
        }
    } else {
        for (int64_t i = 0; i < out_len; ++i) {
            double acc = 0.0;
            for (int t = 0; t < nthreads; ++t) acc += part[(int64_t)t * per_thread + i];
            S_out[i] = pref * acc;
        }
    }
    free(part);
    return 0;
}

/* Number of OpenMP threads the oracle will use (1 without OpenMP). */
int rado_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the OpenMP thread count (ignored without OpenMP). */
void rado_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
