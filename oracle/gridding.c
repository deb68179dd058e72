/* FP64 gridding step of the FIRM oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Nothing in the product may call this file: only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it (through oracle/gridding.py).
 *
 * Ker (eq. kernel) and A*b (eq. backprojection) are sums over every image m and disc
 * frequency k of a weight times exp(+i <n, xi_{m,k}>), with the slice points
 * xi_{m,k} = R_m^T (2 pi k / N, 0) of eq. forward-projector.  At large N the direct
 * sums cost too much, so the oracle also computes them as a type-1 non-uniform FFT
 * (Dutt & Rokhlin 1993; the paper itself uses Fessler's NUFFT, Section 4).  This file
 * is the first step of that method: every weighted point is spread onto a periodic
 * grid of G points per axis with a separable window,
 *
 *     tau[j] = sum_{m,k} w_{m,k} phi(j1 - u1) phi(j2 - u2) phi(j3 - u3),
 *     u = G xi / (2 pi) = (G / N) (k1 * row 0 of R_m + k2 * row 1 of R_m),
 *
 * where along each axis j runs over the W integers with -W/2 < j - u <= W/2, taken
 * modulo G.  The FFT of tau and the division by the window's Fourier transform are
 * done in oracle/gridding.py with a library FFT.
 *
 * Windows (t in [-W/2, W/2], s = sqrt(1 - (2t/W)^2)):
 *   window 0, Kaiser-Bessel:          phi(t) = I0(beta s)
 *   window 1, exponential of semicircle (Barnett, Magland & af Klinteberg 2019):
 *                                     phi(t) = exp(beta (s - 1))
 * I0 is summed from its power series, sum_q ((x/2)^q / q!)^2.
 *
 * Parallel only by ownership of grid planes: thread t adds just the taps that fall in
 * its own block of z-planes, visiting the points in input order, so every grid value
 * is the same sum in the same order whatever the thread count.  Plain C, FP64. */
#include <math.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* 1 / q^2 for q = 1 .. 199 (a multiply per series term, not a divide), filled by
 * oracle_spread_slices before its threads start */
static double inv_q2[200];

static void fill_inv_q2(void) {
    for (int q = 1; q < 200; ++q) inv_q2[q] = 1.0 / ((double)q * (double)q);
}

static double bessel_i0(double x) {
    const double q2 = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int q = 1; q < 200; ++q) {
        term *= q2 * inv_q2[q];
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

static double window_value(double t, int W, int window, double beta) {
    const double a = 2.0 * t / (double)W;
    const double r = 1.0 - a * a;
    const double s = r > 0.0 ? sqrt(r) : 0.0;
    if (window == 0) return bessel_i0(beta * s);
    return exp(beta * (s - 1.0));
}

/* The first tap index (modulo G) and the W window values of one axis for position u:
 * tap a sits at (first + a) modulo G. */
static int axis_taps(double u, int G, int W, int window, double beta, double* val) {
    const double first = floor(u - 0.5 * W) + 1.0;
    for (int a = 0; a < W; ++a) val[a] = window_value(first + a - u, W, window, beta);
    long long j0 = (long long)first % G;
    if (j0 < 0) j0 += G;
    return (int)j0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Spread the weighted slice points of M images onto tau (added to what it holds).
 *   R        M x 9 rotations, row-major (R_m[i][j] at R[9m + 3i + j])
 *   K        nK x 2 disc frequencies (k1, k2)
 *   N        volume size (the frequencies are 2 pi k / N)
 *   w        weights: M x nK doubles (cplx = 0) or M x nK (re, im) pairs (cplx = 1)
 *   G, W     grid points per axis, window width in grid points (W <= 32)
 *   tau      G^3 doubles (cplx = 0) or G^3 (re, im) pairs, stored [j3][j2][j1]
 * Returns 0, or -1 for arguments out of range. */
int oracle_spread_slices(int M, const double* R, int nK, const int* K, int N, const double* w, int cplx, int G,
                         int W, int window, double beta, int nthreads, double* tau) {
    if (M < 0 || nK < 0 || N <= 0 || G <= 0 || W < 1 || W > 32 || W > G || nthreads < 1) return -1;
    if (window != 0 && window != 1) return -1;
    const double scale = (double)G / (double)N;
    fill_inv_q2();
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
#ifdef _OPENMP
        const int t = omp_get_thread_num(), T = omp_get_num_threads();
#else
        const int t = 0, T = 1;
#endif
        const int z_lo = (int)((long long)G * t / T), z_hi = (int)((long long)G * (t + 1) / T);
        double vx[32], vy[32], vz[32];
        for (int m = 0; m < M; ++m) {
            const double* Rm = R + 9 * (size_t)m;
            for (int p = 0; p < nK; ++p) {
                const double k1 = K[2 * p], k2 = K[2 * p + 1];
                const double u3 = scale * (k1 * Rm[2] + k2 * Rm[5]);
                /* does any z tap of this point fall in this thread's planes? */
                long long z0 = (long long)(floor(u3 - 0.5 * W) + 1.0) % G;
                if (z0 < 0) z0 += G;
                int mine = 0;
                for (int c = 0; c < W && !mine; ++c) {
                    const long long jz = z0 + c < G ? z0 + c : z0 + c - G;
                    mine = (jz >= z_lo && jz < z_hi);
                }
                if (!mine) continue;
                const double u1 = scale * (k1 * Rm[0] + k2 * Rm[3]);
                const double u2 = scale * (k1 * Rm[1] + k2 * Rm[4]);
                const int x0 = axis_taps(u1, G, W, window, beta, vx);
                const int y0 = axis_taps(u2, G, W, window, beta, vy);
                axis_taps(u3, G, W, window, beta, vz);
                /* the x taps are x0 .. x0 + nx - 1 and, past the end of the period,
                 * 0 .. W - nx - 1 */
                const int nx = W < G - x0 ? W : G - x0;
                const size_t q = (size_t)m * nK + p;
                const double wr = cplx ? w[2 * q] : w[q];
                const double wi = cplx ? w[2 * q + 1] : 0.0;
                for (int c = 0; c < W; ++c) {
                    const int jz = (int)(z0 + c < G ? z0 + c : z0 + c - G);
                    if (jz < z_lo || jz >= z_hi) continue;
                    for (int b = 0; b < W; ++b) {
                        const int jy = y0 + b < G ? y0 + b : y0 + b - G;
                        const double f = vz[c] * vy[b];
                        double* row = tau + (cplx ? 2 : 1) * (((size_t)jz * G + jy) * G);
                        if (cplx) {
                            const double fr = f * wr, fi = f * wi;
                            double* r0 = row + 2 * (size_t)x0;
                            for (int a = 0; a < nx; ++a) {
                                r0[2 * a] += vx[a] * fr;
                                r0[2 * a + 1] += vx[a] * fi;
                            }
                            for (int a = nx; a < W; ++a) {
                                row[2 * (a - nx)] += vx[a] * fr;
                                row[2 * (a - nx) + 1] += vx[a] * fi;
                            }
                        } else {
                            const double fr = f * wr;
                            double* r0 = row + x0;
                            for (int a = 0; a < nx; ++a) r0[a] += vx[a] * fr;
                            for (int a = nx; a < W; ++a) row[a - nx] += vx[a] * fr;
                        }
                    }
                }
            }
        }
    }
    return 0;
}
