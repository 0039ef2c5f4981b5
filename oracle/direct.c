/*
 * FP64 direct-sum oracle for the Gaussian-regularised Biot-Savart velocity and the
 * vortex-stretching term of a periodic vortex-particle system.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this library.  It shares no code, header or table with the GPU path.
 *
 * Definitions followed (the plain O(N^2) sum, no approximation):
 *   - Eq. (biotsavart): u_i = sum_j gamma_j x grad(G g_sigma), G = 1/(4 pi r).  Written out,
 *     u_i = sum_n sum_j' K(r) gamma_j x r with r = x_i - x_j - n L.
 *   - Eq. (cutoff): q(rho) = erf(rho/sqrt 2) - sqrt(2/pi) rho exp(-rho^2/2), rho = |r|/sigma,
 *     which equals sqrt(2/pi) * int_0^rho s^2 exp(-s^2/2) ds (the Gaussian's enclosed fraction).
 *     K(r) = q(rho) / (4 pi |r|^3).
 *   - Eq. (stretching), read as the classical (gamma_i . grad) u evaluated at x_i:
 *     S_i = sum_n sum_j' [ K gamma_j x gamma_i + F (gamma_i . r)(gamma_j x r) ],
 *     F = K'(|r|)/|r| = [ sqrt(2/pi) exp(-rho^2/2)/(sigma^3 |r|^2) - 3 q/|r|^5 ] / (4 pi).
 *   - Periodic images (Section 4.1, "3^3 x 3^3 x 3^3 - 1" images): a cube of image boxes
 *     n in {-K..K}^3 around the primary box; K = 1 is 27 boxes, K = 13 is 27^3 boxes.
 *   - sum' skips the self pair (j = i, n = 0), which contributes exactly zero anyway.  Any
 *     other pair at r = 0 (coincident distinct particles) takes the finite r -> 0 limit of
 *     the smoothed kernel: K(0) = sqrt(2/pi)/(12 pi sigma^3), F(0) = -sqrt(2/pi)/(20 pi sigma^5).
 *
 * Optional output G (3x3 per target, row a, column k) is the velocity gradient
 * du_a/dx_k = sum eps_abc gamma_jb (K delta_ck + F r_c r_k), used by the gradient oracle.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* q(rho): for rho < 0.5 the integral's power series (term k: (-1)^k rho^(2k+3)/(2^k k! (2k+3))),
 * otherwise the closed form with erf. Both are the definition in Eq. (cutoff). */
static double oracle_q(double rho)
{
    const double c = sqrt(2.0 / ORACLE_PI);
    if (rho < 0.5) {
        double rho2 = rho * rho, pw = rho * rho2, fact = 1.0, sum = 0.0;
        for (int k = 0; k < 30; ++k) {
            double term = pw / (fact * (2.0 * k + 3.0));
            sum += (k & 1) ? -term : term;
            if (term < 1e-20 * fabs(sum)) break;
            pw *= rho2;
            fact *= 2.0 * (k + 1);
        }
        return c * sum;
    }
    return erf(rho / sqrt(2.0)) - c * rho * exp(-0.5 * rho * rho);
}

double oracle_cutoff_q(double rho) { return oracle_q(rho); }

/* Levi-Civita symbol eps_abc. */
static inline int levi_civita(int a, int b, int c)
{
    return ((a - b) * (b - c) * (c - a)) / 2;
}

/* Add the contribution of one source (position already shifted by its image) to a target. */
static inline void pair(const double xt[3], const double gt[3], const double xs[3], const double gs[3],
                        double sigma, double u[3], double S[3], double G[9])
{
    double r[3] = {xt[0] - xs[0], xt[1] - xs[1], xt[2] - xs[2]};
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rr = sqrt(r2);
    double rho = rr / sigma;
    double K, F;
    if (rho < 0.5) {
        /* K = k(rho)/(4 pi sigma^3), F = f(rho)/(4 pi sigma^5) with k = q/rho^3 and
         * f = k'(rho)/rho from the same integral series; finite at r = 0 (the smoothed
         * kernel of two coincident distinct particles). */
        double x = rho * rho, xp = 1.0, xm1 = 1.0, fact = 1.0, k = 0.0, f = 0.0;
        for (int q = 0; q < 30; ++q) {
            double den = fact * (2.0 * q + 3.0);
            k += (q & 1) ? -xp / den : xp / den;
            if (q >= 1) f += (q & 1) ? -2.0 * q * xm1 / den : 2.0 * q * xm1 / den;
            xm1 = xp;
            xp *= x;
            fact *= 2.0 * (q + 1);
        }
        double c = sqrt(2.0 / ORACLE_PI);
        K = c * k / (4.0 * ORACLE_PI * sigma * sigma * sigma);
        F = c * f / (4.0 * ORACLE_PI * sigma * sigma * sigma * sigma * sigma);
    } else {
        double q = oracle_q(rho);
        K = q / (4.0 * ORACLE_PI * rr * r2);
        F = (sqrt(2.0 / ORACLE_PI) * exp(-0.5 * rho * rho) / (sigma * sigma * sigma * r2)
             - 3.0 * q / (r2 * r2 * rr)) / (4.0 * ORACLE_PI);
    }
    double W[3] = {gs[1] * r[2] - gs[2] * r[1], gs[2] * r[0] - gs[0] * r[2], gs[0] * r[1] - gs[1] * r[0]};
    double X[3] = {gs[1] * gt[2] - gs[2] * gt[1], gs[2] * gt[0] - gs[0] * gt[2], gs[0] * gt[1] - gs[1] * gt[0]};
    double gr = gt[0] * r[0] + gt[1] * r[1] + gt[2] * r[2];
    for (int a = 0; a < 3; ++a) {
        u[a] += K * W[a];
        S[a] += K * X[a] + F * gr * W[a];
    }
    if (G) {
        /* du_a/dx_k = eps_abc gs_b (K delta_ck + F r_c r_k) = K eps_abk gs_b + F W_a r_k */
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 3; ++k) {
                double epsterm = 0.0;
                for (int b = 0; b < 3; ++b) epsterm += levi_civita(a, b, k) * gs[b];
                G[3 * a + k] += K * epsterm + F * W[a] * r[k];
            }
    }
}

/*
 * Direct sum at nt targets from ns sources with image boxes n, kmin <= max|n_i| <= kmax.
 * xs, gs: ns x 3 source positions and strengths.  xt, gt: nt x 3 target positions and the
 * target strengths used by the stretching term.  tidx[i] is the source index of target i
 * (excluded at n = 0) or -1.  u, S: nt x 3 outputs (overwritten).  G: nt x 9 or NULL.
 * nthreads <= 0 uses the OpenMP default.
 */
void oracle_direct(int64_t ns, const double *xs, const double *gs,
                   int64_t nt, const double *xt, const double *gt, const int64_t *tidx,
                   double sigma, double L, int kmin, int kmax,
                   double *u, double *S, double *G, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < nt; ++i) {
        double ui[3] = {0, 0, 0}, Si[3] = {0, 0, 0}, Gi[9] = {0};
        const double *x0 = xt + 3 * i, *g0 = gt + 3 * i;
        for (int nx = -kmax; nx <= kmax; ++nx)
            for (int ny = -kmax; ny <= kmax; ++ny)
                for (int nz = -kmax; nz <= kmax; ++nz) {
                    int m = abs(nx); if (abs(ny) > m) m = abs(ny); if (abs(nz) > m) m = abs(nz);
                    if (m < kmin) continue;
                    int primary = (nx == 0 && ny == 0 && nz == 0);
                    for (int64_t j = 0; j < ns; ++j) {
                        if (primary && tidx && tidx[i] == j) continue;
                        double xsj[3] = {xs[3 * j] + nx * L, xs[3 * j + 1] + ny * L, xs[3 * j + 2] + nz * L};
                        pair(x0, g0, xsj, gs + 3 * j, sigma, ui, Si, G ? Gi : NULL);
                    }
                }
        for (int a = 0; a < 3; ++a) { u[3 * i + a] = ui[a]; S[3 * i + a] = Si[a]; }
        if (G) for (int a = 0; a < 9; ++a) G[9 * i + a] = Gi[a];
    }
}

/*
 * The same image-cube sum restricted to the image boxes kmin <= max|n_i| <= kmax with
 * kmin >= 2, for the case where every such pair is at least 10 sigma apart
 * ((kmin - 1) L >= 10 sigma for positions in [0, L)^3).  There q(rho) of Eq. (cutoff) is 1 in
 * FP64 (1 - q(10) < 2e-21) and the Gaussian term of F is below 1e-19 of the 3q/r^5 term, so
 * the definition reduces exactly (to FP64 rounding) to the singular Biot-Savart kernel
 * K = 1/(4 pi r^3), F = -3 K / r^2.  This is the far-image increment of Section 4.1's
 * 3^3 x 3^3 x 3^3 image cube beyond the central 27 boxes.  Targets xt, gt (nt x 3) are
 * positions and strengths, none of them a source of the primary box (n = 0 is excluded).
 * The work is split over image boxes; each thread sums its boxes into its own partial
 * sums, which are added at the end.  u, S: nt x 3 outputs (overwritten).
 * Returns 0, or -1 if the distance condition does not hold (nothing is computed).
 */
int oracle_far_images(int64_t ns, const double *xs, const double *gs,
                      int64_t nt, const double *xt, const double *gt,
                      double sigma, double L, int kmin, int kmax,
                      double *u, double *S, int nthreads)
{
    if (kmin < 2 || kmax < kmin || (kmin - 1) * L < 10.0 * sigma) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    (void)nthreads;
    const double c4pi = 1.0 / (4.0 * ORACLE_PI);
    /* structure-of-arrays copies of the sources */
    double *sx = (double *)malloc(sizeof(double) * 6 * (size_t)ns);
    if (!sx) return -1;
    double *sy = sx + ns, *sz = sy + ns, *ga = sz + ns, *gb = ga + ns, *gc = gb + ns;
    for (int64_t j = 0; j < ns; ++j) {
        sx[j] = xs[3 * j]; sy[j] = xs[3 * j + 1]; sz[j] = xs[3 * j + 2];
        ga[j] = gs[3 * j]; gb[j] = gs[3 * j + 1]; gc[j] = gs[3 * j + 2];
    }
    /* the image boxes of the shell */
    int side = 2 * kmax + 1;
    int *boxes = (int *)malloc(sizeof(int) * 3 * (size_t)side * side * side);
    if (!boxes) { free(sx); return -1; }
    int nb = 0;
    for (int nx = -kmax; nx <= kmax; ++nx)
        for (int ny = -kmax; ny <= kmax; ++ny)
            for (int nz = -kmax; nz <= kmax; ++nz) {
                int m = abs(nx); if (abs(ny) > m) m = abs(ny); if (abs(nz) > m) m = abs(nz);
                if (m < kmin) continue;
                boxes[3 * nb] = nx; boxes[3 * nb + 1] = ny; boxes[3 * nb + 2] = nz;
                ++nb;
            }
    for (int64_t i = 0; i < 3 * nt; ++i) { u[i] = 0.0; S[i] = 0.0; }
#pragma omp parallel
    {
        double *acc = (double *)calloc(6 * (size_t)nt, sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (int b = 0; b < nb; ++b) {
            const double shx = boxes[3 * b] * L, shy = boxes[3 * b + 1] * L, shz = boxes[3 * b + 2] * L;
            for (int64_t i = 0; i < nt; ++i) {
                /* r = x_i - (x_j + n L) */
                const double tx = xt[3 * i] - shx, ty = xt[3 * i + 1] - shy, tz = xt[3 * i + 2] - shz;
                const double t0 = gt[3 * i], t1 = gt[3 * i + 1], t2 = gt[3 * i + 2];
                double u0 = 0, u1 = 0, u2 = 0, s0 = 0, s1 = 0, s2 = 0;
#pragma omp simd reduction(+ : u0, u1, u2, s0, s1, s2)
                for (int64_t j = 0; j < ns; ++j) {
                    double r0 = tx - sx[j], r1 = ty - sy[j], r2 = tz - sz[j];
                    double rr2 = r0 * r0 + r1 * r1 + r2 * r2;
                    double rinv = 1.0 / sqrt(rr2);
                    double K = rinv * rinv * rinv;
                    double F = -3.0 * K * rinv * rinv;
                    double w0 = gb[j] * r2 - gc[j] * r1, w1 = gc[j] * r0 - ga[j] * r2, w2 = ga[j] * r1 - gb[j] * r0;
                    double fg = F * (t0 * r0 + t1 * r1 + t2 * r2);
                    u0 += K * w0; u1 += K * w1; u2 += K * w2;
                    s0 += K * (gb[j] * t2 - gc[j] * t1) + fg * w0;
                    s1 += K * (gc[j] * t0 - ga[j] * t2) + fg * w1;
                    s2 += K * (ga[j] * t1 - gb[j] * t0) + fg * w2;
                }
                acc[6 * i] += u0; acc[6 * i + 1] += u1; acc[6 * i + 2] += u2;
                acc[6 * i + 3] += s0; acc[6 * i + 4] += s1; acc[6 * i + 5] += s2;
            }
        }
#pragma omp critical
        for (int64_t i = 0; i < nt; ++i)
            for (int a = 0; a < 3; ++a) {
                u[3 * i + a] += c4pi * acc[6 * i + a];
                S[3 * i + a] += c4pi * acc[6 * i + 3 + a];
            }
        free(acc);
    }
    free(boxes);
    free(sx);
    return 0;
}
