/*
 * FP64 CPU oracle for the lattice Green's function (LGF) convolution.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code with the CUDA implementation.
 *
 * Everything here is plain, slow and written to be checked against the paper
 * by eye (Liska & Colonius, "A fast lattice Green's function method for
 * solving viscous incompressible flows on unbounded domains"):
 *
 *   - scaled modified Bessel functions  i_n(t) = exp(-2t) I_n(2t)      (App. B)
 *   - the 7-point Laplacian LGF on the unit lattice                      (App. B,
 *       Bessel form of G_L):  G(n) = -int_0^inf prod_i i_{n_i}(t) dt
 *   - the direct convolution u(n) = sum_m G(n-m) f(m)          (Sec. 2.2, eq. dpoisson_conv)
 *   - the integrating-factor convolution with kernel prod_i g_alpha(n_i),
 *       g_alpha(k) = exp(-2 alpha) I_k(2 alpha)               (App. B, eq. lgf_intfac)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------------------
 * Gauss-Legendre rule on [-1, 1]: Newton iteration on the Legendre polynomial
 * P_n, evaluated by its three-term recurrence (Bonnet's formula).
 * ------------------------------------------------------------------------- */
int oracle_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1) return -1;
    for (int i = 0; i < (n + 1) / 2; i++) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double pn = 0.0, pnm1 = 0.0, dp = 1.0;
        for (int it = 0; it < 200; it++) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; k++) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            pn = p0;
            pnm1 = p1;
            dp = n * (z * pn - pnm1) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        /* one more evaluation at the converged z for the weight */
        {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; k++) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Scaled modified Bessel functions of the first kind,
 *     out[n] = exp(-x) I_n(x),  x = 2 t,  n = 0..nmax.
 *
 * Moderate x: Miller's backward recurrence  I_{n-1} = I_{n+1} + (2n/x) I_n,
 * started far above both nmax and the Gaussian width sqrt(x) of n -> I_n(x),
 * and normalised with the generating-function identity
 *     exp(-x) [ I_0(x) + 2 sum_{n>=1} I_n(x) ] = 1.
 * Very large x (x >> nmax^2): the Hankel large-argument series
 *     exp(-x) I_n(x) ~ (2 pi x)^{-1/2} sum_k (-1)^k a_k(n) / x^k,
 *     a_k(n) = prod_{j=1..k} (4 n^2 - (2j-1)^2) / (k! 8^k).
 * ------------------------------------------------------------------------- */
int oracle_bessel_scaled(double t, int nmax, double *out)
{
    if (nmax < 0 || !(t >= 0.0)) return -1;
    const double x = 2.0 * t;
    if (x == 0.0) {
        out[0] = 1.0;
        for (int n = 1; n <= nmax; n++) out[n] = 0.0;
        return 0;
    }
    if (x > 1e8 && 4.0 * (double)nmax * nmax < 1e-3 * x) {
        const double pre = 1.0 / sqrt(2.0 * M_PI * x);
        for (int n = 0; n <= nmax; n++) {
            const double mu = 4.0 * (double)n * n;
            double term = 1.0, sum = 1.0;
            for (int k = 1; k < 60; k++) {
                const double odd = 2.0 * k - 1.0;
                term *= -(mu - odd * odd) / (8.0 * k * x);
                sum += term;
                if (fabs(term) < 1e-20 * fabs(sum)) break;
            }
            out[n] = pre * sum;
        }
        return 0;
    }
    const long nstart = (long)nmax + 40 + (long)(10.0 * sqrt(x)) + 10;
    double bnp1 = 0.0, bn = 1e-280, sum = 0.0, comp = 0.0;
    for (int n = 0; n <= nmax; n++) out[n] = 0.0;
    for (long n = nstart; n >= 1; n--) {
        /* b_n is current; store/accumulate it, then step down to b_{n-1} */
        if (n <= nmax) out[n] = bn;
        {   /* Kahan-compensated sum of 2 b_n */
            double yk = 2.0 * bn - comp;
            double tk = sum + yk;
            comp = (tk - sum) - yk;
            sum = tk;
        }
        const double bnm1 = bnp1 + (2.0 * (double)n / x) * bn;
        bnp1 = bn;
        bn = bnm1;
        if (fabs(bn) > 1e250) {
            const double s = 1e-250;
            bn *= s;
            bnp1 *= s;
            sum *= s;
            comp *= s;
            for (int m = (int)((n - 1 < nmax) ? n - 1 : nmax); m <= nmax; m++) out[m] *= s;
        }
    }
    /* bn now holds b_0 */
    out[0] = bn;
    sum += bn - comp;
    for (int n = 0; n <= nmax; n++) out[n] /= sum;
    return 0;
}

/* index of the sorted octant entry a >= b >= c >= 0 */
static inline int64_t oct_index(int64_t a, int64_t b, int64_t c)
{
    return a * (a + 1) * (a + 2) / 6 + b * (b + 1) / 2 + c;
}

int64_t oracle_octant_size(int K)
{
    return oct_index(K + 1, 0, 0);
}

/* ---------------------------------------------------------------------------
 * Unit-lattice LGF of the 7-point Laplacian on the sorted octant
 * K >= a >= b >= c >= 0 (App. B, Bessel form):
 *     G(a,b,c) = - int_0^inf i_a(t) i_b(t) i_c(t) dt,   i_n(t) = exp(-2t) I_n(2t).
 *
 * Quadrature: substitute t = exp(s); composite Gauss-Legendre in s on
 * [ln t_lo, ln T] with panels of width `panel` and `ngl` nodes each.  The
 * piece [0, t_lo] is below 1e-17 and dropped.  The piece [T, inf) is added in
 * closed form from the large-argument series truncated after its 1/t term:
 *     prod_i i_{n_i}(t) ~ (4 pi t)^{-3/2} [1 - sum_i (4 n_i^2 - 1)/(16 t)],
 *     int_T^inf ... dt = (4 pi)^{-3/2} [ 2 T^{-1/2} - (2/3) c1 T^{-3/2} ],
 *     c1 = sum_i (4 n_i^2 - 1) / 16.
 * Output: out[oct_index(a,b,c)], oracle_octant_size(K) doubles.
 * ------------------------------------------------------------------------- */
int oracle_lgf_octant(int K, double t_lo, double T, double panel, int ngl, double *out)
{
    if (K < 0 || ngl < 2 || ngl > 64 || !(panel > 0.0) || !(T > t_lo) || !(t_lo > 0.0)) return -1;
    double xg[64], wg[64];
    oracle_gauss_legendre(ngl, xg, wg);
    const double s0 = log(t_lo), s1 = log(T);
    const int npan = (int)ceil((s1 - s0) / panel);
    const double h = (s1 - s0) / npan;
    const long nq = (long)npan * ngl;
    double *wt = (double *)malloc(sizeof(double) * nq);
    double *bes = (double *)malloc(sizeof(double) * nq * (K + 1));
    if (!wt || !bes) { free(wt); free(bes); return -2; }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (long q = 0; q < nq; q++) {
        const int p = (int)(q / ngl), g = (int)(q % ngl);
        const double s = s0 + h * (p + 0.5 * (xg[g] + 1.0));
        const double t = exp(s);
        wt[q] = 0.5 * h * wg[g] * t; /* dt = t ds */
        bad |= oracle_bessel_scaled(t, K, bes + q * (K + 1)) != 0;
    }
    if (bad) { free(wt); free(bes); return -3; }
    const double c4pi = pow(4.0 * M_PI, -1.5);
#pragma omp parallel for schedule(dynamic, 1)
    for (int a = K; a >= 0; a--) {
        for (int b = 0; b <= a; b++) {
            for (int c = 0; c <= b; c++) {
                double sum = 0.0, comp = 0.0;
                for (long q = 0; q < nq; q++) {
                    const double *bq = bes + q * (K + 1);
                    double yk = wt[q] * bq[a] * bq[b] * bq[c] - comp;
                    double tk = sum + yk;
                    comp = (tk - sum) - yk;
                    sum = tk;
                }
                const double c1 = ((4.0 * a * a - 1.0) + (4.0 * b * b - 1.0) + (4.0 * c * c - 1.0)) / 16.0;
                const double tail = c4pi * (2.0 / sqrt(T) - (2.0 / 3.0) * c1 * pow(T, -1.5));
                out[oct_index(a, b, c)] = -(sum + tail);
            }
        }
    }
    free(wt);
    free(bes);
    return 0;
}

/* G at an explicit list of offsets (a_i, b_i, c_i) (any signs), same
 * quadrature and tail as oracle_lgf_octant; for offsets too large for a
 * dense table.  nmax must be >= every |offset|. */
int oracle_lgf_points(int64_t n, const int32_t *abc, int nmax, double t_lo, double T, double panel, int ngl,
                      double *out)
{
    if (nmax < 0 || ngl < 2 || ngl > 64 || !(panel > 0.0) || !(T > t_lo) || !(t_lo > 0.0)) return -1;
    double xg[64], wg[64];
    oracle_gauss_legendre(ngl, xg, wg);
    const double s0 = log(t_lo), s1 = log(T);
    const int npan = (int)ceil((s1 - s0) / panel);
    const double h = (s1 - s0) / npan;
    const long nq = (long)npan * ngl;
    double *wt = (double *)malloc(sizeof(double) * nq);
    double *bes = (double *)malloc(sizeof(double) * nq * (nmax + 1));
    if (!wt || !bes) { free(wt); free(bes); return -2; }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (long q = 0; q < nq; q++) {
        const int p = (int)(q / ngl), g = (int)(q % ngl);
        const double t = exp(s0 + h * (p + 0.5 * (xg[g] + 1.0)));
        wt[q] = 0.5 * h * wg[g] * t;
        bad |= oracle_bessel_scaled(t, nmax, bes + q * (nmax + 1)) != 0;
    }
    const double c4pi = pow(4.0 * M_PI, -1.5);
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < n; i++) {
        const int a = abs(abc[3 * i]), b = abs(abc[3 * i + 1]), c = abs(abc[3 * i + 2]);
        if (a > nmax || b > nmax || c > nmax) { bad = 1; continue; }
        double sum = 0.0, comp = 0.0;
        for (long q = 0; q < nq; q++) {
            const double *bq = bes + q * (nmax + 1);
            double yk = wt[q] * bq[a] * bq[b] * bq[c] - comp;
            double tk = sum + yk;
            comp = (tk - sum) - yk;
            sum = tk;
        }
        const double c1 = ((4.0 * a * a - 1.0) + (4.0 * b * b - 1.0) + (4.0 * c * c - 1.0)) / 16.0;
        out[i] = -(sum + c4pi * (2.0 / sqrt(T) - (2.0 / 3.0) * c1 * pow(T, -1.5)));
    }
    free(wt);
    free(bes);
    return bad ? -3 : 0;
}

/* Expand an octant table into the dense cube D[z][y][x] = G(x, y, z),
 * 0 <= x, y, z <= K (the LGF is even in each coordinate and symmetric under
 * permutations, App. B). */
int oracle_octant_to_cube(int K, const double *oct, double *cube)
{
    const int64_t n = K + 1;
#pragma omp parallel for schedule(static)
    for (int z = 0; z <= K; z++)
        for (int y = 0; y <= K; y++)
            for (int x = 0; x <= K; x++) {
                int a = x, b = y, c = z, tmp;
                if (a < b) { tmp = a; a = b; b = tmp; }
                if (b < c) { tmp = b; b = c; c = tmp; }
                if (a < b) { tmp = a; a = b; b = tmp; }
                cube[((int64_t)z * n + y) * n + x] = oct[oct_index(a, b, c)];
            }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Direct convolution (Sec. 2.2, eq. dpoisson_conv):
 *     out[j] = sum_i cube(|t_j - s_i|) * val[i]
 * over an explicit list of source points s_i with values val[i] and target
 * points t_j.  cube is the dense (K+1)^3 table of the kernel indexed
 * [|dz|][|dy|][|dx|]; every |d| must be <= K (checked: returns -1).
 * Kahan-compensated accumulation per target.
 * ------------------------------------------------------------------------- */
int oracle_direct_conv(int K, const double *cube, int64_t nsrc, const int32_t *src_xyz,
                       const double *val, int64_t ntgt, const int32_t *tgt_xyz, double *out)
{
    const int64_t n = K + 1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int64_t j = 0; j < ntgt; j++) {
        const int32_t tx = tgt_xyz[3 * j], ty = tgt_xyz[3 * j + 1], tz = tgt_xyz[3 * j + 2];
        double sum = 0.0, comp = 0.0;
        for (int64_t i = 0; i < nsrc; i++) {
            const int dx = abs(tx - src_xyz[3 * i]);
            const int dy = abs(ty - src_xyz[3 * i + 1]);
            const int dz = abs(tz - src_xyz[3 * i + 2]);
            if (dx > K || dy > K || dz > K) { bad = 1; continue; }
            double yk = cube[((int64_t)dz * n + dy) * n + dx] * val[i] - comp;
            double tk = sum + yk;
            comp = (tk - sum) - yk;
            sum = tk;
        }
        out[j] = sum;
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------------
 * Integrating factor as a plain 3-D sum (App. B eq. lgf_intfac, Sec. 4.4):
 *     y(n) = sum_{m : |n_i - m_i| <= R, m in mask} g[|n1-m1|] g[|n2-m2|] g[|n3-m3|] x(m)
 * on a dense box x[z][y][x] of size nx*ny*nz with zeros outside the box;
 * g[0..R] are the 1-D factors.  Only targets listed in tgt_xyz are evaluated.
 * The source mask is applied by the caller (x already zero outside it).
 * ------------------------------------------------------------------------- */
int oracle_ifactor_direct(int R, const double *g, int nx, int ny, int nz, const double *x,
                          int64_t ntgt, const int32_t *tgt_xyz, double *out)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < ntgt; j++) {
        const int tx = tgt_xyz[3 * j], ty = tgt_xyz[3 * j + 1], tz = tgt_xyz[3 * j + 2];
        double sum = 0.0, comp = 0.0;
        for (int dz = -R; dz <= R; dz++) {
            const int z = tz - dz;
            if (z < 0 || z >= nz) continue;
            for (int dy = -R; dy <= R; dy++) {
                const int y = ty - dy;
                if (y < 0 || y >= ny) continue;
                for (int dx = -R; dx <= R; dx++) {
                    const int xx = tx - dx;
                    if (xx < 0 || xx >= nx) continue;
                    const double w = g[abs(dx)] * g[abs(dy)] * g[abs(dz)];
                    double yk = w * x[((int64_t)z * ny + y) * nx + xx] - comp;
                    double tk = sum + yk;
                    comp = (tk - sum) - yk;
                    sum = tk;
                }
            }
        }
        out[j] = sum;
    }
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
