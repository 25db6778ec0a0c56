// Device FP64 tables of the two lattice kernels (App. B).
//
// 7-point Laplacian LGF on the unit lattice (Bessel form of App. B):
//     G(a,b,c) = - int_0^inf  i_a(t) i_b(t) i_c(t) dt,   i_n(t) = e^{-2t} I_n(2t),
// tabulated on the sorted octant K >= a >= b >= c >= 0.  The integral is taken
// in the variable s = ln t by composite Gauss-Legendre on [ln T_LO, ln T_HI];
// beyond T_HI the large-argument behaviour of the scaled Bessel functions,
//     prod_i i_{n_i}(t) = (4 pi t)^{-3/2} (1 - sum_i (4 n_i^2 - 1)/(16 t) + O(t^-2)),
// is integrated in closed form; below T_LO the integrand is < T_LO.
//
// Scaled Bessel values at each node: for x = 2t up to X_HANKEL, Miller's
// backward recurrence I_{n-1} = I_{n+1} + (2n/x) I_n started well above the
// Gaussian width sqrt(x) of n -> I_n(x), normalised by e^{-x}(I_0 + 2 sum I_n) = 1;
// beyond that, the Hankel series e^{-x} I_n(x) ~ (2 pi x)^{-1/2} sum_k (-1)^k a_k(n)/x^k.
//
// Integrating factor: g(k) = e^{-2 alpha} I_k(2 alpha) (eq. lgf_intfac), k <= R,
// R the largest k with g(k) g(0)^2 >= tol (the 3-D kernel along an axis).
#include <cmath>
#include <vector>

#include "plan.hpp"

namespace lgf {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double T_LO = 1e-19;
constexpr double T_HI = 1e13;
constexpr double PANEL = 0.8;   // width of a panel in ln t
constexpr int NGL = 20;          // Gauss-Legendre nodes per panel
constexpr double X_HANKEL = 2e8; // x = 2t above which the Hankel series is used

// Gauss-Legendre nodes on [-1, 1]: roots of P_n by Newton's method from the
// Tricomi initial guesses, weights 2 / ((1 - x^2) P_n'(x)^2).
void gauss_legendre_rule(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 1; i <= n; i++) {
        const double th = kPi * (4.0 * i - 1.0) / (4.0 * n + 2.0);
        double r = std::cos(th) * (1.0 - (n - 1.0) / (8.0 * n * n * n));
        double dp = 0.0;
        for (int iter = 0; iter < 100; iter++) {
            double p0 = 1.0, p1 = r;  // P_0, P_1
            for (int k = 2; k <= n; k++) {
                const double p2 = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            // p1 = P_n(r), p0 = P_{n-1}(r)
            dp = n * (p0 - r * p1) / (1.0 - r * r);
            const double step = p1 / dp;
            r -= step;
            if (std::fabs(step) <= 1e-16 * std::fabs(r) + 1e-300) {
                double q0 = 1.0, q1 = r;
                for (int k = 2; k <= n; k++) {
                    const double q2 = ((2.0 * k - 1.0) * r * q1 - (k - 1.0) * q0) / k;
                    q0 = q1;
                    q1 = q2;
                }
                dp = n * (q0 - r * q1) / (1.0 - r * r);
                break;
            }
        }
        x[i - 1] = r;
        w[i - 1] = 2.0 / ((1.0 - r * r) * dp * dp);
    }
}

// Scaled Bessel functions e^{-x} I_n(x), n = 0..nmax, written to out[n * stride].
__device__ void scaled_bessel(double x, int nmax, double *out, int stride)
{
    if (x <= 0.0) {
        out[0] = 1.0;
        for (int n = 1; n <= nmax; n++) out[n * stride] = 0.0;
        return;
    }
    if (x > X_HANKEL && 4.0 * nmax * (double)nmax < 1e-3 * x) {
        const double pre = rsqrt(2.0 * kPi * x);
        for (int n = 0; n <= nmax; n++) {
            const double mu = 4.0 * n * (double)n;
            double term = 1.0, sum = 1.0;
            for (int k = 1; k < 40; k++) {
                const double o = 2.0 * k - 1.0;
                term *= -(mu - o * o) / (8.0 * k * x);
                sum += term;
                if (fabs(term) < 1e-19 * fabs(sum)) break;
            }
            out[n * stride] = pre * sum;
        }
        return;
    }
    const int top = nmax + 32 + (int)(12.0 * sqrt(x));
    for (int n = 0; n <= nmax; n++) out[n * stride] = 0.0;
    double hi = 0.0, cur = 1e-300, norm = 0.0;
    for (int n = top; n >= 1; n--) {
        if (n <= nmax) out[n * stride] = cur;
        norm += 2.0 * cur;
        const double lo = hi + (2.0 * n / x) * cur;
        hi = cur;
        cur = lo;
        if (cur > 1e240) {
            hi *= 1e-240;
            cur *= 1e-240;
            norm *= 1e-240;
            const int from = (n - 1 < nmax) ? (n - 1) : nmax;
            for (int m = from; m <= nmax; m++) out[m * stride] *= 1e-240;
        }
    }
    norm += cur;
    out[0] = cur;
    const double inv = 1.0 / norm;
    for (int n = 0; n <= nmax; n++) out[n * stride] *= inv;
}

// one thread per quadrature node: bes[q * (K + 1) + n] = i_n(t_q)
__global__ void k_nodes(const double *__restrict__ tq, int nq, int K, double *__restrict__ bes)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    scaled_bessel(2.0 * tq[q], K, bes + (size_t)q * (K + 1), 1);
}

// one block per leading index a; threads over the (b, c) pairs with a >= b >= c.
// Entry (a, b, c) samples the lattice offset stride * (a, b, c): bes rows hold
// i_n(t_q) for n = 0 .. nrow - 1.  tail: add the closed-form integral beyond T_hi.
__global__ void k_octant(const double *__restrict__ bes, const double *__restrict__ wq, int nq, int nrow, int stride,
                         double *__restrict__ out, double T_hi, int tail)
{
    const int a = blockIdx.x;
    const int npairs = (a + 1) * (a + 2) / 2;
    const double c4 = 1.0 / ((4.0 * kPi) * sqrt(4.0 * kPi));
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
        int b = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
        while ((b + 1) * (b + 2) / 2 <= p) b++;
        while (b * (b + 1) / 2 > p) b--;
        const int c = p - b * (b + 1) / 2;
        const int na = stride * a, nb = stride * b, nc = stride * c;
        double acc = 0.0;
        for (int q = 0; q < nq; q++) {
            const double *row = bes + (size_t)q * nrow;
            acc = fma(wq[q] * row[na], row[nb] * row[nc], acc);
        }
        double tl = 0.0;
        if (tail) {
            const double c1 = ((4.0 * na * (double)na - 1.0) + (4.0 * nb * (double)nb - 1.0) +
                               (4.0 * nc * (double)nc - 1.0)) / 16.0;
            tl = c4 * (2.0 / sqrt(T_hi) - (2.0 / 3.0) * c1 / (T_hi * sqrt(T_hi)));
        }
        const int64_t idx = (int64_t)a * (a + 1) * (a + 2) / 6 + (int64_t)b * (b + 1) / 2 + c;
        out[idx] = -(acc + tl);
    }
}

__global__ void k_if_taps(double alpha, int maxr, double tol, double *__restrict__ taps, int *__restrict__ R_out,
                          double *__restrict__ scratch)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    scaled_bessel(2.0 * alpha, maxr, scratch, 1);
    const double g0 = scratch[0];
    int R = 0;
    while (R + 1 <= maxr && scratch[R + 1] * g0 * g0 >= tol) R++;
    for (int k = 0; k <= maxr; k++) taps[k] = k <= R ? scratch[k] : 0.0;
    *R_out = R;
}

}  // namespace

lgf_status build_lgf_octant(int K, double *d_out, cudaStream_t s)
{
    return build_lgf_octant_part(K, 1, 0.0, 0.0, d_out, s);
}

// Part of the t-integral of the Bessel form: -int_{t0}^{t1} prod_i i_{n_i}(t) dt, with
// t0 = 0 read as T_LO (the integrand is < T_LO below it) and t1 = 0 read as infinity
// (Gauss-Legendre up to T_HI plus the closed-form tail), at the offsets stride * (a, b, c)
// of the sorted octant K >= a >= b >= c >= 0.
lgf_status build_lgf_octant_part(int K, int stride, double t0, double t1, double *d_out, cudaStream_t s)
{
    std::vector<double> xg, wg;
    gauss_legendre_rule(NGL, xg, wg);
    const bool tail = !(t1 > 0.0);
    const double s0 = std::log(t0 > T_LO ? t0 : T_LO), s1 = std::log(tail ? T_HI : t1);
    const int npan = (int)std::ceil((s1 - s0) / PANEL);
    const double h = (s1 - s0) / npan;
    const int nq = npan * NGL;
    std::vector<double> tq(nq), wq(nq);
    for (int p = 0; p < npan; p++)
        for (int g = 0; g < NGL; g++) {
            const double sv = s0 + h * (p + 0.5 * (xg[g] + 1.0));
            const double t = std::exp(sv);
            tq[p * NGL + g] = t;
            wq[p * NGL + g] = 0.5 * h * wg[g] * t;
        }
    double *d_t = nullptr, *d_w = nullptr, *d_bes = nullptr;
    lgf_status st = LGF_OK;
    const int nrow = stride * K + 1;
    if (cudaMalloc(&d_t, nq * sizeof(double)) != cudaSuccess || cudaMalloc(&d_w, nq * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&d_bes, (size_t)nq * nrow * sizeof(double)) != cudaSuccess) {
        set_error("table workspace allocation failed");
        st = LGF_ERR_OOM;
    }
    if (st == LGF_OK && (cudaMemcpyAsync(d_t, tq.data(), nq * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                         cudaMemcpyAsync(d_w, wq.data(), nq * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)) {
        set_error("table upload failed");
        st = LGF_ERR_CUDA;
    }
    if (st == LGF_OK) {
        k_nodes<<<(nq + 63) / 64, 64, 0, s>>>(d_t, nq, nrow - 1, d_bes);
        k_octant<<<K + 1, 256, 0, s>>>(d_bes, d_w, nq, nrow, stride, d_out, T_HI, tail ? 1 : 0);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("LGF table kernels failed: %s", cudaGetErrorString(e));
            st = LGF_ERR_CUDA;
        }
    }
    cudaFree(d_t);
    cudaFree(d_w);
    cudaFree(d_bes);
    return st;
}

lgf_status build_if_taps(double alpha, double tol, double *d_taps, int max_r, int *R_out, cudaStream_t s)
{
    double *scratch = nullptr;
    int *d_R = nullptr;
    lgf_status st = LGF_OK;
    if (cudaMalloc(&scratch, (max_r + 1) * sizeof(double)) != cudaSuccess || cudaMalloc(&d_R, sizeof(int)) != cudaSuccess) {
        set_error("taps workspace allocation failed");
        st = LGF_ERR_OOM;
    }
    if (st == LGF_OK) {
        k_if_taps<<<1, 1, 0, s>>>(alpha, max_r, tol, d_taps, d_R, scratch);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(R_out, d_R, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("IF taps kernel failed: %s", cudaGetErrorString(e));
            st = LGF_ERR_CUDA;
        }
    }
    cudaFree(scratch);
    cudaFree(d_R);
    return st;
}

}  // namespace lgf
