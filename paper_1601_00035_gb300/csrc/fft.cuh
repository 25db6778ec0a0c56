// 1-D complex FFTs of length N = 2^k (16..1024), 3 * 2^k (96, 192, 384, 768),
// 288 = 9 * 2^5 or 432 = 27 * 2^4 with the data held in registers, for batches
// of lines processed by one thread block.  In-register DFTs have lengths 2^k,
// 3 * 2^k (dividing 48) or 9 * 2^k (dividing 36).
//
// A line is transformed by G lanes (threads); lane j holds E = N / G elements.
// Algorithm: Stockham autosort, mixed radix R_0 .. R_{S-1} (product N).  In
// stage s (span L = R_0 ... R_{s-1}) butterfly jb reads the elements at
// positions jb + m N/R_s (m < R_s), multiplies element m by w_{R_s L}^{m (jb mod L)},
// takes a length-R_s DFT and writes output q to position
// (jb div L) R_s L + q L + (jb mod L).  Lane j owns butterflies jb = j + b G,
// b < E / R_s, and keeps them in registers as v[b R_s + m].
//
// Between stages the elements move once through shared memory (write at the
// output positions, barrier, read at the next input positions, barrier).
// Before the first stage the caller loads v[b R_0 + m] = x[jb + m N/R_0]
// directly; after the last stage v[b R + q] holds X[jb + q N/R] (R = R_{S-1}),
// which is exactly the input layout of an inverse transform whose first
// radix is R: a forward transform, a pointwise multiply and an inverse
// transform (radices reversed) therefore chain in registers.  Forward uses
// w = exp(-2 pi i/N), inverse the conjugate (unnormalised).
#pragma once
#include <cmath>
#include <type_traits>

#include "common.cuh"

namespace lgf {
namespace fft {

// w_64^j = exp(-2 pi i j / 64) for the in-register DFTs (indices are compile-time
// constants after unrolling, so these are uniform constant-bank loads).
// (static: each translation unit that includes this header owns and uploads
// its own copy with upload_tw64())
static __constant__ float2 c_tw64f[64];
static __constant__ double2 c_tw64d[64];

static inline cudaError_t upload_tw64()
{
    static thread_local int done_mask = 0;  // bit per device (up to 32 devices)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 32 && (done_mask >> dev) & 1) return cudaSuccess;
    float2 hf[64];
    double2 hd[64];
    for (int j = 0; j < 64; j++) {
        const double a = -2.0 * 3.14159265358979323846 * j / 64.0;
        hd[j] = make_double2(cos(a), sin(a));
        hf[j] = make_float2((float)hd[j].x, (float)hd[j].y);
    }
    e = cudaMemcpyToSymbol(c_tw64f, hf, sizeof(hf));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tw64d, hd, sizeof(hd));
    if (e == cudaSuccess && dev < 32) done_mask |= 1 << dev;
    return e;
}

template <typename T>
__device__ __forceinline__ cx<T> tw64(int j);
template <>
__device__ __forceinline__ cx<float> tw64<float>(int j)
{
    float2 w = c_tw64f[j];
    return {w.x, w.y};
}
template <>
__device__ __forceinline__ cx<double> tw64<double>(int j)
{
    double2 w = c_tw64d[j];
    return {w.x, w.y};
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
__host__ __device__ constexpr int bitrev(int i, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; b++) r = (r << 1) | ((i >> b) & 1);
    return r;
}

// multiply v by w_len^k (conjugated for the inverse); k, len compile-time
template <bool INV, typename T>
__device__ __forceinline__ cx<T> twiddle_len(cx<T> v, int k, int len)
{
    if (k == 0) return v;
    if (4 * k == len) {  // w = -i (forward) or +i (inverse)
        return INV ? cx<T>{-v.y, v.x} : cx<T>{v.y, -v.x};
    }
    if (8 * k == len || 8 * k == 3 * len) {
        // w = h (s - i) forward, h (s + i) inverse, h = 1/sqrt2, s = +1 (k = len/8) or -1 (k = 3 len/8)
        const T h = (T)0.70710678118654752440;
        const T s = (8 * k == len) ? (T)1 : (T)-1;
        if (!INV) return {h * (s * v.x + v.y), h * (s * v.y - v.x)};
        return {h * (s * v.x - v.y), h * (s * v.y + v.x)};
    }
    const cx<T> w = tw64<T>(k * (64 / len));
    return INV ? cmulc(v, w) : cmul(v, w);
}

// Bit-reversal permutation by template recursion (compile-time indices).
template <int R, typename T, int OFF, int I = 0>
__device__ __forceinline__ void bitrev_perm(cx<T> *a)
{
    if constexpr (I < R) {
        constexpr int J = bitrev(I, ilog2(R));
        if constexpr (J > I) {
            const cx<T> t = a[OFF + I];
            a[OFF + I] = a[OFF + J];
            a[OFF + J] = t;
        }
        bitrev_perm<R, T, OFF, I + 1>(a);
    }
}

// One butterfly (u, v) -> (u + w v, u - w v) with w = w_len^k (conjugated for
// the inverse), k and len compile-time.  Where w is not a power of -i the
// multiply is folded into fused multiply-adds: with t the rotated v, u + h t
// and u - h t are two FMAs (w = w_8 type), and for a general w the sum is
// two chained FMAs per component and the difference 2 u - sum is one more.
template <bool INV, typename T>
__device__ __forceinline__ void butterfly(cx<T> &u, cx<T> &v, int k, int len)
{
    if (k == 0 || 4 * k == len) {
        const cx<T> wv = twiddle_len<INV>(v, k, len);
        const cx<T> a = u + wv, b = u - wv;
        u = a;
        v = b;
        return;
    }
    if (8 * k == len || 8 * k == 3 * len) {
        const T h = (T)0.70710678118654752440;
        const T sg = (8 * k == len) ? (T)1 : (T)-1;
        // w v = h t
        const cx<T> t = INV ? cx<T>{sg * v.x - v.y, sg * v.y + v.x} : cx<T>{sg * v.x + v.y, sg * v.y - v.x};
        const cx<T> a = {fma(h, t.x, u.x), fma(h, t.y, u.y)};
        const cx<T> b = {fma(-h, t.x, u.x), fma(-h, t.y, u.y)};
        u = a;
        v = b;
        return;
    }
    const cx<T> w = tw64<T>(k * (64 / len));
    const T ws = INV ? -w.y : w.y;  // imaginary part of the applied twiddle
    cx<T> a;
    a.x = fma(-v.y, ws, fma(v.x, w.x, u.x));
    a.y = fma(v.y, w.x, fma(v.x, ws, u.y));
    const cx<T> b = {fma((T)2, u.x, -a.x), fma((T)2, u.y, -a.y)};
    u = a;
    v = b;
}

// ---------------------------------------------------------------------------
// Two lines per lane.  A packed value holds the same quantity of two lines
// (low half: the first line, high half: the second) and every arithmetic step
// is one .f32x2 instruction (add, sub, mul, fma; sm_100 and later), so a lane
// runs both lines' transforms with one instruction stream.  cx<f32x2> is then
// {(re_a, re_b), (im_a, im_b)}.
struct f32x2 {
    unsigned long long r;
};
}  // namespace fft
// 16-byte aligned, so that a packed complex value moves with one 128-bit access
template <>
struct __align__(16) cx<fft::f32x2> {
    fft::f32x2 x, y;
};
namespace fft {
__device__ __forceinline__ f32x2 pk2(float lo, float hi)
{
    f32x2 o;
    asm("mov.b64 %0, {%1, %2};" : "=l"(o.r) : "f"(lo), "f"(hi));
    return o;
}
__device__ __forceinline__ void unpk2(f32x2 a, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.r));
}
__device__ __forceinline__ f32x2 operator+(f32x2 a, f32x2 b)
{
    f32x2 o;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
    return o;
}
__device__ __forceinline__ f32x2 operator-(f32x2 a, f32x2 b)
{
    f32x2 o;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
    return o;
}
__device__ __forceinline__ f32x2 operator*(f32x2 a, f32x2 b)
{
    f32x2 o;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
    return o;
}
__device__ __forceinline__ f32x2 fma(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 o;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(o.r) : "l"(a.r), "l"(b.r), "l"(c.r));
    return o;
}
__device__ __forceinline__ f32x2 bc2(float c) { return pk2(c, c); }

// cos(2 pi j / 64), j = 0..16 (the other octants by symmetry), as literals so
// that the packed twiddle constants of an unrolled DFT are immediates
__host__ __device__ constexpr double cos64_q(int j)
{
    constexpr double t[17] = {1.0, 0.99518472667219693, 0.98078528040323043, 0.95694033573220882,
                              0.92387953251128674, 0.88192126434835505, 0.83146961230254524, 0.77301045336273699,
                              0.70710678118654757, 0.63439328416364549, 0.55557023301960229, 0.47139673682599781,
                              0.38268343236508984, 0.29028467725446233, 0.19509032201612833, 0.09801714032956077,
                              0.0};
    return t[j];
}
__host__ __device__ constexpr double cos64(int j)
{
    j &= 63;
    return j <= 16 ? cos64_q(j) : (j <= 32 ? -cos64_q(32 - j) : (j <= 48 ? -cos64_q(j - 32) : cos64_q(64 - j)));
}
__host__ __device__ constexpr double sin64(int j) { return cos64(j + 48); }

// complex products on packed values (a w and a conj(w))
__device__ __forceinline__ cx<f32x2> cmul(cx<f32x2> a, cx<f32x2> w)
{
    return {a.x * w.x - a.y * w.y, fma(a.x, w.y, a.y * w.x)};
}
__device__ __forceinline__ cx<f32x2> cmulc(cx<f32x2> a, cx<f32x2> w)
{
    return {fma(a.y, w.y, a.x * w.x), a.y * w.x - a.x * w.y};
}

// The butterfly of the scalar path on packed values.  Negated constants are
// separate immediates, so no step needs a negation instruction.
template <bool INV>
__device__ __forceinline__ void butterfly(cx<f32x2> &u, cx<f32x2> &v, int k, int len)
{
    cx<f32x2> a, b;
    if (k == 0) {
        a = u + v;
        b = u - v;
    } else if (4 * k == len) {  // w v = (v.y, -v.x) forward, (-v.y, v.x) inverse
        if (!INV) {
            a = {u.x + v.y, u.y - v.x};
            b = {u.x - v.y, u.y + v.x};
        } else {
            a = {u.x - v.y, u.y + v.x};
            b = {u.x + v.y, u.y - v.x};
        }
    } else if (8 * k == len || 8 * k == 3 * len) {
        // w v = h (sx Tx, sy Ty) with Tx, Ty sums or differences of v.x, v.y
        const bool s = 8 * k == len;
        f32x2 tx, ty;
        float sx = 1.f, sy = 1.f;
        if (!INV) {
            if (s) { tx = v.x + v.y; ty = v.y - v.x; }
            else { tx = v.y - v.x; ty = v.x + v.y; sy = -1.f; }
        } else {
            if (s) { tx = v.x - v.y; ty = v.x + v.y; }
            else { tx = v.x + v.y; ty = v.x - v.y; sx = -1.f; }
        }
        const float h = 0.70710678118654752440f;
        a = {fma(bc2(sx * h), tx, u.x), fma(bc2(sy * h), ty, u.y)};
        b = {fma(bc2(-sx * h), tx, u.x), fma(bc2(-sy * h), ty, u.y)};
    } else {
        // applied twiddle (wr, ws): w_len^k forward, its conjugate inverse
        const int jj = k * (64 / len);
        const float wr = (float)cos64(jj);
        const float ws = INV ? (float)sin64(jj) : -(float)sin64(jj);
        a = {fma(v.y, bc2(-ws), fma(v.x, bc2(wr), u.x)), fma(v.x, bc2(ws), fma(v.y, bc2(wr), u.y))};
        b = {fma(v.y, bc2(ws), fma(v.x, bc2(-wr), u.x)), fma(v.x, bc2(-ws), fma(v.y, bc2(-wr), u.y))};
    }
    u = a;
    v = b;
}

// Butterflies of one radix-2 level (span LEN) by template recursion over (I, K).
template <int R, bool INV, typename T, int OFF, int LEN, int I = 0, int K = 0>
__device__ __forceinline__ void level(cx<T> *a)
{
    if constexpr (I < R) {
        if constexpr (K < LEN / 2) {
            butterfly<INV>(a[OFF + I + K], a[OFF + I + K + LEN / 2], K, LEN);
            level<R, INV, T, OFF, LEN, I, K + 1>(a);
        } else {
            level<R, INV, T, OFF, LEN, I + LEN, 0>(a);
        }
    }
}

// First level when the upper half of the DFT input is zero: after the
// bit-reversal each pair holds (x_m, x_{m+R/2} = 0), so both outputs are x_m.
template <int R, typename T, int OFF, int I = 0>
__device__ __forceinline__ void level_half(cx<T> *a)
{
    if constexpr (I < R) {
        a[OFF + I + 1] = a[OFF + I];
        level_half<R, T, OFF, I + 2>(a);
    }
}

template <int R, bool INV, typename T, int OFF, bool HALF, int LEN = 2>
__device__ __forceinline__ void levels(cx<T> *a)
{
    if constexpr (LEN <= R) {
        if constexpr (HALF && LEN == 2) level_half<R, T, OFF>(a);
        else level<R, INV, T, OFF, LEN>(a);
        levels<R, INV, T, OFF, HALF, LEN * 2>(a);
    }
}

// In-register DFT of length R on a[OFF .. OFF+R), natural order in and out
// (radix-2 decimation in time).  HALF: inputs R/2 .. R-1 are known to be zero.
__host__ __device__ constexpr bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// cos(2 pi j / 48), j = 0..12 (the other quadrants by symmetry): the twiddles
// of the in-register DFTs whose length has a factor 3 (R divides 48)
__host__ __device__ constexpr double cos48_q(int j)
{
    constexpr double t[13] = {1.0, 0.99144486137381041114, 0.96592582628906828675, 0.92387953251128675613,
                              0.86602540378443864676, 0.79335334029123516458, 0.70710678118654752440,
                              0.60876142900872063942, 0.5, 0.38268343236508977173, 0.25881904510252076235,
                              0.13052619222005159155, 0.0};
    return t[j];
}
__host__ __device__ constexpr double cos48(int j)
{
    j = ((j % 48) + 48) % 48;
    return j <= 12 ? cos48_q(j) : (j <= 24 ? -cos48_q(24 - j) : (j <= 36 ? -cos48_q(j - 24) : cos48_q(48 - j)));
}
__host__ __device__ constexpr double sin48(int j) { return cos48(j - 12); }

// scalar helpers shared by the FP32, FP64 and packed transforms
template <typename T>
__device__ __forceinline__ T cst(double c) { return (T)c; }
template <>
__device__ __forceinline__ f32x2 cst<f32x2>(double c) { return bc2((float)c); }
template <typename T>
__device__ __forceinline__ T neg(T a) { return -a; }
template <>
__device__ __forceinline__ f32x2 neg<f32x2>(f32x2 a) { return bc2(0.f) - a; }
template <typename T>
__device__ __forceinline__ T fmaT(T a, T b, T c) { return ::fma(a, b, c); }
template <>
__device__ __forceinline__ f32x2 fmaT<f32x2>(f32x2 a, f32x2 b, f32x2 c) { return fma(a, b, c); }

// v times w_R^j = exp(-2 pi i j / R) (its conjugate for the inverse); R divides
// 48, j compile-time.  Quarter turns are swaps, the rest complex products with
// literal constants.
template <bool INV, int R, typename T>
__device__ __forceinline__ cx<T> twiddle48(cx<T> v, int j)
{
    j %= R;
    if (j == 0) return v;
    if (2 * j == R) return {neg(v.x), neg(v.y)};
    if (4 * j == R) return INV ? cx<T>{neg(v.y), v.x} : cx<T>{v.y, neg(v.x)};
    if (4 * j == 3 * R) return INV ? cx<T>{v.y, neg(v.x)} : cx<T>{neg(v.y), v.x};
    const int q = j * (48 / R);
    const double sd = INV ? sin48(q) : -sin48(q);  // w = c + i sn
    const T c = cst<T>(cos48(q)), sn = cst<T>(sd), nsn = cst<T>(-sd);
    return {fmaT(v.x, c, v.y * nsn), fmaT(v.x, sn, v.y * c)};
}

// In-register DFT of length R = 3 M (M a power of two), natural order in and
// out: the three stride-3 subsequences x[3 n + r] are transformed by the
// radix-2 DFT of length M, then X[k + m M] = sum_r w_R^{r k} Y_r[k] w_3^{r m}
// (a length-3 DFT per k < M).  HALF: inputs R/2 .. R-1 are zero, which leaves
// the upper half of every subsequence zero.
template <int R, bool INV, typename T, int OFF, bool HALF>
__device__ __forceinline__ void dft_reg3(cx<T> *a)
{
    constexpr int M = R / 3;
    static_assert(R == 3 * M && is_pow2(M) && 48 % R == 0, "R = 3 M, R divides 48");
    cx<T> y[3][M];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int n = 0; n < M; n++) y[r][n] = a[OFF + 3 * n + r];
    if constexpr (M > 1) {
#pragma unroll
        for (int r = 0; r < 3; r++) {
            bitrev_perm<M, T, 0>(y[r]);
            levels<M, INV, T, 0, HALF>(y[r]);
        }
    }
    const T nh = cst<T>(-0.5), s3 = cst<T>(0.86602540378443864676);  // -cos(pi/3), sin(pi/3)
#pragma unroll
    for (int k = 0; k < M; k++) {
        const cx<T> b0 = y[0][k];
        const cx<T> b1 = twiddle48<INV, R>(y[1][k], k);
        const cx<T> b2 = twiddle48<INV, R>(y[2][k], 2 * k);
        // length-3 DFT: X0 = b0 + b1 + b2, X1,2 = b0 - (b1 + b2)/2 -+ i sqrt3/2 (b1 - b2) (forward)
        const cx<T> t1 = b1 + b2;
        const cx<T> t2 = {fmaT(nh, t1.x, b0.x), fmaT(nh, t1.y, b0.y)};
        const cx<T> t3 = {s3 * (b1.x - b2.x), s3 * (b1.y - b2.y)};
        a[OFF + k] = b0 + t1;
        if (!INV) {
            a[OFF + k + M] = {t2.x + t3.y, t2.y - t3.x};
            a[OFF + k + 2 * M] = {t2.x - t3.y, t2.y + t3.x};
        } else {
            a[OFF + k + M] = {t2.x - t3.y, t2.y + t3.x};
            a[OFF + k + 2 * M] = {t2.x + t3.y, t2.y - t3.x};
        }
    }
}

// cos(2 pi j / 36), j = 0..9 (the other quadrants by symmetry): the twiddles of
// the in-register DFTs whose length has the factor 9 (R divides 36)
__host__ __device__ constexpr double cos36_q(int j)
{
    constexpr double t[10] = {1.0, 0.98480775301220805937, 0.93969262078590838405, 0.86602540378443864676,
                              0.76604444311897803520, 0.64278760968653932632, 0.5, 0.34202014332566873304,
                              0.17364817766693034885, 0.0};
    return t[j];
}
__host__ __device__ constexpr double cos36(int j)
{
    j = ((j % 36) + 36) % 36;
    return j <= 9 ? cos36_q(j) : (j <= 18 ? -cos36_q(18 - j) : (j <= 27 ? -cos36_q(j - 18) : cos36_q(36 - j)));
}
__host__ __device__ constexpr double sin36(int j) { return cos36(j - 9); }

// v times w_R^j (its conjugate for the inverse); R divides 36, j compile-time
template <bool INV, int R, typename T>
__device__ __forceinline__ cx<T> twiddle36(cx<T> v, int j)
{
    j %= R;
    if (j == 0) return v;
    if (2 * j == R) return {neg(v.x), neg(v.y)};
    if (4 * j == R) return INV ? cx<T>{neg(v.y), v.x} : cx<T>{v.y, neg(v.x)};
    if (4 * j == 3 * R) return INV ? cx<T>{v.y, neg(v.x)} : cx<T>{neg(v.y), v.x};
    const int q = j * (36 / R);
    const double sd = INV ? sin36(q) : -sin36(q);
    const T c = cst<T>(cos36(q)), sn = cst<T>(sd), nsn = cst<T>(-sd);
    return {fmaT(v.x, c, v.y * nsn), fmaT(v.x, sn, v.y * c)};
}

// length-3 DFT of (a, b, c) in place (forward: w_3 = exp(-2 pi i / 3))
template <bool INV, typename T>
__device__ __forceinline__ void dft3(cx<T> &a, cx<T> &b, cx<T> &c)
{
    const T nh = cst<T>(-0.5), s3 = cst<T>(0.86602540378443864676);
    const cx<T> t1 = b + c;
    const cx<T> t2 = {fmaT(nh, t1.x, a.x), fmaT(nh, t1.y, a.y)};
    const cx<T> t3 = {s3 * (b.x - c.x), s3 * (b.y - c.y)};
    a = a + t1;
    if (!INV) {
        b = {t2.x + t3.y, t2.y - t3.x};
        c = {t2.x - t3.y, t2.y + t3.x};
    } else {
        b = {t2.x - t3.y, t2.y + t3.x};
        c = {t2.x + t3.y, t2.y - t3.x};
    }
}

// length-9 DFT, natural order in and out, as 3 x 3: with n = 3 n1 + n2 and
// k = k1 + 3 k2, X[k] = sum_{n2} w_3^{n2 k2} w_9^{n2 k1} sum_{n1} w_3^{n1 k1} x[3 n1 + n2]
template <bool INV, typename T>
__device__ __forceinline__ void dft9(cx<T> (&b)[9])
{
    cx<T> z[3][3];  // z[n2][k1]
#pragma unroll
    for (int n2 = 0; n2 < 3; n2++) {
        z[n2][0] = b[n2];
        z[n2][1] = b[3 + n2];
        z[n2][2] = b[6 + n2];
        dft3<INV>(z[n2][0], z[n2][1], z[n2][2]);
#pragma unroll
        for (int k1 = 0; k1 < 3; k1++) z[n2][k1] = twiddle36<INV, 9, T>(z[n2][k1], n2 * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < 3; k1++) {
        dft3<INV>(z[0][k1], z[1][k1], z[2][k1]);
        b[k1] = z[0][k1];
        b[k1 + 3] = z[1][k1];
        b[k1 + 6] = z[2][k1];
    }
}

// In-register DFT of length R = 9 M (M a power of two), natural order in and
// out, structured as dft_reg3 with a length-9 DFT in place of the length-3 one:
// the nine stride-9 subsequences are transformed by the radix-2 DFT of length M,
// then X[k + m M] = sum_r w_R^{r k} Y_r[k] w_9^{r m}.  HALF: inputs R/2 .. R-1
// are zero, which leaves the upper half of every subsequence zero (M >= 2).
template <int R, bool INV, typename T, int OFF, bool HALF>
__device__ __forceinline__ void dft_reg9(cx<T> *a)
{
    constexpr int M = R / 9;
    static_assert(R == 9 * M && is_pow2(M) && 36 % R == 0, "R = 9 M, R divides 36");
    cx<T> y[9][M];
#pragma unroll
    for (int r = 0; r < 9; r++)
#pragma unroll
        for (int n = 0; n < M; n++) y[r][n] = a[OFF + 9 * n + r];
    if constexpr (M > 1) {
#pragma unroll
        for (int r = 0; r < 9; r++) {
            bitrev_perm<M, T, 0>(y[r]);
            levels<M, INV, T, 0, HALF>(y[r]);
        }
    }
#pragma unroll
    for (int k = 0; k < M; k++) {
        cx<T> b[9];
#pragma unroll
        for (int r = 0; r < 9; r++) b[r] = twiddle36<INV, R>(y[r][k], r * k);
        dft9<INV>(b);
#pragma unroll
        for (int m = 0; m < 9; m++) a[OFF + k + m * M] = b[m];
    }
}

template <int R, bool INV, typename T, int OFF, bool HALF = false>
__device__ __forceinline__ void dft_reg(cx<T> *a)
{
    if constexpr (is_pow2(R)) {
        bitrev_perm<R, T, OFF>(a);
        levels<R, INV, T, OFF, HALF>(a);
    } else if constexpr (R % 9 == 0) {
        dft_reg9<R, INV, T, OFF, HALF && R / 9 >= 2>(a);
    } else {
        dft_reg3<R, INV, T, OFF, HALF>(a);
    }
}

// G lanes per line, E = N / G elements per lane, radices (forward order).
template <int N>
struct Plan;
template <>
struct Plan<16> {
    static constexpr int G = 1, E = 16, S = 1;
    static constexpr int R[1] = {16};
};
template <>
struct Plan<32> {
    static constexpr int G = 1, E = 32, S = 1;
    static constexpr int R[1] = {32};
};
template <>
struct Plan<64> {
    static constexpr int G = 8, E = 8, S = 2;
    static constexpr int R[2] = {8, 8};
};
template <>
struct Plan<128> {
    static constexpr int G = 8, E = 16, S = 2;
    static constexpr int R[2] = {16, 8};
};
template <>
struct Plan<256> {
    static constexpr int G = 16, E = 16, S = 2;
    static constexpr int R[2] = {16, 16};
};
template <>
struct Plan<512> {
    static constexpr int G = 16, E = 32, S = 2;
    static constexpr int R[2] = {16, 32};
};
// lengths 3 * 2^k: one in-register radix has the factor 3
template <>
struct Plan<96> {
    static constexpr int G = 4, E = 24, S = 2;
    static constexpr int R[2] = {12, 8};
};
template <>
struct Plan<192> {
    static constexpr int G = 8, E = 24, S = 2;
    static constexpr int R[2] = {24, 8};
};
template <>
struct Plan<384> {
    static constexpr int G = 16, E = 24, S = 3;
    static constexpr int R[3] = {8, 6, 8};
};
template <>
struct Plan<768> {
    static constexpr int G = 32, E = 24, S = 3;
    static constexpr int R[3] = {8, 12, 8};
};
// lengths with the factor 9 or 27, two stages each: 288 = 12 x 24 (radices with one
// factor 3) and 432 = 12 x 36 (radix 36 = 4 x 9 in registers); G = 12 is not a
// power of two, only a divisor or multiple of every stage's span
template <>
struct Plan<288> {
    static constexpr int G = 12, E = 24, S = 2;
    static constexpr int R[2] = {12, 24};
};
template <>
struct Plan<432> {
    static constexpr int G = 12, E = 36, S = 2;
    static constexpr int R[2] = {12, 36};
};
template <>
struct Plan<1024> {
    static constexpr int G = 64, E = 16, S = 3;
    static constexpr int R[3] = {16, 16, 4};
};

// Radix and span of stage s of the forward (INV = false) or inverse
// (INV = true, radices reversed) transform.
template <int N, bool INV>
__host__ __device__ constexpr int radix(int s)
{
    return INV ? Plan<N>::R[Plan<N>::S - 1 - s] : Plan<N>::R[s];
}
template <int N, bool INV>
__host__ __device__ constexpr int span(int s)
{
    int L = 1;
    for (int i = 0; i < s; i++) L *= radix<N, INV>(i);
    return L;
}

// Twiddles of the stages s >= 1 in shared memory.  N <= 512: stage-major
// tables; for direction INV, stage s (radix R, span L, STEP = N / (R L))
// holds w_N^(m k STEP) at off(s) + m L + k (k < L, m < R), so a butterfly
// finds its R twiddles at fixed offsets from its k, and lanes with
// consecutive k read consecutive words.  Plans whose radices are not a
// palindrome keep the inverse direction's table behind the forward one.
// N = 1024: the N powers w_N^q (q < N), indexed m k STEP (shared-memory budget).
template <int N>
__host__ __device__ constexpr bool tw_stage_tables() { return N <= 512; }
template <int N, bool INV>
__host__ __device__ constexpr int tw_stage_off(int s)
{
    int off = 0;
    for (int i = 1; i < s; i++) off += span<N, INV>(i) * radix<N, INV>(i);
    return off;
}
template <int N, bool INV>
__host__ __device__ constexpr int tw_dir_size() { return tw_stage_off<N, INV>(Plan<N>::S); }
template <int N>
__host__ __device__ constexpr bool tw_palindrome()
{
    for (int s = 0; s < Plan<N>::S; s++)
        if (radix<N, false>(s) != radix<N, true>(s)) return false;
    return true;
}
template <int N>
__host__ __device__ constexpr int tw_base(bool inv) { return inv && !tw_palindrome<N>() ? tw_dir_size<N, false>() : 0; }
// entries of the shared twiddle array
template <int N>
__host__ __device__ constexpr int tw_size()
{
    if (!tw_stage_tables<N>()) return N;
    const int n = tw_dir_size<N, false>() + (tw_palindrome<N>() ? 0 : tw_dir_size<N, true>());
    return n > 0 ? n : 1;
}

// Shared-memory addressing of element `pos` of line `l`:
//   LINE_FAST (threads of a warp run across lines):  pos * LSP + l
//   lane-fast (threads of a warp run along a line):   l * NP + pos + pos / 32
template <int N, bool LINE_FAST>
struct Smem {
    int LSP;
    static constexpr int NP = N + (N >= 32 ? N / 32 : 1);
    __device__ __forceinline__ int at(int pos, int l) const
    {
        if constexpr (LINE_FAST) return pos * LSP + l;
        else return l * NP + pos + pos / 32;
    }
};

template <int N, bool INV, int s, typename T, bool HALF, int b = 0>
__device__ __forceinline__ void dft_all(cx<T> (&v)[Plan<N>::E])
{
    constexpr int R = radix<N, INV>(s);
    if constexpr (b < Plan<N>::E / R) {
        dft_reg<R, INV, T, b * R, HALF>(v);
        dft_all<N, INV, s, T, HALF, b + 1>(v);
    }
}

// Stage s: twiddles (s > 0) and the DFTs, all in registers.  HALF (stage 0
// only): the input positions >= N/2 are zero, i.e. elements m >= R/2 of every
// stage-0 butterfly (see in_lower_half).
template <int N, bool INV, int s, typename T, bool HALF = false>
__device__ __forceinline__ void stage_compute(cx<T> (&v)[Plan<N>::E], const cx<T> *tw, int j)
{
    static_assert(!HALF || s == 0, "zero upper half only holds for the first stage");
    constexpr int R = radix<N, INV>(s);
    constexpr int L = span<N, INV>(s);
    constexpr int STEP = N / (R * L);
    constexpr int G = Plan<N>::G;
    static_assert(G % L == 0 || L % G == 0, "lane/span layout");
    if constexpr (L > 1) {
#pragma unroll
        for (int b = 0; b < Plan<N>::E / R; b++) {
            // k = (j + b G) mod L, with j < G
            const int k = G % L == 0 ? j % L : j + (b * G) % L;
            if constexpr (tw_stage_tables<N>()) {
                const cx<T> *col = tw + tw_base<N>(INV) + tw_stage_off<N, INV>(s) + k;
#pragma unroll
                for (int m = 1; m < R; m++) {
                    const cx<T> w = col[m * L];
                    v[b * R + m] = INV ? cmulc(v[b * R + m], w) : cmul(v[b * R + m], w);
                }
            } else {
#pragma unroll
                for (int m = 1; m < R; m++) {
                    const cx<T> w = tw[m * k * STEP];
                    v[b * R + m] = INV ? cmulc(v[b * R + m], w) : cmul(v[b * R + m], w);
                }
            }
        }
    }
    dft_all<N, INV, s, T, HALF>(v);
}

// Move from the output layout of stage s to the input layout of stage s+1.
template <int N, bool INV, int s, bool LINE_FAST, typename T>
__device__ __forceinline__ void exchange(cx<T> (&v)[Plan<N>::E], cx<T> *buf, Smem<N, LINE_FAST> sm, int l, int j)
{
    constexpr int R = radix<N, INV>(s);
    constexpr int L = span<N, INV>(s);
    constexpr int R2 = radix<N, INV>(s + 1);
    constexpr int G = Plan<N>::G;
    constexpr int E = Plan<N>::E;
#pragma unroll
    for (int b = 0; b < E / R; b++) {
        const int jb = j + b * G;
        const int base = (jb / L) * R * L + (jb % L);
#pragma unroll
        for (int q = 0; q < R; q++) buf[sm.at(base + q * L, l)] = v[b * R + q];
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < E / R2; b++) {
        const int jb = j + b * G;
#pragma unroll
        for (int m = 0; m < R2; m++) v[b * R2 + m] = buf[sm.at(jb + m * (N / R2), l)];
    }
    __syncthreads();
}

// The whole transform: registers in (input layout of stage 0), registers out
// (output layout of the last stage).  Every thread of the block must call it.
// HALF: the caller left every element with in_lower_half(e) == false at zero.
template <int N, bool INV, bool LINE_FAST, typename T, bool HALF = false, int s = 0>
__device__ __forceinline__ void transform(cx<T> (&v)[Plan<N>::E], cx<T> *buf, const cx<T> *tw,
                                          Smem<N, LINE_FAST> sm, int l, int j)
{
    if constexpr (s < Plan<N>::S) {
        stage_compute<N, INV, s, T, HALF && s == 0>(v, tw, j);
        if constexpr (s + 1 < Plan<N>::S) exchange<N, INV, s, LINE_FAST, T>(v, buf, sm, l, j);
        transform<N, INV, LINE_FAST, T, HALF, s + 1>(v, buf, tw, sm, l, j);
    }
}

// Position of register element e before the first stage / after the last.
template <int N, bool INV>
__host__ __device__ constexpr int in_pos(int e, int j)
{
    constexpr int R = radix<N, INV>(0);
    return (j + (e / R) * Plan<N>::G) + (e % R) * (N / R);
}
template <int N, bool INV>
__host__ __device__ constexpr int out_pos(int e, int j)
{
    constexpr int R = radix<N, INV>(Plan<N>::S - 1);
    return (j + (e / R) * Plan<N>::G) + (e % R) * (N / R);
}
// Whether input element e can be non-zero when only positions < N/2 carry
// data (true for every forward transform here: the data extent is <= N/2).
// Lane-independent when N/R_0 divides N/2, which holds for every plan.
template <int N, bool INV>
__host__ __device__ constexpr bool in_lower_half(int e)
{
    constexpr int R = radix<N, INV>(0);
    return (e % R) * (N / R) < N / 2;
}

// Fill the shared twiddle array (tw_size<N>() entries) from the global table of
// the same precision (float2 for T = float, double2 for double): from its
// w_TW_POW part for every length dividing TW_POW, else from its w_TW_MAX part.
template <typename T>
__device__ __forceinline__ cx<T> tw_global_at(const void *tw_global, int idx)
{
    if constexpr (std::is_same<T, f32x2>::value) {
        const float2 w = __ldg((const float2 *)tw_global + idx);
        return {bc2(w.x), bc2(w.y)};
    } else if constexpr (sizeof(T) == 8) {
        const double2 w = __ldg((const double2 *)tw_global + idx);
        return {w.x, w.y};
    } else {
        const float2 w = __ldg((const float2 *)tw_global + idx);
        return {w.x, w.y};
    }
}
template <int N, bool INV, typename T, int s = 1>
__device__ __forceinline__ void load_dir(cx<T> *tw_s, const void *tw_global)
{
    if constexpr (s < Plan<N>::S) {
        static_assert(TW_MAX % N == 0, "N divides the twiddle table length");
        // lengths dividing TW_POW read the short w_TW_POW part (a few KB, cached across
        // thread blocks); 288 and 432 the w_TW_MAX part
        constexpr bool SHORT = TW_POW % N == 0;
        constexpr int M = SHORT ? TW_POW : TW_MAX, BASE = SHORT ? TW_MAX : 0, SC = M / N;
        constexpr int R = radix<N, INV>(s), L = span<N, INV>(s), STEP = N / (R * L);
        cx<T> *ts = tw_s + tw_base<N>(INV) + tw_stage_off<N, INV>(s);
        for (int q = threadIdx.x; q < L * R; q += blockDim.x) {
            const int m = q / L, k = q - m * L;
            ts[q] = tw_global_at<T>(tw_global, BASE + (m * k * STEP * SC) % M);
        }
        load_dir<N, INV, T, s + 1>(tw_s, tw_global);
    }
}
template <int N, typename T>
__device__ __forceinline__ void load_twiddles(cx<T> *tw_s, const void *tw_global)
{
    static_assert(N <= TW_MAX, "N too large");
    if constexpr (tw_stage_tables<N>()) {
        load_dir<N, false, T>(tw_s, tw_global);
        if constexpr (!tw_palindrome<N>()) load_dir<N, true, T>(tw_s, tw_global);
    } else {
        static_assert(TW_POW % N == 0, "N divides the second twiddle table's length");
        for (int q = threadIdx.x; q < N; q += blockDim.x) tw_s[q] = tw_global_at<T>(tw_global, TW_MAX + q * (TW_POW / N));
    }
}

}  // namespace fft
}  // namespace lgf
