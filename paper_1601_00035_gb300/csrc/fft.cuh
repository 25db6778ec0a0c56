// Batched 1-D complex FFTs of power-of-two length N (16..1024) on data held
// in shared memory, in FP32 or FP64.
//
// Layout: a tile of LS lines, element n of line l at buf[n * LSP + l]
// (LSP = LS + 1 to spread shared-memory banks).  Thread t works on line
// l = t % LS as lane t / LS of G = blockDim / LS lanes.
//
// Algorithm: Stockham autosort with mixed radices (each stage one radix-R
// butterfly per lane, R <= 32, done in registers by an unrolled radix-2
// decimation-in-time DFT).  Stage with span L (product of earlier radices):
// butterfly j reads x[j + m N/R], m < R, multiplies by w_{R L}^{m (j mod L)},
// does a length-R DFT and writes y[(j div L) R L + q L + (j mod L)], q < R.
// Forward transforms use w = exp(-2 pi i / N); inverse ones the conjugate
// (unnormalised).  Every stage ends in __syncthreads(): all threads of the
// block must call the line routines.
#pragma once
#include <cmath>

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

// multiply v by w_len^k (conjugated for the inverse); k, len compile-time after unrolling
template <bool INV, typename T>
__device__ __forceinline__ cx<T> twiddle_len(cx<T> v, int k, int len)
{
    if (k == 0) return v;
    if (4 * k == len) {  // w = -i (forward) or +i (inverse)
        return INV ? cx<T>{-v.y, v.x} : cx<T>{v.y, -v.x};
    }
    const cx<T> w = tw64<T>(k * (64 / len));
    return INV ? cmulc(v, w) : cmul(v, w);
}

// Bit-reversal permutation by template recursion, so every index is a
// compile-time constant and the array stays in registers.
template <int R, typename T, int I = 0>
__device__ __forceinline__ void bitrev_perm(cx<T> (&a)[R])
{
    if constexpr (I < R) {
        constexpr int J = bitrev(I, ilog2(R));
        if constexpr (J > I) {
            const cx<T> t = a[I];
            a[I] = a[J];
            a[J] = t;
        }
        bitrev_perm<R, T, I + 1>(a);
    }
}

// Butterflies of one radix-2 level (span LEN) by template recursion over (I, K).
template <int R, bool INV, typename T, int LEN, int I = 0, int K = 0>
__device__ __forceinline__ void level(cx<T> (&a)[R])
{
    if constexpr (I < R) {
        if constexpr (K < LEN / 2) {
            const cx<T> u = a[I + K];
            const cx<T> v = twiddle_len<INV>(a[I + K + LEN / 2], K, LEN);
            a[I + K] = u + v;
            a[I + K + LEN / 2] = u - v;
            level<R, INV, T, LEN, I, K + 1>(a);
        } else {
            level<R, INV, T, LEN, I + LEN, 0>(a);
        }
    }
}

template <int R, bool INV, typename T, int LEN = 2>
__device__ __forceinline__ void levels(cx<T> (&a)[R])
{
    if constexpr (LEN <= R) {
        level<R, INV, T, LEN>(a);
        levels<R, INV, T, LEN * 2>(a);
    }
}

// In-register DFT of length R (power of two, <= 32), natural order in and out
// (radix-2 decimation in time).
template <int R, bool INV, typename T>
__device__ __forceinline__ void dft_reg(cx<T> (&a)[R])
{
    bitrev_perm<R, T>(a);
    levels<R, INV, T>(a);
}

// One Stockham stage of radix R and span L on every line of the tile.
// tw: shared table of w_N^j, j < N.
template <int N, int R, int L, bool INV, typename T>
__device__ __forceinline__ void stage(cx<T> *buf, const cx<T> *tw, int LSP, int l, int lane, bool line_ok)
{
    constexpr int NB = N / R;
    constexpr int STEP = N / (R * L);
    cx<T> a[R];
    const bool active = line_ok && lane < NB;
    const int j = lane;
    const int k = j % L;
    if (active) {
#pragma unroll
        for (int m = 0; m < R; m++) a[m] = buf[(j + m * NB) * LSP + l];
        if (L > 1) {
#pragma unroll
            for (int m = 1; m < R; m++) {
                const cx<T> w = tw[(m * k * STEP) % N];
                a[m] = INV ? cmulc(a[m], w) : cmul(a[m], w);
            }
        }
        dft_reg<R, INV>(a);
    }
    __syncthreads();
    if (active) {
        const int base = (j / L) * R * L + k;
#pragma unroll
        for (int q = 0; q < R; q++) buf[(base + q * L) * LSP + l] = a[q];
    }
    __syncthreads();
}

template <int N, int L, bool INV, typename T, int R, int... Rest>
__device__ __forceinline__ void stages(cx<T> *buf, const cx<T> *tw, int LSP, int l, int lane, bool line_ok)
{
    stage<N, R, L, INV, T>(buf, tw, LSP, l, lane, line_ok);
    if constexpr (sizeof...(Rest) > 0) stages<N, L * R, INV, T, Rest...>(buf, tw, LSP, l, lane, line_ok);
}

// Radix plans and the lanes each line needs (max butterflies in a stage).
template <int N>
struct Plan;
template <>
struct Plan<16> {
    static constexpr int lanes = 1;
};
template <>
struct Plan<32> {
    static constexpr int lanes = 1;
};
template <>
struct Plan<64> {
    static constexpr int lanes = 8;
};
template <>
struct Plan<128> {
    static constexpr int lanes = 16;
};
template <>
struct Plan<256> {
    static constexpr int lanes = 16;
};
template <>
struct Plan<512> {
    static constexpr int lanes = 64;
};
template <>
struct Plan<1024> {
    static constexpr int lanes = 128;
};

// Transform every line of the tile in place.  line_ok masks partial tiles
// (inactive lines still take part in the barriers).
template <int N, bool INV, typename T>
__device__ __forceinline__ void line_fft(cx<T> *buf, const cx<T> *tw, int LSP, int l, int lane, bool line_ok)
{
    if constexpr (N == 16) stages<N, 1, INV, T, 16>(buf, tw, LSP, l, lane, line_ok);
    else if constexpr (N == 32) stages<N, 1, INV, T, 32>(buf, tw, LSP, l, lane, line_ok);
    else if constexpr (N == 64) stages<N, 1, INV, T, 8, 8>(buf, tw, LSP, l, lane, line_ok);
    else if constexpr (N == 128) stages<N, 1, INV, T, 16, 8>(buf, tw, LSP, l, lane, line_ok);
    else if constexpr (N == 256) stages<N, 1, INV, T, 16, 16>(buf, tw, LSP, l, lane, line_ok);
    else if constexpr (N == 512) stages<N, 1, INV, T, 8, 8, 8>(buf, tw, LSP, l, lane, line_ok);
    else if constexpr (N == 1024) stages<N, 1, INV, T, 16, 8, 8>(buf, tw, LSP, l, lane, line_ok);
    else static_assert(N == 16, "unsupported FFT length");
}

// Load w_N^j (j < N) into shared memory from the 1024-entry global table.
template <int N, typename T>
__device__ __forceinline__ void load_twiddles(cx<T> *tw_s, const void *tw_global)
{
    static_assert(N <= TW_MAX, "N too large");
    constexpr int STRIDE = TW_MAX / N;
    if constexpr (sizeof(T) == 4) {
        const float2 *g = (const float2 *)tw_global;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            float2 w = __ldg(g + j * STRIDE);
            tw_s[j] = {w.x, w.y};
        }
    } else {
        const double2 *g = (const double2 *)tw_global;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            double2 w = __ldg(g + j * STRIDE);
            tw_s[j] = {w.x, w.y};
        }
    }
}

}  // namespace fft
}  // namespace lgf
