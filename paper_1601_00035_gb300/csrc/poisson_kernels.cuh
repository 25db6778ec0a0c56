// Kernels of the five FFT passes of a Poisson solve (the pass structure is
// described in poisson.cu) and their launchers, as templates over the pass
// length N.  Each poisson_len_*.cu translation unit includes this header and
// instantiates PoissonPasses for its lengths, so the lengths compile in parallel.
#pragma once
#include "fft.cuh"
#include "plan.hpp"
#include "poisson_passes.hpp"

namespace lgf {

namespace {

using fft::Plan;

// Lines per block: y/z passes run LS consecutive kx lines (line-fast thread
// mapping, coalesced rows of kx); x passes run whole rows (lane-fast mapping).
// (FP64 tiles are half as wide.)
// Shared-memory budget of a pass's exchange buffer and twiddles: 44 KB, and 100 KB from
// length 432 on (static shared memory beyond 48 KB compiles for this architecture).  On the
// 256^3 ring's step the larger budget, which gives the 432-point y and x passes 16 and 21
// lines per block instead of 8 and 10, took 1.611 ms against 1.644 ms; applied to every
// length it slowed the 64-solve ragged batch (1.806 against 1.763 ms: its 96- and 192-point
// passes went to 64 and 32 lines per block).
template <int N>
constexpr size_t smem_budget() { return (N >= 432 ? 100 : 44) * 1024; }
// largest line count <= want (halving) whose exchange buffer and twiddles fit in the budget
template <int N, typename T>
constexpr int lines_fit(int want, int pad)
{
    int ls = want;
    while (ls > 1 && (size_t)N * (ls + pad) * sizeof(cx<T>) + fft::tw_size<N>() * sizeof(cx<T>) > smem_budget<N>()) ls /= 2;
    return ls;
}
template <int N, typename T>
struct TileY {
    static constexpr int G = Plan<N>::G;
    static constexpr int LS32 = G == 1 ? 64 : (G >= 64 ? (N >= 1024 ? 4 : 8) : (G <= 8 ? 256 / G : 16));
    static constexpr int LS = lines_fit<N, T>(sizeof(T) == 8 ? (G >= 64 ? 2 : LS32 / 2) : LS32, 1);
    static constexpr int LSP = LS + 1;
    static constexpr int threads = LS * G;
    // resident blocks per SM asked of the compiler (a register cap per thread:
    // 48 / 64 for the single / double transform passes in FP32, twice that in FP64)
    static constexpr int cap(int mode)
    {
        return (Plan<N>::E > 32 ? 160 : (G == 1 || Plan<N>::E > 16 ? 128 : (mode == 1 ? 64 : 48) + (N >= 1024 ? 8 : 0))) *
               (sizeof(T) == 8 ? 2 : 1);
    }
    static constexpr int minb(int mode) { return 65536 / (threads * cap(mode)) > 0 ? 65536 / (threads * cap(mode)) : 1; }
    // the z pass's spectrum columns fit beside the exchange buffer and twiddles
    // in the shared-memory budget
    static constexpr bool slab_fits = (size_t)N * LSP * sizeof(cx<T>) + fft::tw_size<N>() * sizeof(cx<T>) +
                                          (size_t)(N / 2 + 1) * LS * sizeof(T) <= smem_budget<N>() + 4 * 1024;
};
template <int N, typename T>
struct TileX {
    static constexpr int G = Plan<N>::G;
    static constexpr int LS = G == 1 ? 64 : lines_fit<N, T>((sizeof(T) == 8 ? 128 : 256) / G, 0);
    static constexpr int threads = LS * G;
    static constexpr int cap = (G == 1 || Plan<N>::E > 16 ? 128 : (N >= 1024 ? 80 : (N == 128 ? 64 : 48))) *
                               (sizeof(T) == 8 ? 2 : 1);
    static constexpr int minb = 65536 / (threads * cap) > 0 ? 65536 / (threads * cap) : 1;
};

// spectrum pointer and factor of the requested precision
template <typename T>
__device__ __forceinline__ const T *kh_of(const Geom &g);
template <>
__device__ __forceinline__ const float *kh_of<float>(const Geom &g) { return g.Kh; }
template <>
__device__ __forceinline__ const double *kh_of<double>(const Geom &g) { return g.Kh64; }
template <typename T>
__device__ __forceinline__ T mul_of(const Geom &g) { return sizeof(T) == 8 ? (T)g.mul64 : (T)g.mul; }

// v mod N in [0, N) for -N <= v < 2N
template <int N>
__device__ __forceinline__ int wrap_mod(int v)
{
    if constexpr ((N & (N - 1)) == 0) return v & (N - 1);
    else return v < 0 ? v + N : (v >= N ? v - N : v);
}

// ---------------------------------------------------------------------------
// x forward: gather two source rows per complex line from the block list, R2C.
// bx: this thread block's tile; c: workspace component (g.c0 + c in the source layout)
template <int N, typename T>
__device__ __forceinline__ void x_fwd_body(const Geom &g, const T *__restrict__ src, cx<T> *__restrict__ out,
                                           const void *tw_g, int bx, int c)
{
    using TL = TileX<N, T>;
    constexpr int E = Plan<N>::E;
    using SM = fft::Smem<N, false>;
    // block-list lookups of the lines' rows: the source extent is <= N/2 and
    // B >= 8, so a row meets at most N/16 blocks
    constexpr int NBX = N / 16;
    __shared__ cx<T> buf[TL::LS * SM::NP + 8];
    __shared__ cx<T> tw[fft::tw_size<N>()];
    __shared__ int lut_s[TL::LS * NBX];
    fft::load_twiddles<N, T>(tw, tw_g);
    const int j = threadIdx.x % TL::G, l = threadIdx.x / TL::G;
    const int nrows = g.Es[1] * g.Es[2];
    const int B = g.B;
    const int lB = g.lB, mB = B - 1;
    // the lookup table is fixed at plan time: read it before waiting
    int mine = 0;  // whether this thread's lookups found a block
    for (int q = threadIdx.x; q < TL::LS * NBX; q += TL::threads) {
        const int ll = q / NBX, xb = q - ll * NBX;
        const int rr = 2 * (bx * TL::LS + ll);
        int b = -1;
        if (rr < nrows && xb < g.nbS[0]) {
            const int zz = rr / g.Es[1], yy = rr - zz * g.Es[1];
            b = __ldg(g.src_lut + ((zz >> lB) * g.nbS[1] + (yy >> lB)) * g.nbS[0] + xb);
        }
        lut_s[q] = b;
        mine |= b >= 0;
    }
    pdl_trigger();
    pdl_wait();  // the previous pass (or the producer of src) is complete
    // twiddles, lookups; a thread block whose rows meet no source block writes
    // its zero rows without transforming them
    if (!__syncthreads_or(mine)) {
        constexpr int KXZ = N / 2 + 1;
        for (int idx = threadIdx.x; idx < TL::LS * KXZ; idx += TL::threads) {
            const int ll = idx / KXZ, k = idx - ll * KXZ;
            const int rr = 2 * (bx * TL::LS + ll);
            if (rr >= nrows) continue;
            const size_t row = ((size_t)c * nrows + rr) * KXZ;
            out[row + k] = {(T)0, (T)0};
            out[row + KXZ + k] = {(T)0, (T)0};
        }
        return;
    }
    const int r0 = 2 * (bx * TL::LS + l);
    const bool row_ok = r0 < nrows;
    const int z = row_ok ? r0 / g.Es[1] : 0, y = row_ok ? r0 - z * g.Es[1] : 0;
    const int in_blk = (((z & mB) << lB) + (y & mB)) << lB;
    const int *lut = lut_s + l * NBX;
    cx<T> v[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        v[e] = {(T)0, (T)0};
        if (fft::in_lower_half<N, false>(e)) {
            const int pos = fft::in_pos<N, false>(e, j);
            if (row_ok && pos < g.Es[0]) {
                const int blk = lut[pos >> lB];
                if (blk >= 0) {
                    const T *p = src + ((size_t)(blk * g.ncomp + g.c0 + c) << (3 * lB)) + in_blk + (pos & mB);
                    v[e] = {__ldg(p), __ldg(p + B)};
                }
            }
        }
    }
    SM sm{0};
    fft::transform<N, false, false, T, true>(v, buf, tw, sm, l, j);
#pragma unroll
    for (int e = 0; e < E; e++) buf[sm.at(fft::out_pos<N, false>(e, j), l)] = v[e];
    __syncthreads();
    // split the two real rows: A(k) = (Z_k + conj Z_{N-k})/2, B(k) = (Z_k - conj Z_{N-k})/(2i)
    constexpr int KX = N / 2 + 1;
    for (int idx = threadIdx.x; idx < TL::LS * KX; idx += TL::threads) {
        const int ll = idx / KX, k = idx - ll * KX;
        const int rr = 2 * (bx * TL::LS + ll);
        if (rr >= nrows) continue;
        const cx<T> zk = buf[sm.at(k, ll)];
        const cx<T> zn = buf[sm.at(k == 0 ? 0 : N - k, ll)];
        const size_t row = ((size_t)c * nrows + rr) * KX;
        const T h = (T)0.5;
        out[row + k] = {h * (zk.x + zn.x), h * (zk.y - zn.y)};
        out[row + KX + k] = {h * (zk.y + zn.y), -h * (zk.x - zn.x)};
    }
}
template <int N, typename T>
__global__ void __launch_bounds__(TileX<N, T>::threads, TileX<N, T>::minb) k_x_fwd(Geom g, const T *__restrict__ src,
                                                                 cx<T> *__restrict__ out, const void *tw_g)
{
    x_fwd_body<N, T>(g, src, out, tw_g, blockIdx.x, blockIdx.y);
}

// y forward (MODE 0), z forward + spectral multiply + z inverse (MODE 1),
// y inverse (MODE 2) over [c][plane][line][kx] arrays.
//   MODE 0: in [c][Es_z][Es_y][KX] -> out [c][Es_z][Ny][KX]
//   MODE 1: in [c][Es_z][Ny][KX]   -> out [c][Et_z][Ny][KX]
//   MODE 2: in [c][Et_z][Ny][KX]   -> out [c][Et_z][Et_y][KX]
// Block tiling: the KX * planes lines of a component are numbered kx-fastest
// (line i = p * KX + kx) and block b takes lines b LS .. b LS + LS - 1.
// Consecutive lines are consecutive kx of one plane, so a block's rows are
// coalesced (at most two contiguous segments, at a plane boundary), and only
// the last block of a component holds padding lines.  KX = Nx/2 + 1 is the x
// extent of the spectrum, independent of this pass's line length N.  (In the
// z pass the [plane][line] offset of line i is i itself.)
template <int MODE>
__host__ __device__ __forceinline__ int line_planes(const Geom &g)
{
    return MODE == 0 ? g.Es[2] : (MODE == 1 ? g.N[1] : g.Et[2]);
}

template <int N, int MODE, typename T>
__device__ __forceinline__ void line_body(const Geom &g, const cx<T> *__restrict__ in, cx<T> *__restrict__ out,
                                          const void *tw_g, int bx, int c)
{
    using TL = TileY<N, T>;
    constexpr int E = Plan<N>::E;
    constexpr int G = Plan<N>::G;
    using SM = fft::Smem<N, true>;
    __shared__ cx<T> buf[N * TL::LSP];
    __shared__ cx<T> tw[fft::tw_size<N>()];
    // z pass: this block's kernel-spectrum columns ks[kz][l] (kz <= N/2), scaled
    constexpr int KZ = N / 2 + 1;
    constexpr bool SLAB = MODE == 1 && TileY<N, T>::slab_fits;
    __shared__ T ks[SLAB ? KZ * TL::LS : 1];
    fft::load_twiddles<N, T>(tw, tw_g);
    const int KX = g.KX;
    const int l = threadIdx.x % TL::LS, j = threadIdx.x / TL::LS;
    const int i = bx * TL::LS + l;  // line p * KX + kx
    const bool ok = i < KX * line_planes<MODE>(g);
    const int Ny = g.N[1];
    pdl_trigger();
    if constexpr (SLAB) {
        // the spectrum is fixed at plan time, so it is read before waiting on
        // the previous pass; thread (l, j) fetches kz = j, j + G, ... of line l
        if (ok) {
            const int p = i / KX, kx = i - p * KX;
            const int kyf = p <= Ny / 2 ? p : Ny - p;
            const int kstride = (Ny / 2 + 1) * KX;
            const T *kcol = kh_of<T>(g) + kyf * KX + kx + j * kstride;
            const T mul = mul_of<T>(g);
#pragma unroll
            for (int kz = j, q = 0; q < (KZ + G - 1) / G; q++, kz += G)
                if (kz < KZ) ks[kz * TL::LS + l] = mul * __ldg(kcol + q * G * kstride);
        }
    }
    pdl_wait();  // the previous pass (or the producer of src) is complete
    const int Es1 = g.Es[1], Es2 = g.Es[2], Et1 = g.Et[1], Et2 = g.Et[2];
    SM sm{TL::LSP};
    cx<T> v[E];
    {
        // element pos of the line sits at ibase[pos * istride]
        const cx<T> *ibase;
        int istride;
        if constexpr (MODE == 1) {
            ibase = in + (size_t)c * Es2 * Ny * KX + i;
            istride = Ny * KX;
        } else {
            const int p = i / KX, kx = i - p * KX;
            ibase = in + ((size_t)c * (MODE == 0 ? Es2 : Et2) + p) * (MODE == 0 ? Es1 : Ny) * KX + kx;
            istride = KX;
        }
        constexpr bool INV0 = MODE == 2;  // first transform direction
        const int ilim = MODE == 0 ? Es1 : (MODE == 1 ? Es2 : N);
#pragma unroll
        for (int e = 0; e < E; e++) {
            v[e] = {(T)0, (T)0};
            const int pos = fft::in_pos<N, INV0>(e, j);
            const bool live = MODE == 2 || fft::in_lower_half<N, false>(e);
            if (live && ok && pos < ilim) v[e] = ibase[pos * istride];
        }
    }
    __syncthreads();  // twiddles
    if constexpr (MODE == 0) {
        fft::transform<N, false, true, T, true>(v, buf, tw, sm, l, j);
        if (ok) {
            const int p = i / KX, kx = i - p * KX;
            cx<T> *obase = out + (((size_t)c * Es2 + p) * N) * KX + kx;
#pragma unroll
            for (int e = 0; e < E; e++) obase[fft::out_pos<N, false>(e, j) * KX] = v[e];
        }
    } else if constexpr (MODE == 1) {
        fft::transform<N, false, true, T, true>(v, buf, tw, sm, l, j);
        if constexpr (SLAB) {
            // element e sits at kz position C + j, C = out_pos(e, 0) a multiple
            // of G; its folded index is C + j below N/2 and N - C - j from N/2 on
            const T *k_lo = ks + j * TL::LS + l;
            const T *k_hi = ks + l - j * TL::LS;
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int C = fft::out_pos<N, false>(e, 0);
                const T w = C < N / 2 ? k_lo[C * TL::LS] : k_hi[(N - C) * TL::LS];
                v[e] = {v[e].x * w, v[e].y * w};
            }
        } else {
            const int p = ok ? i / KX : 0, kx = ok ? i - p * KX : 0;
            const int kyf = p <= Ny / 2 ? p : Ny - p;
            const T *krow = kh_of<T>(g) + kyf * KX + kx;
            const int kstride = (Ny / 2 + 1) * KX;
            const T mul = mul_of<T>(g);
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int pos = fft::out_pos<N, false>(e, j);
                const int kzf = pos <= N / 2 ? pos : N - pos;
                const T w = mul * __ldg(krow + kzf * kstride);
                v[e] = {v[e].x * w, v[e].y * w};
            }
        }
        fft::transform<N, true, true, T>(v, buf, tw, sm, l, j);
        if (ok) {
            const int dz = g.T0[2] - g.S0[2];
            cx<T> *obase = out + (size_t)c * Et2 * Ny * KX + i;
            const int ostride = Ny * KX;
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int zt = wrap_mod<N>(fft::out_pos<N, true>(e, j) - dz);
                if (zt < Et2) obase[zt * ostride] = v[e];
            }
        }
    } else {
        fft::transform<N, true, true, T>(v, buf, tw, sm, l, j);
        if (ok) {
            const int p = i / KX, kx = i - p * KX;
            const int dy = g.T0[1] - g.S0[1];
            cx<T> *obase = out + (((size_t)c * Et2 + p) * Et1) * KX + kx;
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int yt = wrap_mod<N>(fft::out_pos<N, true>(e, j) - dy);
                if (yt < Et1) obase[yt * KX] = v[e];
            }
        }
    }
}
template <int N, int MODE, typename T>
__global__ void __launch_bounds__(TileY<N, T>::threads, TileY<N, T>::minb(MODE))
    k_line(Geom g, const cx<T> *__restrict__ in, cx<T> *__restrict__ out, const void *tw_g)
{
    line_body<N, MODE, T>(g, in, out, tw_g, blockIdx.x, blockIdx.y);
}

// z pass on line pairs (FP32, N = 128, 256 with 16 elements per lane and
// N = 384 with 24): lanes of a packed value carry lines 2q and
// 2q+1, so the forward transform, the spectral multiply and the inverse
// transform of both lines run as one stream of .f32x2 instructions (a third
// fewer instructions than k_line<N, 1, float>).
// Same arrays and results as k_line<N, 1, float>; a 16-byte access moves one
// element of both lines.  The twiddle table holds pairs (w, w) so that a
// stage twiddle is one 128-bit shared load.
template <int N>
struct TileZ2 {
    static constexpr int G = Plan<N>::G;
    // line pairs per block: 24-element lanes take 64-thread blocks; G = 12 (288) takes 8
    // pairs, 96 threads and 55 KB of shared memory, so that an 8-thread phase of a 128-bit
    // access covers one 128-byte exchange row (the pass 138 -> 121 us on the 256^3 step
    // against 5 pairs; 6 pairs: 196 us; 4 pairs: 146 us)
    static constexpr int LS = G == 12 ? 8 : (Plan<N>::E > 16 ? 64 : 128) / G;
    static constexpr int threads = LS * G;
    // 170 / 128 registers per thread (160 for G = 12)
    static constexpr int minb = G == 12 ? 4 : (Plan<N>::E > 16 ? 6 : 4);
};

template <int N>
__device__ __forceinline__ void zmid2_body(const Geom &g, const cx<float> *__restrict__ in,
                                           cx<float> *__restrict__ out, const void *tw_g, int bx, int c)
{
    using TL = TileZ2<N>;
    using P = fft::f32x2;
    constexpr int E = Plan<N>::E;
    constexpr int G = Plan<N>::G;
    constexpr int KZ = N / 2 + 1;
    static_assert(E == 16 || E == 24, "packed z pass: 16 or 24 elements per lane");
    using SM = fft::Smem<N, true>;
    // line-fast exchange rows of LS 16-byte entries: every 8-thread phase of a
    // 128-bit access touches one contiguous 128-byte row, so no padding
    __shared__ cx<P> buf[N * TL::LS];
    __shared__ cx<P> tw[fft::tw_size<N>()];
    __shared__ float2 ks[KZ * TL::LS];  // spectrum columns of both lines, scaled
    fft::load_twiddles<N, P>(tw, tw_g);
    const int KX = g.KX, Ny = g.N[1];
    const int l = threadIdx.x % TL::LS, j = threadIdx.x / TL::LS;
    const int q = bx * TL::LS + l;  // lines 2q, 2q+1 (numbered as in k_line)
    const int half = KX * Ny / 2;           // KX * Ny is even (Ny a power of two)
    const bool ok = q < half;
    pdl_trigger();
    if (ok) {
        // fixed at plan time: read before waiting on the previous pass
        const int kstride = (Ny / 2 + 1) * KX;
        const float *kc[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int i = 2 * q + h;
            const int p = i / KX, kx = i - p * KX;
            const int kyf = p <= Ny / 2 ? p : Ny - p;
            kc[h] = g.Kh + kyf * KX + kx;
        }
        const float mul = g.mul;
#pragma unroll
        for (int kz = j, t = 0; t < (KZ + G - 1) / G; t++, kz += G)
            if (kz < KZ)
                ks[kz * TL::LS + l] = make_float2(mul * __ldg(kc[0] + kz * kstride), mul * __ldg(kc[1] + kz * kstride));
    }
    pdl_wait();  // the previous pass is complete
    const int Es2 = g.Es[2], Et2 = g.Et[2];
    const size_t pstride = (size_t)Ny * KX / 2;  // float4 per z plane
    SM sm{TL::LS};
    cx<P> v[E];
    {
        const float4 *ibase = reinterpret_cast<const float4 *>(in + (size_t)c * Es2 * Ny * KX) + q;
#pragma unroll
        for (int e = 0; e < E; e++) {
            const int pos = fft::in_pos<N, false>(e, j);
            float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
            if (fft::in_lower_half<N, false>(e) && ok && pos < Es2) d = ibase[pos * pstride];
            v[e] = {fft::pk2(d.x, d.z), fft::pk2(d.y, d.w)};
        }
    }
    __syncthreads();  // twiddles, spectrum columns
    fft::transform<N, false, true, P, true>(v, buf, tw, sm, l, j);
    {
        // element e sits at kz position C + j, C = out_pos(e, 0) a multiple of G;
        // its folded index is C + j below N/2 and N - C - j from N/2 on
        const float2 *k_lo = ks + j * TL::LS + l;
        const float2 *k_hi = ks + l - j * TL::LS;
#pragma unroll
        for (int e = 0; e < E; e++) {
            const int C = fft::out_pos<N, false>(e, 0);
            const float2 w = C < N / 2 ? k_lo[C * TL::LS] : k_hi[(N - C) * TL::LS];
            const P W = fft::pk2(w.x, w.y);
            v[e] = {v[e].x * W, v[e].y * W};
        }
    }
    fft::transform<N, true, true, P>(v, buf, tw, sm, l, j);
    if (ok) {
        const int dz = g.T0[2] - g.S0[2];
        float4 *obase = reinterpret_cast<float4 *>(out + (size_t)c * Et2 * Ny * KX) + q;
#pragma unroll
        for (int e = 0; e < E; e++) {
            const int zt = wrap_mod<N>(fft::out_pos<N, true>(e, j) - dz);
            if (zt < Et2) {
                float ra, rb, ia, ib;
                fft::unpk2(v[e].x, ra, rb);
                fft::unpk2(v[e].y, ia, ib);
                obase[zt * pstride] = make_float4(ra, ia, rb, ib);
            }
        }
    }
}
template <int N>
__global__ void __launch_bounds__(TileZ2<N>::threads, TileZ2<N>::minb)
    k_zmid2(Geom g, const cx<float> *__restrict__ in, cx<float> *__restrict__ out, const void *tw_g)
{
    zmid2_body<N>(g, in, out, tw_g, blockIdx.x, blockIdx.y);
}

// x inverse: two target rows per complex line (Z = A + i B with Hermitian
// extension), C2R, scatter into the target block list.
// bx: this thread block's tile; c: workspace component (g.c0 + c in the target layout)
template <int N, typename T>
__device__ __forceinline__ void x_inv_body(const Geom &g, const cx<T> *__restrict__ in, T *__restrict__ dst,
                                           const void *tw_g, int bx, int c)
{
    using TL = TileX<N, T>;
    constexpr int E = Plan<N>::E;
    using SM = fft::Smem<N, false>;
    // block-list lookups of the lines' rows: the target extent is < N and
    // B >= 8, so a row meets at most N/8 blocks
    constexpr int NBX = N / 8;
    __shared__ cx<T> buf[TL::LS * SM::NP + 8];
    __shared__ cx<T> tw[fft::tw_size<N>()];
    __shared__ int lut_d[TL::LS * NBX];
    fft::load_twiddles<N, T>(tw, tw_g);
    constexpr int KX = N / 2 + 1;
    const int j = threadIdx.x % TL::G, l = threadIdx.x / TL::G;
    const int nrows = g.Et[1] * g.Et[2];
    const int lB = g.lB;
    // the lookup table is fixed at plan time: read it before waiting
    int mine = 0;  // whether this thread's lookups found a block
    for (int q = threadIdx.x; q < TL::LS * NBX; q += TL::threads) {
        const int ll = q / NBX, xb = q - ll * NBX;
        const int rr = 2 * (bx * TL::LS + ll);
        int b = -1;
        if (rr < nrows && xb < g.nbT[0]) {
            const int zz = rr / g.Et[1], yy = rr - zz * g.Et[1];
            b = __ldg(g.dst_lut + ((zz >> lB) * g.nbT[1] + (yy >> lB)) * g.nbT[0] + xb);
        }
        lut_d[q] = b;
        mine |= b >= 0;
    }
    // a thread block whose rows meet no target block has nothing to write
    if (!__syncthreads_or(mine)) return;
    pdl_trigger();
    pdl_wait();  // the previous pass (or the producer of src) is complete
    const int r0 = 2 * (bx * TL::LS + l);
    const bool row_ok = r0 < nrows;
    const size_t row = ((size_t)c * nrows + (row_ok ? r0 : 0)) * KX;
    cx<T> v[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        v[e] = {(T)0, (T)0};
        if (row_ok) {
            const int pos = fft::in_pos<N, true>(e, j);
            cx<T> a, b;
            if (pos <= N / 2) {
                a = in[row + pos];
                b = in[row + KX + pos];
            } else {
                a = conj(in[row + (N - pos)]);
                b = conj(in[row + KX + (N - pos)]);
            }
            v[e] = {a.x - b.y, a.y + b.x};
        }
    }
    __syncthreads();  // twiddles
    SM sm{0};
    fft::transform<N, true, false, T>(v, buf, tw, sm, l, j);
    if (!row_ok) return;
    const int B = g.B;
    const int zt = r0 / g.Et[1], yt = r0 - zt * g.Et[1];
    const int mB = B - 1;
    const int *lut = lut_d + l * NBX;
    const int out_blk = (((zt & mB) << lB) + (yt & mB)) << lB;
    const int dx0 = g.T0[0] - g.S0[0];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int xt = wrap_mod<N>(fft::out_pos<N, true>(e, j) - dx0);
        if (xt < g.Et[0]) {
            const int blk = lut[xt >> lB];
            if (blk >= 0) {
                T *p = dst + ((size_t)(blk * g.ncomp + g.c0 + c) << (3 * lB)) + out_blk + (xt & mB);
                p[0] = v[e].x;
                p[B] = v[e].y;
            }
        }
    }
}
template <int N, typename T>
__global__ void __launch_bounds__(TileX<N, T>::threads, TileX<N, T>::minb) k_x_inv(Geom g, const cx<T> *__restrict__ in,
                                                                 T *__restrict__ dst, const void *tw_g)
{
    x_inv_body<N, T>(g, in, dst, tw_g, blockIdx.x, blockIdx.y);
}

template <typename T>
const void *tw_table() { return sizeof(T) == 8 ? (const void *)twiddle_table_f64() : (const void *)twiddle_table_f32(); }

template <int N, typename T>
lgf_status launch_x_fwd(const Geom &g, const T *src, cx<T> *out, cudaStream_t s)
{
    using TL = TileX<N, T>;
    const int nrows = g.Es[1] * g.Es[2];
    dim3 grid(ceil_div(nrows / 2, TL::LS), g.nc);
    LGF_CUDA_TRY(launch_pdl(k_x_fwd<N, T>, grid, dim3(TL::threads), s, g, src, out, tw_table<T>()));
    return LGF_OK;
}
template <int N, int MODE, typename T>
lgf_status launch_line(const Geom &g, const cx<T> *in, cx<T> *out, cudaStream_t s)
{
    using TL = TileY<N, T>;
    const int planes = MODE == 0 ? g.Es[2] : (MODE == 1 ? g.N[1] : g.Et[2]);
    dim3 grid(ceil_div(g.KX * planes, TL::LS), g.nc);
    LGF_CUDA_TRY(launch_pdl(k_line<N, MODE, T>, grid, dim3(TL::threads), s, g, in, out, tw_table<T>()));
    return LGF_OK;
}
template <int N>
lgf_status launch_zmid2(const Geom &g, const cx<float> *in, cx<float> *out, cudaStream_t s)
{
    using TL = TileZ2<N>;
    dim3 grid(ceil_div(g.KX * g.N[1] / 2, TL::LS), g.nc);
    LGF_CUDA_TRY(launch_pdl(k_zmid2<N>, grid, dim3(TL::threads), s, g, in, out, tw_table<float>()));
    return LGF_OK;
}
// the packed z pass covers the FP32 plans with 16 elements per lane, 288 and
// 384 (measured faster there; 96 and 192 keep the scalar pass)
template <int N, typename T>
constexpr bool use_zmid2()
{
    return sizeof(T) == 4 && (Plan<N>::E == 16 || N == 288 || N == 384) && Plan<N>::G > 1 &&
           fft::tw_stage_tables<N>();
}
template <int N, typename T>
lgf_status launch_x_inv(const Geom &g, const cx<T> *in, T *dst, cudaStream_t s)
{
    using TL = TileX<N, T>;
    const int nrows = g.Et[1] * g.Et[2];
    dim3 grid(ceil_div(nrows / 2, TL::LS), g.nc);
    LGF_CUDA_TRY(launch_pdl(k_x_inv<N, T>, grid, dim3(TL::threads), s, g, in, dst, tw_table<T>()));
    return LGF_OK;
}

// Grouped launches (poisson_passes.hpp): the thread block finds its task, then runs
// the same body on that unit's geometry and buffers.
template <int N, typename T>
__global__ void __launch_bounds__(TileX<N, T>::threads, TileX<N, T>::minb)
    k_x_fwd_grp(const GroupTask<T> *__restrict__ tasks, const int *__restrict__ cta_task, SolvePtrs<T> ptrs,
                const void *tw_g)
{
    const GroupTask<T> &t = tasks[__ldg(cta_task + blockIdx.x)];
    const Geom g = t.g;
    x_fwd_body<N, T>(g, ptrs.src[t.solve], t.wa, tw_g, blockIdx.x - t.first, 0);
}
template <int N, int MODE, typename T>
__global__ void __launch_bounds__(TileY<N, T>::threads, TileY<N, T>::minb(MODE))
    k_line_grp(const GroupTask<T> *__restrict__ tasks, const int *__restrict__ cta_task, const void *tw_g)
{
    const GroupTask<T> &t = tasks[__ldg(cta_task + blockIdx.x)];
    const Geom g = t.g;
    // y forward wa -> wb, z wb -> wa, y inverse wa -> wb
    line_body<N, MODE, T>(g, MODE == 1 ? t.wb : t.wa, MODE == 1 ? t.wa : t.wb, tw_g, blockIdx.x - t.first, 0);
}
template <int N>
__global__ void __launch_bounds__(TileZ2<N>::threads, TileZ2<N>::minb)
    k_zmid2_grp(const GroupTask<float> *__restrict__ tasks, const int *__restrict__ cta_task, const void *tw_g)
{
    const GroupTask<float> &t = tasks[__ldg(cta_task + blockIdx.x)];
    const Geom g = t.g;
    zmid2_body<N>(g, t.wb, t.wa, tw_g, blockIdx.x - t.first, 0);
}
template <int N, typename T>
__global__ void __launch_bounds__(TileX<N, T>::threads, TileX<N, T>::minb)
    k_x_inv_grp(const GroupTask<T> *__restrict__ tasks, const int *__restrict__ cta_task, SolvePtrs<T> ptrs,
                const void *tw_g)
{
    const GroupTask<T> &t = tasks[__ldg(cta_task + blockIdx.x)];
    const Geom g = t.g;
    x_inv_body<N, T>(g, t.wb, ptrs.dst[t.solve], tw_g, blockIdx.x - t.first, 0);
}

}  // namespace

template <int N, typename T>
int PoissonPasses<N, T>::tiles(int pass, const Geom &g)
{
    switch (pass) {
        case 0: return ceil_div(g.Es[1] * g.Es[2] / 2, TileX<N, T>::LS);
        case 1: return ceil_div((long long)g.KX * g.Es[2], TileY<N, T>::LS);
        case 2:
            if constexpr (use_zmid2<N, T>()) return ceil_div((long long)g.KX * g.N[1] / 2, TileZ2<N>::LS);
            else return ceil_div((long long)g.KX * g.N[1], TileY<N, T>::LS);
        case 3: return ceil_div((long long)g.KX * g.Et[2], TileY<N, T>::LS);
        default: return ceil_div(g.Et[1] * g.Et[2] / 2, TileX<N, T>::LS);
    }
}

template <int N, typename T>
lgf_status PoissonPasses<N, T>::grouped(int pass, const GroupTask<T> *tasks, const int *cta_task, int ncta,
                                        const SolvePtrs<T> &ptrs, cudaStream_t s)
{
    const void *tw = tw_table<T>();
    switch (pass) {
        case 0:
            LGF_CUDA_TRY(launch_pdl(k_x_fwd_grp<N, T>, dim3(ncta), dim3(TileX<N, T>::threads), s, tasks, cta_task,
                                    ptrs, tw));
            break;
        case 1:
            LGF_CUDA_TRY(launch_pdl(k_line_grp<N, 0, T>, dim3(ncta), dim3(TileY<N, T>::threads), s, tasks, cta_task, tw));
            break;
        case 2:
            if constexpr (use_zmid2<N, T>())
                LGF_CUDA_TRY(launch_pdl(k_zmid2_grp<N>, dim3(ncta), dim3(TileZ2<N>::threads), s, tasks, cta_task, tw));
            else
                LGF_CUDA_TRY(
                    launch_pdl(k_line_grp<N, 1, T>, dim3(ncta), dim3(TileY<N, T>::threads), s, tasks, cta_task, tw));
            break;
        case 3:
            LGF_CUDA_TRY(launch_pdl(k_line_grp<N, 2, T>, dim3(ncta), dim3(TileY<N, T>::threads), s, tasks, cta_task, tw));
            break;
        default:
            LGF_CUDA_TRY(launch_pdl(k_x_inv_grp<N, T>, dim3(ncta), dim3(TileX<N, T>::threads), s, tasks, cta_task,
                                    ptrs, tw));
    }
    return LGF_OK;
}

template <int N, typename T>
lgf_status PoissonPasses<N, T>::x_fwd(const Geom &g, const T *src, cx<T> *out, cudaStream_t s)
{
    return launch_x_fwd<N, T>(g, src, out, s);
}
template <int N, typename T>
lgf_status PoissonPasses<N, T>::y_fwd(const Geom &g, const cx<T> *in, cx<T> *out, cudaStream_t s)
{
    return launch_line<N, 0, T>(g, in, out, s);
}
template <int N, typename T>
lgf_status PoissonPasses<N, T>::z_mid(const Geom &g, const cx<T> *in, cx<T> *out, cudaStream_t s)
{
    if constexpr (use_zmid2<N, T>()) return launch_zmid2<N>(g, (const cx<float> *)in, (cx<float> *)out, s);
    else return launch_line<N, 1, T>(g, in, out, s);
}
template <int N, typename T>
lgf_status PoissonPasses<N, T>::y_inv(const Geom &g, const cx<T> *in, cx<T> *out, cudaStream_t s)
{
    return launch_line<N, 2, T>(g, in, out, s);
}
template <int N, typename T>
lgf_status PoissonPasses<N, T>::x_inv(const Geom &g, const cx<T> *in, T *dst, cudaStream_t s)
{
    return launch_x_inv<N, T>(g, in, dst, s);
}

}  // namespace lgf
