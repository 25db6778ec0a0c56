// Block-sparse Poisson solve: the LGF split into a compact near part and a smooth
// far part, the near part convolved block pair by block pair and the far part on a
// coarse lattice through Lagrange interpolation (the near-field / far-field
// structure of the LGF-FMM the paper uses, Sec. 2.2 "evaluated to tolerance eps").
//
// Split.  In the Bessel form of App. B, G(n) = -int_0^inf prod_i i_{n_i}(t) dt with
// i_n(t) = e^{-2t} I_n(2t).  With a split time a:
//     G_near(n) = -int_0^a  prod_i i_{n_i}(t) dt,   G_far(n) = -int_a^inf prod_i i_{n_i}(t) dt,
// G = G_near + G_far exactly.  G_far = e^{a L} G (the semigroup of Sec. 2.3), so it is
// smooth on the scale sqrt(2a); G_near decays like the heat kernel at time a.
//
// Near field.  Blocks of 16^3 cells.  For a target block t and a source block
// s = t - d, the pair's offsets n - m = 16 d + j, |j_i| <= 15, fit a circular
// convolution of length 32: the source block zero-padded to 32^3 (R2C, kept
// spectrum 32 x 32 x 17) times the spectrum of the window w_d(j) = G_near(16 d + j)
// (computed once per plan in FP64).  Per target, the spectra of all kept offsets d
// in [-2, 2]^3 are summed (spectral multiply-accumulate), then one C2R returns the
// 16^3 result.  Spectra are stored frequency-major in chunks of 32 frequencies,
// [chunk][block][32], so that the multiply-accumulate reads 256-byte rows.
//
// Far field.  Coarse lattice nodes c at fine positions 2c.  Interpolation phi_c(n):
// an even fine index takes its node; an odd index n = 2j + 1 takes the 10-point
// Lagrange midpoint rule on nodes j-4 .. j+5.  Then
//     u_far(n) ~ sum_c phi_c(n) v(c),  v(c) = sum_c' G_far(2 (c - c')) q(c'),
//     q(c') = sum_m phi_c'(m) f(m)            (anterpolation, the transpose),
// i.e. G_far(x - y) is replaced by its tensor-product interpolant in x and y.  The
// coarse convolution v = G_far(2 .) * q runs as a whole-box zero-padded FFT
// convolution (the exact embedding of the library's plain plans) on coarse blocks of
// 16^3 nodes.  Per fine block of 16 cells the 1-D interpolation touches the 17 nodes
// 8b - 4 .. 8b + 12 (its window), so interpolation and anterpolation are 16 x 17
// matrices applied along x, y and z.
//
// u = scale dx^2 (u_near + u_far).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <unordered_map>
#include <vector>

#include "fft.cuh"
#include "plan.hpp"
#include "tc.cuh"

namespace lgf {
namespace {

constexpr int BN = 16;                 // near-field block edge
constexpr int NF = 32;                 // near-field FFT length
constexpr int KXN = NF / 2 + 1;        // kept x frequencies
constexpr int NFREQ = NF * NF * KXN;   // 17408
constexpr int CH = 32;                 // frequencies per chunk
constexpr int NCHUNK = NFREQ / CH;     // 544
constexpr int RNEAR = 2;               // near offsets d in [-RNEAR, RNEAR]^3
constexpr int KNEAR = RNEAR * BN + BN - 1;  // largest |offset| a near window samples (47)
constexpr int PINT = 10;               // interpolation points per axis (Lagrange order PINT - 1)
constexpr int WOFF = PINT / 2 - 1;     // a block's window starts at node 8 b - WOFF
constexpr int W = BN / 2 - 1 + PINT;   // nodes per window and axis (17)
constexpr int W3 = W * W * W;

__host__ __device__ inline int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

__device__ __forceinline__ int64_t oct_index(int a, int b, int c)
{
    int t;
    if (a < b) { t = a; a = b; b = t; }
    if (b < c) { t = b; b = c; c = t; }
    if (a < b) { t = a; a = b; b = t; }
    return (int64_t)a * (a + 1) * (a + 2) / 6 + (int64_t)b * (b + 1) / 2 + c;
}

// ---------------------------------------------------------------------------
// Plan-time kernels (FP64): windows of G_near and their DFTs.
// ---------------------------------------------------------------------------
// win[d][z][y][x] = G_near(16 d + j) at circular index (x, y, z) = j mod 32, |j_i| <= 15;
// index 16 (j = +-16) stays zero.
__global__ void k_near_windows(const double *__restrict__ oct, const int *__restrict__ offs, int noff,
                               double *__restrict__ win)
{
    const int64_t total = (int64_t)noff * NF * NF * NF;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % NF), y = (int)((i / NF) % NF), z = (int)((i / (NF * NF)) % NF);
        const int d = (int)(i / (NF * NF * NF));
        double v = 0.0;
        if (x != NF / 2 && y != NF / 2 && z != NF / 2) {
            const int jx = x < NF / 2 ? x : x - NF, jy = y < NF / 2 ? y : y - NF, jz = z < NF / 2 ? z : z - NF;
            const int nx = abs(BN * offs[3 * d] + jx), ny = abs(BN * offs[3 * d + 1] + jy),
                      nz = abs(BN * offs[3 * d + 2] + jz);
            v = oct[oct_index(nx, ny, nz)];
        }
        win[i] = v;
    }
}

// DFT along x of real windows: out[d][z][y][kx] (kx < 17), complex FP64
__global__ void k_near_dft_x(const double *__restrict__ win, int noff, double2 *__restrict__ out,
                             const double2 *__restrict__ tw)
{
    const int64_t total = (int64_t)noff * NF * NF * KXN;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % KXN);
        const int64_t row = i / KXN;
        const double *r = win + row * NF;
        double re = 0.0, im = 0.0;
        for (int x = 0; x < NF; x++) {
            const double2 w = tw[(kx * x) % NF];
            re = fma(r[x], w.x, re);
            im = fma(r[x], w.y, im);
        }
        out[i] = make_double2(re, im);
    }
}

// complex DFT along y (axis 1) or z (axis 2) of [d][z][y][kx] arrays
__global__ void k_near_dft_yz(const double2 *__restrict__ in, int noff, int axis, double2 *__restrict__ out,
                              const double2 *__restrict__ tw)
{
    const int64_t total = (int64_t)noff * NF * NF * KXN;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % KXN), y = (int)((i / KXN) % NF), z = (int)((i / (KXN * NF)) % NF);
        const int64_t d = i / ((int64_t)KXN * NF * NF);
        const int k = axis == 1 ? y : z;
        const int64_t stride = axis == 1 ? KXN : (int64_t)KXN * NF;
        const int64_t base = d * NF * NF * KXN + (axis == 1 ? (int64_t)z * NF * KXN + kx : (int64_t)y * KXN + kx);
        double re = 0.0, im = 0.0;
        for (int m = 0; m < NF; m++) {
            const double2 w = tw[(k * m) % NF];
            const double2 v = in[base + m * stride];
            re += v.x * w.x - v.y * w.y;
            im += v.x * w.y + v.y * w.x;
        }
        out[i] = make_double2(re, im);
    }
}

// [d][kz][ky][kx] FP64 -> chunked FP32 [chunk][d][32], frequency f = (kz * 32 + ky) * 17 + kx
__global__ void k_near_pack(const double2 *__restrict__ in, int noff, float2 *__restrict__ out)
{
    const int64_t total = (int64_t)noff * NFREQ;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(i % NFREQ);
        const int d = (int)(i / NFREQ);
        const double2 v = in[i];
        out[((int64_t)(f / CH) * noff + d) * CH + (f % CH)] = make_float2((float)v.x, (float)v.y);
    }
}

// ---------------------------------------------------------------------------
// Near field, per execution.
// ---------------------------------------------------------------------------
constexpr int SM_S1 = BN * BN * KXN;       // [z < 16][y < 16][kx]
constexpr int SM_S2 = BN * NF * KXN;       // [z < 16][ky < 32][kx]
constexpr size_t NEAR_SMEM = (size_t)(SM_S1 + SM_S2) * sizeof(float2);

// Forward: one thread block per (source block, component).  R2C of the 16^3 block
// zero-padded to 32^3: x (two real rows per complex line), y, z; the spectrum is
// written chunked: S[((c * NCHUNK + chunk) * nsrc + b) * 32 + j].
__global__ void __launch_bounds__(256) k_near_fwd(const float *__restrict__ src, int ncomp, int c0, int nsrc,
                                                   float2 *__restrict__ S)
{
    extern __shared__ float2 sm[];
    float2 *S1 = sm;
    float2 *S2 = sm + SM_S1;
    const int b = blockIdx.x, c = blockIdx.y;
    const int t = threadIdx.x;
    const float *f = src + ((size_t)b * ncomp + c0 + c) * (BN * BN * BN);
    pdl_wait();
    if (t < 128) {
        cx<float> a[NF];
        const float4 *r0 = reinterpret_cast<const float4 *>(f + (2 * t) * BN);
        const float4 *r1 = reinterpret_cast<const float4 *>(f + (2 * t + 1) * BN);
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const float4 u = r0[i], v = r1[i];
            a[4 * i + 0] = {u.x, v.x};
            a[4 * i + 1] = {u.y, v.y};
            a[4 * i + 2] = {u.z, v.z};
            a[4 * i + 3] = {u.w, v.w};
        }
#pragma unroll
        for (int i = BN; i < NF; i++) a[i] = {0.f, 0.f};
        fft::dft_reg<NF, false, float, 0, true>(a);
        // rows 2t (real part) and 2t + 1 (imaginary part) from Z = X0 + i X1
#pragma unroll
        for (int k = 0; k < KXN; k++) {
            const cx<float> zk = a[k], zm = a[(NF - k) & (NF - 1)];
            S1[(2 * t) * KXN + k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            S1[(2 * t + 1) * KXN + k] = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
        }
    }
    __syncthreads();
    for (int l = t; l < BN * KXN; l += 256) {  // y lines (z, kx)
        const int z = l / KXN, kx = l % KXN;
        cx<float> a[NF];
#pragma unroll
        for (int y = 0; y < BN; y++) {
            const float2 v = S1[(z * BN + y) * KXN + kx];
            a[y] = {v.x, v.y};
        }
#pragma unroll
        for (int y = BN; y < NF; y++) a[y] = {0.f, 0.f};
        fft::dft_reg<NF, false, float, 0, true>(a);
#pragma unroll
        for (int ky = 0; ky < NF; ky++) S2[(z * NF + ky) * KXN + kx] = make_float2(a[ky].x, a[ky].y);
    }
    __syncthreads();
    pdl_trigger();
    float2 *out = S + (size_t)c * NCHUNK * nsrc * CH;
    for (int l = t; l < NF * KXN; l += 256) {  // z lines (ky, kx), l = ky * 17 + kx
        cx<float> a[NF];
#pragma unroll
        for (int z = 0; z < BN; z++) {
            const float2 v = S2[z * NF * KXN + l];
            a[z] = {v.x, v.y};
        }
#pragma unroll
        for (int z = BN; z < NF; z++) a[z] = {0.f, 0.f};
        fft::dft_reg<NF, false, float, 0, true>(a);
#pragma unroll
        for (int kz = 0; kz < NF; kz++) {
            const int fq = kz * (NF * KXN) + l;
            out[((size_t)(fq / CH) * nsrc + b) * CH + (fq % CH)] = make_float2(a[kz].x, a[kz].y);
        }
    }
}

// The window spectra of a chunk ([noff][32] complex, contiguous) are staged in shared
// memory by one bulk copy (TMA) that completes on an mbarrier; every thread waits on the
// barrier with a bounded poll count and, if the copy has not landed by then, the block
// records the error flag (LGF_ERR_TIMEOUT on the next check) and returns.
constexpr int STAGE_WAIT = 1 << 18;
template <typename WT>
__device__ __forceinline__ bool stage_windows(WT *Kc, const WT *src, int noff, unsigned long long *bar_s, int *err)
{
    const uint32_t bar = tc::smem_addr(bar_s);
    const uint32_t bytes = (uint32_t)noff * CH * sizeof(WT);
    if (threadIdx.x == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::mbar_expect_tx(bar, bytes);
        tc::bulk_g2s(tc::smem_addr(Kc), src, bytes, bar);
    }
    const bool ok = tc::mbar_wait(bar, 0, STAGE_WAIT);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicExch(err, 1);
            tc::mbar_wait(bar, 0, STAGE_WAIT);  // let a late copy land before the block exits
        }
        return false;
    }
    return true;
}

// Spectral multiply-accumulate: U_t(k) = sum_d W_d(k) S_{t-d}(k) over the kept offsets
// present for target t.  One thread block per (chunk, group of 64 targets, component);
// a warp per target, lane = frequency in the chunk.  pairs[off[t] .. off[t+1]) lists
// (d, s) for target t.
__global__ void __launch_bounds__(256) k_near_mac(const float2 *__restrict__ W, int noff, const float2 *__restrict__ S,
                                                   int nsrc, const int *__restrict__ off, const int2 *__restrict__ pairs,
                                                   int ndst, float2 *__restrict__ U, int *err)
{
    extern __shared__ __align__(128) float2 Kc[];  // [noff][32]
    __shared__ __align__(8) unsigned long long kbar;
    const int chunk = blockIdx.x, c = blockIdx.z;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (!stage_windows(Kc, W + (size_t)chunk * noff * CH, noff, &kbar, err)) return;
    pdl_wait();
    const float2 *Sc = S + ((size_t)c * NCHUNK + chunk) * nsrc * CH;
    float2 *Uc = U + ((size_t)c * NCHUNK + chunk) * ndst * CH;
    for (int i = 0; i < 8; i++) {
        const int t = blockIdx.y * 64 + warp * 8 + i;
        if (t >= ndst) break;
        const int beg = off[t], end = off[t + 1];
        float ar = 0.f, ai = 0.f;
        for (int base = beg; base < end; base += 32) {
            const int2 my = base + lane < end ? pairs[base + lane] : make_int2(0, 0);
            const int n = min(32, end - base);
            for (int k = 0; k < n; k++) {
                const int d = __shfl_sync(0xffffffffu, my.x, k);
                const int s = __shfl_sync(0xffffffffu, my.y, k);
                const float2 sv = Sc[(size_t)s * CH + lane];
                const float2 kv = Kc[d * CH + lane];
                ar = fmaf(kv.x, sv.x, ar);
                ar = fmaf(-kv.y, sv.y, ar);
                ai = fmaf(kv.x, sv.y, ai);
                ai = fmaf(kv.y, sv.x, ai);
            }
        }
        Uc[(size_t)t * CH + lane] = make_float2(ar, ai);
    }
    pdl_trigger();
}

// The same sum over runs of 4 x-adjacent target slots t_i = (x0 + i, y, z): for each
// (oy, oz) row the warp loads the 8 source rows x0 - 2 .. x0 + 5 once and the 5 window
// rows of ox = -2..2, and accumulates acc_i += W_(ox,oy,oz) S_(x0 + i - ox, y - oy, z - oz)
// for all 20 (i, ox): 13 row loads per 20 complex multiply-adds.  W row noff is zero
// (offsets without a window, and sources or targets that are absent).
// Packed arithmetic: each source value is broadcast once into (Re S, Re S) and (Im S, Im S),
// so a complex multiply-add is two .f32x2 FMAs on the window as loaded,
// P_i += (Re S, Re S) W and Q_i += (Im S, Im S) W, and W S = (P.re - Q.im, P.im + Q.re) at
// the end (40 packed FMAs per row where the scalar form issues 80).  A warp takes the runs
// r = blockIdx.y * 8 + warp + k * 8 gridDim.y, so one staging of a chunk's windows serves
// several runs.
__global__ void __launch_bounds__(256) k_near_mac_runs(const float2 *__restrict__ W, int noff,
                                                        const float2 *__restrict__ S, int nsrc,
                                                        const int4 *__restrict__ run_tgt,
                                                        const int *__restrict__ run_row,
                                                        const int4 *__restrict__ rows, int nruns, int ndst,
                                                        float2 *__restrict__ U, int *err)
{
    extern __shared__ __align__(128) float2 Kc[];  // [noff + 1][32]
    __shared__ __align__(8) unsigned long long kbar;
    const int chunk = blockIdx.x, c = blockIdx.z;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < CH) Kc[noff * CH + threadIdx.x] = make_float2(0.f, 0.f);
    if (!stage_windows(Kc, W + (size_t)chunk * noff * CH, noff, &kbar, err)) return;  // (its barrier orders the zero row)
    pdl_wait();
    const float2 *Sc = S + ((size_t)c * NCHUNK + chunk) * nsrc * CH;
    float2 *Uc = U + ((size_t)c * NCHUNK + chunk) * ndst * CH;
    const fft::f32x2 zero = fft::pk2(0.f, 0.f);
    for (int r = blockIdx.y * 8 + warp; r < nruns; r += gridDim.y * 8) {
        fft::f32x2 P[4] = {zero, zero, zero, zero}, Q[4] = {zero, zero, zero, zero};
        const int r0 = __ldg(run_row + r), r1 = __ldg(run_row + r + 1);
        for (int q = r0; q < r1; q++) {
            const int4 a = __ldg(rows + 4 * q), b = __ldg(rows + 4 * q + 1), cc = __ldg(rows + 4 * q + 2),
                       dd = __ldg(rows + 4 * q + 3);
            const int wrow[5] = {a.x, a.y, a.z, a.w, b.x};
            const int src[8] = {b.y, b.z, b.w, cc.x, cc.y, cc.z, cc.w, dd.x};
            fft::f32x2 sr[8], si[8];
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const float2 v = src[k] >= 0 ? Sc[(size_t)src[k] * CH + lane] : make_float2(0.f, 0.f);
                sr[k] = fft::bc2(v.x);
                si[k] = fft::bc2(v.y);
            }
#pragma unroll
            for (int o = 0; o < 5; o++) {  // ox = o - 2
                fft::f32x2 w;
                w.r = *(const unsigned long long *)(Kc + wrow[o] * CH + lane);
#pragma unroll
                for (int i = 0; i < 4; i++) {  // source x0 + i - ox = x0 - 2 + (i - o + 4)
                    P[i] = fft::fma(sr[i - o + 4], w, P[i]);  // (Re S Re W, Re S Im W)
                    Q[i] = fft::fma(si[i - o + 4], w, Q[i]);  // (Im S Re W, Im S Im W)
                }
            }
        }
        const int4 tg = __ldg(run_tgt + r);
        const int t4[4] = {tg.x, tg.y, tg.z, tg.w};
#pragma unroll
        for (int i = 0; i < 4; i++)
            if (t4[i] >= 0) {
                float pr, pi, qr, qi;
                fft::unpk2(P[i], pr, pi);
                fft::unpk2(Q[i], qr, qi);
                Uc[(size_t)t4[i] * CH + lane] = make_float2(pr - qi, pi + qr);
            }
    }
    pdl_trigger();
}

// Quads of 4 x 2 target slots t_ij = (x0 + i, y0 + j, z), y0 even: a source row (y', z - oz)
// serves slot row j = 0 with oy = y0 - y' and j = 1 with oy = y0 + 1 - y', so the 8 source rows
// a row-step loads feed up to 40 complex multiply-adds (against 20 in the run form), with the
// 5 window rows of each valid half read from shared memory.  The windows are the plan's 125
// offsets in canonical order, (ox + 2) + 5 (oy + 2) + 25 (oz + 2); a row-step names the first
// window row of each half (its ox = -2), or -1 where that half has no target.
// Row-step entry: int4 sources 0-3, int4 sources 4-7, int4 (wa, wb, 0, 0).
__global__ void __launch_bounds__(256, 4) k_near_mac_quads(const float2 *__restrict__ W, int noff,
                                                         const float2 *__restrict__ S, int nsrc,
                                                         const int4 *__restrict__ quad_tgt,
                                                         const int *__restrict__ quad_row,
                                                         const int4 *__restrict__ qrows, int nquads, int ndst,
                                                         float2 *__restrict__ U, int *err)
{
    extern __shared__ __align__(128) float2 Kc[];  // [noff][32]
    __shared__ __align__(8) unsigned long long kbar;
    const int chunk = blockIdx.x, c = blockIdx.z;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (!stage_windows(Kc, W + (size_t)chunk * noff * CH, noff, &kbar, err)) return;
    pdl_wait();
    const float2 *Sc = S + ((size_t)c * NCHUNK + chunk) * nsrc * CH;
    float2 *Uc = U + ((size_t)c * NCHUNK + chunk) * ndst * CH;
    const fft::f32x2 zero = fft::pk2(0.f, 0.f);
    for (int r = blockIdx.y * 8 + warp; r < nquads; r += gridDim.y * 8) {
        fft::f32x2 PA[4] = {zero, zero, zero, zero}, QA[4] = {zero, zero, zero, zero};
        fft::f32x2 PB[4] = {zero, zero, zero, zero}, QB[4] = {zero, zero, zero, zero};
        const int r0 = __ldg(quad_row + r), r1 = __ldg(quad_row + r + 1);
        for (int q = r0; q < r1; q++) {
            const int4 a = __ldg(qrows + 3 * q), b = __ldg(qrows + 3 * q + 1), m = __ldg(qrows + 3 * q + 2);
            const int src[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            fft::f32x2 sr[8], si[8];
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const float2 v = src[k] >= 0 ? Sc[(size_t)src[k] * CH + lane] : make_float2(0.f, 0.f);
                sr[k] = fft::bc2(v.x);
                si[k] = fft::bc2(v.y);
            }
            if (m.x >= 0) {
#pragma unroll
                for (int o = 0; o < 5; o++) {  // ox = o - 2; source x0 + i - ox
                    fft::f32x2 w;
                    w.r = *(const unsigned long long *)(Kc + (m.x + o) * CH + lane);
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        PA[i] = fft::fma(sr[i - o + 4], w, PA[i]);
                        QA[i] = fft::fma(si[i - o + 4], w, QA[i]);
                    }
                }
            }
            if (m.y >= 0) {
#pragma unroll
                for (int o = 0; o < 5; o++) {
                    fft::f32x2 w;
                    w.r = *(const unsigned long long *)(Kc + (m.y + o) * CH + lane);
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        PB[i] = fft::fma(sr[i - o + 4], w, PB[i]);
                        QB[i] = fft::fma(si[i - o + 4], w, QB[i]);
                    }
                }
            }
        }
        const int4 ta = __ldg(quad_tgt + 2 * r), tb = __ldg(quad_tgt + 2 * r + 1);
        const int t8[8] = {ta.x, ta.y, ta.z, ta.w, tb.x, tb.y, tb.z, tb.w};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            float pr, pi, qr, qi;
            if (t8[i] >= 0) {
                fft::unpk2(PA[i], pr, pi);
                fft::unpk2(QA[i], qr, qi);
                Uc[(size_t)t8[i] * CH + lane] = make_float2(pr - qi, pi + qr);
            }
            if (t8[4 + i] >= 0) {
                fft::unpk2(PB[i], pr, pi);
                fft::unpk2(QB[i], qr, qi);
                Uc[(size_t)t8[4 + i] * CH + lane] = make_float2(pr - qi, pi + qr);
            }
        }
    }
    pdl_trigger();
}

// Inverse: one thread block per (target block, component): z, y (keeping the first
// 16 outputs of each), then C2R in x with two rows per complex line; adds
// mul * result (the target window of the circular convolution) to dst, which holds the
// far field.
__global__ void __launch_bounds__(256) k_near_inv(const float2 *__restrict__ U, int ndst, float *__restrict__ dst,
                                                   int ncomp, int c0, float mul)
{
    extern __shared__ float2 sm[];
    float2 *S1 = sm;          // [z][y][kx]
    float2 *S2 = sm + SM_S1;  // [z][ky][kx]
    const int b = blockIdx.x, c = blockIdx.y;
    const int t = threadIdx.x;
    const float2 *in = U + (size_t)c * NCHUNK * ndst * CH;
    pdl_wait();
    for (int l = t; l < NF * KXN; l += 256) {  // z lines (ky, kx)
        cx<float> a[NF];
#pragma unroll
        for (int kz = 0; kz < NF; kz++) {
            const int fq = kz * (NF * KXN) + l;
            const float2 v = in[((size_t)(fq / CH) * ndst + b) * CH + (fq % CH)];
            a[kz] = {v.x, v.y};
        }
        fft::dft_reg<NF, true, float, 0, false>(a);
#pragma unroll
        for (int z = 0; z < BN; z++) S2[z * NF * KXN + l] = make_float2(a[z].x, a[z].y);
    }
    __syncthreads();
    for (int l = t; l < BN * KXN; l += 256) {  // y lines (z, kx)
        const int z = l / KXN, kx = l % KXN;
        cx<float> a[NF];
#pragma unroll
        for (int ky = 0; ky < NF; ky++) {
            const float2 v = S2[(z * NF + ky) * KXN + kx];
            a[ky] = {v.x, v.y};
        }
        fft::dft_reg<NF, true, float, 0, false>(a);
#pragma unroll
        for (int y = 0; y < BN; y++) S1[(z * BN + y) * KXN + kx] = make_float2(a[y].x, a[y].y);
    }
    __syncthreads();
    pdl_trigger();
    if (t < 128) {  // x: rows 2t, 2t + 1 as Z = X0 + i X1 with the Hermitian halves filled in
        cx<float> a[NF];
#pragma unroll
        for (int k = 0; k < KXN; k++) {
            const float2 p = S1[(2 * t) * KXN + k], q = S1[(2 * t + 1) * KXN + k];
            a[k] = {p.x - q.y, p.y + q.x};
        }
#pragma unroll
        for (int k = KXN; k < NF; k++) {
            const float2 p = S1[(2 * t) * KXN + (NF - k)], q = S1[(2 * t + 1) * KXN + (NF - k)];
            a[k] = {p.x + q.y, q.x - p.y};  // conj(p) + i conj(q)
        }
        fft::dft_reg<NF, true, float, 0, false>(a);
        float *o = dst + ((size_t)b * ncomp + c0 + c) * (BN * BN * BN);
        float4 *w0 = reinterpret_cast<float4 *>(o + (2 * t) * BN);
        float4 *w1 = reinterpret_cast<float4 *>(o + (2 * t + 1) * BN);
#pragma unroll
        for (int i = 0; i < 4; i++) {  // added to the far field the interpolation wrote
            const float4 f0 = w0[i], f1 = w1[i];
            w0[i] = make_float4(f0.x + mul * a[4 * i].x, f0.y + mul * a[4 * i + 1].x, f0.z + mul * a[4 * i + 2].x,
                                f0.w + mul * a[4 * i + 3].x);
            w1[i] = make_float4(f1.x + mul * a[4 * i].y, f1.y + mul * a[4 * i + 1].y, f1.z + mul * a[4 * i + 2].y,
                                f1.w + mul * a[4 * i + 3].y);
        }
    }
}

// ---------------------------------------------------------------------------
// Far field: anterpolation, coarse charge gather, interpolation (SIMT).
// The 1-D matrix P[i][l] (fine i < 16 of a block, node l < 17 of its window
// 8b - 4 + l) is in constant memory.
// ---------------------------------------------------------------------------
__constant__ float c_P[BN * W];
// threads per block of the two SIMT kernels: one thread block per (block, component), whose
// three passes are short loops over the block's points; 512 threads keep every block of a
// few-hundred-block set resident at once
constexpr int FAR_THREADS = 512;

// Q_b[lz][ly][lx] = sum_i P[iz][lz] P[iy][ly] P[ix][lx] f_b[iz][iy][ix] (a W^3 window), per
// (source block, component)
__global__ void __launch_bounds__(FAR_THREADS) k_far_anterp(const float *__restrict__ src, int ncomp, int c0,
                                                     float *__restrict__ Q, int ncq)
{
    __shared__ float A[W3];
    __shared__ float T[W3];
    __shared__ float sP[BN * W];
    const int b = blockIdx.x, c = blockIdx.y, t = threadIdx.x;
    const float *f = src + ((size_t)b * ncomp + c0 + c) * (BN * BN * BN);
    for (int i = t; i < BN * W; i += FAR_THREADS) sP[i] = c_P[i];
    pdl_wait();
    for (int i = t; i < BN * BN * BN; i += FAR_THREADS) A[i] = f[i];
    __syncthreads();
    // x: T[z][y][lx] = sum_x P[x][lx] A[z][y][x]      (16 x 16 x W)
    for (int i = t; i < BN * BN * W; i += FAR_THREADS) {
        const int lx = i % W, row = i / W;
        float acc = 0.f;
#pragma unroll
        for (int x = 0; x < BN; x++) acc = fmaf(sP[x * W + lx], A[row * BN + x], acc);
        T[i] = acc;
    }
    __syncthreads();
    // y: A[z][ly][lx] = sum_y P[y][ly] T[z][y][lx]    (16 x W x W)
    for (int i = t; i < BN * W * W; i += FAR_THREADS) {
        const int lx = i % W, ly = (i / W) % W, z = i / (W * W);
        float acc = 0.f;
#pragma unroll
        for (int y = 0; y < BN; y++) acc = fmaf(sP[y * W + ly], T[(z * BN + y) * W + lx], acc);
        A[i] = acc;
    }
    __syncthreads();
    // z: Q[lz][ly][lx] = sum_z P[z][lz] A[z][ly][lx]  (W^3)
    float *out = Q + ((size_t)b * ncq + c) * W3;
    for (int i = t; i < W3; i += FAR_THREADS) {
        const int r = i % (W * W), lz = i / (W * W);
        float acc = 0.f;
#pragma unroll
        for (int z = 0; z < BN; z++) acc = fmaf(sP[z * W + lz], A[z * W * W + r], acc);
        out[i] = acc;
    }
    pdl_trigger();
}

// Coarse charges q on coarse block C: node n = 16 C + l receives Q_b[n - (8 b - 4)] from
// each source block b whose window holds n (up to three per axis, fixed order).
// flut: dense lookup of the fine source blocks over [fmin, fmin + fext).
constexpr int GATHER_PARTS = 8;
__global__ void __launch_bounds__(256) k_far_gather(const float *__restrict__ Q, int ncq,
                                                     const int *__restrict__ ccoords, const int *__restrict__ flut,
                                                     int3 fmin, int3 fext, float *__restrict__ q)
{
    // GATHER_PARTS thread blocks per coarse block (a slab of 16 / GATHER_PARTS planes each):
    // the coarse source blocks are few (hundreds), so one thread block each would leave
    // most SMs idle
    const int C = blockIdx.x / GATHER_PARTS, part = blockIdx.x % GATHER_PARTS, c = blockIdx.y;
    const int Cx = ccoords[3 * C], Cy = ccoords[3 * C + 1], Cz = ccoords[3 * C + 2];
    float *out = q + ((size_t)C * ncq + c) * (BN * BN * BN);
    pdl_wait();
    constexpr int PART = BN * BN * BN / GATHER_PARTS;
    for (int i = part * PART + threadIdx.x; i < (part + 1) * PART; i += 256) {
        const int nx = 16 * Cx + i % BN, ny = 16 * Cy + (i / BN) % BN, nz = 16 * Cz + i / (BN * BN);
        const int bx1 = floordiv(nx + WOFF, 8), by1 = floordiv(ny + WOFF, 8), bz1 = floordiv(nz + WOFF, 8);
        float acc = 0.f;
        for (int dz = -2; dz <= 0; dz++) {
            const int bz = bz1 + dz, lz = nz - (8 * bz - WOFF);
            if (lz >= W || bz - fmin.z < 0 || bz - fmin.z >= fext.z) continue;
            for (int dy = -2; dy <= 0; dy++) {
                const int by = by1 + dy, ly = ny - (8 * by - WOFF);
                if (ly >= W || by - fmin.y < 0 || by - fmin.y >= fext.y) continue;
                for (int dx = -2; dx <= 0; dx++) {
                    const int bx = bx1 + dx, lx = nx - (8 * bx - WOFF);
                    if (lx >= W || bx - fmin.x < 0 || bx - fmin.x >= fext.x) continue;
                    const int s = flut[((size_t)(bz - fmin.z) * fext.y + (by - fmin.y)) * fext.x + (bx - fmin.x)];
                    if (s < 0) continue;
                    acc += Q[((size_t)s * ncq + c) * W3 + (lz * W + ly) * W + lx];
                }
            }
        }
        out[i] = acc;
    }
    pdl_trigger();
}

// dst_b = mul * sum_l P[iz][lz] P[iy][ly] P[ix][lx] v(8 b - 4 + l), per (target block, component);
// v on coarse blocks through clut (dense lookup over [cmin, cmin + cext)), ncv components.
__global__ void __launch_bounds__(FAR_THREADS) k_far_interp(const float *__restrict__ v, int ncv, const int *__restrict__ tcoords,
                                                     const int *__restrict__ clut, int3 cmin, int3 cext,
                                                     float *__restrict__ dst, int ncomp, int c0, float mul)
{
    __shared__ float A[W3];
    __shared__ float T[W3];
    __shared__ float sP[BN * W];
    const int b = blockIdx.x, c = blockIdx.y, t = threadIdx.x;
    const int bx = tcoords[3 * b], by = tcoords[3 * b + 1], bz = tcoords[3 * b + 2];
    for (int i = t; i < BN * W; i += FAR_THREADS) sP[i] = c_P[i];
    pdl_wait();
    for (int i = t; i < W3; i += FAR_THREADS) {
        const int nx = 8 * bx - WOFF + i % W, ny = 8 * by - WOFF + (i / W) % W, nz = 8 * bz - WOFF + i / (W * W);
        const int Cx = floordiv(nx, 16) - cmin.x, Cy = floordiv(ny, 16) - cmin.y, Cz = floordiv(nz, 16) - cmin.z;
        float val = 0.f;
        if (Cx >= 0 && Cy >= 0 && Cz >= 0 && Cx < cext.x && Cy < cext.y && Cz < cext.z) {
            const int C = clut[((size_t)Cz * cext.y + Cy) * cext.x + Cx];
            if (C >= 0) {
                const int lx = nx - 16 * (Cx + cmin.x), ly = ny - 16 * (Cy + cmin.y), lz = nz - 16 * (Cz + cmin.z);
                val = v[((size_t)C * ncv + c) * (BN * BN * BN) + (lz * BN + ly) * BN + lx];
            }
        }
        A[i] = val;
    }
    __syncthreads();
    // x: T[lz][ly][ix] = sum_lx P[ix][lx] A[lz][ly][lx]   (W x W x 16)
    for (int i = t; i < W * W * BN; i += FAR_THREADS) {
        const int ix = i % BN, row = i / BN;
        float acc = 0.f;
#pragma unroll
        for (int l = 0; l < W; l++) acc = fmaf(sP[ix * W + l], A[row * W + l], acc);
        T[i] = acc;
    }
    __syncthreads();
    for (int i = t; i < W * BN * BN; i += FAR_THREADS) {  // y: A[lz][iy][ix]   (W x 16 x 16)
        const int ix = i % BN, iy = (i / BN) % BN, lz = i / (BN * BN);
        float acc = 0.f;
#pragma unroll
        for (int l = 0; l < W; l++) acc = fmaf(sP[iy * W + l], T[(lz * W + l) * BN + ix], acc);
        A[i] = acc;
    }
    __syncthreads();
    float *o = dst + ((size_t)b * ncomp + c0 + c) * (BN * BN * BN);
    for (int i = t; i < BN * BN * BN; i += FAR_THREADS) {  // z: the far field, to which the near field is added
        const int r = i % (BN * BN), iz = i / (BN * BN);
        float acc = 0.f;
#pragma unroll
        for (int l = 0; l < W; l++) acc = fmaf(sP[iz * W + l], A[l * BN * BN + r], acc);
        o[i] = mul * acc;
    }
    pdl_trigger();
}

// ---------------------------------------------------------------------------
// Far field on the tensor cores.  Each 1-D interpolation step is a GEMM: with the
// block's data as the A operand (rows = the two other axes, K = the axis transformed)
// and the 16 x 17 matrix P as B, D = A B^T lands in TMEM; the next step reads D back
// (one row per thread), writes it transposed as its own A operand, and so on for x, y,
// z.  Data and weights are split into two TF32 parts, x = hi + lo; each product keeps
// hi*hi + hi*lo + lo*hi (three MMAs per K step).  The tensor cores add each MMA's
// products into the FP32 accumulator with truncation, so the steps are not quite FP32
// accurate: measured ~1e-6 relative on the far field (this is the reduced-precision far
// field, held to 1e-5; a three-part split adds MMAs and measured worse).
//   anterpolation: 16^3 -> 17^3: K = 16 each step, N = 17 padded to 32, rows 256, 272, 289
//   interpolation: 17^3 -> 16^3: K = 17 padded to 24, N = 16, rows 289, 272, 256
// One 128-thread block (one warpgroup, so every TMEM lane has its thread) per block and
// component; M = 128 per MMA, up to three row tiles; TMEM: 128 columns.
// ---------------------------------------------------------------------------
constexpr int TC_THREADS = 128;
constexpr int TC_ROWS = 384;           // three 128-row tiles
constexpr int TC_TMEM_COLS = 128;
constexpr int TC_WAIT = 1 << 18;       // mbarrier polls before a wait gives up

template <int K>
struct TcSmem {
    uint32_t a_hi[TC_ROWS * K], a_lo[TC_ROWS * K];  // A operand, core-matrix layout
    uint32_t b_hi[32 * K], b_lo[32 * K];            // B operand (P), core-matrix layout
    uint64_t mbar;
    uint32_t tmem_base;
};

// Issue D[tile] = A[tile] B^T for every row tile (three MMAs per K step), commit to the
// mbarrier and wait for it (phase `ph`).  Thread 0 issues; everyone waits.  Returns false
// if the wait gave up.
template <int K, int N>
__device__ __forceinline__ bool tc_pass(TcSmem<K> &sm, int ntiles, uint32_t ph)
{
    tc::fence_smem_to_async();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::fence_after_sync();
        const uint32_t idesc = tc::idesc_tf32(128, N);
        const uint32_t sbo = K * 32;
        const uint32_t ah = tc::smem_addr(sm.a_hi), al = tc::smem_addr(sm.a_lo);
        const uint32_t bh = tc::smem_addr(sm.b_hi), bl = tc::smem_addr(sm.b_lo);
        for (int mt = 0; mt < ntiles; mt++) {
            const uint32_t d = sm.tmem_base + mt * N;
            for (int ks = 0; ks < K / 8; ks++) {
                const uint32_t ao = mt * 16 * sbo + ks * 256, bo = ks * 256;
                tc::mma_tf32(d, tc::smem_desc(ah + ao, 128, sbo), tc::smem_desc(bh + bo, 128, sbo), idesc, ks > 0);
                tc::mma_tf32(d, tc::smem_desc(ah + ao, 128, sbo), tc::smem_desc(bl + bo, 128, sbo), idesc, 1);
                tc::mma_tf32(d, tc::smem_desc(al + ao, 128, sbo), tc::smem_desc(bh + bo, 128, sbo), idesc, 1);
            }
        }
        tc::mma_commit(tc::smem_addr(&sm.mbar));
    }
    bool ok = tc::mbar_wait(tc::smem_addr(&sm.mbar), ph, TC_WAIT);
    ok = __syncthreads_and(ok) != 0;  // uniform across the block
    tc::fence_after_sync();
    return ok;
}

// this thread's row `row` of tile `mt` of the last pass: N (16 or 32) columns
template <int N>
__device__ __forceinline__ void tc_row(uint32_t tmem_base, int mt, float v[N])
{
    const int w = threadIdx.x >> 5;
    const uint32_t t = tmem_base + ((uint32_t)(32 * w) << 16) + mt * N;
    tc::tmem_ld16(t, v);
    if constexpr (N == 32) tc::tmem_ld16(t + 16, v + 16);
}

template <int K>
__device__ __forceinline__ void tc_put(TcSmem<K> &sm, int r, int k, float x)
{
    uint32_t hi, lo;
    tc::split_tf32(x, hi, lo);
    const int o = tc::core_byte(r, k, K) >> 2;
    sm.a_hi[o] = hi;
    sm.a_lo[o] = lo;
}

template <int K>
__device__ __forceinline__ void tc_setup(TcSmem<K> &sm, const uint32_t *__restrict__ Bhl)
{
    for (int i = threadIdx.x; i < 32 * K; i += TC_THREADS) {
        sm.b_hi[i] = Bhl[i];
        sm.b_lo[i] = Bhl[32 * K + i];
    }
    for (int i = threadIdx.x; i < TC_ROWS * K; i += TC_THREADS) sm.a_hi[i] = sm.a_lo[i] = 0u;
    if (threadIdx.x == 0) {
        tc::mbar_init(tc::smem_addr(&sm.mbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) tc::tmem_alloc(tc::smem_addr(&sm.tmem_base), TC_TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// ok = false: a wait gave up on phase `ph` with MMAs possibly in flight; wait for them
// once more (bounded) before the TMEM is freed
template <int K>
__device__ __forceinline__ void tc_teardown(TcSmem<K> &sm, bool ok, uint32_t ph)
{
    if (!ok && threadIdx.x == 0) tc::mbar_wait(tc::smem_addr(&sm.mbar), ph, TC_WAIT);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(sm.tmem_base, TC_TMEM_COLS);
}

__global__ void __launch_bounds__(TC_THREADS) k_far_anterp_tc(const float *__restrict__ src, int ncomp, int c0,
                                                               float *__restrict__ Q, int ncq,
                                                               const uint32_t *__restrict__ Bhl, int *err)
{
    extern __shared__ __align__(128) unsigned char tc_raw[];
    TcSmem<16> &sm = *reinterpret_cast<TcSmem<16> *>(tc_raw);
    const int b = blockIdx.x, c = blockIdx.y, t = threadIdx.x;
    tc_setup<16>(sm, Bhl);
    const float *f = src + ((size_t)b * ncomp + c0 + c) * (BN * BN * BN);
    pdl_wait();
    for (int i = t; i < BN * BN * BN; i += TC_THREADS) tc_put<16>(sm, i / BN, i % BN, f[i]);  // rows (z, y), k = x
    uint32_t ph = 0;
    bool ok = tc_pass<16, 32>(sm, 2, ph);
    float v[32];
    // D1 rows (z, y), cols lx  ->  A2 rows (z, lx), k = y
    for (int mt = 0; mt < 2 && ok; mt++) {
        const int r = mt * 128 + t;
        tc_row<32>(sm.tmem_base, mt, v);
        const int z = r / BN, y = r % BN;
        for (int l = 0; l < W; l++) tc_put<16>(sm, z * W + l, y, v[l]);
    }
    tc::fence_before_sync();
    if (ok) ok = tc_pass<16, 32>(sm, 3, ph = 1);
    // D2 rows (z, lx), cols ly  ->  A3 rows (ly, lx), k = z
    for (int mt = 0; mt < 3 && ok; mt++) {
        const int r = mt * 128 + t;
        tc_row<32>(sm.tmem_base, mt, v);
        if (r < BN * W) {
            const int z = r / W, lx = r % W;
            for (int l = 0; l < W; l++) tc_put<16>(sm, l * W + lx, z, v[l]);
        }
    }
    tc::fence_before_sync();
    if (ok) ok = tc_pass<16, 32>(sm, 3, ph = 0);
    // D3 rows (ly, lx), cols lz  ->  Q[lz][ly][lx]
    float *out = Q + ((size_t)b * ncq + c) * W3;
    for (int mt = 0; mt < 3 && ok; mt++) {
        const int r = mt * 128 + t;
        tc_row<32>(sm.tmem_base, mt, v);
        if (r < W * W)
            for (int l = 0; l < W; l++) out[l * W * W + r] = v[l];
    }
    if (!ok && t == 0) atomicExch(err, 1);
    tc_teardown<16>(sm, ok, ph);
    pdl_trigger();
}

__global__ void __launch_bounds__(TC_THREADS) k_far_interp_tc(const float *__restrict__ vc, int ncv,
                                                               const int *__restrict__ tcoords,
                                                               const int *__restrict__ clut, int3 cmin, int3 cext,
                                                               float *__restrict__ dst, int ncomp, int c0, float mul,
                                                               const uint32_t *__restrict__ Bhl, int *err)
{
    extern __shared__ __align__(128) unsigned char tc_raw[];
    TcSmem<24> &sm = *reinterpret_cast<TcSmem<24> *>(tc_raw);
    const int b = blockIdx.x, c = blockIdx.y, t = threadIdx.x;
    tc_setup<24>(sm, Bhl);
    const int bx = tcoords[3 * b], by = tcoords[3 * b + 1], bz = tcoords[3 * b + 2];
    pdl_wait();
    // the block's window of the coarse potential: rows (lz, ly), k = lx
    for (int i = t; i < W3; i += TC_THREADS) {
        const int nx = 8 * bx - WOFF + i % W, ny = 8 * by - WOFF + (i / W) % W, nz = 8 * bz - WOFF + i / (W * W);
        const int Cx = floordiv(nx, 16) - cmin.x, Cy = floordiv(ny, 16) - cmin.y, Cz = floordiv(nz, 16) - cmin.z;
        float val = 0.f;
        if (Cx >= 0 && Cy >= 0 && Cz >= 0 && Cx < cext.x && Cy < cext.y && Cz < cext.z) {
            const int C = clut[((size_t)Cz * cext.y + Cy) * cext.x + Cx];
            if (C >= 0) {
                const int lx = nx - 16 * (Cx + cmin.x), ly = ny - 16 * (Cy + cmin.y), lz = nz - 16 * (Cz + cmin.z);
                val = vc[((size_t)C * ncv + c) * (BN * BN * BN) + (lz * BN + ly) * BN + lx];
            }
        }
        tc_put<24>(sm, i / W, i % W, val);
    }
    uint32_t ph = 0;
    bool ok = tc_pass<24, 16>(sm, 3, ph);
    float v[16];
    // D1 rows (lz, ly), cols ix  ->  A2 rows (lz, ix), k = ly
    for (int mt = 0; mt < 3 && ok; mt++) {
        const int r = mt * 128 + t;
        tc_row<16>(sm.tmem_base, mt, v);
        if (r < W * W) {
            const int lz = r / W, ly = r % W;
            for (int i = 0; i < BN; i++) tc_put<24>(sm, lz * BN + i, ly, v[i]);
        }
    }
    tc::fence_before_sync();
    if (ok) ok = tc_pass<24, 16>(sm, 3, ph = 1);
    // D2 rows (lz, ix), cols iy  ->  A3 rows (iy, ix), k = lz
    for (int mt = 0; mt < 3 && ok; mt++) {
        const int r = mt * 128 + t;
        tc_row<16>(sm.tmem_base, mt, v);
        if (r < W * BN) {
            const int lz = r / BN, ix = r % BN;
            for (int i = 0; i < BN; i++) tc_put<24>(sm, i * BN + ix, lz, v[i]);
        }
    }
    tc::fence_before_sync();
    if (ok) ok = tc_pass<24, 16>(sm, 2, ph = 0);
    // D3 rows (iy, ix), cols iz: the far field, to which the near field is added
    float *o = dst + ((size_t)b * ncomp + c0 + c) * (BN * BN * BN);
    for (int mt = 0; mt < 2 && ok; mt++) {
        const int r = mt * 128 + t;
        tc_row<16>(sm.tmem_base, mt, v);
        for (int i = 0; i < BN; i++) o[i * BN * BN + r] = mul * v[i];
    }
    if (!ok && t == 0) atomicExch(err, 1);
    tc_teardown<24>(sm, ok, ph);
    pdl_trigger();
}

// The bounded wait of the tensor-core kernels, run on an mbarrier that nothing arrives on:
// after `polls` polls the wait gives up and the kernel records it in *err (no fault, no trap).
__global__ void k_wait_probe(int polls, int *err)
{
    __shared__ uint64_t mbar;
    if (threadIdx.x == 0) {
        tc::mbar_init(tc::smem_addr(&mbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = tc::mbar_wait(tc::smem_addr(&mbar), 0, polls);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
template <typename T>
lgf_status dalloc_n(T **p, size_t n, size_t &bytes)
{
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc(p, n * sizeof(T));
    if (e != cudaSuccess) {
        set_error("device allocation of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
        return LGF_ERR_OOM;
    }
    bytes += n * sizeof(T);
    return LGF_OK;
}
template <typename T>
lgf_status upload_v(T *d, const std::vector<T> &h, cudaStream_t s)
{
    if (h.empty()) return LGF_OK;
    LGF_CUDA_TRY(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return LGF_OK;
}

inline int64_t key3(int x, int y, int z)
{
    const int64_t off = 1 << 20, m = (1 << 21) - 1;
    return (((int64_t)x + off) & m) << 42 | (((int64_t)y + off) & m) << 21 | (((int64_t)z + off) & m);
}

// PINT-point Lagrange weights at the midpoint of nodes PINT/2 - 1 and PINT/2 of 0 .. PINT-1
void midpoint_weights(double w[PINT])
{
    for (int k = 0; k < PINT; k++) {
        double v = 1.0;
        for (int m = 0; m < PINT; m++)
            if (m != k) v *= (0.5 * (PINT - 1) - m) / (double)(k - m);
        w[k] = v;
    }
}

// the 1-D interpolation matrix P[i][l]: fine i of a block, node l of its window 8b - WOFF + l.
// Even i: its own node i/2; odd i = 2j + 1: nodes j - (PINT/2 - 1) .. j + PINT/2.
void interp_matrix(float P[BN * W])
{
    double w[PINT];
    midpoint_weights(w);
    for (int i = 0; i < BN * W; i++) P[i] = 0.f;
    for (int i = 0; i < BN; i++) {
        if (i % 2 == 0) {
            P[i * W + i / 2 + WOFF] = 1.f;
        } else {
            const int j = i / 2;
            for (int k = 0; k < PINT; k++) P[i * W + j - (PINT / 2 - 1) + k + WOFF] = (float)w[k];
        }
    }
}

// B operands of the tensor-core steps, split into TF32 hi / lo parts, in the core-matrix
// layout: anterpolation B[n = l][k = i] = P[i][l] (32 rows x K 16), interpolation
// B[n = i][k = l] = P[i][l] (rows 16..31 zero, K 24).  out: [2][32 * K] (hi, then lo).
void tc_weights(const float P[BN * W], bool anterp, std::vector<uint32_t> &out)
{
    const int K = anterp ? 16 : 24;
    out.assign(2 * 32 * K, 0u);
    for (int n = 0; n < 32; n++)
        for (int k = 0; k < K; k++) {
            float v = 0.f;
            if (anterp && n < W) v = P[k * W + n];
            if (!anterp && n < BN && k < W) v = P[n * W + k];
            // TF32: round to nearest on the top 10 mantissa bits (ties away), as cvt.rna.tf32
            auto tf32 = [](float x) {
                uint32_t u;
                std::memcpy(&u, &x, 4);
                u = (u + 0x1000u) & 0xFFFFE000u;
                float y;
                std::memcpy(&y, &u, 4);
                return y;
            };
            const float hi = tf32(v), lo = tf32(v - hi);
            const int idx = ((n >> 3) * (K * 32) + (k >> 2) * 128 + (n & 7) * 16 + (k & 3) * 4) >> 2;
            std::memcpy(&out[idx], &hi, 4);
            std::memcpy(&out[32 * K + idx], &lo, 4);
        }
}

}  // namespace

void free_split(SplitPlan *sp)
{
    if (!sp) return;
    cudaFree(sp->d_W);
    cudaFree(sp->d_S);
    cudaFree(sp->d_U);
    cudaFree(sp->d_off);
    cudaFree(sp->d_pairs);
    cudaFree(sp->d_run_tgt);
    cudaFree(sp->d_run_row);
    cudaFree(sp->d_rows);
    cudaFree(sp->d_quad_tgt);
    cudaFree(sp->d_quad_row);
    cudaFree(sp->d_qrows);
    cudaFree(sp->d_Q);
    cudaFree(sp->d_q);
    cudaFree(sp->d_v);
    cudaFree(sp->d_ccoords);
    cudaFree(sp->d_flut);
    cudaFree(sp->d_tcoords);
    cudaFree(sp->d_clut);
    cudaFree(sp->d_stage_src);
    cudaFree(sp->d_stage_dst);
    cudaFree(sp->d_Ba);
    cudaFree(sp->d_Bi);
    cudaFree(sp->d_err);
    if (sp->coarse) lgf_plan_destroy(sp->coarse);
    if (sp->far_table) lgf_table_destroy(sp->far_table);
    if (sp->far_stream) cudaStreamDestroy(sp->far_stream);
    if (sp->ev_fork) cudaEventDestroy(sp->ev_fork);
    if (sp->ev_far) cudaEventDestroy(sp->ev_far);
    if (sp->ev_src) cudaEventDestroy(sp->ev_src);
    delete sp;
}

static lgf_status choose_near_mac(SplitPlan *sp, int near_form, cudaStream_t s);

// One level of the split on the lattice of spacing `stride` (in unit cells; the level's own
// block coordinates are in units of 16 of its points): the near part of the kernel is the
// Bessel-form integral over t in [t_lo, alpha] (t_lo = 0: the LGF's own split), the far part
// the integral from alpha on, sampled on the lattice of spacing 2 stride.  The far part's
// coarse convolution is a whole-box plan, or, where that box is beyond the FFT lengths or
// large (a 512^3 grid or more), the next level: a split plan on the coarse lattice with
// t in [alpha, 4 alpha] near and [4 alpha, inf) far (the same near radius and interpolation
// error in that level's units, since the heat kernel's width grows as sqrt t).
static lgf_status plan_split_level(lgf_plan *p, const lgf_solve_desc &d, double t_lo, double alpha, int stride,
                                   int far_precision, int near_form, cudaStream_t s);

lgf_status plan_split(lgf_plan *p, const lgf_solve_desc &d, double alpha, int far_precision, int near_form,
                      cudaStream_t s)
{
    LGF_CHECK_ARG(alpha >= 1.0 && alpha <= 64.0, "block-sparse method: split time %g outside [1, 64]", alpha);
    return plan_split_level(p, d, 0.0, alpha, 1, far_precision, near_form, s);
}

static lgf_status plan_split_level(lgf_plan *p, const lgf_solve_desc &d, double t_lo, double alpha, int stride,
                                   int far_precision, int near_form, cudaStream_t s)
{
    LGF_CHECK_ARG(d.B == BN, "block-sparse method: B=%d (the near-field blocks are 16^3)", d.B);
    LGF_CHECK_ARG(stride <= 16, "block-sparse method: more than five levels");
    SplitPlan *sp = new (std::nothrow) SplitPlan();
    if (!sp) {
        set_error("host allocation failed");
        return LGF_ERR_OOM;
    }
    p->split = sp;
    sp->alpha = alpha;
    sp->far_tensor_cores = far_precision == 1;
    sp->ncomp = d.ncomp;
    sp->nsrc = d.n_src;
    sp->ndst = d.n_dst;
    sp->dx = d.dx;
    sp->scale = d.scale;
    size_t &bytes = p->bytes;
    // device error flag of the bounded waits (window staging, tensor-core completions)
    LGF_TRY(dalloc_n(&sp->d_err, 1, bytes));
    LGF_CUDA_TRY(cudaMemsetAsync(sp->d_err, 0, sizeof(int), s));
    LGF_CUDA_TRY(fft::upload_tw64());

    // --- near field: G_near table, kept offsets, window spectra ---
    double *d_near = nullptr;
    const int64_t noct = (int64_t)(KNEAR + 1) * (KNEAR + 2) * (KNEAR + 3) / 6;
    LGF_TRY(dalloc_n(&d_near, (size_t)noct, bytes));
    lgf_status st = build_lgf_octant_part(KNEAR, stride, t_lo, alpha, d_near, s);
    std::vector<double> h_near(noct);
    if (st == LGF_OK && cudaMemcpy(h_near.data(), d_near, noct * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        st = LGF_ERR_CUDA;
    if (st != LGF_OK) {
        cudaFree(d_near);
        bytes -= noct * sizeof(double);
        return st == LGF_ERR_CUDA ? (set_error("near table download failed"), st) : st;
    }
    // keep an offset when its window holds a value above 1e-12 |G(0)| (|G(0)| ~ 0.2527)
    auto oct_h = [&](int a, int b, int c) {
        a = std::abs(a), b = std::abs(b), c = std::abs(c);
        if (a < b) std::swap(a, b);
        if (b < c) std::swap(b, c);
        if (a < b) std::swap(a, b);
        return h_near[(int64_t)a * (a + 1) * (a + 2) / 6 + (int64_t)b * (b + 1) / 2 + c];
    };
    std::vector<int> offs;
    for (int dz = -RNEAR; dz <= RNEAR; dz++)
        for (int dy = -RNEAR; dy <= RNEAR; dy++)
            for (int dxo = -RNEAR; dxo <= RNEAR; dxo++) {
                // the window's largest |G_near| sits at its point nearest the origin
                auto nearest = [](int o) { return o == 0 ? 0 : (o > 0 ? BN * o - (BN - 1) : BN * o + (BN - 1)); };
                const double g = std::fabs(oct_h(nearest(dxo), nearest(dy), nearest(dz)));
                if (g >= 1e-12 * 0.2527) {
                    offs.push_back(dxo);
                    offs.push_back(dy);
                    offs.push_back(dz);
                }
            }
    sp->noff = (int)offs.size() / 3;
    sp->offs = offs;
    {
        int *d_offs = nullptr;
        double *d_win = nullptr;
        double2 *d_a = nullptr, *d_b = nullptr, *d_tw = nullptr;
        size_t tmp = 0;
        const size_t nwin = (size_t)sp->noff * NF * NF * NF, nspec = (size_t)sp->noff * NF * NF * KXN;
        st = dalloc_n(&d_offs, offs.size(), tmp);
        if (st == LGF_OK) st = dalloc_n(&d_win, nwin, tmp);
        if (st == LGF_OK) st = dalloc_n(&d_a, nspec, tmp);
        if (st == LGF_OK) st = dalloc_n(&d_b, nspec, tmp);
        if (st == LGF_OK) st = dalloc_n(&d_tw, (size_t)NF, tmp);
        if (st == LGF_OK) st = dalloc_n(&sp->d_W, (size_t)sp->noff * NFREQ, bytes);
        std::vector<double2> tw(NF);
        for (int j = 0; j < NF; j++) tw[j] = make_double2(std::cos(-2.0 * M_PI * j / NF), std::sin(-2.0 * M_PI * j / NF));
        if (st == LGF_OK) st = upload_v(d_offs, offs, s);
        if (st == LGF_OK) st = upload_v(d_tw, tw, s);
        if (st == LGF_OK) {
            k_near_windows<<<1024, 256, 0, s>>>(d_near, d_offs, sp->noff, d_win);
            k_near_dft_x<<<1024, 256, 0, s>>>(d_win, sp->noff, d_a, d_tw);
            k_near_dft_yz<<<1024, 256, 0, s>>>(d_a, sp->noff, 1, d_b, d_tw);
            k_near_dft_yz<<<1024, 256, 0, s>>>(d_b, sp->noff, 2, d_a, d_tw);
            k_near_pack<<<1024, 256, 0, s>>>(d_a, sp->noff, sp->d_W);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                set_error("near-field spectra: %s", cudaGetErrorString(e));
                st = LGF_ERR_CUDA;
            }
        }
        cudaFree(d_offs);
        cudaFree(d_win);
        cudaFree(d_a);
        cudaFree(d_b);
        cudaFree(d_tw);
    }
    cudaFree(d_near);
    bytes -= noct * sizeof(double);
    if (st != LGF_OK) return st;

    // target -> (offset, source) pairs
    std::unordered_map<int64_t, int> smap;
    for (int i = 0; i < d.n_src; i++) smap[key3(d.src_blocks[3 * i], d.src_blocks[3 * i + 1], d.src_blocks[3 * i + 2])] = i;
    std::vector<int> off(d.n_dst + 1, 0);
    std::vector<int2> pairs;
    for (int t = 0; t < d.n_dst; t++) {
        off[t] = (int)pairs.size();
        for (int k = 0; k < sp->noff; k++) {
            auto it = smap.find(key3(d.dst_blocks[3 * t] - offs[3 * k], d.dst_blocks[3 * t + 1] - offs[3 * k + 1],
                                     d.dst_blocks[3 * t + 2] - offs[3 * k + 2]));
            if (it != smap.end()) pairs.push_back(make_int2(k, it->second));
        }
    }
    off[d.n_dst] = (int)pairs.size();
    sp->npairs = (int64_t)pairs.size();
    LGF_TRY(dalloc_n(&sp->d_off, off.size(), bytes));
    LGF_TRY(dalloc_n(&sp->d_pairs, pairs.size(), bytes));
    LGF_TRY(upload_v(sp->d_off, off, s));
    LGF_TRY(upload_v(sp->d_pairs, pairs, s));
    {
        // runs of 4 x-adjacent target slots (x0 a multiple of 4) and their (oy, oz) rows
        std::unordered_map<int, int> dmap;  // (ox+2) + 5 (oy+2) + 25 (oz+2) -> W row
        for (int k = 0; k < sp->noff; k++)
            dmap[(offs[3 * k] + 2) + 5 * (offs[3 * k + 1] + 2) + 25 * (offs[3 * k + 2] + 2)] = k;
        auto wrow = [&](int ox, int oy, int oz) {
            auto it = dmap.find((ox + 2) + 5 * (oy + 2) + 25 * (oz + 2));
            return it == dmap.end() ? sp->noff : it->second;
        };
        auto fdiv4 = [](int v) { return v >= 0 ? v / 4 : -((-v + 3) / 4); };
        std::unordered_map<int64_t, int> rmap;
        std::vector<int4> rt;
        for (int t = 0; t < d.n_dst; t++) {
            const int x = d.dst_blocks[3 * t], y = d.dst_blocks[3 * t + 1], z = d.dst_blocks[3 * t + 2];
            const int x0 = 4 * fdiv4(x);
            auto it = rmap.find(key3(x0, y, z));
            if (it == rmap.end()) {
                it = rmap.emplace(key3(x0, y, z), (int)rt.size()).first;
                rt.push_back(make_int4(-1, -1, -1, -1));
            }
            int *slot = &rt[it->second].x;
            slot[x - x0] = t;
        }
        // run coordinates back from any of its targets
        std::vector<int> run_row(rt.size() + 1, 0);
        std::vector<int4> rows;
        for (size_t r = 0; r < rt.size(); r++) {
            run_row[r] = (int)(rows.size() / 4);
            const int *slot = &rt[r].x;
            int t = -1;
            for (int i = 0; i < 4 && t < 0; i++) t = slot[i];
            const int x0 = 4 * fdiv4(d.dst_blocks[3 * t]), y = d.dst_blocks[3 * t + 1], z = d.dst_blocks[3 * t + 2];
            for (int oz = -RNEAR; oz <= RNEAR; oz++)
                for (int oy = -RNEAR; oy <= RNEAR; oy++) {
                    int src[8];
                    bool any = false;
                    for (int k = 0; k < 8; k++) {
                        auto it = smap.find(key3(x0 - 2 + k, y - oy, z - oz));
                        src[k] = it == smap.end() ? -1 : it->second;
                        any = any || src[k] >= 0;
                    }
                    if (!any) continue;
                    int w[5];
                    bool anyw = false;
                    for (int o = 0; o < 5; o++) {
                        w[o] = wrow(o - 2, oy, oz);
                        anyw = anyw || w[o] < sp->noff;
                    }
                    if (!anyw) continue;
                    rows.push_back(make_int4(w[0], w[1], w[2], w[3]));
                    rows.push_back(make_int4(w[4], src[0], src[1], src[2]));
                    rows.push_back(make_int4(src[3], src[4], src[5], src[6]));
                    rows.push_back(make_int4(src[7], -1, -1, -1));
                }
        }
        run_row[rt.size()] = (int)(rows.size() / 4);
        sp->nruns = (int)rt.size();
        sp->nrows = (int)(rows.size() / 4);
        LGF_TRY(dalloc_n(&sp->d_run_tgt, rt.size(), bytes));
        LGF_TRY(dalloc_n(&sp->d_run_row, run_row.size(), bytes));
        LGF_TRY(dalloc_n(&sp->d_rows, std::max<size_t>(rows.size(), 4), bytes));
        LGF_TRY(upload_v(sp->d_run_tgt, rt, s));
        LGF_TRY(upload_v(sp->d_run_row, run_row, s));
        if (!rows.empty()) LGF_TRY(upload_v(sp->d_rows, rows, s));

        // quads of 4 x 2 target slots (x0 a multiple of 4, y0 even), when the windows are the
        // 125 offsets in canonical order: row-steps over (oz, y') with y' = y0 - 2 .. y0 + 3
        bool canonical = sp->noff == 125;
        for (int k = 0; canonical && k < 125; k++)
            canonical = offs[3 * k] == k % 5 - 2 && offs[3 * k + 1] == (k / 5) % 5 - 2 && offs[3 * k + 2] == k / 25 - 2;
        if (canonical) {
            auto fdiv2 = [](int v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); };
            std::unordered_map<int64_t, int> qmap;
            std::vector<int4> qt;  // 2 per quad
            for (int t = 0; t < d.n_dst; t++) {
                const int x = d.dst_blocks[3 * t], y = d.dst_blocks[3 * t + 1], z = d.dst_blocks[3 * t + 2];
                const int x0 = 4 * fdiv4(x), y0 = 2 * fdiv2(y);
                auto it = qmap.find(key3(x0, y0, z));
                if (it == qmap.end()) {
                    it = qmap.emplace(key3(x0, y0, z), (int)(qt.size() / 2)).first;
                    qt.push_back(make_int4(-1, -1, -1, -1));
                    qt.push_back(make_int4(-1, -1, -1, -1));
                }
                int *slot = &qt[2 * (size_t)it->second].x;
                slot[(y - y0) * 4 + (x - x0)] = t;
            }
            const size_t nq = qt.size() / 2;
            std::vector<int> quad_row(nq + 1, 0);
            std::vector<int4> qrows;
            for (size_t r = 0; r < nq; r++) {
                quad_row[r] = (int)(qrows.size() / 3);
                const int *slot = &qt[2 * r].x;
                int t = -1;
                bool rowj[2] = {false, false};
                for (int k = 0; k < 8; k++)
                    if (slot[k] >= 0) {
                        t = slot[k];
                        rowj[k / 4] = true;
                    }
                const int x0 = 4 * fdiv4(d.dst_blocks[3 * t]), y0 = 2 * fdiv2(d.dst_blocks[3 * t + 1]),
                          z = d.dst_blocks[3 * t + 2];
                for (int oz = -RNEAR; oz <= RNEAR; oz++)
                    for (int yp = y0 - RNEAR; yp <= y0 + 1 + RNEAR; yp++) {
                        int src[8];
                        bool any = false;
                        for (int k = 0; k < 8; k++) {
                            auto it = smap.find(key3(x0 - 2 + k, yp, z - oz));
                            src[k] = it == smap.end() ? -1 : it->second;
                            any = any || src[k] >= 0;
                        }
                        if (!any) continue;
                        int wb[2];
                        for (int j = 0; j < 2; j++) {
                            const int oy = y0 + j - yp;
                            wb[j] = rowj[j] && oy >= -RNEAR && oy <= RNEAR ? 5 * (oy + 2) + 25 * (oz + 2) : -1;
                        }
                        if (wb[0] < 0 && wb[1] < 0) continue;
                        qrows.push_back(make_int4(src[0], src[1], src[2], src[3]));
                        qrows.push_back(make_int4(src[4], src[5], src[6], src[7]));
                        qrows.push_back(make_int4(wb[0], wb[1], 0, 0));
                    }
            }
            quad_row[nq] = (int)(qrows.size() / 3);
            sp->nquads = (int)nq;
            sp->nqrows = (int)(qrows.size() / 3);
            LGF_TRY(dalloc_n(&sp->d_quad_tgt, qt.size(), bytes));
            LGF_TRY(dalloc_n(&sp->d_quad_row, quad_row.size(), bytes));
            LGF_TRY(dalloc_n(&sp->d_qrows, std::max<size_t>(qrows.size(), 3), bytes));
            LGF_TRY(upload_v(sp->d_quad_tgt, qt, s));
            LGF_TRY(upload_v(sp->d_quad_row, quad_row, s));
            if (!qrows.empty()) LGF_TRY(upload_v(sp->d_qrows, qrows, s));
        }
    }
    LGF_TRY(dalloc_n(&sp->d_S, (size_t)d.ncomp * NFREQ * d.n_src, bytes));

    LGF_TRY(dalloc_n(&sp->d_U, (size_t)d.ncomp * NFREQ * d.n_dst, bytes));
    LGF_TRY(choose_near_mac(sp, near_form, s));

    // --- far field: coarse block sets, G_far table, coarse plan ---
    float P[BN * W];
    interp_matrix(P);
    LGF_CUDA_TRY(cudaMemcpyToSymbol(c_P, P, sizeof(P)));
    {
        std::vector<uint32_t> ba, bi;
        tc_weights(P, true, ba);
        tc_weights(P, false, bi);
        LGF_TRY(dalloc_n(&sp->d_Ba, ba.size(), bytes));
        LGF_TRY(dalloc_n(&sp->d_Bi, bi.size(), bytes));
        LGF_TRY(upload_v(sp->d_Ba, ba, s));
        LGF_TRY(upload_v(sp->d_Bi, bi, s));
    }
    auto coarse_of = [&](const int32_t *bl, int n) {
        std::map<int64_t, int> m;  // ordered: deterministic coarse block order
        std::vector<int> out;
        for (int i = 0; i < n; i++) {
            int lo[3], hi[3];
            for (int a = 0; a < 3; a++) {  // the block's window: nodes 8 b - WOFF .. 8 b - WOFF + W - 1
                lo[a] = floordiv(8 * bl[3 * i + a] - WOFF, 16);
                hi[a] = floordiv(8 * bl[3 * i + a] - WOFF + W - 1, 16);
            }
            for (int z = lo[2]; z <= hi[2]; z++)
                for (int y = lo[1]; y <= hi[1]; y++)
                    for (int x = lo[0]; x <= hi[0]; x++) m.emplace(key3(z, y, x), 0);
        }
        for (auto &kv : m) {
            const int64_t k = kv.first, off20 = 1 << 20, msk = (1 << 21) - 1;
            const int z = (int)(((k >> 42) & msk) - off20), y = (int)(((k >> 21) & msk) - off20), x = (int)((k & msk) - off20);
            out.push_back(x);
            out.push_back(y);
            out.push_back(z);
        }
        return out;
    };
    std::vector<int> csrc = coarse_of(d.src_blocks, d.n_src), cdst = coarse_of(d.dst_blocks, d.n_dst);
    sp->ncsrc = (int)csrc.size() / 3;
    sp->ncdst = (int)cdst.size() / 3;
    // the coarse plan's table must cover half its FFT length: same size rule as lgf_conv_plan
    int Kc = 1;
    bool beyond = false;  // a whole-box coarse plan would need an FFT longer than 1024
    double vol = 1.0;     // its FFT grid points
    for (int a = 0; a < 3; a++) {
        int smin = 1 << 30, smax = -(1 << 30), tmin = 1 << 30, tmax = -(1 << 30);
        for (int i = 0; i < sp->ncsrc; i++) smin = std::min(smin, csrc[3 * i + a]), smax = std::max(smax, csrc[3 * i + a]);
        for (int i = 0; i < sp->ncdst; i++) tmin = std::min(tmin, cdst[3 * i + a]), tmax = std::max(tmax, cdst[3 * i + a]);
        const long S0 = 16L * smin, S1 = 16L * (smax + 1) - 1, T0 = 16L * tmin, T1 = 16L * (tmax + 1) - 1;
        const long m = std::max(std::labs(T0 - S1), std::labs(T1 - S0));
        const int n = poisson_pick_n((int)std::min<long>(std::max(2 * m + 2, 2 * (S1 - S0 + 1)), 1 << 20));
        beyond = beyond || n == 0;
        vol *= n;
        Kc = std::max(Kc, n / 2 - 1);
    }
    lgf_solve_desc cd;
    std::memset(&cd, 0, sizeof(cd));
    cd.B = BN;
    cd.ncomp = d.ncomp;
    cd.n_src = sp->ncsrc;
    cd.n_dst = sp->ncdst;
    cd.src_blocks = csrc.data();
    cd.dst_blocks = cdst.data();
    cd.dx = 1.0;
    cd.scale = 1.0;
    if (beyond || vol >= (double)(1 << 28)) {
        // the next level: a split plan on the coarse lattice (convolves the coarse charges
        // with G_far(2 stride .) as its own near part t in [alpha, 4 alpha] and far part)
        lgf_plan *q = new (std::nothrow) lgf_plan();
        if (!q) {
            set_error("host allocation failed");
            return LGF_ERR_OOM;
        }
        q->kind = LGF_KERNEL_LAPLACE7;
        q->device = p->device;
        q->method = 1;
        sp->coarse = q;
        LGF_TRY(plan_split_level(q, cd, alpha, 4.0 * alpha, 2 * stride, far_precision, near_form, s));
        sp->levels = 1 + q->split->levels;
        bytes += q->bytes;
    } else {
    lgf_table *ft = new (std::nothrow) lgf_table();
    if (!ft) {
        set_error("host allocation failed");
        return LGF_ERR_OOM;
    }
    sp->far_table = ft;
    ft->kind = LGF_KERNEL_LAPLACE7;
    ft->alpha = 0.0;
    ft->K = Kc;
    ft->R = 0;
    ft->device = p->device;
    ft->n = (int64_t)(Kc + 1) * (Kc + 2) * (Kc + 3) / 6;
    ft->d_vals = nullptr;
    ft->d_taps32 = nullptr;
    if (cudaMalloc(&ft->d_vals, ft->n * sizeof(double)) != cudaSuccess) {
        set_error("far table allocation failed");
        return LGF_ERR_OOM;
    }
    LGF_TRY(build_lgf_octant_part(Kc, 2 * stride, alpha, 0.0, ft->d_vals, s));
    lgf_plan_opts co;
    std::memset(&co, 0, sizeof(co));
    LGF_TRY(lgf_conv_plan(ft, &cd, 1, &co, (void *)s, &sp->coarse));
    bytes += sp->coarse->bytes;
    sp->levels = 1;
    }
    // lookups: fine source blocks (dense over their box + 1), coarse target blocks
    int fmin[3], fmax[3], cmin[3], cmax[3];
    for (int a = 0; a < 3; a++) {
        fmin[a] = 1 << 30, fmax[a] = -(1 << 30), cmin[a] = 1 << 30, cmax[a] = -(1 << 30);
        for (int i = 0; i < d.n_src; i++) fmin[a] = std::min(fmin[a], d.src_blocks[3 * i + a]),
                                           fmax[a] = std::max(fmax[a], d.src_blocks[3 * i + a]);
        for (int i = 0; i < sp->ncdst; i++) cmin[a] = std::min(cmin[a], cdst[3 * i + a]), cmax[a] = std::max(cmax[a], cdst[3 * i + a]);
    }
    sp->fmin = make_int3(fmin[0], fmin[1], fmin[2]);
    sp->fext = make_int3(fmax[0] - fmin[0] + 1, fmax[1] - fmin[1] + 1, fmax[2] - fmin[2] + 1);
    sp->cmin = make_int3(cmin[0], cmin[1], cmin[2]);
    sp->cext = make_int3(cmax[0] - cmin[0] + 1, cmax[1] - cmin[1] + 1, cmax[2] - cmin[2] + 1);
    std::vector<int> flut((size_t)sp->fext.x * sp->fext.y * sp->fext.z, -1);
    for (int i = 0; i < d.n_src; i++)
        flut[((size_t)(d.src_blocks[3 * i + 2] - fmin[2]) * sp->fext.y + (d.src_blocks[3 * i + 1] - fmin[1])) * sp->fext.x +
             (d.src_blocks[3 * i] - fmin[0])] = i;
    std::vector<int> clut((size_t)sp->cext.x * sp->cext.y * sp->cext.z, -1);
    for (int i = 0; i < sp->ncdst; i++)
        clut[((size_t)(cdst[3 * i + 2] - cmin[2]) * sp->cext.y + (cdst[3 * i + 1] - cmin[1])) * sp->cext.x +
             (cdst[3 * i] - cmin[0])] = i;
    std::vector<int> tco(d.dst_blocks, d.dst_blocks + 3 * d.n_dst);
    LGF_TRY(dalloc_n(&sp->d_flut, flut.size(), bytes));
    LGF_TRY(dalloc_n(&sp->d_clut, clut.size(), bytes));
    LGF_TRY(dalloc_n(&sp->d_ccoords, csrc.size(), bytes));
    LGF_TRY(dalloc_n(&sp->d_tcoords, tco.size(), bytes));
    LGF_TRY(upload_v(sp->d_flut, flut, s));
    LGF_TRY(upload_v(sp->d_clut, clut, s));
    LGF_TRY(upload_v(sp->d_ccoords, csrc, s));
    LGF_TRY(upload_v(sp->d_tcoords, tco, s));
    const size_t B3 = (size_t)BN * BN * BN;
    LGF_TRY(dalloc_n(&sp->d_Q, (size_t)d.n_src * d.ncomp * W3, bytes));
    LGF_TRY(dalloc_n(&sp->d_q, (size_t)sp->ncsrc * d.ncomp * B3, bytes));
    LGF_TRY(dalloc_n(&sp->d_v, (size_t)sp->ncdst * d.ncomp * B3, bytes));
    LGF_CUDA_TRY(cudaStreamCreateWithFlags(&sp->far_stream, cudaStreamNonBlocking));
    LGF_CUDA_TRY(cudaEventCreateWithFlags(&sp->ev_fork, cudaEventDisableTiming));
    LGF_CUDA_TRY(cudaEventCreateWithFlags(&sp->ev_far, cudaEventDisableTiming));
    LGF_CUDA_TRY(cudaEventCreateWithFlags(&sp->ev_src, cudaEventDisableTiming));
    static bool attr_done[64] = {false};
    if (p->device >= 0 && p->device < 64 && !attr_done[p->device]) {
        LGF_CUDA_TRY(cudaFuncSetAttribute(k_near_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NEAR_SMEM));
        LGF_CUDA_TRY(cudaFuncSetAttribute(k_near_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NEAR_SMEM));
        LGF_CUDA_TRY(cudaFuncSetAttribute(k_far_anterp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sizeof(TcSmem<16>)));
        LGF_CUDA_TRY(cudaFuncSetAttribute(k_far_interp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sizeof(TcSmem<24>)));
        attr_done[p->device] = true;
    }
    LGF_CUDA_TRY(cudaStreamSynchronize(s));
    return LGF_OK;
}

// The status of the split solve's bounded device waits (synchronises s).
lgf_status split_check(lgf_plan *p, cudaStream_t s)
{
    SplitPlan *sp = p->split;
    int h = 0;
    LGF_CUDA_TRY(cudaMemcpyAsync(&h, sp->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    LGF_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) {
        LGF_CUDA_TRY(cudaMemsetAsync(sp->d_err, 0, sizeof(int), s));
        set_error("a bounded device wait of the split solve gave up (its result is not valid)");
        return LGF_ERR_TIMEOUT;
    }
    return LGF_OK;
}

// The near-field multiply-accumulate in the form the plan chose (0 pairs: one target per
// warp over its (offset, source) list; 1 runs: 4 x-adjacent targets per warp; 2 quads: 4 x 2
// targets per warp; RUNS_PER_WARP runs or quads per warp).
constexpr int RUNS_PER_WARP = 2;
static lgf_status launch_near_mac(const SplitPlan *sp, int form, cudaStream_t s)
{
    const int nc = sp->ncomp;
    if (form == 2)
        LGF_CUDA_TRY(launch_pdl_smem(k_near_mac_quads,
                                     dim3(NCHUNK, (sp->nquads + 8 * RUNS_PER_WARP - 1) / (8 * RUNS_PER_WARP), nc),
                                     dim3(256), (size_t)sp->noff * CH * sizeof(float2), s, (const float2 *)sp->d_W,
                                     sp->noff, (const float2 *)sp->d_S, sp->nsrc, (const int4 *)sp->d_quad_tgt,
                                     (const int *)sp->d_quad_row, (const int4 *)sp->d_qrows, sp->nquads, sp->ndst,
                                     sp->d_U, sp->d_err));
    else if (form == 1)
        LGF_CUDA_TRY(launch_pdl_smem(k_near_mac_runs,
                                     dim3(NCHUNK, (sp->nruns + 8 * RUNS_PER_WARP - 1) / (8 * RUNS_PER_WARP), nc),
                                     dim3(256), (size_t)(sp->noff + 1) * CH * sizeof(float2), s,
                                     (const float2 *)sp->d_W, sp->noff, (const float2 *)sp->d_S, sp->nsrc,
                                     (const int4 *)sp->d_run_tgt, (const int *)sp->d_run_row,
                                     (const int4 *)sp->d_rows, sp->nruns, sp->ndst, sp->d_U, sp->d_err));
    else
        LGF_CUDA_TRY(launch_pdl_smem(k_near_mac, dim3(NCHUNK, (sp->ndst + 63) / 64, nc), dim3(256),
                                     (size_t)sp->noff * CH * sizeof(float2), s, (const float2 *)sp->d_W, sp->noff,
                                     (const float2 *)sp->d_S, sp->nsrc, (const int *)sp->d_off,
                                     (const int2 *)sp->d_pairs, sp->ndst, sp->d_U, sp->d_err));
    return LGF_OK;
}

// Plan time (near_form 0): time the forms (three launches each, on zeroed spectra) and keep
// the fastest; near_form 1 / 2 / 3 takes the pair / run / quad form.  The run and quad forms
// do their multiply-adds dense over each run's or quad's rows, so they win where targets fill
// them (the 256^3 shell) and can lose where they are sparse.  The quad form needs the 125
// offsets in canonical order (without them near_form 3 takes the run form).
static lgf_status choose_near_mac(SplitPlan *sp, int near_form, cudaStream_t s)
{
    if (near_form != 0) {  // the caller's choice
        sp->mac_form = near_form - 1;
        if (sp->mac_form == 2 && sp->nquads == 0) sp->mac_form = 1;
        return LGF_OK;
    }
    LGF_CUDA_TRY(cudaMemsetAsync(sp->d_S, 0, (size_t)sp->ncomp * NFREQ * sp->nsrc * sizeof(float2), s));
    cudaEvent_t e[2];
    LGF_CUDA_TRY(cudaEventCreate(&e[0]));
    if (cudaEventCreate(&e[1]) != cudaSuccess) {
        cudaEventDestroy(e[0]);
        set_error("event creation failed");
        return LGF_ERR_CUDA;
    }
    lgf_status st = LGF_OK;
    const int nforms = sp->nquads > 0 ? 3 : 2;
    for (int form = 0; form < nforms && st == LGF_OK; form++) {
        st = launch_near_mac(sp, form, s);  // warm-up
        if (st == LGF_OK && cudaEventRecord(e[0], s) != cudaSuccess) st = LGF_ERR_CUDA;
        for (int k = 0; k < 3 && st == LGF_OK; k++) st = launch_near_mac(sp, form, s);
        if (st == LGF_OK && cudaEventRecord(e[1], s) != cudaSuccess) st = LGF_ERR_CUDA;
        if (st == LGF_OK && cudaEventSynchronize(e[1]) != cudaSuccess) st = LGF_ERR_CUDA;
        float ms = 0.f;
        if (st == LGF_OK && cudaEventElapsedTime(&ms, e[0], e[1]) != cudaSuccess) st = LGF_ERR_CUDA;
        sp->mac_ms[form] = ms / 3.f;
    }
    cudaEventDestroy(e[0]);
    cudaEventDestroy(e[1]);
    if (st != LGF_OK) {
        if (st == LGF_ERR_CUDA) set_error("timing the near-field forms failed");
        return st;
    }
    sp->mac_form = 0;
    for (int form = 1; form < nforms; form++)
        if (sp->mac_ms[form] < sp->mac_ms[sp->mac_form]) sp->mac_form = form;
    return LGF_OK;
}

// One split solve.  prof: per-kernel event timing (then all launches go to s, one after
// another).
lgf_status run_split(lgf_plan *p, const float *src, float *dst, cudaStream_t s, Profiler *prof)
{
    // The far field runs on its own stream beside the near field and ends with the
    // interpolation writing dst = u_far; the near field's inverse then adds u_near, so only
    // that last kernel waits for both.  The interpolation first waits for the near field's
    // forward transform, so that dst may share memory with src.
    SplitPlan *sp = p->split;
    const bool P = prof && prof->on;
    const int nc = sp->ncomp;
    const float mul_near = (float)(sp->scale * sp->dx * sp->dx / ((double)NF * NF * NF));
    const float mul_far = (float)(sp->scale * sp->dx * sp->dx);
    cudaStream_t fs = P ? s : sp->far_stream;
    if (!P) {
        LGF_CUDA_TRY(cudaEventRecord(sp->ev_fork, s));
        LGF_CUDA_TRY(cudaStreamWaitEvent(fs, sp->ev_fork, 0));
    }
    // far field: anterpolation, coarse charges, coarse convolution
    if (P) prof->begin(fs);
    if (!sp->far_tensor_cores) {
        k_far_anterp<<<dim3(sp->nsrc, nc), FAR_THREADS, 0, fs>>>(src, nc, 0, sp->d_Q, nc);
        LGF_LAUNCH_CHECK("k_far_anterp");
    } else {
        LGF_CUDA_TRY(launch_pdl_smem(k_far_anterp_tc, dim3(sp->nsrc, nc), dim3(TC_THREADS), sizeof(TcSmem<16>), fs, src,
                                     nc, 0, sp->d_Q, nc, (const uint32_t *)sp->d_Ba, sp->d_err));
    }
    if (P) prof->end("far_anterp", fs);
    if (P) prof->begin(fs);
    k_far_gather<<<dim3(sp->ncsrc * GATHER_PARTS, nc), 256, 0, fs>>>(sp->d_Q, nc, sp->d_ccoords, sp->d_flut, sp->fmin,
                                                                     sp->fext, sp->d_q);
    LGF_LAUNCH_CHECK("k_far_gather");
    if (P) prof->end("far_gather", fs);
    {
        const float *cs[1] = {sp->d_q};
        float *cd[1] = {sp->d_v};
        if (P) prof->begin(fs);
        LGF_TRY(lgf_conv_execute(sp->coarse, cs, cd, (void *)fs));
        if (P) prof->end("far_coarse_conv", fs);
    }
    // near field: forward transforms of the source blocks, multiply-accumulate
    if (P) prof->begin(s);
    LGF_CUDA_TRY(launch_pdl_smem(k_near_fwd, dim3(sp->nsrc, nc), dim3(256), NEAR_SMEM, s, src, nc, 0, sp->nsrc, sp->d_S));
    if (P) prof->end("near_fwd", s);
    if (!P) {
        LGF_CUDA_TRY(cudaEventRecord(sp->ev_src, s));
        LGF_CUDA_TRY(cudaStreamWaitEvent(fs, sp->ev_src, 0));
    }
    // far field: interpolation, dst = u_far
    if (P) prof->begin(fs);
    if (!sp->far_tensor_cores) {
        k_far_interp<<<dim3(sp->ndst, nc), FAR_THREADS, 0, fs>>>(sp->d_v, nc, sp->d_tcoords, sp->d_clut, sp->cmin,
                                                                 sp->cext, dst, nc, 0, mul_far);
        LGF_LAUNCH_CHECK("k_far_interp");
    } else {
        LGF_CUDA_TRY(launch_pdl_smem(k_far_interp_tc, dim3(sp->ndst, nc), dim3(TC_THREADS), sizeof(TcSmem<24>), fs,
                                     (const float *)sp->d_v, nc, (const int *)sp->d_tcoords, (const int *)sp->d_clut,
                                     sp->cmin, sp->cext, dst, nc, 0, mul_far, (const uint32_t *)sp->d_Bi, sp->d_err));
    }
    if (P) prof->end("far_interp", fs);
    if (!P) LGF_CUDA_TRY(cudaEventRecord(sp->ev_far, fs));
    if (P) prof->begin(s);
    LGF_TRY(launch_near_mac(sp, sp->mac_form, s));
    if (P) prof->end("near_mac", s);
    // near field: inverse transforms, dst += u_near
    if (!P) LGF_CUDA_TRY(cudaStreamWaitEvent(s, sp->ev_far, 0));
    if (P) prof->begin(s);
    LGF_CUDA_TRY(launch_pdl_smem(k_near_inv, dim3(sp->ndst, nc), dim3(256), NEAR_SMEM, s, (const float2 *)sp->d_U,
                                 sp->ndst, dst, nc, 0, mul_near));
    if (P) prof->end("near_inv", s);
    return LGF_OK;
}

}  // namespace lgf

extern "C" lgf_status lgf_wait_probe(int polls, void *stream)
{
    lgf::clear_error();
    LGF_CHECK_ARG(polls >= 1 && polls <= (1 << 20), "lgf_wait_probe: polls %d outside [1, 2^20]", polls);
    cudaStream_t s = (cudaStream_t)stream;
    int *d_err = nullptr, h = 0;
    LGF_CUDA_TRY(cudaMalloc(&d_err, sizeof(int)));
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        lgf::k_wait_probe<<<1, 32, 0, s>>>(polls, d_err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_err);
    if (e != cudaSuccess) {
        lgf::set_error("lgf_wait_probe: %s", cudaGetErrorString(e));
        return LGF_ERR_CUDA;
    }
    if (h) {
        lgf::set_error("bounded device wait gave up after %d polls", polls);
        return LGF_ERR_TIMEOUT;
    }
    return LGF_OK;
}
