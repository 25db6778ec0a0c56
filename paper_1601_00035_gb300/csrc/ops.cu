// Local operators of the staggered grid (App. A point forms) on a block set,
// with the mask semantics of Sec. 4.2: values outside the listed blocks are
// zero.  Axis map: component (1),(2),(3) = x, y, z; position index n = (i, j, k).
//
//   G^T f  (faces -> cells):   sum_q (f^q_{n-e_q} - f^q_n) / dx            (G^T = -Dbar)
//   G c    (cells -> faces):   (c_{n+e_q} - c_n) / dx
//   C f    (faces -> edges):   (f^r_n - f^r_{n+e_s} + f^s_{n+e_r} - f^s_n) / dx,  (q,r,s) cyclic
//   C^T e  (edges -> faces):   (e^r_{n-e_s} - e^r_n + e^s_n - e^s_{n-e_r}) / dx
//   N~(f)  (faces -> faces, eq. opr_def_nonlin, e = C f):
//     1/4 sum_{m in {-1,0}} [ e^r_{n+m e_s} (f^s + f^s_{+e_q})_{n+m e_s} - e^s_{n+m e_r} (f^r + f^r_{+e_q})_{n+m e_r} ]
//
// One thread block per block of the set, one thread per (x, y) column looping
// over z; neighbour values come through the 27-neighbour table (L1/L2).
#include <algorithm>

#include "plan.hpp"

namespace lgf {
namespace {

template <int B>
struct Fetch {
    const float *f;
    int ncomp;
    const int *nb;  // 27 neighbours of this block
    // value of component c at local position (x, y, z), which may lie in a neighbour
    __device__ __forceinline__ float operator()(int c, int x, int y, int z) const
    {
        const int dx = x < 0 ? -1 : (x >= B ? 1 : 0);
        const int dy = y < 0 ? -1 : (y >= B ? 1 : 0);
        const int dz = z < 0 ? -1 : (z >= B ? 1 : 0);
        const int n = nb[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
        if (n < 0) return 0.f;
        return __ldg(f + ((size_t)(n * ncomp + c) * B + (z - dz * B)) * B * B + (y - dy * B) * B + (x - dx * B));
    }
};

__device__ __forceinline__ void axis_shift(int q, int d, int &x, int &y, int &z)
{
    if (q == 0) x += d;
    else if (q == 1) y += d;
    else z += d;
}

// OP: 0 curl (faces->edges), 1 curl^T (edges->faces), 2 G^T (faces->cells),
//     3 G (cells->faces), 4 nonlinear (faces->faces)
template <int B, int OP>
__global__ void __launch_bounds__(B *B) k_op(const float *__restrict__ in, float *__restrict__ out,
                                             const int *__restrict__ nbr27, const unsigned char *__restrict__ out_keep,
                                             float inv_dx, float coef, float u0, float u1, float u2)
{
    const int blk = blockIdx.x;
    __shared__ int nb[27];
    if (threadIdx.x < 27) nb[threadIdx.x] = nbr27[blk * 27 + threadIdx.x];
    __syncthreads();
    const int x = threadIdx.x % B, y = threadIdx.x / B;
    constexpr int nin = (OP == 3) ? 1 : 3;
    constexpr int nout = (OP == 2) ? 1 : 3;
    Fetch<B> F{in, nin, nb};
    const float uinf[3] = {u0, u1, u2};
    const bool keep = (OP != 4) || out_keep == nullptr || out_keep[blk];
    for (int z = 0; z < B; z++) {
        if constexpr (OP == 0) {
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const int r = (q + 1) % 3, s = (q + 2) % 3;
                int xs = x, ys = y, zs = z, xr = x, yr = y, zr = z;
                axis_shift(s, 1, xs, ys, zs);
                axis_shift(r, 1, xr, yr, zr);
                const float v = F(r, x, y, z) - F(r, xs, ys, zs) + F(s, xr, yr, zr) - F(s, x, y, z);
                out[((size_t)(blk * 3 + q) * B + z) * B * B + y * B + x] = v * inv_dx;
            }
        } else if constexpr (OP == 1) {
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const int r = (q + 1) % 3, s = (q + 2) % 3;
                int xs = x, ys = y, zs = z, xr = x, yr = y, zr = z;
                axis_shift(s, -1, xs, ys, zs);
                axis_shift(r, -1, xr, yr, zr);
                const float v = F(r, xs, ys, zs) - F(r, x, y, z) + F(s, x, y, z) - F(s, xr, yr, zr);
                out[((size_t)(blk * 3 + q) * B + z) * B * B + y * B + x] = v * inv_dx;
            }
        } else if constexpr (OP == 2) {
            float v = 0.f;
#pragma unroll
            for (int q = 0; q < 3; q++) {
                int xm = x, ym = y, zm = z;
                axis_shift(q, -1, xm, ym, zm);
                v += F(q, xm, ym, zm) - F(q, x, y, z);
            }
            out[((size_t)blk * B + z) * B * B + y * B + x] = v * inv_dx;
        } else if constexpr (OP == 3) {
            const float c0 = F(0, x, y, z);
#pragma unroll
            for (int q = 0; q < 3; q++) {
                int xp = x, yp = y, zp = z;
                axis_shift(q, 1, xp, yp, zp);
                out[((size_t)(blk * 3 + q) * B + z) * B * B + y * B + x] = (F(0, xp, yp, zp) - c0) * inv_dx;
            }
        } else {
            // f = M(u + u_inf): u_inf added only inside the block set
            auto fv = [&](int c, int px, int py, int pz) -> float {
                const int dx = px < 0 ? -1 : (px >= B ? 1 : 0);
                const int dy = py < 0 ? -1 : (py >= B ? 1 : 0);
                const int dz = pz < 0 ? -1 : (pz >= B ? 1 : 0);
                const int n = nb[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
                if (n < 0) return 0.f;
                return __ldg(in + ((size_t)(n * 3 + c) * B + (pz - dz * B)) * B * B + (py - dy * B) * B +
                             (px - dx * B)) + uinf[c];
            };
            // component c of e = C f at a position
            auto ev = [&](int c, int px, int py, int pz) -> float {
                const int r = (c + 1) % 3, s = (c + 2) % 3;
                int xs = px, ys = py, zs = pz, xr = px, yr = py, zr = pz;
                axis_shift(s, 1, xs, ys, zs);
                axis_shift(r, 1, xr, yr, zr);
                return (fv(r, px, py, pz) - fv(r, xs, ys, zs) + fv(s, xr, yr, zr) - fv(s, px, py, pz)) * inv_dx;
            };
#pragma unroll
            for (int q = 0; q < 3; q++) {
                float v = 0.f;
                if (keep) {
                    const int r = (q + 1) % 3, s = (q + 2) % 3;
#pragma unroll
                    for (int m = -1; m <= 0; m++) {
                        int xa = x, ya = y, za = z;
                        axis_shift(s, m, xa, ya, za);
                        int xa1 = xa, ya1 = ya, za1 = za;
                        axis_shift(q, 1, xa1, ya1, za1);
                        v += ev(r, xa, ya, za) * (fv(s, xa, ya, za) + fv(s, xa1, ya1, za1));
                        int xb = x, yb = y, zb = z;
                        axis_shift(r, m, xb, yb, zb);
                        int xb1 = xb, yb1 = yb, zb1 = zb;
                        axis_shift(q, 1, xb1, yb1, zb1);
                        v -= ev(s, xb, yb, zb) * (fv(r, xb, yb, zb) + fv(r, xb1, yb1, zb1));
                    }
                    v *= 0.25f * coef;
                }
                out[((size_t)(blk * 3 + q) * B + z) * B * B + y * B + x] = v;
            }
        }
    }
}

// N~(f) with shared-memory planes (replaces the per-point neighbour fetches of
// k_op<B, 4>): thread (x, y) walks z; plane z' of f = M(u + u_inf) with a
// one-cell halo in x and y lives in a ring of three slots, and plane z' of
// e = C f at in-plane positions -1 .. B-1 in a ring of two, so every stencil
// value is one shared-memory read.  Same arithmetic as eq. opr_def_nonlin.
// rv (optional): also writes rv = u + out (the first stage's r = u + g without a separate
// linear combination; the same single FP32 addition).
template <int B>
__global__ void __launch_bounds__(B *B) k_nonlinear(const float *__restrict__ in, float *__restrict__ out,
                                                    const int *__restrict__ nbr27,
                                                    const unsigned char *__restrict__ out_keep, float inv_dx,
                                                    float coef, float u0, float u1, float u2, float *__restrict__ rv)
{
    constexpr int H = B + 2;  // f plane edge (halo -1 .. B)
    constexpr int HE = B + 1; // e plane edge (-1 .. B-1)
    __shared__ int nb[27];
    __shared__ float Fs[3][3][H * H];   // [slot][component][(y+1) H + (x+1)]
    __shared__ float Es[2][3][HE * HE]; // [slot][component][(y+1) HE + (x+1)]
    // thread block (blk, zs) walks output planes z0 .. z1 - 1 of block blk
    constexpr int ZS = B >= 16 ? 2 : 1;
    const int blk = blockIdx.x / ZS;
    const int z0 = (blockIdx.x % ZS) * (B / ZS), z1 = z0 + B / ZS;
    const int x = threadIdx.x % B, y = threadIdx.x / B;
    const bool keep = out_keep == nullptr || out_keep[blk];
    if (!keep) {
        for (int z = z0; z < z1; z++)
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const size_t o = ((size_t)(blk * 3 + q) * B + z) * B * B + y * B + x;
                out[o] = 0.f;
                if (rv) rv[o] = __ldg(in + o);
            }
        return;
    }
    if (threadIdx.x < 27) nb[threadIdx.x] = nbr27[blk * 27 + threadIdx.x];
    __syncthreads();
    const float uinf[3] = {u0, u1, u2};
    // f plane zp (-1 .. B): fetch_f reads it from global memory into registers
    // (each thread holds at most 2 points x 3 components: (B + 2)^2 < 2 B^2),
    // commit_f stores it into its slot, so a plane's loads can be in flight
    // while the previous plane is computed
    constexpr int PT = (H * H + B * B - 1) / (B * B);
    static_assert(PT <= 2, "halo plane points per thread");
    float pre[PT][3];
    auto fetch_f = [&](int zp) {
        const int dz = zp < 0 ? -1 : (zp >= B ? 1 : 0);
        const int lz = zp - dz * B;
#pragma unroll
        for (int t = 0; t < PT; t++) {
            const int idx = threadIdx.x + t * B * B;
            const int hx = idx % H - 1, hy = idx / H - 1;
            const int dx = hx < 0 ? -1 : (hx >= B ? 1 : 0);
            const int dy = hy < 0 ? -1 : (hy >= B ? 1 : 0);
            const int n = idx < H * H ? nb[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] : -1;
            const size_t base = n >= 0 ? ((size_t)n * 3 * B + lz) * B * B + (hy - dy * B) * B + (hx - dx * B) : 0;
#pragma unroll
            for (int c = 0; c < 3; c++) pre[t][c] = n >= 0 ? __ldg(in + base + (size_t)c * B * B * B) + uinf[c] : 0.f;
        }
    };
    auto commit_f = [&](int zp) {
        float *dst = &Fs[(zp + 1) % 3][0][0];
#pragma unroll
        for (int t = 0; t < PT; t++) {
            const int idx = threadIdx.x + t * B * B;
            if (idx < H * H)
#pragma unroll
                for (int c = 0; c < 3; c++) dst[c * H * H + idx] = pre[t][c];
        }
    };
    auto load_f = [&](int zp) {
        fetch_f(zp);
        commit_f(zp);
    };
    auto F = [&](int c, int px, int py, int pz) -> float { return Fs[(pz + 1) % 3][c][(py + 1) * H + (px + 1)]; };
    // e plane zp (-1 .. B-1): e^c(p) = f^r(p) - f^r(p + e_s) + f^s(p + e_r) - f^s(p), (c, r, s) cyclic
    auto make_e = [&](int zp) {
        float *dst = &Es[(zp + 1) % 2][0][0];
        for (int idx = threadIdx.x; idx < HE * HE; idx += B * B) {
            const int px = idx % HE - 1, py = idx / HE - 1;
            const float f0 = F(0, px, py, zp), f1 = F(1, px, py, zp), f2 = F(2, px, py, zp);
            // c = 0 (r = y, s = z); c = 1 (r = z, s = x); c = 2 (r = x, s = y)
            dst[0 * HE * HE + idx] = (f1 - F(1, px, py, zp + 1) + F(2, px, py + 1, zp) - f2) * inv_dx;
            dst[1 * HE * HE + idx] = (f2 - F(2, px + 1, py, zp) + F(0, px, py, zp + 1) - f0) * inv_dx;
            dst[2 * HE * HE + idx] = (f0 - F(0, px, py + 1, zp) + F(1, px + 1, py, zp) - f1) * inv_dx;
        }
    };
    auto Ev = [&](int c, int px, int py, int pz) -> float { return Es[(pz + 1) % 2][c][(py + 1) * HE + (px + 1)]; };
    load_f(z0 - 1);
    load_f(z0);
    load_f(z0 + 1);
    __syncthreads();
    make_e(z0 - 1);
    fetch_f(z0 + 2);  // B / ZS >= 8
    for (int z = z0; z < z1; z++) {
        make_e(z);  // reads f planes z, z + 1
        __syncthreads();
        const int o[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};  // unit offsets e_q
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const int r = (q + 1) % 3, s2 = (q + 2) % 3;
            float v = 0.f;
#pragma unroll
            for (int m = -1; m <= 0; m++) {
                const int ax = x + m * o[s2][0], ay = y + m * o[s2][1], az = z + m * o[s2][2];
                v += Ev(r, ax, ay, az) * (F(s2, ax, ay, az) + F(s2, ax + o[q][0], ay + o[q][1], az + o[q][2]));
                const int bx = x + m * o[r][0], by = y + m * o[r][1], bz = z + m * o[r][2];
                v -= Ev(s2, bx, by, bz) * (F(r, bx, by, bz) + F(r, bx + o[q][0], by + o[q][1], bz + o[q][2]));
            }
            const size_t o = ((size_t)(blk * 3 + q) * B + z) * B * B + y * B + x;
            const float gv = v * 0.25f * coef;
            out[o] = gv;
            if (rv) rv[o] = __ldg(in + o) + gv;
        }
        __syncthreads();  // plane z - 1 of f and of e are no longer read
        if (z + 2 <= z1) {
            commit_f(z + 2);                   // into plane z - 1's slot
            if (z + 3 <= z1) fetch_f(z + 3);   // in flight during plane z + 1
        }
        __syncthreads();
    }
}

// Projection tail fused with the gradient: gd_q(n) = (dhat(n + e_q) - dhat(n)) / dx
// on faces (App. A, G), then out1 = rv - gd and optionally out2 = c2 (g - gd);
// gd itself is never stored.  One block per block of the set, thread (x, y)
// walks z with the scalar dhat plane and its +x/+y neighbours in registers
// from neighbour-table reads.
template <int B>
__global__ void __launch_bounds__(B *B) k_grad_combine(const float *__restrict__ dhat, const float *__restrict__ rv,
                                                       const float *__restrict__ g, float *__restrict__ out1,
                                                       float *__restrict__ out2, const int *__restrict__ nbr27,
                                                       float inv_dx, float c2)
{
    const int blk = blockIdx.x;
    __shared__ int nb[27];
    if (threadIdx.x < 27) nb[threadIdx.x] = nbr27[blk * 27 + threadIdx.x];
    __syncthreads();
    const int x = threadIdx.x % B, y = threadIdx.x / B;
    Fetch<B> D{dhat, 1, nb};
    float d0 = D(0, x, y, 0);
    for (int z = 0; z < B; z++) {
        const float dpx = D(0, x + 1, y, z), dpy = D(0, x, y + 1, z), dpz = D(0, x, y, z + 1);
        const float gq[3] = {(dpx - d0) * inv_dx, (dpy - d0) * inv_dx, (dpz - d0) * inv_dx};
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const size_t o = ((size_t)(blk * 3 + q) * B + z) * B * B + y * B + x;
            out1[o] = __ldg(rv + o) - gq[q];
            if (out2) out2[o] = c2 * (__ldg(g + o) - gq[q]);
        }
        d0 = dpz;
    }
}

// Ring diagnostics (Sec. 6 eq. int_quantities) over the first n_soln blocks of
// the set (D_soln): 15 FP64 sums, acc[0..2] = sum (x cross w) / 2, acc[3] = sum
// u . (x cross w) at cell centres, acc[4] = sum |w|^2 / 2, acc[5] = sum u . w at
// cell centres, acc[6 + 3a + b] = sum (x cross w)_a x_b / 2 (all without dx^3).
// w = C u on edges (computed here in FP64 from u), counted only on D_soln edges;
// edge (q) of cell index n sits at n - e_q / 2, cell n at n - (1,1,1)/2 (units
// of dx); cell values average the 2 faces / 4 edges around the cell.
template <int B>
__global__ void __launch_bounds__(B *B) k_diag(const float *__restrict__ u, const float *__restrict__ w,
                                               const int *__restrict__ nbr27, const int *__restrict__ coords,
                                               int n_soln, double dx, double *__restrict__ acc)
{
    const int blk = blockIdx.x;
    __shared__ int nb[27];
    __shared__ double red[15][B * B / 32];
    if (threadIdx.x < 27) {
        const int n = nbr27[blk * 27 + threadIdx.x];
        nb[threadIdx.x] = n < n_soln ? n : -1;  // w counts on D_soln only
    }
    __syncthreads();
    const int x = threadIdx.x % B, y = threadIdx.x / B;
    Fetch<B> U{u, 3, nbr27 + blk * 27};  // u: the whole set (global table)
    // w = C u at edge (q) of index (px, py, pz) in FP64 (App. A), zero off D_soln
    const double idx = 1.0 / dx;
    auto W = [&](int q, int px, int py, int pz) -> double {
        const int bx = px < 0 ? -1 : (px >= B ? 1 : 0);
        const int by = py < 0 ? -1 : (py >= B ? 1 : 0);
        const int bz = pz < 0 ? -1 : (pz >= B ? 1 : 0);
        if (nb[(bz + 1) * 9 + (by + 1) * 3 + (bx + 1)] < 0) return 0.0;
        const int r = (q + 1) % 3, s2 = (q + 2) % 3;
        const int o[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        return ((double)U(r, px, py, pz) - U(r, px + o[s2][0], py + o[s2][1], pz + o[s2][2]) +
                U(s2, px + o[r][0], py + o[r][1], pz + o[r][2]) - U(s2, px, py, pz)) * idx;
    };
    (void)w;
    const double ox = (double)coords[3 * blk] * B, oy = (double)coords[3 * blk + 1] * B,
                 oz = (double)coords[3 * blk + 2] * B;
    double a[15];
#pragma unroll
    for (int k = 0; k < 15; k++) a[k] = 0.0;
    for (int z = 0; z < B; z++) {
        const double vx = (ox + x) * dx, vy = (oy + y) * dx, vz = (oz + z) * dx;  // vertex of index n
        const double h = 0.5 * dx;
        // own-block edges
        const double w0 = W(0, x, y, z), w1 = W(1, x, y, z), w2 = W(2, x, y, z);
        // edge (q) positions: coordinate q shifted by -1/2
        const double e[3][3] = {{vx - h, vy, vz}, {vx, vy - h, vz}, {vx, vy, vz - h}};  // e[q][a]
        const double wv[3] = {w0, w1, w2};
#pragma unroll
        for (int ai = 0; ai < 3; ai++) {
            const int bi = (ai + 1) % 3, ci = (ai + 2) % 3;
            const double t1 = e[ci][bi] * wv[ci], t2 = e[bi][ci] * wv[bi];  // (x cross w)_a = x_b w_c - x_c w_b
            a[ai] += 0.5 * (t1 - t2);
#pragma unroll
            for (int bb = 0; bb < 3; bb++) a[6 + 3 * ai + bb] += 0.5 * (t1 * e[ci][bb] - t2 * e[bi][bb]);
        }
        a[4] += 0.5 * (w0 * w0 + w1 * w1 + w2 * w2);
        // cell-centred u and w
        const double uc[3] = {0.5 * ((double)U(0, x, y, z) + U(0, x - 1, y, z)),
                              0.5 * ((double)U(1, x, y, z) + U(1, x, y - 1, z)),
                              0.5 * ((double)U(2, x, y, z) + U(2, x, y, z - 1))};
        const double wc[3] = {
            0.25 * ((double)w0 + W(0, x, y - 1, z) + W(0, x, y, z - 1) + W(0, x, y - 1, z - 1)),
            0.25 * ((double)w1 + W(1, x, y, z - 1) + W(1, x - 1, y, z) + W(1, x - 1, y, z - 1)),
            0.25 * ((double)w2 + W(2, x - 1, y, z) + W(2, x, y - 1, z) + W(2, x - 1, y - 1, z))};
        const double px = vx - h, py = vy - h, pz = vz - h;
        const double xw[3] = {py * wc[2] - pz * wc[1], pz * wc[0] - px * wc[2], px * wc[1] - py * wc[0]};
        a[3] += uc[0] * xw[0] + uc[1] * xw[1] + uc[2] * xw[2];
        a[5] += uc[0] * wc[0] + uc[1] * wc[1] + uc[2] * wc[2];
    }
    // block reduction: warp shuffles, then one partial per warp in shared memory
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
#pragma unroll
    for (int k = 0; k < 15; k++) {
        double v = a[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 15) {
        double v = 0.0;
        for (int i = 0; i < B * B / 32; i++) v += red[threadIdx.x][i];
        atomicAdd(acc + threadIdx.x, v);
    }
}

// Regrid weights' raw maxima (Sec. 5 eq. weight_fun): mu[b] = max |w| (3 edge
// components) and nu[b] = max |q| (cells) over block b, leaving out the cells within
// RIM = 3 cells of a block outside the set: the masked curl is spurious on the last
// layer, and N~ and G^T carry that one cell further each.
template <int B>
__global__ void __launch_bounds__(B *B) k_block_max(const float *__restrict__ w, const float *__restrict__ q,
                                                    const int *__restrict__ nbr27, float *__restrict__ mu,
                                                    float *__restrict__ nu)
{
    const int blk = blockIdx.x;
    __shared__ int nb[27];
    __shared__ float red[2][B * B / 32];
    if (threadIdx.x < 27) nb[threadIdx.x] = nbr27[blk * 27 + threadIdx.x];
    __syncthreads();
    const int x = threadIdx.x % B, y = threadIdx.x / B;
    const size_t b3 = (size_t)B * B * B;
    float m1 = 0.f, m2 = 0.f;
    for (int z = 0; z < B; z++) {
        bool inner = true;
        constexpr int RIM = 3;
        for (int oz = (z < RIM ? -1 : 0); oz <= (z >= B - RIM ? 1 : 0); oz++)
            for (int oy = (y < RIM ? -1 : 0); oy <= (y >= B - RIM ? 1 : 0); oy++)
                for (int ox = (x < RIM ? -1 : 0); ox <= (x >= B - RIM ? 1 : 0); ox++)
                    if (nb[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)] < 0) inner = false;
        if (!inner) continue;
        const size_t o = (size_t)z * B * B + y * B + x;
#pragma unroll
        for (int c = 0; c < 3; c++) m1 = fmaxf(m1, fabsf(__ldg(w + ((size_t)blk * 3 + c) * b3 + o)));
        m2 = fmaxf(m2, fabsf(__ldg(q + (size_t)blk * b3 + o)));
    }
    for (int off = 16; off > 0; off >>= 1) {
        m1 = fmaxf(m1, __shfl_down_sync(0xffffffffu, m1, off));
        m2 = fmaxf(m2, __shfl_down_sync(0xffffffffu, m2, off));
    }
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    if (lane == 0) {
        red[0][warp] = m1;
        red[1][warp] = m2;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        float m = 0.f;
        for (int i = 0; i < B * B / 32; i++) m = fmaxf(m, red[threadIdx.x][i]);
        (threadIdx.x == 0 ? mu : nu)[blk] = m;
    }
}

// Zero a vector field on the cells within RIM = 3 cells of a block outside the set
// (the mask edge's contaminated layer; the same cells the regrid weights leave out).
template <int B>
__global__ void __launch_bounds__(B *B) k_zero_rim(float *__restrict__ f, const int *__restrict__ nbr27)
{
    const int blk = blockIdx.x;
    __shared__ int nb[27];
    if (threadIdx.x < 27) nb[threadIdx.x] = nbr27[blk * 27 + threadIdx.x];
    __syncthreads();
    const int x = threadIdx.x % B, y = threadIdx.x / B;
    const size_t b3 = (size_t)B * B * B;
    constexpr int RIM = 3;
    for (int z = 0; z < B; z++) {
        bool inner = true;
        for (int oz = (z < RIM ? -1 : 0); oz <= (z >= B - RIM ? 1 : 0); oz++)
            for (int oy = (y < RIM ? -1 : 0); oy <= (y >= B - RIM ? 1 : 0); oy++)
                for (int ox = (x < RIM ? -1 : 0); ox <= (x >= B - RIM ? 1 : 0); ox++)
                    if (nb[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)] < 0) inner = false;
        if (inner) continue;
        const size_t o = (size_t)z * B * B + y * B + x;
#pragma unroll
        for (int c = 0; c < 3; c++) f[((size_t)blk * 3 + c) * b3 + o] = 0.f;
    }
}

// out = sum_t c_t x_t over n floats (up to 4 terms; null x_t skipped).  out may
// alias an input (each element is read and written by the same thread), so no
// __restrict__ and no read-only-cache loads here.
__global__ void k_lincomb(float *out, int64_t n, const float *x0, float c0, const float *x1, float c1,
                          const float *x2, float c2, const float *x3, float c3)
{
    const int64_t n4 = n / 4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        auto acc = [&](const float *x, float c) {
            if (!x) return;
            const float4 v = reinterpret_cast<const float4 *>(x)[i];
            a.x = fmaf(c, v.x, a.x);
            a.y = fmaf(c, v.y, a.y);
            a.z = fmaf(c, v.z, a.z);
            a.w = fmaf(c, v.w, a.w);
        };
        acc(x0, c0);
        acc(x1, c1);
        acc(x2, c2);
        acc(x3, c3);
        reinterpret_cast<float4 *>(out)[i] = a;
    }
}

// out[i] = in[idx[i]] block by block ([n][ncomp][B^3] each)
__global__ void k_gather_blocks(const float *__restrict__ in, float *__restrict__ out, const int *__restrict__ idx,
                                int block_floats)
{
    const int i = blockIdx.x;
    const float4 *src = reinterpret_cast<const float4 *>(in + (size_t)__ldg(idx + i) * block_floats);
    float4 *dst = reinterpret_cast<float4 *>(out + (size_t)i * block_floats);
    for (int t = threadIdx.x; t < block_floats / 4; t += blockDim.x) dst[t] = __ldg(src + t);
}

}  // namespace

lgf_status op_launch(int op, int B, int nblk, const int *d_nbr27, const unsigned char *d_keep, const float *in,
                     float *out, double dx, double coef, const double uinf[3], cudaStream_t s, float *out2)
{
    if (out2 && op != 4) {
        set_error("a second output is only for the nonlinear term");
        return LGF_ERR_ARG;
    }
    const float inv_dx = (float)(1.0 / dx);
    const float u0 = uinf ? (float)uinf[0] : 0.f, u1 = uinf ? (float)uinf[1] : 0.f, u2 = uinf ? (float)uinf[2] : 0.f;
    const float cf = (float)coef;
#define LGF_OPCASE(BB, OPV)                                                                                     \
    if constexpr (OPV == 4)                                                                                     \
        k_nonlinear<BB><<<nblk * (BB >= 16 ? 2 : 1), BB * BB, 0, s>>>(in, out, d_nbr27, d_keep, inv_dx, cf, u0,  \
                                                                       u1, u2, out2);                          \
    else                                                                                                        \
        k_op<BB, OPV><<<nblk, BB * BB, 0, s>>>(in, out, d_nbr27, d_keep, inv_dx, cf, u0, u1, u2);
#define LGF_OPSWITCH(BB)                                                                                        \
    switch (op) {                                                                                               \
        case 0: LGF_OPCASE(BB, 0) break;                                                                        \
        case 1: LGF_OPCASE(BB, 1) break;                                                                        \
        case 2: LGF_OPCASE(BB, 2) break;                                                                        \
        case 3: LGF_OPCASE(BB, 3) break;                                                                        \
        case 4: LGF_OPCASE(BB, 4) break;                                                                        \
        default: set_error("unknown operator %d", op); return LGF_ERR_ARG;                                      \
    }
    if (B == 8) {
        LGF_OPSWITCH(8)
    } else if (B == 16) {
        LGF_OPSWITCH(16)
    } else {
        set_error("operators support B in {8, 16} (got %d)", B);
        return LGF_ERR_ARG;
    }
#undef LGF_OPSWITCH
#undef LGF_OPCASE
    LGF_LAUNCH_CHECK("local operator");
    return LGF_OK;
}

lgf_status lincomb_launch(float *out, int64_t n, const float *x0, double c0, const float *x1, double c1, const float *x2,
                          double c2, const float *x3, double c3, cudaStream_t s)
{
    if (n % 4 != 0) {
        set_error("lincomb length %lld not a multiple of 4", (long long)n);
        return LGF_ERR_ARG;
    }
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n / 4 + threads - 1) / threads, 152 * 16);
    k_lincomb<<<blocks, threads, 0, s>>>(out, n, x0, (float)c0, x1, (float)c1, x2, (float)c2, x3, (float)c3);
    LGF_LAUNCH_CHECK("lincomb");
    return LGF_OK;
}

lgf_status diag_launch(int B, int n_soln, const int *d_nbr27, const int *d_coords, const float *u, const float *w,
                       double dx, double *d_acc, cudaStream_t s)
{
    if (B == 8)
        k_diag<8><<<n_soln, 64, 0, s>>>(u, w, d_nbr27, d_coords, n_soln, dx, d_acc);
    else if (B == 16)
        k_diag<16><<<n_soln, 256, 0, s>>>(u, w, d_nbr27, d_coords, n_soln, dx, d_acc);
    else {
        set_error("operators support B in {8, 16} (got %d)", B);
        return LGF_ERR_ARG;
    }
    LGF_LAUNCH_CHECK("diagnostics");
    return LGF_OK;
}

lgf_status block_max_launch(int B, int nblk, const int *d_nbr27, const float *w, const float *q, float *mu, float *nu,
                            cudaStream_t s)
{
    if (B == 8)
        k_block_max<8><<<nblk, 64, 0, s>>>(w, q, d_nbr27, mu, nu);
    else if (B == 16)
        k_block_max<16><<<nblk, 256, 0, s>>>(w, q, d_nbr27, mu, nu);
    else {
        set_error("operators support B in {8, 16} (got %d)", B);
        return LGF_ERR_ARG;
    }
    LGF_LAUNCH_CHECK("block_max");
    return LGF_OK;
}

lgf_status zero_rim_launch(int B, int nblk, const int *d_nbr27, float *f, cudaStream_t s)
{
    if (B == 8)
        k_zero_rim<8><<<nblk, 64, 0, s>>>(f, d_nbr27);
    else if (B == 16)
        k_zero_rim<16><<<nblk, 256, 0, s>>>(f, d_nbr27);
    else {
        set_error("operators support B in {8, 16} (got %d)", B);
        return LGF_ERR_ARG;
    }
    LGF_LAUNCH_CHECK("zero_rim");
    return LGF_OK;
}

lgf_status grad_combine_launch(int B, int nblk, const int *d_nbr27, const float *dhat, const float *rv, const float *g,
                               float *out1, float *out2, double c2, double dx, cudaStream_t s)
{
    const float inv_dx = (float)(1.0 / dx);
    if (B == 8)
        k_grad_combine<8><<<nblk, 64, 0, s>>>(dhat, rv, g, out1, out2, d_nbr27, inv_dx, (float)c2);
    else if (B == 16)
        k_grad_combine<16><<<nblk, 256, 0, s>>>(dhat, rv, g, out1, out2, d_nbr27, inv_dx, (float)c2);
    else {
        set_error("operators support B in {8, 16} (got %d)", B);
        return LGF_ERR_ARG;
    }
    LGF_LAUNCH_CHECK("grad_combine");
    return LGF_OK;
}

lgf_status gather_launch(const float *in, float *out, const int *d_idx, int n, int block_floats, cudaStream_t s)
{
    if (n == 0) return LGF_OK;
    k_gather_blocks<<<n, 256, 0, s>>>(in, out, d_idx, block_floats);
    LGF_LAUNCH_CHECK("gather");
    return LGF_OK;
}

}  // namespace lgf
