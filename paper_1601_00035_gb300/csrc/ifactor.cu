// Integrating factor y = M E_Q(alpha) M x (Sec. 2.3 eq. if_def; Sec. 4.4),
// evaluated in real space as the convolution with the separable kernel
// prod_i g(n_i), g(k) = e^{-2 alpha} I_k(2 alpha) (App. B eq. lgf_intfac),
// truncated to the box |n_i| <= R (R <= min(B, 16); B in {8, 16}).  M keeps the block set S
// and zeroes everything else.
//
// The box kernel factorises, so the sum is taken as three 1-D passes
//   y1 = g *_z x,   y2 = g *_y y1,   y = g *_x y2,
// which is the same finite sum in another order.  With x zero outside S the
// intermediates are needed, and non-zero, only on small dilations of S:
//   y1 on L1 = (S + {dx,dy}) n (S + {dz}),
//   y2 on L2 = (S + {dx})    n (S + {dy,dz}),
//   y  on S,
// (block offsets in {-1,0,1}); the plan builds L1, L2 and the neighbour
// tables along each pass axis.  A block missing from a pass's input list is
// zero there.
//
// Each pass: one thread block per output block, one thread per line along the
// pass axis; the thread loads its B + 2R inputs (own block plus both
// neighbours) into registers and produces its B outputs with the symmetric
// taps (g0 v + sum_d g_d (v_{+d} + v_{-d})).  Taps travel as kernel parameters
// (constant bank), padded with zeros up to the instantiated radius RM.
#include "plan.hpp"

namespace lgf {
namespace {

template <int RM>
struct Taps {
    float g[RM + 1];
};

// AXIS 2: z pass (thread per (x, y)), AXIS 1: y pass (thread per (x, z)),
// AXIS 0: x pass (thread per (y, z), rows read as aligned float4 groups).
// EXTRA (optional linear combinations folded into the first and last pass):
// the z pass reads ca in + cb in2 instead of in, the x pass writes r + add.
template <int B, int RM, int AXIS, bool EXTRA>
__global__ void __launch_bounds__(B *B) k_if_pass(const float *__restrict__ in, float *__restrict__ out,
                                                  const int *__restrict__ nbr3, int ncomp, Taps<RM> t,
                                                  const float *__restrict__ in2, float ca, float cb,
                                                  const float *__restrict__ add)
{
    const int ob = blockIdx.x;  // output block
    const int c = blockIdx.y;
    const int a = threadIdx.x % B, b = threadIdx.x / B;
    const int n_lo = __ldg(nbr3 + 3 * ob), n_mid = __ldg(nbr3 + 3 * ob + 1), n_hi = __ldg(nbr3 + 3 * ob + 2);
    constexpr int W = B + 2 * RM;
    float v[W];
    if constexpr (AXIS == 0) {
        // v[k] = value at x = k - RM of row (y = a, z = b); rows of neighbours as float4
        constexpr int Q = B / 4;
        float rl[B], rm[B], rh[B];
        auto row = [&](int n, float *r) {
            if (n >= 0) {
                const float4 *p = reinterpret_cast<const float4 *>(in + ((size_t)(n * ncomp + c) * B + b) * B * B + a * B);
#pragma unroll
                for (int q = 0; q < Q; q++) {
                    const float4 w = __ldg(p + q);
                    r[4 * q] = w.x;
                    r[4 * q + 1] = w.y;
                    r[4 * q + 2] = w.z;
                    r[4 * q + 3] = w.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < B; q++) r[q] = 0.f;
            }
        };
        row(n_mid, rm);
        row(RM > 0 ? n_lo : -1, rl);
        row(RM > 0 ? n_hi : -1, rh);
#pragma unroll
        for (int k = 0; k < W; k++) {
            const int x = k - RM;
            v[k] = x < 0 ? rl[x + B] : (x < B ? rm[x] : rh[x - B]);
        }
    } else {
        const size_t cs = (size_t)B * B * B;
        const size_t om = (size_t)(n_mid >= 0 ? n_mid : 0) * ncomp * cs + (size_t)c * cs;
        const size_t ol = (size_t)(n_lo >= 0 ? n_lo : 0) * ncomp * cs + (size_t)c * cs;
        const size_t oh = (size_t)(n_hi >= 0 ? n_hi : 0) * ncomp * cs + (size_t)c * cs;
        const float *pm = in + om, *pl = in + ol, *ph = in + oh;
        // value at element offset q of the block at offset o: in, or ca in + cb in2
        auto val_at = [&](const float *p, size_t o, int q) -> float {
            if constexpr (EXTRA && AXIS == 2) return ca * __ldg(p + q) + cb * __ldg(in2 + o + q);
            else return __ldg(p + q);
        };
        // element (line index j along the axis) of this thread's line
        auto off = [&](int j) -> int {
            if constexpr (AXIS == 2) return j * B * B + b * B + a;  // (x=a, y=b, z=j)
            else return b * B * B + j * B + a;                     // (x=a, y=j, z=b)
        };
#pragma unroll
        for (int k = 0; k < W; k++) {
            const int j = k - RM;
            float val = 0.f;
            if (j < 0) {
                if (n_lo >= 0) val = val_at(pl, ol, off(j + B));
            } else if (j < B) {
                if (n_mid >= 0) val = val_at(pm, om, off(j));
            } else {
                if (n_hi >= 0) val = val_at(ph, oh, off(j - B));
            }
            v[k] = val;
        }
    }
    float r[B];
#pragma unroll
    for (int j = 0; j < B; j++) {
        float s = t.g[0] * v[j + RM];
#pragma unroll
        for (int d = 1; d <= RM; d++) s = fmaf(t.g[d], v[j + RM + d] + v[j + RM - d], s);
        r[j] = s;
    }
    float *o = out + (size_t)(ob * ncomp + c) * B * B * B;
    if constexpr (AXIS == 0) {
        const size_t ro = (size_t)(ob * ncomp + c) * B * B * B + (size_t)b * B * B + a * B;
        float4 *p = reinterpret_cast<float4 *>(out + ro);
        if constexpr (EXTRA) {
            const float4 *ad = reinterpret_cast<const float4 *>(add + ro);
#pragma unroll
            for (int q = 0; q < B / 4; q++) {
                const float4 w = __ldg(ad + q);
                r[4 * q] += w.x;
                r[4 * q + 1] += w.y;
                r[4 * q + 2] += w.z;
                r[4 * q + 3] += w.w;
            }
        }
#pragma unroll
        for (int q = 0; q < B / 4; q++) p[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < B; j++) {
            if constexpr (AXIS == 2) o[(size_t)j * B * B + b * B + a] = r[j];
            else o[(size_t)b * B * B + j * B + a] = r[j];
        }
    }
}

template <int B, int RM>
lgf_status launch3(const IfPlan &ip, int ncomp, const float *taps, const IfIO &io, float *y, cudaStream_t s,
                   Profiler *prof)
{
    Taps<RM> t;
    for (int i = 0; i <= RM; i++) t.g[i] = i <= ip.R ? taps[i] : 0.f;
    const bool P = prof && prof->on;
    const bool lin = io.x1 != nullptr || io.c0 != 1.0;
    const float ca = (float)io.c0, cb = (float)io.c1;
    if (P) prof->begin(s);
    if (lin)
        k_if_pass<B, RM, 2, true><<<dim3(ip.n1, ncomp), B * B, 0, s>>>(io.x0, ip.y1, ip.nbz, ncomp, t,
                                                                       io.x1 ? io.x1 : io.x0, ca, io.x1 ? cb : 0.f,
                                                                       nullptr);
    else
        k_if_pass<B, RM, 2, false><<<dim3(ip.n1, ncomp), B * B, 0, s>>>(io.x0, ip.y1, ip.nbz, ncomp, t, nullptr, 1.f,
                                                                        0.f, nullptr);
    LGF_LAUNCH_CHECK("if_z_pass");
    if (P) prof->end("if_z_pass", s);
    if (P) prof->begin(s);
    k_if_pass<B, RM, 1, false><<<dim3(ip.n2, ncomp), B * B, 0, s>>>(ip.y1, ip.y2, ip.nby, ncomp, t, nullptr, 1.f, 0.f,
                                                                    nullptr);
    LGF_LAUNCH_CHECK("if_y_pass");
    if (P) prof->end("if_y_pass", s);
    if (P) prof->begin(s);
    if (io.add)
        k_if_pass<B, RM, 0, true><<<dim3(ip.n0, ncomp), B * B, 0, s>>>(ip.y2, y, ip.nbx, ncomp, t, nullptr, 1.f, 0.f,
                                                                       io.add);
    else
        k_if_pass<B, RM, 0, false><<<dim3(ip.n0, ncomp), B * B, 0, s>>>(ip.y2, y, ip.nbx, ncomp, t, nullptr, 1.f, 0.f,
                                                                        nullptr);
    LGF_LAUNCH_CHECK("if_x_pass");
    if (P) prof->end("if_x_pass", s);
    return LGF_OK;
}

}  // namespace

lgf_status ifactor_launch(const IfPlan &ip, int ncomp, const float *h_taps, const float *x, float *y, cudaStream_t s,
                          Profiler *prof)
{
    IfIO io;
    io.x0 = x;
    return ifactor_launch_ex(ip, ncomp, h_taps, io, y, s, prof);
}

lgf_status ifactor_launch_ex(const IfPlan &ip, int ncomp, const float *h_taps, const IfIO &x, float *y, cudaStream_t s,
                             Profiler *prof)
{
    const int B = ip.B, R = ip.R;
    if (R > B || R > 16) {
        set_error("integrating-factor radius %d exceeds min(B=%d, 16)", R, B);
        return LGF_ERR_ARG;
    }
    const int RM = R <= 4 ? 4 : (R <= 8 ? 8 : (R <= 12 ? 12 : 16));
    switch (B) {
        case 8:
            if (RM == 4) return launch3<8, 4>(ip, ncomp, h_taps, x, y, s, prof);
            return launch3<8, 8>(ip, ncomp, h_taps, x, y, s, prof);
        case 16:
            if (RM == 4) return launch3<16, 4>(ip, ncomp, h_taps, x, y, s, prof);
            if (RM == 8) return launch3<16, 8>(ip, ncomp, h_taps, x, y, s, prof);
            if (RM == 12) return launch3<16, 12>(ip, ncomp, h_taps, x, y, s, prof);
            return launch3<16, 16>(ip, ncomp, h_taps, x, y, s, prof);
        default:
            set_error("unsupported block size %d", B);
            return LGF_ERR_ARG;
    }
}

}  // namespace lgf
