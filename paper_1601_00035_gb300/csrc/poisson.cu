// Poisson solve u = scale * dx^2 * G * f (Sec. 2.2, eq. dpoisson_conv) by the
// free-space zero-padding embedding: a circular convolution on an N^3 grid
// with N >= 2 * (largest source-target offset) + 2 reproduces the linear sum
// exactly, because every offset that occurs lands on a distinct wrapped index.
// The kernel samples G(wrap(j)) are real and even, so their spectrum is real
// and even and only its octant is stored (built in FP64, spectrum.cu).
//
// Five passes, each a batch of 1-D FFTs on shared-memory tiles (fft.cuh):
//   x_fwd : gather source rows from the block list (two real rows packed into
//           one complex line), R2C along x                 src -> A[c][z][y][kx]
//   y_fwd : along y (input rows beyond the source box are zero)  A -> B[c][z][ky][kx]
//   z_mid : along z, multiply by the kernel spectrum, inverse along z, keep
//           the target planes                               B -> A[c][zt][ky][kx]
//   y_inv : inverse along y, keep the target rows           A -> B[c][zt][yt][kx]
//   x_inv : C2R along x (two rows per complex line), scatter into the target
//           block list                                      B -> dst
// The gather, the spectral multiply and the scatter are fused into the first,
// middle and last pass, so no padded real array ever exists in memory.
#include "fft.cuh"
#include "plan.hpp"

namespace lgf {

namespace {

constexpr int kThreads = 256;

template <int N>
struct Tile {
    static constexpr int G = fft::Plan<N>::lanes;          // lanes per line
    static constexpr int LS = (kThreads / G) < 64 ? (kThreads / G) : 64;  // lines per block
    static constexpr int LSP = LS + 1;
    static constexpr int threads = LS * G;
};

__device__ __forceinline__ int wrap_mod(int v, int n)
{
    int r = v % n;
    return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Tile<N>::threads) k_x_fwd(Geom g, const float *__restrict__ src,
                                                             cx<float> *__restrict__ out, const float2 *tw_g)
{
    using TL = Tile<N>;
    __shared__ cx<float> buf[N * TL::LSP];
    __shared__ cx<float> tw[N];
    fft::load_twiddles<N, float>(tw, tw_g);
    const int c = blockIdx.y;
    const int t = threadIdx.x;
    const int nrows = g.Es[1] * g.Es[2];
    const int pair0 = blockIdx.x * TL::LS;
    const int B = g.B;
    for (int idx = t; idx < TL::LS * N; idx += TL::threads) {
        const int ll = idx / N, n = idx - ll * N;
        const int r0 = 2 * (pair0 + ll);
        cx<float> v = {0.f, 0.f};
        if (n < g.Es[0] && r0 < nrows) {
            const int z = r0 / g.Es[1], y = r0 - z * g.Es[1];
            const int blk = g.src_lut[((z / B) * g.nbS[1] + y / B) * g.nbS[0] + n / B];
            if (blk >= 0) {
                const float *p = src + ((size_t)(blk * g.ncomp + c) * B + (z % B)) * B * B + (y % B) * B + (n % B);
                v.x = __ldg(p);
                v.y = __ldg(p + B);
            }
        }
        buf[n * TL::LSP + ll] = v;
    }
    __syncthreads();
    fft::line_fft<N, false, float>(buf, tw, TL::LSP, t % TL::LS, t / TL::LS, true);
    constexpr int KX = N / 2 + 1;
    for (int idx = t; idx < TL::LS * KX; idx += TL::threads) {
        const int ll = idx / KX, k = idx - ll * KX;
        const int r0 = 2 * (pair0 + ll);
        if (r0 >= nrows) continue;
        const cx<float> zk = buf[k * TL::LSP + ll];
        const cx<float> zn = buf[((N - k) & (N - 1)) * TL::LSP + ll];
        const cx<float> a = {0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y)};
        const cx<float> b = {0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x)};
        const size_t row = ((size_t)c * nrows + r0) * KX;
        out[row + k] = a;
        out[row + KX + k] = b;
    }
}

// Generic line pass over [c][plane][line-axis][kx] arrays, lines along the
// middle axis, LS consecutive kx per block.
//   MODE 0 (y_fwd): in  [c][Es_z][Es_y][KX] (n < Es_y), out [c][Es_z][Ny][KX]
//   MODE 1 (z_mid): in  [c][Es_z][Ny][KX] lines along z, out [c][Et_z][Ny][KX]
//   MODE 2 (y_inv): in  [c][Et_z][Ny][KX], out [c][Et_z][Et_y][KX]
template <int N, int MODE>
__global__ void __launch_bounds__(Tile<N>::threads) k_line(Geom g, const cx<float> *__restrict__ in,
                                                            cx<float> *__restrict__ out, const float2 *tw_g)
{
    using TL = Tile<N>;
    __shared__ cx<float> buf[N * TL::LSP];
    __shared__ cx<float> tw[N];
    fft::load_twiddles<N, float>(tw, tw_g);
    const int KX = g.KX;
    const int kx0 = blockIdx.x * TL::LS;
    const int p = blockIdx.y;  // plane: z (MODE 0), ky (MODE 1), zt (MODE 2)
    const int c = blockIdx.z;
    const int t = threadIdx.x;
    const int Ny = g.N[1];

    int nin;
    if (MODE == 0) nin = g.Es[1];
    else if (MODE == 1) nin = g.Es[2];
    else nin = Ny;
    for (int idx = t; idx < TL::LS * N; idx += TL::threads) {
        const int n = idx / TL::LS, ll = idx - n * TL::LS;
        const int kx = kx0 + ll;
        cx<float> v = {0.f, 0.f};
        if (n < nin && kx < KX) {
            size_t off;
            if (MODE == 0) off = (((size_t)c * g.Es[2] + p) * g.Es[1] + n) * KX + kx;
            else if (MODE == 1) off = (((size_t)c * g.Es[2] + n) * Ny + p) * KX + kx;
            else off = (((size_t)c * g.Et[2] + p) * Ny + n) * KX + kx;
            v = in[off];
        }
        buf[n * TL::LSP + ll] = v;
    }
    __syncthreads();
    const int l = t % TL::LS, lane = t / TL::LS;
    if (MODE == 0) {
        fft::line_fft<N, false, float>(buf, tw, TL::LSP, l, lane, true);
        for (int idx = t; idx < TL::LS * N; idx += TL::threads) {
            const int n = idx / TL::LS, ll = idx - n * TL::LS;
            const int kx = kx0 + ll;
            if (kx < KX) out[(((size_t)c * g.Es[2] + p) * N + n) * KX + kx] = buf[n * TL::LSP + ll];
        }
    } else if (MODE == 1) {
        fft::line_fft<N, false, float>(buf, tw, TL::LSP, l, lane, true);
        // multiply by the real, even kernel spectrum (octant storage)
        const int ky = p;
        const int kyf = ky <= Ny / 2 ? ky : Ny - ky;
        const int NyH = Ny / 2 + 1;
        for (int idx = t; idx < TL::LS * N; idx += TL::threads) {
            const int n = idx / TL::LS, ll = idx - n * TL::LS;
            const int kx = kx0 + ll;
            if (kx < KX) {
                const int kzf = n <= N / 2 ? n : N - n;
                const float w = g.mul * __ldg(g.Kh + ((size_t)kzf * NyH + kyf) * KX + kx);
                cx<float> v = buf[n * TL::LSP + ll];
                buf[n * TL::LSP + ll] = {v.x * w, v.y * w};
            }
        }
        __syncthreads();
        fft::line_fft<N, true, float>(buf, tw, TL::LSP, l, lane, true);
        const int dz = g.T0[2] - g.S0[2];
        for (int idx = t; idx < TL::LS * g.Et[2]; idx += TL::threads) {
            const int zt = idx / TL::LS, ll = idx - zt * TL::LS;
            const int kx = kx0 + ll;
            if (kx < KX) {
                const int n = wrap_mod(dz + zt, N);
                out[(((size_t)c * g.Et[2] + zt) * Ny + p) * KX + kx] = buf[n * TL::LSP + ll];
            }
        }
    } else {
        fft::line_fft<N, true, float>(buf, tw, TL::LSP, l, lane, true);
        const int dy = g.T0[1] - g.S0[1];
        for (int idx = t; idx < TL::LS * g.Et[1]; idx += TL::threads) {
            const int yt = idx / TL::LS, ll = idx - yt * TL::LS;
            const int kx = kx0 + ll;
            if (kx < KX) {
                const int n = wrap_mod(dy + yt, N);
                out[(((size_t)c * g.Et[2] + p) * g.Et[1] + yt) * KX + kx] = buf[n * TL::LSP + ll];
            }
        }
    }
}

template <int N>
__global__ void __launch_bounds__(Tile<N>::threads) k_x_inv(Geom g, const cx<float> *__restrict__ in,
                                                             float *__restrict__ dst, const float2 *tw_g)
{
    using TL = Tile<N>;
    __shared__ cx<float> buf[N * TL::LSP];
    __shared__ cx<float> tw[N];
    fft::load_twiddles<N, float>(tw, tw_g);
    constexpr int KX = N / 2 + 1;
    const int c = blockIdx.y;
    const int t = threadIdx.x;
    const int nrows = g.Et[1] * g.Et[2];
    const int pair0 = blockIdx.x * TL::LS;
    for (int idx = t; idx < TL::LS * N; idx += TL::threads) {
        const int ll = idx / N, k = idx - ll * N;
        const int r0 = 2 * (pair0 + ll);
        cx<float> zv = {0.f, 0.f};
        if (r0 < nrows) {
            const size_t row = ((size_t)c * nrows + r0) * KX;
            cx<float> a, b;
            if (k <= N / 2) {
                a = in[row + k];
                b = in[row + KX + k];
            } else {
                a = conj(in[row + (N - k)]);
                b = conj(in[row + KX + (N - k)]);
            }
            zv = {a.x - b.y, a.y + b.x};  // a + i b
        }
        buf[k * TL::LSP + ll] = zv;
    }
    __syncthreads();
    fft::line_fft<N, true, float>(buf, tw, TL::LSP, t % TL::LS, t / TL::LS, true);
    const int B = g.B;
    const int dx0 = g.T0[0] - g.S0[0];
    for (int idx = t; idx < TL::LS * g.Et[0]; idx += TL::threads) {
        const int ll = idx / g.Et[0], xt = idx - ll * g.Et[0];
        const int r0 = 2 * (pair0 + ll);
        if (r0 >= nrows) continue;
        const int zt = r0 / g.Et[1], yt = r0 - zt * g.Et[1];
        const int blk = g.dst_lut[((zt / B) * g.nbT[1] + yt / B) * g.nbT[0] + xt / B];
        if (blk < 0) continue;
        const cx<float> zv = buf[wrap_mod(dx0 + xt, N) * TL::LSP + ll];
        float *p = dst + ((size_t)(blk * g.ncomp + c) * B + (zt % B)) * B * B + (yt % B) * B + (xt % B);
        p[0] = zv.x;
        p[B] = zv.y;
    }
}

template <int N>
lgf_status launch_x_fwd(const Geom &g, const float *src, cx<float> *out, cudaStream_t s)
{
    using TL = Tile<N>;
    const int nrows = g.Es[1] * g.Es[2];
    dim3 grid(ceil_div(nrows / 2, TL::LS), g.ncomp);
    k_x_fwd<N><<<grid, TL::threads, 0, s>>>(g, src, out, twiddle_table_f32());
    LGF_LAUNCH_CHECK("x_fwd");
    return LGF_OK;
}
template <int N, int MODE>
lgf_status launch_line(const Geom &g, const cx<float> *in, cx<float> *out, cudaStream_t s)
{
    using TL = Tile<N>;
    int planes = MODE == 0 ? g.Es[2] : (MODE == 1 ? g.N[1] : g.Et[2]);
    dim3 grid(ceil_div(g.KX, TL::LS), planes, g.ncomp);
    k_line<N, MODE><<<grid, TL::threads, 0, s>>>(g, in, out, twiddle_table_f32());
    LGF_LAUNCH_CHECK(MODE == 0 ? "y_fwd" : (MODE == 1 ? "z_mid" : "y_inv"));
    return LGF_OK;
}
template <int N>
lgf_status launch_x_inv(const Geom &g, const cx<float> *in, float *dst, cudaStream_t s)
{
    using TL = Tile<N>;
    const int nrows = g.Et[1] * g.Et[2];
    dim3 grid(ceil_div(nrows / 2, TL::LS), g.ncomp);
    k_x_inv<N><<<grid, TL::threads, 0, s>>>(g, in, dst, twiddle_table_f32());
    LGF_LAUNCH_CHECK("x_inv");
    return LGF_OK;
}

#define LGF_DISPATCH_N(n, CALL)            \
    switch (n) {                           \
        case 16: { constexpr int NN = 16; CALL; } break;     \
        case 32: { constexpr int NN = 32; CALL; } break;     \
        case 64: { constexpr int NN = 64; CALL; } break;     \
        case 128: { constexpr int NN = 128; CALL; } break;   \
        case 256: { constexpr int NN = 256; CALL; } break;   \
        case 512: { constexpr int NN = 512; CALL; } break;   \
        case 1024: { constexpr int NN = 1024; CALL; } break; \
        default: set_error("unsupported FFT length %d", n); return LGF_ERR_ARG; \
    }

}  // namespace

lgf_status poisson_prepare()
{
    if (fft::upload_tw64() != cudaSuccess) {
        set_error("twiddle upload failed");
        return LGF_ERR_CUDA;
    }
    return ensure_twiddles();
}

bool poisson_supported_n(int n)
{
    return n == 16 || n == 32 || n == 64 || n == 128 || n == 256 || n == 512 || n == 1024;
}

int poisson_pick_n(int need)
{
    for (int n = 16; n <= 1024; n *= 2)
        if (n >= need) return n;
    return 0;
}

lgf_status poisson_launch(const Geom &g, const float *src, float *dst, cx<float> *wsA, cx<float> *wsB,
                          cudaStream_t s)
{
    if (fft::upload_tw64() != cudaSuccess) {
        set_error("twiddle upload failed");
        return LGF_ERR_CUDA;
    }
    LGF_DISPATCH_N(g.N[0], LGF_TRY((launch_x_fwd<NN>(g, src, wsA, s))));
    LGF_DISPATCH_N(g.N[1], LGF_TRY((launch_line<NN, 0>(g, wsA, wsB, s))));
    LGF_DISPATCH_N(g.N[2], LGF_TRY((launch_line<NN, 1>(g, wsB, wsA, s))));
    LGF_DISPATCH_N(g.N[1], LGF_TRY((launch_line<NN, 2>(g, wsA, wsB, s))));
    LGF_DISPATCH_N(g.N[0], LGF_TRY((launch_x_inv<NN>(g, wsB, dst, s))));
    return LGF_OK;
}

}  // namespace lgf
