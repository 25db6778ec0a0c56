// Poisson solve u = scale * dx^2 * G * f (Sec. 2.2, eq. dpoisson_conv) by the
// free-space zero-padding embedding: a circular convolution on an N^3 grid
// with N >= 2 * (largest source-target offset) + 2 reproduces the linear sum
// exactly, because every offset that occurs lands on a distinct wrapped index.
// The kernel samples G(wrap(j)) are real and even, so their spectrum is real
// and even and only its octant is stored (built in FP64, spectrum.cu).
//
// Five passes, each a batch of register-resident 1-D FFTs (fft.cuh):
//   x_fwd : gather source rows from the block list (two real rows packed into
//           one complex line), R2C along x                 src -> A[c][z][y][kx]
//   y_fwd : along y (input rows beyond the source box are zero)  A -> B[c][z][ky][kx]
//   z_mid : along z, multiply by the kernel spectrum, inverse along z, keep
//           the target planes                               B -> A[c][zt][ky][kx]
//           (FP32 plans with 16 elements per lane run two lines per lane in
//           packed .f32x2 arithmetic: k_zmid2)
//   y_inv : inverse along y, keep the target rows           A -> B[c][zt][yt][kx]
//   x_inv : C2R along x (two rows per complex line), scatter into the target
//           block list                                      B -> dst
// The gather, the spectral multiply and the scatter are fused into the first,
// middle and last pass, so no padded real array ever exists in memory.
// The kernels are templates over the pass length (poisson_kernels.cuh),
// instantiated per length in the poisson_len_*.cu units; this unit dispatches.
#include "plan.hpp"
#include "poisson_passes.hpp"

namespace lgf {

namespace {

// N-dispatch; FP64 transforms stop at N = 512 (shared-memory budget).
#define LGF_DISPATCH_N(T, n, CALL)                                                          \
    switch (n) {                                                                            \
        case 16: { constexpr int NN = 16; CALL; } break;                                    \
        case 32: { constexpr int NN = 32; CALL; } break;                                    \
        case 64: { constexpr int NN = 64; CALL; } break;                                    \
        case 96: { constexpr int NN = 96; CALL; } break;                                    \
        case 128: { constexpr int NN = 128; CALL; } break;                                  \
        case 192: { constexpr int NN = 192; CALL; } break;                                  \
        case 256: { constexpr int NN = 256; CALL; } break;                                  \
        case 288: { constexpr int NN = 288; CALL; } break;                                  \
        case 384: { constexpr int NN = 384; CALL; } break;                                  \
        case 432: { constexpr int NN = 432; CALL; } break;                                  \
        case 512: { constexpr int NN = 512; CALL; } break;                                  \
        case 768:                                                                           \
            if constexpr (sizeof(T) == 4) { constexpr int NN = 768; CALL; }                 \
            else { set_error("FP64 transforms are limited to N <= 512"); return LGF_ERR_ARG; } \
            break;                                                                          \
        case 1024:                                                                          \
            if constexpr (sizeof(T) == 4) { constexpr int NN = 1024; CALL; }                \
            else { set_error("FP64 transforms are limited to N <= 512"); return LGF_ERR_ARG; } \
            break;                                                                          \
        default: set_error("unsupported FFT length %d", n); return LGF_ERR_ARG;             \
    }

// every unit's copy of the in-register DFT twiddles on the current device
lgf_status upload_all_tw()
{
    const cudaError_t e[4] = {poisson_tw_upload_a(), poisson_tw_upload_b(), poisson_tw_upload_c(),
                              poisson_tw_upload_d()};
    for (cudaError_t x : e)
        if (x != cudaSuccess) {
            set_error("twiddle upload failed: %s", cudaGetErrorString(x));
            return LGF_ERR_CUDA;
        }
    return LGF_OK;
}

template <typename T>
lgf_status launch_all(const Geom &g, const T *src, T *dst, cx<T> *wsA, cx<T> *wsB, cudaStream_t s, Profiler *prof,
                      cudaEvent_t mark = nullptr, int mark_after = -1)
{
    auto MARK = [&](int pass) -> lgf_status {
        if (mark && mark_after == pass) LGF_CUDA_TRY(cudaEventRecord(mark, s));
        return LGF_OK;
    };
    LGF_TRY(upload_all_tw());
    const bool P = prof && prof->on;
    if (P) prof->begin(s);
    LGF_DISPATCH_N(T, g.N[0], LGF_TRY((PoissonPasses<NN, T>::x_fwd(g, src, wsA, s))));
    if (P) prof->end("x_fwd_gather_r2c", s);
    LGF_TRY(MARK(0));
    if (P) prof->begin(s);
    LGF_DISPATCH_N(T, g.N[1], LGF_TRY((PoissonPasses<NN, T>::y_fwd(g, wsA, wsB, s))));
    if (P) prof->end("y_fwd", s);
    LGF_TRY(MARK(1));
    if (P) prof->begin(s);
    LGF_DISPATCH_N(T, g.N[2], LGF_TRY((PoissonPasses<NN, T>::z_mid(g, wsB, wsA, s))));
    if (P) prof->end("z_fwd_mul_inv", s);
    LGF_TRY(MARK(2));
    if (P) prof->begin(s);
    LGF_DISPATCH_N(T, g.N[1], LGF_TRY((PoissonPasses<NN, T>::y_inv(g, wsA, wsB, s))));
    if (P) prof->end("y_inv", s);
    if (P) prof->begin(s);
    LGF_DISPATCH_N(T, g.N[0], LGF_TRY((PoissonPasses<NN, T>::x_inv(g, wsB, dst, s))));
    if (P) prof->end("x_inv_c2r_scatter", s);
    return LGF_OK;
}

}  // namespace

lgf_status poisson_prepare()
{
    LGF_TRY(upload_all_tw());
    return ensure_twiddles();
}

// supported FFT lengths, ascending: powers of two, 3 times a power of two,
// 288 = 9 * 32 and 432 = 27 * 16
static const int kLengths[] = {16, 32, 64, 96, 128, 192, 256, 288, 384, 432, 512, 768, 1024};

bool poisson_supported_n(int n)
{
    for (int v : kLengths)
        if (v == n) return true;
    return false;
}

int poisson_pick_n(int need)
{
    for (int v : kLengths)
        if (v >= need) return v;
    return 0;
}

int poisson_tiles(int pass, const Geom &g)
{
    switch (g.N[pass_axis(pass)]) {
#define LGF_TILES_CASE(n) \
    case n: return PoissonPasses<n, float>::tiles(pass, g);
        LGF_POISSON_LENGTHS_A(LGF_TILES_CASE)
        LGF_POISSON_LENGTHS_B(LGF_TILES_CASE)
        LGF_POISSON_LENGTHS_C(LGF_TILES_CASE)
        LGF_POISSON_LENGTHS_D(LGF_TILES_CASE)
#undef LGF_TILES_CASE
        default: return -1;
    }
}

lgf_status poisson_launch_grouped(int pass, int n, const GroupTask<float> *tasks, const int *cta_task, int ncta,
                                  const SolvePtrs<float> &ptrs, cudaStream_t s)
{
    LGF_TRY(upload_all_tw());
    LGF_DISPATCH_N(float, n, LGF_TRY((PoissonPasses<NN, float>::grouped(pass, tasks, cta_task, ncta, ptrs, s))));
    return LGF_OK;
}

lgf_status poisson_launch(const Geom &g, const float *src, float *dst, cx<float> *wsA, cx<float> *wsB,
                          cudaStream_t s, Profiler *prof, cudaEvent_t mark, int mark_after)
{
    return launch_all<float>(g, src, dst, wsA, wsB, s, prof, mark, mark_after);
}

lgf_status poisson_launch64(const Geom &g, const double *src, double *dst, cx<double> *wsA, cx<double> *wsB,
                            cudaStream_t s, Profiler *prof)
{
    return launch_all<double>(g, src, dst, wsA, wsB, s, prof);
}

}  // namespace lgf
