// The five FFT passes of one Poisson solve at FFT length N along the pass
// axis (kernels in poisson_kernels.cuh).  PoissonPasses<N, T> is instantiated
// once per supported length and precision, in the poisson_len_*.cu units:
//   a: 16, 32, 64, 96, 128     b: 192, 256, 288     c: 384, 432, 512 (FP32 and FP64)
//   d: 768, 1024 (FP32 only)
#pragma once
#include "plan.hpp"

namespace lgf {

// Grouped execution of a plan with many units (solve, component): one launch per
// (pass, FFT length of that pass's axis) covers every unit with that length.
// Thread block b of a grouped launch runs tile b - first of task cta_task[b].
constexpr int kGroupMaxSolves = 128;  // solves of a plan that runs grouped
template <typename T>
struct GroupTask {
    Geom g;          // the unit's geometry (c0 = its component, nc = 1)
    cx<T> *wa, *wb;  // the unit's two workspaces
    int solve;       // index of the unit's buffers in SolvePtrs
    int first;       // first thread block of this task in its launch
};
template <typename T>
struct SolvePtrs {  // the buffers of one execution (kernel parameter)
    const T *src[kGroupMaxSolves];
    T *dst[kGroupMaxSolves];
};
// pass index: 0 x forward, 1 y forward, 2 z, 3 y inverse, 4 x inverse; its axis
constexpr int pass_axis(int pass) { return pass == 0 || pass == 4 ? 0 : (pass == 2 ? 2 : 1); }

template <int N, typename T>
struct PoissonPasses {
    static int tiles(int pass, const Geom &g);  // thread blocks of one unit's pass
    static lgf_status grouped(int pass, const GroupTask<T> *tasks, const int *cta_task, int ncta,
                              const SolvePtrs<T> &ptrs, cudaStream_t s);
    static lgf_status x_fwd(const Geom &g, const T *src, cx<T> *out, cudaStream_t s);     // gather, R2C in x
    static lgf_status y_fwd(const Geom &g, const cx<T> *in, cx<T> *out, cudaStream_t s);  // forward in y
    static lgf_status z_mid(const Geom &g, const cx<T> *in, cx<T> *out, cudaStream_t s);  // z: fwd, multiply, inv
    static lgf_status y_inv(const Geom &g, const cx<T> *in, cx<T> *out, cudaStream_t s);  // inverse in y
    static lgf_status x_inv(const Geom &g, const cx<T> *in, T *dst, cudaStream_t s);      // C2R in x, scatter
};

// Each unit holds its own constant-bank copy of the in-register DFT twiddles
// (fft.cuh); these upload it on the current device (once per device).
cudaError_t poisson_tw_upload_a();
cudaError_t poisson_tw_upload_b();
cudaError_t poisson_tw_upload_c();
cudaError_t poisson_tw_upload_d();

// thread blocks of a unit's pass (-1: unsupported length); one grouped launch (poisson.cu)
int poisson_tiles(int pass, const Geom &g);
lgf_status poisson_launch_grouped(int pass, int n, const GroupTask<float> *tasks, const int *cta_task, int ncta,
                                  const SolvePtrs<float> &ptrs, cudaStream_t s);

#define LGF_POISSON_LENGTHS_A(X) X(16) X(32) X(64) X(96) X(128)
#define LGF_POISSON_LENGTHS_B(X) X(192) X(256) X(288)
#define LGF_POISSON_LENGTHS_C(X) X(384) X(432) X(512)
#define LGF_POISSON_LENGTHS_D(X) X(768) X(1024)
#define LGF_POISSON_EXTERN_FD(n) extern template struct PoissonPasses<n, float>; extern template struct PoissonPasses<n, double>;
#define LGF_POISSON_EXTERN_F(n) extern template struct PoissonPasses<n, float>;
LGF_POISSON_LENGTHS_A(LGF_POISSON_EXTERN_FD)
LGF_POISSON_LENGTHS_B(LGF_POISSON_EXTERN_FD)
LGF_POISSON_LENGTHS_C(LGF_POISSON_EXTERN_FD)
LGF_POISSON_LENGTHS_D(LGF_POISSON_EXTERN_F)
#undef LGF_POISSON_EXTERN_FD
#undef LGF_POISSON_EXTERN_F

}  // namespace lgf
