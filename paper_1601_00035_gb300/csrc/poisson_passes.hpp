// The five FFT passes of one Poisson solve at FFT length N along the pass
// axis (kernels in poisson_kernels.cuh).  PoissonPasses<N, T> is instantiated
// once per supported length and precision, in the poisson_len_*.cu units:
//   a: 16, 32, 64, 96, 128     b: 192, 256, 288     c: 384, 432, 512 (FP32 and FP64)
//   d: 768, 1024 (FP32 only)
#pragma once
#include "plan.hpp"

namespace lgf {

template <int N, typename T>
struct PoissonPasses {
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
