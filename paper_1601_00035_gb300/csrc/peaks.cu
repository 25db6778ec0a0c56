// lgf_measure_peak: the arithmetic rates of this GPU that bound the FFT, spectral
// multiply and integrating-factor passes (the roofline denominators for work that is
// not HBM-bound).  Every thread of a grid of 8 x 256-thread blocks per SM runs eight
// independent register-resident FMA chains; the rate is FMAs x flops per FMA / time,
// with the time taken by CUDA events on the caller's stream.
#include <cmath>

#include "plan.hpp"

namespace lgf {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void k_peak_f32(int iters, float b, float c, float *out)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = 1e-3f * (threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    if (s == -1.0f) out[blockIdx.x] = s;  // never true for these operands; keeps the chains live
}

__global__ void k_peak_f32x2(int iters, float b, float c, float *out)
{
    unsigned long long a[kChains], bb, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int k = 0; k < kChains; k++) {
        const float v = 1e-3f * (threadIdx.x + k);
        asm("mov.b64 %0, {%1, %1};" : "=l"(a[k]) : "f"(v));
    }
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
#pragma unroll
            for (int k = 0; k < kChains; k++) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(bb), "l"(cc));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[k]));
        s += lo + hi;
    }
    if (s == -1.0f) out[blockIdx.x] = s;
}

__global__ void k_peak_f64(int iters, double b, double c, float *out)
{
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    if (s == -1.0) out[blockIdx.x] = (float)s;
}

lgf_status run_peak(int kind, int iters, int grid, cudaStream_t s, float *sink, float *ms)
{
    cudaEvent_t e0, e1;
    LGF_CUDA_TRY(cudaEventCreate(&e0));
    LGF_CUDA_TRY(cudaEventCreate(&e1));
    cudaEventRecord(e0, s);
    if (kind == 0)
        k_peak_f32<<<grid, 256, 0, s>>>(iters, 0.9999999f, 1e-7f, sink);
    else if (kind == 1)
        k_peak_f32x2<<<grid, 256, 0, s>>>(iters, 0.9999999f, 1e-7f, sink);
    else
        k_peak_f64<<<grid, 256, 0, s>>>(iters, 0.9999999999, 1e-9, sink);
    cudaError_t e = cudaGetLastError();
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        set_error("peak kernel failed: %s", cudaGetErrorString(e));
        return LGF_ERR_CUDA;
    }
    return LGF_OK;
}

}  // namespace
}  // namespace lgf

using namespace lgf;

extern "C" lgf_status lgf_measure_peak(int kind, double ms, double *tflops, void *stream)
{
    clear_error();
    LGF_CHECK_ARG(kind >= 0 && kind <= 2, "lgf_measure_peak: kind %d not in 0..2", kind);
    LGF_CHECK_ARG(tflops && ms > 0.0 && ms <= 10000.0, "lgf_measure_peak: bad output pointer or ms %g", ms);
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    LGF_CUDA_TRY(cudaGetDevice(&dev));
    LGF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = 8 * nsm;
    float *sink = nullptr;
    LGF_CUDA_TRY(cudaMalloc(&sink, grid * sizeof(float)));
    // calibrate the iteration count on a short run, then time one run of about `ms`
    int iters = 64;
    float t = 0.f;
    lgf_status st = run_peak(kind, iters, grid, s, sink, &t);
    for (int k = 0; st == LGF_OK && k < 4 && t < 0.05f * (float)ms; k++) {
        iters *= 8;
        st = run_peak(kind, iters, grid, s, sink, &t);
    }
    if (st == LGF_OK) {
        const double scale = ms / fmax((double)t, 1e-3);
        iters = (int)fmin(fmax(iters * scale, 64.0), 2.0e9 / (kChains * kUnroll));
        st = run_peak(kind, iters, grid, s, sink, &t);
    }
    cudaFree(sink);
    if (st != LGF_OK) return st;
    const double fmas = (double)grid * 256 * iters * kUnroll * kChains;
    const double flops_per_fma = kind == 1 ? 4.0 : 2.0;
    *tflops = fmas * flops_per_fma / ((double)t * 1e-3) / 1e12;
    return LGF_OK;
}
