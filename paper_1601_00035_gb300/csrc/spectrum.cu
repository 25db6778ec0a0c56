// Spectrum of the zero-padded LGF kernel (the LGF tables are pre-processed
// once per simulation, App. B last paragraph).
//
// On an N-periodic grid the kernel is K(j) = G(wrap(j)), wrap(j) = j for
// j < N/2, j - N for j > N/2, and K(N/2) = 0.  K is real and even in every
// axis, so its DFT is real, even, and separable into cosine sums:
//   Khat(k) = sum_{j=0}^{N/2-1} c_j cos(2 pi j k / N) K(j),  c_0 = 1, c_j = 2,
// applied along x, y and z in turn on the octant j, k in [0, N/2].  Computed
// in FP64 by direct summation (no FFT), rounded once to FP32 at the end.
#include <algorithm>
#include <cmath>
#include <vector>

#include "plan.hpp"

namespace lgf {
namespace {

__device__ __forceinline__ int64_t oct_idx(int a, int b, int c)
{
    // sorted a >= b >= c
    return (int64_t)a * (a + 1) * (a + 2) / 6 + (int64_t)b * (b + 1) / 2 + c;
}

// in[z][y][x], x,y,z in [0, N/2]; zero where any index == N/2
__global__ void k_fill(const double *__restrict__ oct, int K, int hx, int hy, int hz, double *__restrict__ out)
{
    const int64_t total = (int64_t)(hx + 1) * (hy + 1) * (hz + 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % (hx + 1));
        const int y = (int)((i / (hx + 1)) % (hy + 1));
        const int z = (int)(i / ((int64_t)(hx + 1) * (hy + 1)));
        double v = 0.0;
        if (x < hx && y < hy && z < hz) {
            int a = x, b = y, c = z, t;
            if (a < b) { t = a; a = b; b = t; }
            if (b < c) { t = b; b = c; c = t; }
            if (a < b) { t = a; a = b; b = t; }
            if (a <= K) v = oct[oct_idx(a, b, c)];
        }
        out[i] = v;
    }
}

// Apply the cosine sum along one axis of a [nz][ny][nx] array (all dims N_a/2+1).
// axis 0: x, 1: y, 2: z.  cos table ct[m] = cos(2 pi m / Na), m < Na.
__global__ void k_cos_axis(const double *__restrict__ in, double *__restrict__ out, int nx, int ny, int nz, int axis,
                           int Na, const double *__restrict__ ct)
{
    const int64_t total = (int64_t)nx * ny * nz;
    const int h = Na / 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const int y = (int)((i / nx) % ny);
        const int z = (int)(i / ((int64_t)nx * ny));
        const int k = axis == 0 ? x : (axis == 1 ? y : z);
        int64_t base, stride;
        if (axis == 0) { base = ((int64_t)z * ny + y) * nx; stride = 1; }
        else if (axis == 1) { base = (int64_t)z * ny * nx + x; stride = nx; }
        else { base = (int64_t)y * nx + x; stride = (int64_t)nx * ny; }
        double acc = in[base];  // j = 0, weight 1
        int m = 0;
        for (int j = 1; j < h; j++) {
            m += k;
            if (m >= Na) m -= Na;
            acc += 2.0 * ct[m] * in[base + j * stride];
        }
        out[i] = acc;
    }
}

__global__ void k_to_f32(const double *__restrict__ in, float *__restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

}  // namespace

lgf_status build_spectrum(const double *d_octant, int K, const int N[3], float *d_Kh, double *d_Kh64,
                          cudaStream_t s)
{
    const int hx = N[0] / 2, hy = N[1] / 2, hz = N[2] / 2;
    if (hx - 1 > K || hy - 1 > K || hz - 1 > K) {
        set_error("table max_offset %d too small for FFT grid (%d,%d,%d): need %d", K, N[0], N[1], N[2],
                  (N[0] > N[1] ? (N[0] > N[2] ? N[0] : N[2]) : (N[1] > N[2] ? N[1] : N[2])) / 2 - 1);
        return LGF_ERR_ARG;
    }
    const int nx = hx + 1, ny = hy + 1, nz = hz + 1;
    const int64_t total = (int64_t)nx * ny * nz;
    double *a = nullptr, *b = nullptr, *ct = nullptr;
    lgf_status st = LGF_OK;
    std::vector<double> hct;
    if (cudaMalloc(&a, total * sizeof(double)) != cudaSuccess || cudaMalloc(&b, total * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ct, (size_t)std::max(N[0], std::max(N[1], N[2])) * sizeof(double)) != cudaSuccess) {
        set_error("spectrum workspace allocation failed (%lld doubles)", (long long)total);
        st = LGF_ERR_OOM;
        goto done;
    }
    {
        const int threads = 256;
        const int blocks = (int)std::min<int64_t>((total + threads - 1) / threads, 152 * 32);
        k_fill<<<blocks, threads, 0, s>>>(d_octant, K, hx, hy, hz, a);
        if (cudaGetLastError() != cudaSuccess) { set_error("k_fill launch failed"); st = LGF_ERR_CUDA; goto done; }
        double *cur = a, *nxt = b;
        for (int axis = 0; axis < 3; axis++) {
            const int Na = N[axis];
            hct.assign(Na, 0.0);
            for (int m = 0; m < Na; m++) hct[m] = std::cos(2.0 * 3.14159265358979323846 * (double)m / (double)Na);
            if (cudaMemcpyAsync(ct, hct.data(), Na * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                set_error("cos table upload failed");
                st = LGF_ERR_CUDA;
                goto done;
            }
            k_cos_axis<<<blocks, threads, 0, s>>>(cur, nxt, nx, ny, nz, axis, Na, ct);
            if (cudaGetLastError() != cudaSuccess) { set_error("k_cos_axis launch failed"); st = LGF_ERR_CUDA; goto done; }
            double *tmp = cur; cur = nxt; nxt = tmp;
        }
        if (d_Kh64 && cudaMemcpyAsync(d_Kh64, cur, total * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            set_error("FP64 spectrum copy failed");
            st = LGF_ERR_CUDA;
            goto done;
        }
        k_to_f32<<<blocks, threads, 0, s>>>(cur, d_Kh, total);
        if (cudaGetLastError() != cudaSuccess) { set_error("k_to_f32 launch failed"); st = LGF_ERR_CUDA; goto done; }
        if (cudaStreamSynchronize(s) != cudaSuccess) { set_error("spectrum build failed on the device"); st = LGF_ERR_CUDA; goto done; }
    }
done:
    cudaFree(a);
    cudaFree(b);
    cudaFree(ct);
    return st;
}

}  // namespace lgf
