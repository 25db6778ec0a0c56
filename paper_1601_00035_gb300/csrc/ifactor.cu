// Integrating factor y = M E_Q(alpha) M x (Sec. 2.3 eq. if_def; Sec. 4.4),
// evaluated in real space as the convolution with the separable kernel
// prod_i g(n_i), g(k) = e^{-2 alpha} I_k(2 alpha) (App. B eq. lgf_intfac),
// truncated to |n_i| <= R (R <= B).  M keeps the block set and zeroes the rest.
//
// One thread block per (block, component); one thread per (x, y) column.
// The kernel marches through the input slices z_in in [-R, B + R): each slice
// of (B + 2R)^2 values is staged in shared memory from the up-to-9 blocks
// that cover it at that height (zeros where no block exists), filtered along
// x, then along y, and the resulting value is scattered into the B outputs
// of the thread's column with the z taps (kept in registers).  HBM traffic is
// one read of every input block (halo reads hit L2) and one write.
#include "plan.hpp"

namespace lgf {
namespace {

template <int B>
__global__ void __launch_bounds__(B *B) k_ifactor(const float *__restrict__ x, float *__restrict__ y,
                                                  const int *__restrict__ nbr, const float *__restrict__ taps,
                                                  int ncomp, int R)
{
    extern __shared__ float sm[];
    const int W = B + 2 * R;
    float *S = sm;                 // [W][W] input slice
    float *T = S + W * W;          // [W][B] after the x pass
    float *g = T + W * B;          // [R + 1] taps
    const int blk = blockIdx.x;
    const int c = blockIdx.y;
    const int tx = threadIdx.x % B, ty = threadIdx.x / B;
    for (int i = threadIdx.x; i <= R; i += blockDim.x) g[i] = taps[i];
    __shared__ int nb[27];
    if (threadIdx.x < 27) nb[threadIdx.x] = nbr[blk * 27 + threadIdx.x];

    float acc[B];
#pragma unroll
    for (int z = 0; z < B; z++) acc[z] = 0.f;
    __syncthreads();

    for (int zin = -R; zin < B + R; zin++) {
        const int dz = zin < 0 ? -1 : (zin >= B ? 1 : 0);
        const int zl = zin - dz * B;
        for (int i = threadIdx.x; i < W * W; i += blockDim.x) {
            const int yy = i / W - R, xx = i % W - R;
            const int dy = yy < 0 ? -1 : (yy >= B ? 1 : 0);
            const int dxb = xx < 0 ? -1 : (xx >= B ? 1 : 0);
            const int n = nb[(dz + 1) * 9 + (dy + 1) * 3 + (dxb + 1)];
            float v = 0.f;
            if (n >= 0) v = __ldg(x + ((size_t)(n * ncomp + c) * B + zl) * B * B + (yy - dy * B) * B + (xx - dxb * B));
            S[i] = v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < W * B; i += blockDim.x) {
            const int yy = i / B, xo = i % B;
            const float *row = S + yy * W + xo + R;
            float s = g[0] * row[0];
            for (int d = 1; d <= R; d++) s = fmaf(g[d], row[d] + row[-d], s);
            T[i] = s;
        }
        __syncthreads();
        {
            const float *col = T + (ty + R) * B + tx;
            float v = g[0] * col[0];
            for (int d = 1; d <= R; d++) v = fmaf(g[d], col[d * B] + col[-d * B], v);
#pragma unroll
            for (int z = 0; z < B; z++) {
                const int d = z - zin;
                const int ad = d < 0 ? -d : d;
                if (ad <= R) acc[z] = fmaf(g[ad], v, acc[z]);
            }
        }
        __syncthreads();
    }
    float *out = y + ((size_t)(blk * ncomp + c) * B) * B * B + ty * B + tx;
#pragma unroll
    for (int z = 0; z < B; z++) out[(size_t)z * B * B] = acc[z];
}

}  // namespace

lgf_status ifactor_launch(int B, int ncomp, int nblk, int R, const int *d_nbr, const float *d_taps, const float *x,
                          float *y, cudaStream_t s)
{
    if (R > B) {
        set_error("integrating-factor radius %d exceeds the block size %d", R, B);
        return LGF_ERR_ARG;
    }
    const int W = B + 2 * R;
    const size_t smem = (size_t)(W * W + W * B + R + 1) * sizeof(float);
    dim3 grid(nblk, ncomp);
    switch (B) {
        case 8:
            k_ifactor<8><<<grid, 64, smem, s>>>(x, y, d_nbr, d_taps, ncomp, R);
            break;
        case 16:
            k_ifactor<16><<<grid, 256, smem, s>>>(x, y, d_nbr, d_taps, ncomp, R);
            break;
        case 32:
            if (smem > 48 * 1024) {
                if (cudaFuncSetAttribute(k_ifactor<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
                    set_error("cannot raise shared memory for B=32");
                    return LGF_ERR_CUDA;
                }
            }
            k_ifactor<32><<<grid, 1024, smem, s>>>(x, y, d_nbr, d_taps, ncomp, R);
            break;
        default:
            set_error("unsupported block size %d", B);
            return LGF_ERR_ARG;
    }
    LGF_LAUNCH_CHECK("ifactor");
    return LGF_OK;
}

}  // namespace lgf
