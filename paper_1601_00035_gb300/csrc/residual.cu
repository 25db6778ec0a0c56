// FP64 residual of a Poisson result (App. A 7-point stencil; Sec. 4.3 residual):
//   num = sum (L u - scale f)^2,  den = sum (scale f)^2
// over target points whose six neighbours are target points, with
// L u = (sum of the six neighbours - 6 u) / dx^2 evaluated in FP64 from the
// FP32 values.  One thread block per target block, one thread per (x, y)
// column marching in z; block reduction, then one double atomicAdd per block.
#include "plan.hpp"

namespace lgf {
namespace {

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void k_residual(const float *__restrict__ u, const float *__restrict__ f, const int *__restrict__ nbr,
                           const int *__restrict__ dst2src, int B, int ncomp, double inv_dx2, double scale,
                           double *__restrict__ acc)
{
    const int blk = blockIdx.x;
    const int c = blockIdx.y;
    const int tx = threadIdx.x % B, ty = threadIdx.x / B;
    const int *nb = nbr + blk * 27;
    const int sblk = dst2src[blk];
    auto at = [&](int x, int y, int z, bool &ok) -> double {
        const int dxb = x < 0 ? -1 : (x >= B ? 1 : 0);
        const int dyb = y < 0 ? -1 : (y >= B ? 1 : 0);
        const int dzb = z < 0 ? -1 : (z >= B ? 1 : 0);
        const int n = nb[(dzb + 1) * 9 + (dyb + 1) * 3 + (dxb + 1)];
        if (n < 0) {
            ok = false;
            return 0.0;
        }
        return (double)u[((size_t)(n * ncomp + c) * B + (z - dzb * B)) * B * B + (y - dyb * B) * B + (x - dxb * B)];
    };
    double num = 0.0, den = 0.0;
    if (threadIdx.x < B * B) {
        for (int z = 0; z < B; z++) {
            bool ok = true;
            const double c0 = at(tx, ty, z, ok);
            const double s = at(tx - 1, ty, z, ok) + at(tx + 1, ty, z, ok) + at(tx, ty - 1, z, ok) +
                             at(tx, ty + 1, z, ok) + at(tx, ty, z - 1, ok) + at(tx, ty, z + 1, ok);
            if (!ok) continue;
            const double fv = sblk >= 0 ? scale * (double)f[((size_t)(sblk * ncomp + c) * B + z) * B * B + ty * B + tx] : 0.0;
            const double r = (s - 6.0 * c0) * inv_dx2 - fv;
            num += r * r;
            den += fv * fv;
        }
    }
    __shared__ double red[2][32];
    num = warp_sum(num);
    den = warp_sum(den);
    const int w = threadIdx.x / 32, ln = threadIdx.x % 32;
    if (ln == 0) {
        red[0][w] = num;
        red[1][w] = den;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) / 32;
        num = ln < nw ? red[0][ln] : 0.0;
        den = ln < nw ? red[1][ln] : 0.0;
        num = warp_sum(num);
        den = warp_sum(den);
        if (ln == 0) {
            atomicAdd(acc, num);
            atomicAdd(acc + 1, den);
        }
    }
}

}  // namespace

lgf_status residual_launch(const PoissonSolve &ps, const float *src, const float *dst, double *d_acc, cudaStream_t s)
{
    const int B = ps.g.B;
    const int threads = B * B < 32 ? 32 : B * B;
    if (threads > 1024) {
        set_error("block size too large for the residual kernel");
        return LGF_ERR_ARG;
    }
    dim3 grid(ps.ndst, ps.g.ncomp);
    k_residual<<<grid, threads, 0, s>>>(dst, src, ps.d_dst_nbr, ps.d_dst2src, B, ps.g.ncomp, 1.0 / (ps.dx * ps.dx),
                                         ps.scale, d_acc);
    LGF_LAUNCH_CHECK("residual");
    return LGF_OK;
}

}  // namespace lgf
