// Shared helpers of liblgf: status/error plumbing, device complex type,
// launch checking.  No numerics of the method live here.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "lgf.h"

namespace lgf {

// Thread-local last-error message (lgf_last_error).
void set_error(const char *fmt, ...);
void clear_error();

#define LGF_CHECK_ARG(cond, ...)                                                              \
    do {                                                                                      \
        if (!(cond)) {                                                                        \
            ::lgf::set_error(__VA_ARGS__);                                                    \
            return LGF_ERR_ARG;                                                               \
        }                                                                                     \
    } while (0)

#define LGF_CUDA_TRY(expr)                                                                    \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            ::lgf::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                             __LINE__);                                                       \
            return e_ == cudaErrorMemoryAllocation ? LGF_ERR_OOM : LGF_ERR_CUDA;              \
        }                                                                                     \
    } while (0)

#define LGF_LAUNCH_CHECK(name)                                                                \
    do {                                                                                      \
        cudaError_t e_ = cudaGetLastError();                                                  \
        if (e_ != cudaSuccess) {                                                              \
            ::lgf::set_error("launch of %s failed: %s", name, cudaGetErrorString(e_));        \
            return LGF_ERR_CUDA;                                                              \
        }                                                                                     \
    } while (0)

#define LGF_TRY(expr)                                                                         \
    do {                                                                                      \
        lgf_status s_ = (expr);                                                               \
        if (s_ != LGF_OK) return s_;                                                          \
    } while (0)

template <typename T>
struct cx {
    T x, y;
};

template <typename T>
__host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b)
{
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> conj(cx<T> a) { return {a.x, -a.y}; }

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Twiddle table w_M^j = exp(-2 pi i j / M), M = 27648 = 2^10 * 27, j < M, computed
// on the host in double precision and uploaded once per device (FP32 and FP64
// copies); every FFT length (2^k <= 1024, 3 * 2^k <= 768, 288, 432) divides M.
// Behind it follow the powers of w_3072 (TW_POW entries), read by every length
// that divides 3072 (all but 288 and 432): a few KB that stay cached across
// thread blocks, and short strides that keep the loads coalesced.
const float2 *twiddle_table_f32();   // device pointer, current device
const double2 *twiddle_table_f64();  // device pointer, current device
lgf_status ensure_twiddles();
constexpr int TW_MAX = 27648;
constexpr int TW_POW = 3072;

// Programmatic dependent launch (sm_90 and later).  A kernel launched by
// launch_pdl may begin while its predecessor on the stream is still draining:
// pdl_wait() blocks until that predecessor has completed and its writes are
// visible, so every read of a predecessor's output and every global write
// comes after it; pdl_trigger() lets the successor begin launching once every
// block of this grid has started.  Without a programmatic dependency both
// return at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// launch_pdl with dynamic shared memory
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                   Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace lgf
