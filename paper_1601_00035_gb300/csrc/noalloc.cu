// ifactor_apply_noalloc: the integrating factor for callers that cannot
// allocate device memory (for example code running under a device-memory
// budget owned by someone else, or a framework that forbids cudaMalloc
// after start-up).  It does the same three passes as ifactor_apply but keeps
// the neighbour tables and both intermediate fields in one file-scope device
// array of fixed size, reached through cudaGetSymbolAddress, and it uses no
// host heap either (fixed host staging arrays below).
//
// Limits: the dilated block lists and the intermediates must fit in
// LGF_NOALLOC_SCRATCH_BYTES (64 MiB), and the block set's bounding box grown
// by one block per side must have at most LGF_NOALLOC_MAX_BBOX cells.
// Every call shares the array (and the host staging): calls that overlap on
// the GPU, or run concurrently from several host threads, race.  Each call
// rewrites everything it reads, so nothing needs clearing between calls.
// The first call on a device resolves the array's device address there.  No
// call may be made while its stream is being captured: each call copies its
// tables from static host staging that the next call overwrites, so a
// captured copy would replay stale tables (checked: LGF_ERR_ARG).
#include <cmath>
#include <cstring>

#include "plan.hpp"

namespace lgf {
namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;
constexpr int kMaxBBox = 1 << 21;   // cells of the dilated bounding box (block units)
constexpr int kMaxBlocks = 1 << 16; // blocks in any of the three lists
constexpr int kMaxTaps = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// per-device address of g_scratch (resolved once per device)
static void *g_scratch_addr[64] = {nullptr};

// host staging (no heap): dense membership LUT and the three neighbour tables
static int32_t g_lut_S[kMaxBBox], g_lut_1[kMaxBBox], g_lut_2[kMaxBBox];
static int32_t g_nb[3 * 3 * kMaxBlocks];

}  // namespace

// e^{-x} I_n(x), n = 0..nmax, by Miller's backward recurrence normalised with
// e^{-x} (I_0 + 2 sum_{n>=1} I_n) = 1 (host copy for the taps).
void host_scaled_bessel(double x, int nmax, double *out)
{
    for (int n = 0; n <= nmax; n++) out[n] = 0.0;
    if (x <= 0.0) {
        out[0] = 1.0;
        return;
    }
    const int top = nmax + 32 + (int)(12.0 * std::sqrt(x));
    double hi = 0.0, cur = 1e-300, norm = 0.0;
    for (int n = top; n >= 1; n--) {
        if (n <= nmax) out[n] = cur;
        norm += 2.0 * cur;
        const double lo = hi + (2.0 * n / x) * cur;
        hi = cur;
        cur = lo;
        if (cur > 1e240) {
            hi *= 1e-240;
            cur *= 1e-240;
            norm *= 1e-240;
            for (int m = (n - 1 < nmax ? n - 1 : nmax); m <= nmax; m++) out[m] *= 1e-240;
        }
    }
    norm += cur;
    out[0] = cur;
    for (int n = 0; n <= nmax; n++) out[n] /= norm;
}

namespace {

lgf_status scratch_base(unsigned char **base)
{
    int dev = -1;
    LGF_CUDA_TRY(cudaGetDevice(&dev));
    LGF_CHECK_ARG(dev >= 0 && dev < 64, "ifactor_apply_noalloc: device index %d out of range", dev);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            set_error("ifactor_apply_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return LGF_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *base = (unsigned char *)g_scratch_addr[dev];
    return LGF_OK;
}

inline size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace
}  // namespace lgf

using namespace lgf;

extern "C" lgf_status ifactor_apply_noalloc(double alpha, int B, int ncomp, int n_blocks, const int32_t *blocks,
                                            const float *x, float *y, void *stream)
{
    clear_error();
    LGF_CHECK_ARG(blocks && x && y && x != y, "ifactor_apply_noalloc: NULL or aliasing buffer");
    LGF_CHECK_ARG(B == 8 || B == 16, "ifactor_apply_noalloc: B=%d not in {8,16}", B);
    LGF_CHECK_ARG(ncomp >= 1 && ncomp <= 3, "ifactor_apply_noalloc: ncomp=%d not in 1..3", ncomp);
    LGF_CHECK_ARG(n_blocks >= 1 && n_blocks <= kMaxBlocks / 27, "ifactor_apply_noalloc: n_blocks=%d not in [1, %d]",
                  n_blocks, kMaxBlocks / 27);
    LGF_CHECK_ARG(alpha > 0.0 && alpha <= 50.0, "ifactor_apply_noalloc: alpha %g outside (0, 50]", alpha);

    // taps g(k) = e^{-2 alpha} I_k(2 alpha), radius from the 1e-14 rule
    double gd[kMaxTaps + 1];
    host_scaled_bessel(2.0 * alpha, kMaxTaps, gd);
    int R = 0;
    while (R + 1 <= kMaxTaps && gd[R + 1] * gd[0] * gd[0] >= 1e-14) R++;
    LGF_CHECK_ARG(R <= B && R <= 16, "ifactor_apply_noalloc: radius %d exceeds min(B=%d, 16)", R, B);
    float gf[kMaxTaps + 1];
    for (int i = 0; i <= kMaxTaps; i++) gf[i] = (float)gd[i];

    // bounding box grown by one block per side
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = blocks[a];
        hi[a] = blocks[a];
    }
    for (int i = 0; i < n_blocks; i++)
        for (int a = 0; a < 3; a++) {
            LGF_CHECK_ARG(blocks[3 * i + a] > -(1 << 20) && blocks[3 * i + a] < (1 << 20),
                          "ifactor_apply_noalloc: block coordinate out of range");
            lo[a] = blocks[3 * i + a] < lo[a] ? blocks[3 * i + a] : lo[a];
            hi[a] = blocks[3 * i + a] > hi[a] ? blocks[3 * i + a] : hi[a];
        }
    const long dx = hi[0] - lo[0] + 3, dy = hi[1] - lo[1] + 3, dz = hi[2] - lo[2] + 3;
    // each extent is bounded first, so that the product below cannot overflow
    LGF_CHECK_ARG(dx <= kMaxBBox && dy <= kMaxBBox && dz <= kMaxBBox,
                  "ifactor_apply_noalloc: bounding box extent (%ld, %ld, %ld) exceeds %d blocks", dx, dy, dz, kMaxBBox);
    LGF_CHECK_ARG(dx * dy <= kMaxBBox && dx * dy * dz <= kMaxBBox,
                  "ifactor_apply_noalloc: bounding box of %ld cells exceeds %d", dx * dy * dz, kMaxBBox);
    const long ncell = dx * dy * dz;
    auto cell = [&](int bx, int by, int bz) -> long {
        return ((long)(bz - lo[2] + 1) * dy + (by - lo[1] + 1)) * dx + (bx - lo[0] + 1);
    };
    for (long i = 0; i < ncell; i++) g_lut_S[i] = g_lut_1[i] = g_lut_2[i] = -1;
    for (int i = 0; i < n_blocks; i++) {
        const long c = cell(blocks[3 * i], blocks[3 * i + 1], blocks[3 * i + 2]);
        LGF_CHECK_ARG(g_lut_S[c] < 0, "ifactor_apply_noalloc: duplicate block");
        g_lut_S[c] = i;
    }
    // L1 = (S + {dx,dy}) n (S + {dz}),  L2 = (S + {dx}) n (S + {dy,dz}); mark candidates with -2
    auto inS = [&](long bx, long by, long bz) -> bool {
        if (bx < lo[0] || bx > hi[0] || by < lo[1] || by > hi[1] || bz < lo[2] || bz > hi[2]) return false;
        return g_lut_S[cell((int)bx, (int)by, (int)bz)] >= 0;
    };
    int n1 = 0, n2 = 0;
    // deterministic order: scan the grown box in (z, y, x) order
    for (int bz = lo[2] - 1; bz <= hi[2] + 1; bz++)
        for (int by = lo[1] - 1; by <= hi[1] + 1; by++)
            for (int bx = lo[0] - 1; bx <= hi[0] + 1; bx++) {
                bool a1 = false, z1 = false, a2 = false, yz = false;
                for (int a = -1; a <= 1 && !(a1 && z1 && a2 && yz); a++) {
                    z1 = z1 || inS(bx, by, bz - a);
                    a2 = a2 || inS(bx - a, by, bz);
                    for (int b = -1; b <= 1; b++) {
                        a1 = a1 || inS(bx - a, by - b, bz);
                        yz = yz || inS(bx, by - a, bz - b);
                    }
                }
                const long c = cell(bx, by, bz);
                if (a1 && z1) g_lut_1[c] = n1++;
                if (a2 && yz) g_lut_2[c] = n2++;
            }
    LGF_CHECK_ARG(n1 <= kMaxBlocks / 3 && n2 <= kMaxBlocks / 3, "ifactor_apply_noalloc: too many blocks");
    // neighbour tables: nbz over L1 -> S, nby over L2 -> L1, nbx over S -> L2
    int32_t *nbz = g_nb, *nby = g_nb + 3 * n1, *nbx = g_nb + 3 * (n1 + n2);
    auto get = [&](const int32_t *lut, long bx, long by, long bz) -> int32_t {
        if (bx < lo[0] - 1 || bx > hi[0] + 1 || by < lo[1] - 1 || by > hi[1] + 1 || bz < lo[2] - 1 || bz > hi[2] + 1)
            return -1;
        return lut[cell((int)bx, (int)by, (int)bz)];
    };
    for (int bz = lo[2] - 1; bz <= hi[2] + 1; bz++)
        for (int by = lo[1] - 1; by <= hi[1] + 1; by++)
            for (int bx = lo[0] - 1; bx <= hi[0] + 1; bx++) {
                const long c = cell(bx, by, bz);
                if (g_lut_1[c] >= 0)
                    for (int a = -1; a <= 1; a++) nbz[3 * g_lut_1[c] + a + 1] = get(g_lut_S, bx, by, bz + a);
                if (g_lut_2[c] >= 0)
                    for (int a = -1; a <= 1; a++) nby[3 * g_lut_2[c] + a + 1] = get(g_lut_1, bx, by + a, bz);
            }
    for (int i = 0; i < n_blocks; i++)
        for (int a = -1; a <= 1; a++)
            nbx[3 * i + a + 1] = get(g_lut_2, blocks[3 * i] + a, blocks[3 * i + 1], blocks[3 * i + 2]);

    // scratch layout: [tables][y1][y2], 256-byte aligned pieces
    const size_t B3 = (size_t)B * B * B;
    const size_t tab_bytes = up256(sizeof(int32_t) * 3 * (size_t)(n1 + n2 + n_blocks));
    const size_t y1_bytes = up256(sizeof(float) * (size_t)n1 * ncomp * B3);
    const size_t y2_bytes = up256(sizeof(float) * (size_t)n2 * ncomp * B3);
    LGF_CHECK_ARG(tab_bytes + y1_bytes + y2_bytes <= kScratchBytes,
                  "ifactor_apply_noalloc: needs %zu bytes of scratch, the static limit is %zu",
                  tab_bytes + y1_bytes + y2_bytes, kScratchBytes);
    cudaStream_t s = (cudaStream_t)stream;
    {
        // the tables are copied from static host staging that the next call overwrites, so a
        // captured call would replay stale tables: refuse capture outright
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        LGF_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
        LGF_CHECK_ARG(cap == cudaStreamCaptureStatusNone,
                      "ifactor_apply_noalloc: must not be called while the stream is being captured");
    }
    unsigned char *base = nullptr;
    LGF_TRY(scratch_base(&base));
    LGF_CUDA_TRY(cudaMemcpyAsync(base, g_nb, sizeof(int32_t) * 3 * (size_t)(n1 + n2 + n_blocks),
                                 cudaMemcpyHostToDevice, s));
    IfPlan ip;
    ip.B = B;
    ip.R = R;
    ip.n0 = n_blocks;
    ip.n1 = n1;
    ip.n2 = n2;
    ip.nbz = (int *)base;
    ip.nby = (int *)base + 3 * n1;
    ip.nbx = (int *)base + 3 * (n1 + n2);
    ip.y1 = (float *)(base + tab_bytes);
    ip.y2 = (float *)(base + tab_bytes + y1_bytes);
    return ifactor_launch(ip, ncomp, gf, x, y, s, nullptr);
}
