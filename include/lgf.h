/*
 * lgf.h -- C-ABI of liblgf.so, a GB300 (sm_103a) implementation of the
 * lattice-Green's-function (LGF) convolutions of Liska & Colonius,
 * "A fast lattice Green's function method for solving viscous incompressible
 * flows on unbounded domains".
 *
 * Two operations are provided, each the convolution of block-structured,
 * compactly supported sources with a lattice Green's function:
 *
 *   Poisson   u(n) = scale * dx^2 * sum_m G(n - m) f(m)             (Sec. 2.2,
 *             eq. dpoisson_conv), G the unit-lattice LGF of the 7-point
 *             Laplacian (App. B, Bessel form), i.e. u = scale * L^{-1} f with
 *             L = L_unit / dx^2 and zero values at infinity.  Vector problems
 *             are solved per component (Sec. 2.2).
 *   IF        y = M E_Q(alpha) M x                                 (Sec. 2.3
 *             eq. if_def, App. B eq. lgf_intfac, Sec. 4.4): convolution with
 *             the kernel prod_i exp(-2 alpha) I_{n_i}(2 alpha), truncated to the
 *             box |n_i| <= R_alpha outside which the 3-D kernel is < 1e-14;
 *             M is the mask of the block set (zero outside it).
 *
 * Data layout (all user buffers are caller-owned):
 *   A block is B^3 cells at block coordinate (bx, by, bz) covering cells
 *   [bx*B, bx*B + B) x [by*B, ...) x [bz*B, ...).  A field over a block list
 *   is FP32, block-contiguous: index ((blk * ncomp + c) * B + z) * B * B + y * B + x,
 *   i.e. [nblk][ncomp][B][B][B] with x fastest.  Block coordinates are int32
 *   triples (bx, by, bz), [n][3], host memory, copied at plan time; the lists
 *   must not contain duplicates.
 *
 * Conventions: every call returns an lgf_status; no call aborts, throws or
 * exits.  On a non-OK status, lgf_last_error() returns a thread-local message.
 * Library objects (tables, plans) are library-owned; destroy functions accept
 * NULL.  A plan is not thread-safe; distinct plans are.  Streams are passed
 * as `void *` holding a cudaStream_t (NULL = legacy default stream).
 * Execute calls are asynchronous on the given stream, allocate nothing and
 * synchronise nothing (so they may be captured in a CUDA graph), except where
 * stated otherwise.  The library runs on the device that is current at
 * plan/table creation; later calls must be made with that device current.
 */
#ifndef LGF_H
#define LGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LGF_OK = 0,
    LGF_ERR_ARG = -1,     /* invalid argument (NULL pointer, bad size, unsupported shape) */
    LGF_ERR_OOM = -2,     /* device or host allocation failed */
    LGF_ERR_CUDA = -3,    /* a CUDA runtime call or kernel launch failed */
    LGF_ERR_TIMEOUT = -4, /* a bounded device-side wait gave up */
    LGF_ERR_TOL = -5,     /* requested tolerance not reachable with the given options */
    LGF_ERR_STATE = -6    /* object used in the wrong state (e.g. wrong kind of table) */
} lgf_status;

typedef enum {
    LGF_KERNEL_LAPLACE7 = 0, /* G_L: LGF of the 7-point Laplacian (App. B) */
    LGF_KERNEL_IFACTOR = 1   /* G_E(alpha): integrating-factor kernel (App. B eq. lgf_intfac) */
} lgf_kernel;

typedef struct lgf_table lgf_table; /* opaque: device FP64 kernel values */
typedef struct lgf_plan lgf_plan;   /* opaque: block lookups, spectra, workspaces */

/* One independent problem.  For a Poisson plan: sources live on src_blocks
 * (D_supp of Sec. 4.2), results are produced on dst_blocks (D_xsoln).  For an
 * IF plan: src_blocks is the block set of the mask, dst_blocks/n_dst are
 * ignored (output on the same set). */
typedef struct {
    int B;                      /* block edge in cells: 8, 16 or 32 */
    int ncomp;                  /* components per point, 1..3 (solved independently) */
    int n_src;                  /* number of source blocks (>= 1) */
    int n_dst;                  /* number of target blocks (>= 1; Poisson only) */
    const int32_t *src_blocks;  /* [n_src][3] block coordinates (host) */
    const int32_t *dst_blocks;  /* [n_dst][3] block coordinates (host) */
    double dx;                  /* grid spacing; the Poisson kernel is dx^2 * G */
    double scale;               /* result multiplier, e.g. -1 for a = -L^{-1} w (eq. vel_refresh) */
} lgf_solve_desc;

typedef struct {
    int use_graph;      /* 1: lgf_conv_execute captures its launch sequence in a CUDA graph on first
                           use per set of buffers (FP32 plans; FP64 plans launch directly) */
    int precision;      /* 0: FP32 data and transforms (lgf_conv_execute);
                           1: FP64 data and transforms, FP64 spectrum (lgf_conv_execute_f64 only;
                              FFT lengths up to 512; method 0 only) */
    int method;         /* 0: whole-box zero-padded FFT convolution (exact up to rounding);
                           1: block-sparse split solve (Sec. 2.2 "to tolerance eps"): the LGF
                              split as G = G_near + G_far at split time a of its Bessel form,
                              G_near convolved block pair by block pair (16^3 blocks, offsets
                              up to 2 blocks), G_far on the coarse lattice of spacing 2 through
                              10-point Lagrange interpolation and anterpolation, the coarse sum
                              by a whole-box convolution or, where that box is large (a 512^3 FFT
                              grid or more, or beyond 1024-point FFTs), by the next split level
                              (near t in [a, 4a], far on the spacing-4 lattice); one solve, B = 16;
                              cost follows the active blocks; relative L2 error ~1e-7..1e-6;
                           2: autotune: plan both and keep the faster (one timed execution each) */
    int far_precision;  /* method 1: 0 = far-field interpolation and anterpolation in FP32 on the
                           CUDA cores (the solve held to 1e-6 relative L2);
                           1 = the same as GEMMs on the tensor cores (tcgen05 kind::tf32 MMAs,
                           operands split into two TF32 parts, FP32 accumulation: the
                           reduced-precision far field, held to 1e-5) */
    double split_alpha; /* method 1: the split time a in [1, 64]; 0 takes 20, which keeps G_near
                           within two blocks and the spacing-2 far field within 1e-6 */
    int near_form;      /* method 1: the near-field multiply-accumulate: 0 = time the forms at
                           plan time and keep the fastest; 1 = one target per warp over its
                           (offset, source) pairs; 2 = runs of 4 x-adjacent targets per warp
                           (13 row loads per 20 multiply-adds, dense over each run); 3 = quads
                           of 4 x 2 targets per warp (a source row serves two rows of targets:
                           up to 18 row loads per 40 multiply-adds; needs all 125 near offsets,
                           else the run form) */
    int reserved[1];    /* must be zero */
} lgf_plan_opts;

/* ---------------------------------------------------------------------------
 * Tables.
 *
 * LGF_KERNEL_LAPLACE7: tabulates the unit-lattice LGF on the sorted octant
 *   max_offset >= a >= b >= c >= 0 from its Bessel form (App. B)
 *     G(a,b,c) = -int_0^inf e^{-6t} I_a(2t) I_b(2t) I_c(2t) dt
 *   in FP64 on the device (Gauss-Legendre in log t plus the closed-form
 *   large-t tail).  max_offset must cover every offset a plan will sample:
 *   lgf_conv_plan reports LGF_ERR_ARG with the required value otherwise.
 *   alpha is ignored.  1 <= max_offset <= 1024.
 * LGF_KERNEL_IFACTOR: tabulates g(k) = exp(-2 alpha) I_k(2 alpha), k = 0..R,
 *   R = largest k with g(k) g(0)^2 >= 1e-14 (App. B eq. lgf_intfac; the
 *   Bessel argument is 2 alpha as fixed by the decay values of the Sec. 2.3
 *   footnote).  0 < alpha <= 50; max_offset is ignored.
 * Synchronises `stream` before returning.  *out receives a new table.
 * ------------------------------------------------------------------------- */
lgf_status lgf_table_build(lgf_kernel kind, double alpha, int max_offset, void *stream, lgf_table **out);

/* kind, alpha, max_offset (Laplace) and radius R (IF; 0 for Laplace). Any out pointer may be NULL. */
lgf_status lgf_table_info(const lgf_table *t, int *kind, double *alpha, int *max_offset, int *radius);

/* Copy the FP64 table to host memory: the octant entries in the order
 * index(a,b,c) = a(a+1)(a+2)/6 + b(b+1)/2 + c (Laplace), or g(0..R) (IF).
 * n = number of doubles available at host_out; LGF_ERR_ARG if too small.
 * Synchronous. */
lgf_status lgf_table_copy(const lgf_table *t, double *host_out, int64_t n);
int64_t lgf_table_size(const lgf_table *t);

void lgf_table_destroy(lgf_table *t);

/* ---------------------------------------------------------------------------
 * Plans.  lgf_conv_plan analyses n_solves independent problems, uploads the
 * block lookups, builds (Poisson) the real, even spectrum of the LGF on the
 * zero-padded FFT grid of each distinct grid size (Hockney's free-space
 * embedding of eq. dpoisson_conv: exact up to FP32 rounding, no far-field
 * approximation), and allocates every workspace.  Per axis the FFT length is
 * the smallest of 16, 32, 64, 96, 128, 192, 256, 288, 384, 432, 512, 768, 1024 that is
 * >= max(2 m + 2, 2 E), m the largest |target - source| offset and E the
 * source extent (points); at most 1024 (FP32) or 512 (FP64), else
 * LGF_ERR_ARG.  The table must outlive the
 * plan.  Synchronises `stream`.  opts may be NULL (defaults).
 * ------------------------------------------------------------------------- */
lgf_status lgf_conv_plan(const lgf_table *t, const lgf_solve_desc *solves, int n_solves,
                         const lgf_plan_opts *opts, void *stream, lgf_plan **out);

/* The method a Poisson plan executes (0 whole box, 1 block-sparse split; -1 for NULL).  For
 * an autotuned plan (opts->method = 2), *ms_whole_box and *ms_split receive the device times
 * of the two candidates measured at plan time (-1 where not timed); either pointer may be NULL. */
int lgf_plan_method(const lgf_plan *p, double *ms_whole_box, double *ms_split);

/* Synchronises `stream` and reports LGF_ERR_TIMEOUT if a bounded device-side wait of the
 * plan's kernels gave up since the last check (the flag is then cleared; the results of
 * the executions since then are not valid), LGF_OK otherwise.  Only the block-sparse
 * method waits on the device (its window-spectrum staging by bulk copy and its tensor-core
 * completions); lgf_conv_execute_host checks on its own. */
lgf_status lgf_plan_check(lgf_plan *p, void *stream);

/* Failure detection of the bounded device waits (the paper has no counterpart): runs the
 * wait the tensor-core kernels use on an mbarrier that nothing arrives on, for `polls` polls
 * (1..2^20), and returns LGF_ERR_TIMEOUT when it gives up, as a kernel whose dependency never
 * completes reports through lgf_plan_check.  Nothing faults or hangs; the context stays usable.
 * Allocates 4 bytes of device memory; synchronises `stream`. */
lgf_status lgf_wait_probe(int polls, void *stream);

/* Device bytes held by the plan (workspaces + spectra + lookups). */
lgf_status lgf_plan_workspace_bytes(const lgf_plan *p, size_t *bytes);

/* Poisson: for every solve i, dst[i] (device, [n_dst][ncomp][B^3] FP32,
 * overwritten on every target point) = scale * dx^2 * G * src[i] (device,
 * [n_src][ncomp][B^3] FP32).  Asynchronous on `stream`; no allocation.  A
 * plan with more than one (solve, component) unit runs the units on its own
 * worker streams, forked from and joined back to `stream` with events; with
 * opts->use_graph the whole sequence is captured once per set of buffers
 * and replayed.  dst[i] may be the buffer src[i] for a solve with ncomp = 1
 * (every source value is read before the first result is written; the
 * IF-HERK projection solves in place this way), and for a split plan; the
 * buffers of different solves must not overlap. */
lgf_status lgf_conv_execute(lgf_plan *p, const float *const *src, float *const *dst, void *stream);

/* FP64 variant for plans built with opts->precision = 1: src[i], dst[i] are
 * device FP64 arrays with the same layout.  Asynchronous; no allocation. */
lgf_status lgf_conv_execute_f64(lgf_plan *p, const double *const *src, double *const *dst, void *stream);

/* Same as lgf_conv_execute with HOST buffers: copies every src[i] to
 * plan-owned device staging, executes, copies the results to dst[i] and
 * synchronises `stream` before returning.  Each unit copies its own
 * component slice in and out on its worker stream, so copies overlap the
 * other units' passes.  Host buffers should be pinned for full copy
 * bandwidth.  With opts->use_graph and every buffer page-locked, the copies
 * and passes are captured once per set of host pointers and replayed as one
 * graph (pageable buffers take the launch-by-launch path). */
lgf_status lgf_conv_execute_host(lgf_plan *p, const float *const *src, float *const *dst, void *stream);

/* IF plan (table of kind LGF_KERNEL_IFACTOR, one solve): y = M E_Q(alpha) M x
 * on the block set, x and y device [n_src][ncomp][B^3] FP32 (must not alias).
 * Requires R_alpha <= B.  Asynchronous; no allocation. */
lgf_status ifactor_apply(lgf_plan *p, const float *x, float *y, void *stream);

/* No-allocation variant of ifactor_apply, for callers that cannot allocate
 * device memory: code that runs under a memory budget owned by another
 * component, or inside frameworks that forbid cudaMalloc once they are
 * running.  The paper has no counterpart; it is a deployment convenience.
 * Computes the same y = M E_Q(alpha) M x as an IF plan built from
 * lgf_table_build(LGF_KERNEL_IFACTOR, alpha) over `blocks` ([n_blocks][3]
 * host int32 coordinates), with x, y device [n_blocks][ncomp][B^3] FP32.
 * Nothing is allocated: the block tables and intermediate fields live in one
 * static device array of 64 MiB that every GPU loading the library holds
 * until exit; LGF_ERR_ARG if a problem needs more (or if the block set's
 * bounding box, grown by one block per side, exceeds 2^21 blocks).  Host
 * staging is static too.  Every call shares that storage and keeps the last
 * call's contents (each call overwrites all it reads), so calls that overlap
 * on the GPU, or that run concurrently from several host threads, race.
 * The first call on a device looks up the array's device address.  The call
 * must not be made while `stream` is being captured into a CUDA graph (it
 * copies its tables from static host staging that the next call overwrites):
 * it returns LGF_ERR_ARG if it is.  B in {8, 16}; radius R_alpha <= min(B, 16).
 * Asynchronous on `stream` except for a host-to-device copy of the tables
 * from pageable memory. */
lgf_status ifactor_apply_noalloc(double alpha, int B, int ncomp, int n_blocks, const int32_t *blocks,
                                 const float *x, float *y, void *stream);

/* FP64 residual of a Poisson result (App. A stencil, Sec. 4.3 definition):
 *   ||L u - scale f||_2 / ||scale f||_2
 * over target points whose six neighbours are target points (L = 7-point
 * Laplacian / dx^2).  src/dst as for lgf_conv_execute, solve = index.
 * Synchronises `stream`. */
lgf_status lgf_residual_fp64(lgf_plan *p, int solve, const float *src, const float *dst,
                             double *rel_residual, void *stream);

/* Diagnostics.  While profiling is enabled on a plan, every kernel launch made
 * by lgf_conv_execute / lgf_conv_execute_host / ifactor_apply is bracketed by
 * a pair of CUDA events recorded on the launching stream, and its device time
 * and launch count are accumulated per kernel name (graph capture is bypassed
 * while enabled).  enable = 0 stops recording; 2 also clears the totals. */
lgf_status lgf_plan_set_profiling(lgf_plan *p, int enable);
/* Number of kernel names with accumulated times (waits for pending events). */
lgf_status lgf_plan_kernel_count(lgf_plan *p, int *count);
/* Totals of kernel i (0 <= i < count): name (library-owned string, valid
 * until the plan is destroyed), launches and summed device milliseconds. */
lgf_status lgf_plan_kernel_times(lgf_plan *p, int i, const char **name, long long *launches, double *total_ms);

/* Measured arithmetic rate of the current GPU, the compute roofline of the FFT,
 * spectral-multiply and integrating-factor passes (the paper has no counterpart:
 * a measurement helper).  kind 0: FP32 fused multiply-add (2 flops each);
 * 1: paired FP32 fused multiply-add, fma.rn.f32x2 (4 flops each); 2: FP64 fused
 * multiply-add (2 flops each).  Eight independent register-resident FMA chains
 * per thread on 8 x 256-thread blocks per SM run for about `ms` milliseconds
 * (0 < ms <= 10000), timed with CUDA events on `stream`; *tflops receives the
 * rate in TFLOP/s.  Allocates a small device buffer; synchronises `stream`. */
lgf_status lgf_measure_peak(int kind, double ms, double *tflops, void *stream);

/* ---------------------------------------------------------------------------
 * One time step of the IF-HERK scheme on a finite block set (Sec. 3.2
 * algorithm, Sec. 3.3 eq. proj_final, Sec. 5 xIF-HERK masks), Scheme A of
 * eq. ifherk_schemes.  D_soln = D_supp = soln_blocks (Sec. 6); D_xsoln is
 * D_soln dilated by N_b = 1 block (eq. def_xsoln).  Fields live on D_xsoln in
 * the order returned by lgf_rk_blocks(p, 0, ...) (the soln blocks first):
 * face velocity u is [n_xsoln][3][B^3] FP32 (component q is the x_q-face value).
 * ------------------------------------------------------------------------- */
typedef struct {
    int B;                       /* 8 or 16 */
    int n_soln;                  /* number of D_soln (= D_supp) blocks */
    const int32_t *soln_blocks;  /* [n_soln][3] block coordinates (host) */
    double dx, dt, re;           /* grid spacing, time step, Reynolds number: alpha = dt / (dx^2 re) */
    int scheme;                  /* tableau of eq. ifherk_schemes: 0 = Scheme A, 1 = Scheme B, 2 = Scheme C */
    int use_graph;               /* 1: lgf_rk_step captures its launch sequence in a CUDA graph on first
                                    use for a given (u_in, u_out, u_inf) and replays it (two cached) */
    int poisson_method;          /* the Poisson solves D_supp -> D_xsoln: 0 = the whole-box FFT
                                    convolution where its FFT lengths (<= 1024) reach, else the
                                    block-sparse split solve (B = 16; boxes beyond 1024 cells, e.g. the
                                    thin ring of Sec. 6); 1 = whole box; 2 = split */
    int reserved[1];             /* must be zero */
} lgf_rk_desc;

/* Builds the LGF table, a scalar Poisson plan D_supp -> D_xsoln, the
 * integrating-factor plans H^i = E((c~_i - c~_{i-1}) alpha) on D_xsoln of the
 * scheme's shifted nodes (Sec. 3.2; c~_0 = c_1: A: E(a/2), E(a/2), I;
 * B: E(a/3), E(2a/3), I; C: E(8a/15), E(2a/15), E(a/3)), and all workspaces.
 * LGF_ERR_ARG if an integrating-factor radius exceeds min(B, 16), or if the whole box
 * is asked for (or, with B = 8, needed) beyond its FFT lengths.
 * Synchronises `stream`.  The result is used only with the lgf_rk_* and
 * lgf_op_apply calls (and destroyed with lgf_plan_destroy). */
lgf_status lgf_rk_plan(const lgf_rk_desc *d, void *stream, lgf_plan **out);
/* Number of blocks of D_xsoln (which = 0) or D_soln (which = 1); -1 if p is not an RK plan. */
int lgf_rk_block_count(const lgf_plan *p, int which);
/* Copy the block coordinates of D_xsoln (which = 0) or D_soln (which = 1) to coords ([n][3], host). */
lgf_status lgf_rk_blocks(const lgf_plan *p, int which, int32_t *coords, int n);
/* u_out = IF-HERK(u_in) over one step, freestream uinf (host, 3 doubles, constant over the step);
 * u_in and u_out device buffers [n_xsoln][3][B^3], must not alias.  Three scalar Poisson solves,
 * five integrating-factor applications (six for Scheme C, whose H^3 is not the identity), three
 * nonlinear terms.  Asynchronous; no allocation. */
lgf_status lgf_rk_step(lgf_plan *p, const float *u_in, float *u_out, const double uinf[3], void *stream);
/* One step of the vorticity formulation of Sec. 4.1 (the discrete curl of eq. dnstp,
 * dw/dt = L w / Re - C N~(u + u_inf) with u = -C^T L^{-1} w, eq. vel_vor), integrated with the
 * plan's IF-HERK tableau and integrating factors (Sec. 3.2; no constraint, so no projection).
 * w_in, w_out: edge vorticity on D_xsoln, device [n_xsoln][3][B^3] (component q is the x_q-edge
 * value), must not alias.  Each stage solves a VECTOR Poisson problem D_supp -> D_xsoln for the
 * velocity (the cost the paper cites for not pursuing this form) and applies
 * g^i = -a~_ii dt M^soln C M^soln N~(M^xsoln (u + u_inf)).  Algebraically the curl of lgf_rk_step.
 * Asynchronous; no allocation. */
lgf_status lgf_rk_step_vorticity(lgf_plan *p, const float *w_in, float *w_out, const double uinf[3], void *stream);
/* Velocity refresh of Sec. 5 (eq. vel_refresh): u_out = M^xsoln C^T M^xsoln a with
 * a = -M^xsoln L^{-1} M^supp w and w = M^xsoln C M^xsoln u_in (a vector Poisson solve
 * D_supp -> D_xsoln).  u_in, u_out device [n_xsoln][3][B^3]; u_out may equal u_in.
 * Asynchronous; no allocation. */
lgf_status lgf_rk_refresh(lgf_plan *p, const float *u_in, float *u_out, void *stream);
/* Largest number of steps q over which the composed integrating factors E(q alpha) keep the
 * error the D_xsoln mask causes at depth B (one buffer block) below eps relative to max |u|
 * (App. D, with the truncation error read as the kernel mass beyond that depth); 0 if not
 * even one step does; -1 (lgf_last_error set) for a bad argument.  Host only. */
int lgf_rk_qmax(const lgf_plan *p, double eps);
/* Grid update query of Sec. 5 (eq. d_supp with the weight function eq. weight_fun): from
 * w = M C M u and q = -M G^T M N~(M (u + uinf)) on D_xsoln, with the cells within 3 cells
 * of the outside of D_xsoln zeroed (the mask edge's contaminated layer), the blocks with
 * W = max(max|w| / max_global|w|, max|q| / max_global|q|) > eps_supp.  Writes up to `capacity`
 * block coordinates ([n][3], host) in D_xsoln order and returns their count (which may exceed
 * capacity); -1 on a bad argument.  Synchronises `stream`. */
int lgf_rk_regrid_blocks(lgf_plan *p, const float *u, const double uinf[3], double eps_supp, int32_t *blocks_out,
                         int capacity, void *stream);
/* Vorticity copy and velocity refresh onto a new grid (Sec. 5 grid update): w = C u_from on
 * `from`'s D_xsoln, zeroed within 3 cells of its outside (the mask edge's spurious vortex
 * sheet), copied to the D_supp blocks of `to` (every one of which must lie in
 * `from`'s D_xsoln, else LGF_ERR_ARG), then u_to = Vor2Vel(w) on `to`'s D_xsoln
 * (eq. vel_refresh).  Same B and dx.  Synchronises `stream`. */
lgf_status lgf_rk_transfer(lgf_plan *from, const float *u_from, lgf_plan *to, float *u_to, void *stream);
/* Ring diagnostics of Sec. 6 (eq. int_quantities) of the velocity perturbation u (device
 * [n_xsoln][3][B^3]) over D_soln, with w = C u on edges: out[0..2] impulse I = 1/2 sum x cross w,
 * out[3] K = sum u . (x cross w), out[4] enstrophy E = 1/2 sum |w|^2, out[5] helicity
 * J = sum u . w, out[6..8] centroid X = 1/2 sum ((x cross w) . I / |I|^2) x without the
 * freestream term (its component along I is the ring position); all times dx^3, positions
 * in the lattice's absolute coordinates (block coordinate times B, times dx).  I, E and X sum
 * over edges, each component at its own edge (n - e_q / 2); K and J pair u and w at cell
 * centres (n - (1,1,1)/2), averaging the 2 faces / 4 edges around the cell.  FP64 sums;
 * synchronises `stream` (out is host memory). */
lgf_status lgf_rk_diagnostics(lgf_plan *p, const float *u, double out[9], void *stream);
/* nsteps IF-HERK steps u_in -> u_out with a velocity refresh before every step k > 0 with
 * k % qmax == 0 (qmax = 0: never); u_in is not modified; u_in and u_out must not alias.
 * Asynchronous; no allocation. */
lgf_status lgf_rk_run(lgf_plan *p, const float *u_in, float *u_out, int nsteps, const double uinf[3], int qmax,
                      void *stream);
/* One App. A operator on the D_xsoln block set (zero outside it):
 *   op 0: e = C f (faces -> edges)      op 1: f = C^T e (edges -> faces)
 *   op 2: c = G^T f (faces -> cells)    op 3: f = G c (cells -> faces)
 *   op 4: f = coef * M^soln N~(M^xsoln (u + uinf)) (faces -> faces, eq. opr_def_nonlin)
 * Vector fields [n_xsoln][3][B^3], scalar fields [n_xsoln][1][B^3]; uinf only for op 4. */
lgf_status lgf_op_apply(lgf_plan *p, int op, const float *in, float *out, double coef, const double uinf[3],
                        void *stream);

void lgf_plan_destroy(lgf_plan *p);

/* Thread-local description of the last non-OK status ("" if none). */
const char *lgf_last_error(void);

/* Library version string. */
const char *lgf_version(void);

/* The FFT length a Poisson plan takes for an axis that needs at least `need`
 * points (the size rule of lgf_conv_plan): the smallest supported length
 * >= need, 0 if none.  Host only; no CUDA call. */
int lgf_fft_length(int need);

#ifdef __cplusplus
}
#endif
#endif /* LGF_H */
