// Host-side objects behind the opaque lgf_table / lgf_plan handles.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "common.cuh"

// Geometry of one Poisson solve as seen by the FFT passes (POD, passed by value).
// Axis order everywhere: 0 = x, 1 = y, 2 = z.  Positions in cells.
namespace lgf {
struct Geom {
    int B, ncomp;      // block edge; components per point (the stride of the block layout)
    int c0, nc;        // components c0 .. c0+nc-1 in this launch (grid.y = nc; workspaces hold nc)
    int lB;            // log2(B)
    int S0[3], Es[3];  // source bounding box: origin, extent (multiples of B)
    int T0[3], Et[3];  // target bounding box
    int N[3];          // zero-padded FFT length per axis
    int nbS[3], nbT[3];
    const int *src_lut;  // [nbS_z][nbS_y][nbS_x] -> source block index, -1 if none
    const int *dst_lut;  // [nbT_z][nbT_y][nbT_x] -> target block index, -1 if none
    const float *Kh;     // real even spectrum octant [Nz/2+1][Ny/2+1][Nx/2+1]
    float mul;           // scale * dx^2 / (Nx Ny Nz)
    const double *Kh64;  // FP64 copy (precision = FP64 plans only)
    double mul64;
    int KX;              // Nx/2 + 1
};

struct PoissonSolve {
    Geom g;
    int nsrc, ndst;
    double dx, scale;
    std::vector<int32_t> src_coords, dst_coords;  // host copies
    int spec;                                     // index into lgf_plan::spectra
    size_t elemsA, elemsB;                        // complex elements needed in workspaces A and B
    int *d_src_lut = nullptr, *d_dst_lut = nullptr;
    int *d_dst_nbr = nullptr;   // [ndst][27] target-block neighbours (residual)
    int *d_dst2src = nullptr;   // [ndst] source block at the same coordinates, -1 if none
    float *d_stage_src = nullptr, *d_stage_dst = nullptr;  // staging for lgf_conv_execute_host
};

struct Spectrum {
    int N[3];
    float *d_Kh = nullptr;
    double *d_Kh64 = nullptr;  // FP64 plans
};

// Optional per-kernel event timing (lgf_plan_set_profiling).
struct Profiler {
    bool on = false;
    struct Rec {
        std::string name;
        long long launches = 0;
        double ms = 0.0;
    };
    std::vector<Rec> recs;
    struct Pending {
        int rec;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t cur_a = nullptr;
    int rec_of(const char *name);
    cudaEvent_t take();
    void begin(cudaStream_t s);               // before a launch
    void end(const char *name, cudaStream_t s);  // after it
    lgf_status collect();                     // wait for pending pairs, accumulate
    void clear();
    ~Profiler();
};

// launchers (poisson.cu)
// mark (optional): recorded on s right after pass mark_after (0 x forward, 1 y forward, 2 z)
lgf_status poisson_launch(const Geom &g, const float *src, float *dst, cx<float> *wsA, cx<float> *wsB,
                          cudaStream_t s, Profiler *prof = nullptr, cudaEvent_t mark = nullptr, int mark_after = -1);
lgf_status poisson_launch64(const Geom &g, const double *src, double *dst, cx<double> *wsA, cx<double> *wsB,
                            cudaStream_t s, Profiler *prof = nullptr);
bool poisson_supported_n(int n);
lgf_status poisson_prepare();  // per-device constant tables; call outside stream capture
int poisson_pick_n(int need);  // smallest supported FFT length >= need, 0 if none

// spectrum construction (spectrum.cu): FP64 cosine transforms of the table samples
lgf_status build_spectrum(const double *d_octant, int K, const int N[3], float *d_Kh, double *d_Kh64,
                          cudaStream_t s);

// tables (table.cu)
lgf_status build_lgf_octant(int K, double *d_out, cudaStream_t s);
// -int_{t0}^{t1} of the Bessel form at offsets stride * (a, b, c) (t0 = 0: from 0; t1 = 0: to infinity)
lgf_status build_lgf_octant_part(int K, int stride, double t0, double t1, double *d_out, cudaStream_t s);
lgf_status build_if_taps(double alpha, double tol, double *d_taps, int max_r, int *R_out, cudaStream_t s);

// integrating factor (ifactor.cu): block lists of the three passes
struct IfPlan {
    int B = 0, R = 0;
    int n0 = 0, n1 = 0, n2 = 0;          // |S|, |L1|, |L2|
    int *nbz = nullptr;                  // [n1][3]: S index of block L1[i] + (0,0,-1..1), -1 if absent
    int *nby = nullptr;                  // [n2][3]: L1 index of block L2[i] + (0,-1..1,0)
    int *nbx = nullptr;                  // [n0][3]: L2 index of block S[i] + (-1..1,0,0)
    float *y1 = nullptr, *y2 = nullptr;  // intermediates [n1|n2][ncomp][B^3]
};
lgf_status ifactor_launch(const IfPlan &ip, int ncomp, const float *h_taps, const float *x, float *y, cudaStream_t s,
                          Profiler *prof = nullptr);
// y = H(c0 x0 + c1 x1) + add (x1, add optional; c0 x0 alone when x1 is null):
// the linear combination is read by the first pass, add joins in the last
struct IfIO {
    const float *x0 = nullptr;
    double c0 = 1.0;
    const float *x1 = nullptr;
    double c1 = 0.0;
    const float *add = nullptr;
};
lgf_status ifactor_launch_ex(const IfPlan &ip, int ncomp, const float *h_taps, const IfIO &x, float *y, cudaStream_t s,
                             Profiler *prof = nullptr);
}  // namespace lgf
struct lgf_plan;
namespace lgf {
// y = H(c0 x0 + c1 x1) + add on an integrating-factor plan (abi.cu)
lgf_status ifactor_apply_io(lgf_plan *p, const IfIO &io, float *y, cudaStream_t s);

// local operators (ops.cu): op 0 curl, 1 curl^T, 2 G^T, 3 G, 4 nonlinear
// out2 (op 4 only, optional): also out2 = in + out
lgf_status op_launch(int op, int B, int nblk, const int *d_nbr27, const unsigned char *d_keep, const float *in,
                     float *out, double dx, double coef, const double uinf[3], cudaStream_t s, float *out2 = nullptr);
lgf_status lincomb_launch(float *out, int64_t n, const float *x0, double c0, const float *x1, double c1,
                          const float *x2, double c2, const float *x3, double c3, cudaStream_t s);
lgf_status gather_launch(const float *in, float *out, const int *d_idx, int n, int block_floats, cudaStream_t s);
// per-block maxima of |w| (3 components) and |q| off the mask-edge layer (regrid weights)
lgf_status block_max_launch(int B, int nblk, const int *d_nbr27, const float *w, const float *q, float *mu, float *nu,
                            cudaStream_t s);
// zero a vector field on the mask edge's contaminated layer (3 cells)
lgf_status zero_rim_launch(int B, int nblk, const int *d_nbr27, float *f, cudaStream_t s);
// ring diagnostics sums over D_soln (the first n_soln blocks): 15 FP64 accumulators
lgf_status diag_launch(int B, int n_soln, const int *d_nbr27, const int *d_coords, const float *u, const float *w,
                       double dx, double *d_acc, cudaStream_t s);
// projection tail of a stage: with gd = G dhat (cells -> faces),
// out1 = rv - gd and, when out2 != nullptr, out2 = c2 (g - gd)
lgf_status grad_combine_launch(int B, int nblk, const int *d_nbr27, const float *dhat, const float *rv, const float *g,
                               float *out1, float *out2, double c2, double dx, cudaStream_t s);

// e^{-x} I_n(x), n = 0..nmax, on the host (noalloc.cu)
void host_scaled_bessel(double x, int nmax, double *out);

// one IF-HERK step on a block set (rk.cu)
struct RkPlan {
    int B = 0, n_soln = 0, n_x = 0;
    double dx = 0, dt = 0, re = 0, alpha = 0;
    std::vector<int32_t> xsoln;  // [n_x][3]; the first n_soln blocks are D_soln = D_supp
    lgf_table *lgf_table = nullptr;
    // H^i = E((c~_i - c~_{i-1}) alpha), i = 1..3: tables and plans (nullptr where the
    // exponent is zero, H^i = identity; a stage whose exponent equals an earlier one
    // shares that plan and owns nothing)
    struct lgf_table *if_table[3] = {nullptr, nullptr, nullptr};
    lgf_plan *ifp[3] = {nullptr, nullptr, nullptr};
    bool if_owned[3] = {false, false, false};
    int scheme = 0;
    double at[4][4] = {};  // shifted tableau a~_{i,j}, 1-based
    // lgf_rk_step as a replayed CUDA graph (use_graph): one per (u_in, u_out, u_inf),
    // at most two (a loop alternates two buffers)
    int use_graph = 0;
    struct StepGraph {
        const void *in, *out;
        double uinf[3];
        cudaGraphExec_t exec;
    };
    std::vector<StepGraph> graphs;
    lgf_plan *poisson = nullptr;
    lgf_plan *poisson3 = nullptr;  // vector Poisson supp -> xsoln (velocity refresh)
    int poisson_method = 0;        // as in lgf_rk_desc; split = the sub-plans are block-sparse split solves
    bool split = false;
    int *d_nbr27 = nullptr;
    int *d_coords = nullptr;   // [n_x][3] block coordinates
    double *d_acc = nullptr;   // diagnostics accumulators
    float *d_mu = nullptr;     // [2][n_x] regrid maxima
    int *d_tidx = nullptr;     // [n_soln] transfer gather indices
    unsigned char *d_soln_keep = nullptr;
    int *d_supp_idx = nullptr;
    float *work = nullptr;
    size_t vec = 0, scal_x = 0, scal_s = 0;
    size_t bytes = 0;
};
void free_rk(RkPlan *r);
constexpr int LGF_PLAN_RK = 2;

// block-sparse split solve (split.cu): G = G_near + G_far, near field by block-pair
// spectra, far field on the coarse lattice through Lagrange interpolation
struct SplitPlan {
    double alpha = 0, dx = 0, scale = 0;
    int ncomp = 0, nsrc = 0, ndst = 0;
    int noff = 0;
    std::vector<int> offs;       // [noff][3] kept near offsets d (target - source)
    int64_t npairs = 0;
    float2 *d_W = nullptr;       // window spectra [chunk][noff][32]
    float2 *d_S = nullptr;       // source spectra [nc][chunk][nsrc][32]
    float2 *d_U = nullptr;       // target spectra [nc][chunk][ndst][32]
    int *d_off = nullptr;        // [ndst + 1]
    int2 *d_pairs = nullptr;     // (offset index, source block)
    // runs of 4 x-adjacent target slots: targets [nruns] (int4, -1 = empty slot); rows
    // [run_row[r] .. run_row[r+1]): per (oy, oz) the W rows of ox = -2..2 and the 8
    // sources x0 - 2 .. x0 + 5 (int4 x 4: w0..w3 | w4 s0 s1 s2 | s3..s6 | s7)
    int levels = 1;              // split levels (1: the coarse convolution is a whole-box plan)
    int nruns = 0, nrows = 0;
    int mac_form = 0;            // the multiply-accumulate form kept: 0 pairs, 1 runs, 2 quads
    float mac_ms[3] = {-1.f, -1.f, -1.f};  // plan-time times of the three forms (ms per launch; -1 not timed)
    int4 *d_run_tgt = nullptr;
    int *d_run_row = nullptr;
    int4 *d_rows = nullptr;
    // quads of 4 x 2 target slots (x0 = 4 k, y0 = 2 l): targets [nquads][2] (int4, slot j * 4 + i,
    // -1 = empty), row-steps [quad_row[r] .. quad_row[r+1]) of 3 int4 each (sources 0-3 | 4-7 |
    // first window row of slot row 0 and of slot row 1, -1 = none); only with the 125 offsets
    // in canonical order (nquads = 0 otherwise)
    int nquads = 0, nqrows = 0;
    int4 *d_quad_tgt = nullptr;
    int *d_quad_row = nullptr;
    int4 *d_qrows = nullptr;
    // far field
    int ncsrc = 0, ncdst = 0;
    struct lgf_table *far_table = nullptr;  // G_far at even offsets (coarse octant)
    lgf_plan *coarse = nullptr;             // whole-box plan on the coarse blocks
    float *d_Q = nullptr;        // per source block anterpolated windows [nsrc][nc][16^3]
    float *d_q = nullptr;        // coarse charges [ncsrc][nc][16^3]
    float *d_v = nullptr;        // coarse potential [ncdst][nc][16^3]
    int *d_ccoords = nullptr;    // coarse source block coordinates
    int *d_flut = nullptr;       // fine source block lookup
    int *d_tcoords = nullptr;    // fine target block coordinates
    int *d_clut = nullptr;       // coarse target block lookup
    int3 fmin, fext, cmin, cext;
    float *d_stage_src = nullptr, *d_stage_dst = nullptr;  // lgf_conv_execute_host staging
    bool far_tensor_cores = false;  // far-field interpolation on the tensor cores (tcgen05, reduced precision)
    uint32_t *d_Ba = nullptr, *d_Bi = nullptr;  // tensor-core B operands (TF32 hi, lo)
    int *d_err = nullptr;                       // set by a tensor-core wait that gave up
    cudaStream_t far_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_far = nullptr, ev_src = nullptr;
};
void free_split(SplitPlan *sp);
lgf_status plan_split(lgf_plan *p, const lgf_solve_desc &d, double alpha, int far_precision, int near_form,
                      cudaStream_t s);
// device error flag of a split plan (a bounded tensor-core wait gave up): LGF_ERR_TIMEOUT, cleared
lgf_status split_check(lgf_plan *p, cudaStream_t s);
lgf_status run_split(lgf_plan *p, const float *src, float *dst, cudaStream_t s, Profiler *prof);

// residual (residual.cu)
lgf_status residual_launch(const PoissonSolve &ps, const float *src, const float *dst, double *d_acc,
                           cudaStream_t s);

}  // namespace lgf

struct lgf_table {
    int kind;
    double alpha;
    int K;  // max offset (Laplace)
    int R;  // radius (IF)
    int device;
    int64_t n;       // number of doubles
    double *d_vals;  // FP64 values on the device
    float *d_taps32; // IF: FP32 copy of the taps
    std::vector<float> h_taps32;  // IF: host copy (kernel parameters)
};

struct lgf_plan {
    int kind;
    int device;
    const lgf_table *table;
    // Poisson
    std::vector<lgf::PoissonSolve> solves;
    std::vector<lgf::Spectrum> spectra;
    lgf::cx<float> *d_wsA = nullptr, *d_wsB = nullptr;
    size_t wsA = 0, wsB = 0;
    int precision = 0;  // 0 FP32, 1 FP64
    lgf::cx<double> *d_wsA64 = nullptr, *d_wsB64 = nullptr;
    // several solves: worker streams ("lanes"), each with its own workspaces;
    // execute forks them off the caller's stream with events and joins back
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> lane_done;
    cudaEvent_t fork = nullptr;
    std::vector<lgf::cx<float> *> lane_wsA, lane_wsB;
    // FP32 work units: one per (solve, component) when a plan has more than one
    // unit, so that the components of a vector solve also run on separate lanes
    struct Unit {
        int solve, c0, nc, lane;
        size_t elemsA, elemsB;
    };
    std::vector<Unit> units;
    std::vector<cudaEvent_t> unit_mark;  // per unit: recorded after one of its passes (staggered start)
    // grouped execution (many units): the units with the same FFT grid form a group
    // whose five passes are five launches over device task tables; the groups run on
    // the worker streams (lanes); every unit has its own workspaces
    bool grouped = false;
    std::vector<lgf::cx<float> *> unit_wa, unit_wb;
    struct GroupLaunch {
        int pass, n, ncta;
        void *d_tasks;  // GroupTask<float>[]
        int *d_cta;     // task of every thread block
    };
    struct Group {
        int lane;
        std::vector<int> units;
        GroupLaunch pass[5];
    };
    std::vector<Group> groups;
    double *d_acc = nullptr;  // residual accumulators
    // IF
    int B = 0, ncomp = 0, nblk = 0, R = 0;
    lgf::IfPlan ifp;
    // graph capture
    int use_graph = 0;
    cudaGraphExec_t graph = nullptr;
    std::vector<const void *> graph_key;
    // lgf_conv_execute_host with page-locked host buffers: copies and passes as one graph
    cudaGraphExec_t host_graph = nullptr;
    std::vector<const void *> host_graph_key;
    lgf::Profiler prof;
    lgf::RkPlan *rk = nullptr;  // kind == LGF_PLAN_RK
    int method = 0;                 // 0 whole-box FFT, 1 block-sparse split
    lgf::SplitPlan *split = nullptr;
    lgf_plan *sub = nullptr;        // autotuned plan: the executing plan it chose
    double auto_ms[2] = {-1.0, -1.0};  // autotune times: whole box, split (-1: not timed)
    size_t bytes = 0;
};
