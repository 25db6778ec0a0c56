// One step of the IF-HERK scheme on the finite block set (Sec. 3.2 algorithm,
// Sec. 3.3 eq. proj_final, Sec. 5 xIF-HERK) with Scheme A, B or C of
// eq. ifherk_schemes.
//
// Domains (Sec. 4.2): D_soln = D_supp (Sec. 6) = the caller's block list,
// D_xsoln = D_soln dilated by N_b = 1 block (eq. def_xsoln).  Fields live on
// D_xsoln: face velocity u [n_x][3][B^3]; the pressure-like d^ on cells [n_x][1][B^3].
//
// Shifted tableau (eq. herk_shift): a~_{i,j} = a_{i+1,j} (i < 3), b_j (i = 3);
// c~_i = c_{i+1} (i < 3), c~_3 = 1, and c~_0 = c_1 = 0 (the first stage starts at
// t_k).  H^i = E((c~_i - c~_{i-1}) alpha), alpha = dt / (dx^2 Re): Scheme A
// E(a/2), E(a/2), I; Scheme B E(a/3), E(2a/3), I; Scheme C E(8a/15), E(2a/15), E(a/3).
// Carrying the q and w recursions through the integrating factors (linearity of
// E) gives the step with at most six integrating-factor applications:
//   stage 1:  g1 = -a~11 dt M^soln N~(M(u0 + u_inf));  r1 = u0 + g1
//             gd1 = G d^1, d^1 = -L^{-1} M^supp G^T r1;  u1 = H1(r1 - gd1)
//             w11 = (g1 - gd1) / (a~11 dt)
//   stage 2:  g2 = -a~22 dt M^soln N~(M(u1 + u_inf));  r2 = H1(u0 + dt a~21 w11) + g2
//             gd2 = G d^2;  u2 = H2(r2 - gd2);  w22 = (g2 - gd2) / (a~22 dt)
//   stage 3:  g3 = -a~33 dt M^soln N~(M(u2 + u_inf))
//             r3 = H2(H1(u0 + dt a~31 w11) + dt a~32 w22) + g3
//             gd3 = G d^3;  u_{k+1} = H3(r3 - gd3)
// (Hi = M^xsoln H^i M^xsoln).  The sign of g follows eq. ifherk_g.
// The oracle runs the paper's form (explicit q and w recursions) instead, so
// the parity test also checks this rearrangement.
#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <cstring>
#include <utility>
#include <vector>

#include "plan.hpp"

namespace lgf {
namespace {

inline int64_t pack3(int32_t x, int32_t y, int32_t z)
{
    const int64_t off = 1 << 20;
    return ((int64_t)(x + off) << 42) | ((int64_t)(y + off) << 21) | (int64_t)(z + off);
}

template <typename T>
lgf_status alloc_upload(T **d, const std::vector<T> &h, size_t &bytes)
{
    *d = nullptr;
    if (h.empty()) return LGF_OK;
    LGF_CUDA_TRY(cudaMalloc((void **)d, h.size() * sizeof(T)));
    bytes += h.size() * sizeof(T);
    LGF_CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return LGF_OK;
}

}  // namespace

void free_rk(RkPlan *r)
{
    if (!r) return;
    for (auto &g : r->graphs) cudaGraphExecDestroy(g.exec);
    lgf_plan_destroy(r->poisson);
    lgf_plan_destroy(r->poisson3);
    for (int i = 0; i < 3; i++)
        if (r->if_owned[i]) {
            lgf_plan_destroy(r->ifp[i]);
            lgf_table_destroy(r->if_table[i]);
        }
    lgf_table_destroy(r->lgf_table);
    cudaFree(r->d_nbr27);
    cudaFree(r->d_coords);
    cudaFree(r->d_acc);
    cudaFree(r->d_mu);
    cudaFree(r->d_tidx);
    cudaFree(r->d_soln_keep);
    cudaFree(r->d_supp_idx);
    cudaFree(r->work);
    delete r;
}

// run a launch between two profiling events of the plan (when enabled)
template <typename F>
lgf_status timed(Profiler &pr, const char *name, cudaStream_t s, F &&f)
{
    if (pr.on) pr.begin(s);
    lgf_status st = f();
    if (pr.on && st == LGF_OK) pr.end(name, s);
    return st;
}

// Projection of a stage: with gd = G d^, d^ = -M^xsoln L^{-1} M^supp G^T M^xsoln r,
// writes out1 = r - gd and (out2 != nullptr) out2 = c2 (g - gd).
lgf_status rk_project(RkPlan *r, Profiler &pr, const float *rv, const float *g, float *out1, float *out2, double c2,
                      cudaStream_t s)
{
    float *sx = r->work + 8 * r->vec;  // G^T r on xsoln cells
    LGF_TRY(timed(pr, "op_div_t", s, [&] { return op_launch(2, r->B, r->n_x, r->d_nbr27, nullptr, rv, sx, r->dx, 1.0, nullptr, s); }));
    // The D_supp blocks are the first n_soln blocks of D_xsoln, so the xsoln array is
    // the solve's source array as it stands (M^supp: the plan reads only those blocks).
    // d^ overwrites G^T r: the whole-box passes read their source only in the first
    // pass and write their result only in the last, which starts after it has completed.
    // The split solve reads its source on two streams, so it gets a copy of its own.
    const float *srcs[1] = {sx};
    float *dsts[1] = {sx};
    if (r->split) {
        float *ss = sx + r->scal_x;
        const int B3 = r->B * r->B * r->B;
        LGF_TRY(timed(pr, "gather_supp", s, [&] { return gather_launch(sx, ss, r->d_supp_idx, r->n_soln, B3, s); }));
        srcs[0] = ss;
    }
    LGF_TRY(lgf_conv_execute(r->poisson, srcs, dsts, s));
    LGF_TRY(timed(pr, "grad_combine", s, [&] {
        return grad_combine_launch(r->B, r->n_x, r->d_nbr27, sx, rv, g, out1, out2, c2, r->dx, s);
    }));
    return LGF_OK;
}

}  // namespace lgf

using namespace lgf;

extern "C" {

lgf_status lgf_rk_plan(const lgf_rk_desc *d, void *stream, lgf_plan **out)
{
    clear_error();
    LGF_CHECK_ARG(d && out, "lgf_rk_plan: NULL argument");
    *out = nullptr;
    LGF_CHECK_ARG(d->B == 8 || d->B == 16, "lgf_rk_plan: B=%d not in {8,16}", d->B);
    LGF_CHECK_ARG(d->n_soln >= 1 && d->soln_blocks, "lgf_rk_plan: empty soln block list");
    LGF_CHECK_ARG(d->dx > 0 && d->dt > 0 && d->re > 0, "lgf_rk_plan: dx, dt, re must be positive");
    LGF_CHECK_ARG(d->scheme >= 0 && d->scheme <= 2, "lgf_rk_plan: scheme %d not in {0 (A), 1 (B), 2 (C)}",
                  d->scheme);
    LGF_CHECK_ARG(d->reserved[0] == 0, "lgf_rk_plan: reserved fields must be zero");
    LGF_CHECK_ARG(d->poisson_method >= 0 && d->poisson_method <= 2, "lgf_rk_plan: poisson_method %d not in {0, 1, 2}",
                  d->poisson_method);
    LGF_CHECK_ARG(d->poisson_method != 2 || d->B == 16, "lgf_rk_plan: the split Poisson solve takes B = 16");
    const int B = d->B;
    // blocks: soln as given, xsoln = soln dilated by one block, soln first
    std::unordered_map<int64_t, int> xi;
    std::vector<int32_t> xs;
    for (int i = 0; i < d->n_soln; i++) {
        const int32_t *c = d->soln_blocks + 3 * i;
        LGF_CHECK_ARG(c[0] > -(1 << 19) && c[0] < (1 << 19) && c[1] > -(1 << 19) && c[1] < (1 << 19) &&
                          c[2] > -(1 << 19) && c[2] < (1 << 19),
                      "lgf_rk_plan: block coordinate out of range");
        LGF_CHECK_ARG(xi.emplace(pack3(c[0], c[1], c[2]), (int)(xs.size() / 3)).second, "lgf_rk_plan: duplicate block");
        xs.insert(xs.end(), c, c + 3);
    }
    const int nsoln = d->n_soln;
    for (int i = 0; i < nsoln; i++)
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const int32_t x = xs[3 * i] + dx, y = xs[3 * i + 1] + dy, z = xs[3 * i + 2] + dz;
                    if (xi.emplace(pack3(x, y, z), (int)(xs.size() / 3)).second) {
                        xs.push_back(x);
                        xs.push_back(y);
                        xs.push_back(z);
                    }
                }
    const int nx = (int)(xs.size() / 3);
    RkPlan *r = new (std::nothrow) RkPlan();
    if (!r) {
        set_error("host allocation failed");
        return LGF_ERR_OOM;
    }
    r->B = B;
    r->n_soln = nsoln;
    r->n_x = nx;
    r->dx = d->dx;
    r->dt = d->dt;
    r->re = d->re;
    r->alpha = d->dt / (d->dx * d->dx * d->re);
    r->xsoln = xs;
    lgf_status st = LGF_OK;
    auto fail = [&](lgf_status e) {
        free_rk(r);
        return e;
    };
    // neighbour table, soln flags, supp (= soln) indices
    std::vector<int> nbr((size_t)nx * 27, -1);
    for (int i = 0; i < nx; i++)
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    auto it = xi.find(pack3(xs[3 * i] + dx, xs[3 * i + 1] + dy, xs[3 * i + 2] + dz));
                    if (it != xi.end()) nbr[(size_t)i * 27 + (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = it->second;
                }
    std::vector<unsigned char> keep(nx, 0);
    std::vector<int> supp(nsoln);
    for (int i = 0; i < nsoln; i++) {
        keep[i] = 1;
        supp[i] = i;
    }
    if ((st = alloc_upload(&r->d_nbr27, nbr, r->bytes)) != LGF_OK) return fail(st);
    if ((st = alloc_upload(&r->d_coords, xs, r->bytes)) != LGF_OK) return fail(st);
    if (cudaMalloc(&r->d_acc, 15 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&r->d_mu, 2 * (size_t)nx * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&r->d_tidx, (size_t)nsoln * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        set_error("lgf_rk_plan: allocation failed");
        return fail(LGF_ERR_OOM);
    }
    if ((st = alloc_upload(&r->d_soln_keep, keep, r->bytes)) != LGF_OK) return fail(st);
    if ((st = alloc_upload(&r->d_supp_idx, supp, r->bytes)) != LGF_OK) return fail(st);
    // Poisson sub-plan: supp -> xsoln, scalar, d^ = -L^{-1} f (scale -1)
    const int K = [&] {
        int need = 0;
        int slo[3], shi[3], tlo[3], thi[3];
        for (int a = 0; a < 3; a++) {
            slo[a] = tlo[a] = 1 << 30;
            shi[a] = thi[a] = -(1 << 30);
        }
        for (int i = 0; i < nx; i++)
            for (int a = 0; a < 3; a++) {
                const int v = xs[3 * i + a];
                if (i < nsoln) {
                    slo[a] = std::min(slo[a], v);
                    shi[a] = std::max(shi[a], v);
                }
                tlo[a] = std::min(tlo[a], v);
                thi[a] = std::max(thi[a], v);
            }
        for (int a = 0; a < 3; a++) {
            const long m = std::max(std::labs((long)tlo[a] * B - ((long)shi[a] * B + B - 1)),
                                    std::labs(((long)thi[a] * B + B - 1) - (long)slo[a] * B));
            // the Poisson plan's length rule: max(2 m + 2, 2 E_s)
            const long len = std::max<long>(2 * m + 2, 2L * (shi[a] - slo[a] + 1) * B);
            const int n = poisson_pick_n((int)std::min<long>(len, 1 << 20));
            need = n == 0 ? (1 << 20) : std::max(need, n / 2 - 1);  // 0: beyond the longest FFT
        }
        return need;
    }();
    // whole box where its FFT lengths reach (K <= 511 means every length <= 1024), else the split
    // solve (which builds its own near- and far-field tables; the plan's table is then small)
    const bool whole_fits = K >= 1 && K <= 511;
    r->poisson_method = d->poisson_method;
    r->split = d->poisson_method == 2 || (d->poisson_method == 0 && !whole_fits);
    if (r->split && B != 16) {
        set_error("lgf_rk_plan: the block set needs FFTs longer than 1024 and the split solve takes B = 16");
        return fail(LGF_ERR_ARG);
    }
    if (!r->split && !whole_fits) {
        set_error("lgf_rk_plan: block set too large for the whole-box FFT lengths (use poisson_method 0 or 2)");
        return fail(LGF_ERR_ARG);
    }
    if ((st = lgf_table_build(LGF_KERNEL_LAPLACE7, 0.0, r->split ? 63 : K, stream, &r->lgf_table)) != LGF_OK)
        return fail(st);
    lgf_plan_opts po;
    std::memset(&po, 0, sizeof(po));
    po.method = r->split ? 1 : 0;
    lgf_solve_desc pd;
    pd.B = B;
    pd.ncomp = 1;
    pd.n_src = nsoln;
    pd.n_dst = nx;
    pd.src_blocks = xs.data();
    pd.dst_blocks = xs.data();
    pd.dx = d->dx;
    pd.scale = -1.0;
    if ((st = lgf_conv_plan(r->lgf_table, &pd, 1, &po, stream, &r->poisson)) != LGF_OK) return fail(st);
    {
        lgf_solve_desc pv = pd;  // vector potential a = -L^{-1} w (velocity refresh)
        pv.ncomp = 3;
        if ((st = lgf_conv_plan(r->lgf_table, &pv, 1, &po, stream, &r->poisson3)) != LGF_OK) return fail(st);
    }
    // shifted tableau of the scheme (eq. ifherk_schemes, eq. herk_shift)
    {
        const double r3 = std::sqrt(3.0);
        double A[3][3] = {}, b[3] = {}, c[3] = {};
        if (d->scheme == 0) {
            A[1][0] = 0.5;
            A[2][0] = r3 / 3.0;
            A[2][1] = (3.0 - r3) / 3.0;
            b[0] = (3.0 + r3) / 6.0;
            b[1] = -r3 / 3.0;
            b[2] = (3.0 + r3) / 6.0;
        } else if (d->scheme == 1) {
            A[1][0] = 1.0 / 3.0;
            A[2][0] = -1.0;
            A[2][1] = 2.0;
            b[1] = 0.75;
            b[2] = 0.25;
        } else {
            A[1][0] = 8.0 / 15.0;
            A[2][0] = 0.25;
            A[2][1] = 5.0 / 12.0;
            b[0] = 0.25;
            b[2] = 0.75;
        }
        for (int i = 0; i < 3; i++) c[i] = A[i][0] + A[i][1] + A[i][2];
        r->scheme = d->scheme;
        r->use_graph = d->use_graph ? 1 : 0;
        for (int i = 1; i <= 3; i++)
            for (int j = 1; j <= i; j++) r->at[i][j] = i < 3 ? A[i][j - 1] : b[j - 1];
        const double ct[4] = {c[0], c[1], c[2], 1.0};  // c~_0 = c_1, c~_i = c_{i+1}, c~_3 = 1
        // integrating factors on D_xsoln, three components
        lgf_solve_desc id = pd;
        id.ncomp = 3;
        id.n_src = nx;
        id.src_blocks = xs.data();
        id.n_dst = 0;
        id.dst_blocks = nullptr;
        double expo[3];
        for (int i = 0; i < 3; i++) {
            expo[i] = (ct[i + 1] - ct[i]) * r->alpha;
            if (expo[i] <= 0.0) continue;  // identity
            bool shared = false;
            for (int k = 0; k < i; k++)
                if (r->ifp[k] && std::fabs(expo[k] - expo[i]) <= 1e-15 * expo[i]) {
                    r->ifp[i] = r->ifp[k];
                    r->if_table[i] = r->if_table[k];
                    shared = true;
                    break;
                }
            if (shared) continue;
            r->if_owned[i] = true;
            if ((st = lgf_table_build(LGF_KERNEL_IFACTOR, expo[i], 0, stream, &r->if_table[i])) != LGF_OK)
                return fail(st);
            if ((st = lgf_conv_plan(r->if_table[i], &id, 1, nullptr, stream, &r->ifp[i])) != LGF_OK) return fail(st);
        }
    }
    // workspaces: vector fields g, r, w11, w22, t1, t2, u1, u2 ; scalars s_supp, dhat
    const size_t B3 = (size_t)B * B * B;
    r->vec = (size_t)nx * 3 * B3;
    r->scal_x = (size_t)nx * B3;
    r->scal_s = (size_t)nsoln * B3;
    // 8 vectors (slot 5 holds a multi-step run's intermediate state), d^ on D_xsoln and
    // D_supp, w on D_supp (3 components) for the refresh, and 2 more vectors for the
    // vorticity-formulation step
    const size_t total = 8 * r->vec + r->scal_x + r->scal_s + 3 * r->scal_s + 2 * r->vec;
    if (cudaMalloc(&r->work, total * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        set_error("lgf_rk_plan: workspace allocation of %zu bytes failed", total * sizeof(float));
        return fail(LGF_ERR_OOM);
    }
    r->bytes += total * sizeof(float);
    lgf_plan *p = new (std::nothrow) lgf_plan();
    if (!p) return fail(LGF_ERR_OOM);
    p->kind = LGF_PLAN_RK;
    p->rk = r;
    int dev = 0;
    cudaGetDevice(&dev);
    p->device = dev;
    p->bytes = r->bytes;
    *out = p;
    return LGF_OK;
}

int lgf_rk_block_count(const lgf_plan *p, int which)
{
    if (!p || p->kind != LGF_PLAN_RK) return -1;
    return which == 0 ? p->rk->n_x : p->rk->n_soln;
}

lgf_status lgf_rk_blocks(const lgf_plan *p, int which, int32_t *coords, int n)
{
    clear_error();
    LGF_CHECK_ARG(p && coords && p->kind == LGF_PLAN_RK, "lgf_rk_blocks: not an RK plan");
    const int cnt = which == 0 ? p->rk->n_x : p->rk->n_soln;
    LGF_CHECK_ARG(n >= cnt, "lgf_rk_blocks: need room for %d blocks", cnt);
    std::copy(p->rk->xsoln.begin(), p->rk->xsoln.begin() + 3 * (size_t)cnt, coords);
    return LGF_OK;
}

lgf_status lgf_op_apply(lgf_plan *p, int op, const float *in, float *out, double coef, const double uinf[3],
                        void *stream)
{
    clear_error();
    LGF_CHECK_ARG(p && in && out && in != out, "lgf_op_apply: NULL or aliasing argument");
    LGF_CHECK_ARG(p->kind == LGF_PLAN_RK, "lgf_op_apply: needs a plan from lgf_rk_plan");
    LGF_CHECK_ARG(op >= 0 && op <= 4, "lgf_op_apply: unknown operator %d", op);
    RkPlan *r = p->rk;
    return op_launch(op, r->B, r->n_x, r->d_nbr27, op == 4 ? r->d_soln_keep : nullptr, in, out, r->dx, coef, uinf,
                     (cudaStream_t)stream);
}

}  // extern "C"

// the launch sequence of one step (no host synchronisation: capturable)
static lgf_status rk_step_launches(lgf_plan *p, const float *u_in, float *u_out, const double uinf[3], cudaStream_t s)
{
    RkPlan *r = p->rk;
    const double dt = r->dt;
    const double a11 = r->at[1][1], a21 = r->at[2][1], a22 = r->at[2][2];
    const double a31 = r->at[3][1], a32 = r->at[3][2], a33 = r->at[3][3];
    const size_t V = r->vec;
    // slots 0-7: g, rv, w11, w22, t1, (lgf_rk_run's state), u1, u2
    float *g = r->work, *rv = g + V, *w11 = rv + V, *w22 = w11 + V, *t1 = w22 + V, *u1 = t1 + 2 * V,
          *u2 = u1 + V;
    const int B = r->B;
    const float *u0 = u_in;
    Profiler &pr = p->prof;
    // g = -a dt M^soln N~(u + u_inf); with rvo also rvo = u + g
    auto NL = [&](const float *u, double a, float *rvo = nullptr) {
        return timed(pr, "op_nonlinear", s, [&] {
            return op_launch(4, B, r->n_x, r->d_nbr27, r->d_soln_keep, u, g, r->dx, -a * dt, uinf, s, rvo);
        });
    };
    // y = Hk(x0 + c1 x1) + add, the combinations folded into the integrating factor's
    // passes; an identity Hk is one linear combination
    auto H = [&](int k, const float *x, float *y, const float *x1 = nullptr, double c1 = 0.0,
                 const float *add = nullptr) -> lgf_status {
        if (!r->ifp[k - 1])
            return timed(pr, "lincomb", s, [&] {
                return lincomb_launch(y, (int64_t)V, x, 1.0, x1, x1 ? c1 : 0.0, add, add ? 1.0 : 0.0, nullptr, 0.0, s);
            });
        IfIO io;
        io.x0 = x;
        io.x1 = x1;
        io.c1 = c1;
        io.add = add;
        return ifactor_apply_io(r->ifp[k - 1], io, y, s);
    };
    // project(r, t, w, c): t = r - G d^ (the projected stage value) and w = c (g - G d^)
    auto project = [&](const float *rvv, float *t, float *w, double c) { return rk_project(r, pr, rvv, g, t, w, c, s); };
    // stage 1
    LGF_TRY(NL(u0, a11, rv));  // g and rv = u0 + g
    LGF_TRY(project(rv, t1, w11, 1.0 / (a11 * dt)));
    LGF_TRY(H(1, t1, u1));
    // stage 2: r2 = H1(u0 + dt a21 w11) + g2
    LGF_TRY(NL(u1, a22));
    LGF_TRY(H(1, u0, rv, w11, dt * a21, g));
    LGF_TRY(project(rv, t1, w22, 1.0 / (a22 * dt)));
    LGF_TRY(H(2, t1, u2));
    // stage 3: r3 = H2(H1(u0 + dt a31 w11) + dt a32 w22) + g3
    LGF_TRY(NL(u2, a33));
    LGF_TRY(H(1, u0, u1, w11, dt * a31));  // u1 no longer needed
    LGF_TRY(H(2, u1, rv, w22, dt * a32, g));
    if (r->ifp[2]) {
        LGF_TRY(project(rv, t1, nullptr, 0.0));
        LGF_TRY(H(3, t1, u_out));
    } else {
        LGF_TRY(project(rv, u_out, nullptr, 0.0));
    }
    return LGF_OK;
}

extern "C" {

lgf_status lgf_rk_step(lgf_plan *p, const float *u_in, float *u_out, const double uinf[3], void *stream)
{
    clear_error();
    LGF_CHECK_ARG(p && u_in && u_out && uinf && u_in != u_out, "lgf_rk_step: NULL or aliasing argument");
    LGF_CHECK_ARG(p->kind == LGF_PLAN_RK, "lgf_rk_step: needs a plan from lgf_rk_plan");
    RkPlan *r = p->rk;
    cudaStream_t s = (cudaStream_t)stream;
    if (!r->use_graph || p->prof.on) return rk_step_launches(p, u_in, u_out, uinf, s);
    for (auto &g : r->graphs)
        if (g.in == u_in && g.out == u_out && g.uinf[0] == uinf[0] && g.uinf[1] == uinf[1] && g.uinf[2] == uinf[2]) {
            LGF_CUDA_TRY(cudaGraphLaunch(g.exec, s));
            return LGF_OK;
        }
    // capture this buffer set's step on a private stream, then replay it on s
    cudaStream_t cs;
    LGF_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ex = nullptr;
    lgf_status st = LGF_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        set_error("stream capture failed to start");
        st = LGF_ERR_CUDA;
    } else {
        st = rk_step_launches(p, u_in, u_out, uinf, cs);
        const cudaError_t e = cudaStreamEndCapture(cs, &gr);
        if (st == LGF_OK && e != cudaSuccess) {
            set_error("stream capture failed: %s", cudaGetErrorString(e));
            st = LGF_ERR_CUDA;
        }
        if (st == LGF_OK && cudaGraphInstantiate(&ex, gr, 0) != cudaSuccess) {
            set_error("graph instantiation failed");
            st = LGF_ERR_CUDA;
            ex = nullptr;
        }
    }
    if (gr) cudaGraphDestroy(gr);
    cudaStreamDestroy(cs);
    if (st != LGF_OK) return st;
    if (r->graphs.size() == 2) {
        cudaGraphExecDestroy(r->graphs.front().exec);
        r->graphs.erase(r->graphs.begin());
    }
    r->graphs.push_back({u_in, u_out, {uinf[0], uinf[1], uinf[2]}, ex});
    LGF_CUDA_TRY(cudaGraphLaunch(ex, s));
    return LGF_OK;
}

}  // extern "C"

namespace lgf {
// u_out = M^xsoln C^T M^xsoln (-M^xsoln L^{-1} M^supp w); w: a 3-component array whose first
// n_soln blocks are the D_supp blocks (a D_xsoln field, or the plan's D_supp staging buffer)
lgf_status rk_vor2vel_supp(lgf_plan *p, const float *w, float *u_out, cudaStream_t s)
{
    RkPlan *r = p->rk;
    float *ax = r->work + r->vec;
    const float *srcs[1] = {w};
    float *dsts[1] = {ax};
    LGF_TRY(lgf_conv_execute(r->poisson3, srcs, dsts, s));
    return timed(p->prof, "op_curl_t", s,
                 [&] { return op_launch(1, r->B, r->n_x, r->d_nbr27, nullptr, ax, u_out, r->dx, 1.0, nullptr, s); });
}
}  // namespace lgf

namespace lgf {
// One step of the vorticity formulation (Sec. 4.1): the curl of eq. dnstp,
// dw/dt = L w / Re - C N~(u + u_inf) with u = -C^T L^{-1} w (eq. vel_vor), by the IF-HERK
// recursion of Sec. 3.2 without a constraint.  Per stage: the velocity of the previous stage
// value (a vector Poisson solve D_supp -> D_xsoln and C^T), g^i = -a~_ii dt M^soln C M^soln
// N~(M^xsoln (u + u_inf)), and the integrating factors applied to q and to the w^{i,j}
// (linearity gives the stage value from them); the last stage applies H^s to r^s.
static lgf_status rk_step_vorticity_launches(lgf_plan *p, const float *w_in, float *w_out, const double uinf[3],
                                             cudaStream_t s)
{
    RkPlan *r = p->rk;
    const double dt = r->dt;
    const size_t V = r->vec;
    const int B = r->B, B3 = B * B * B;
    // q, w^{i,1}, w^{i,2} and one spare buffer rotate through slots 2-5 (the integrating
    // factor does not work in place)
    float *g = r->work, *q = r->work + 2 * V, *z[2] = {r->work + 3 * V, r->work + 4 * V}, *spare = r->work + 5 * V;
    float *u = r->work + 6 * V, *f = r->work + 7 * V;
    float *ws = r->work + 8 * V + r->scal_x + r->scal_s;  // w on D_supp (Poisson source)
    float *wi = ws + 3 * r->scal_s, *rv = wi + V;          // stage value, r^s
    Profiler &pr = p->prof;
    auto H = [&](int k, const float *x, float *y) -> lgf_status {
        if (!r->ifp[k - 1])
            return timed(pr, "lincomb", s, [&] {
                return lincomb_launch(y, (int64_t)V, x, 1.0, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0, s);
            });
        IfIO io;
        io.x0 = x;
        return ifactor_apply_io(r->ifp[k - 1], io, y, s);
    };
    auto LC = [&](float *o, const float *x0, double c0, const float *x1 = nullptr, double c1 = 0,
                  const float *x2 = nullptr, double c2 = 0, const float *x3 = nullptr, double c3 = 0) {
        return timed(pr, "lincomb", s, [&] { return lincomb_launch(o, (int64_t)V, x0, c0, x1, c1, x2, c2, x3, c3, s); });
    };
    const float *wprev = w_in;
    for (int i = 1; i <= 3; i++) {
        const double aii = r->at[i][i];
        // velocity of the previous stage value (eq. vel_vor, source on D_supp)
        LGF_TRY(rk_vor2vel_supp(p, wprev, u, s));
        // g = -a~_ii dt M^soln C M^soln N~(M^xsoln (u + u_inf)); the D_soln blocks come first
        LGF_TRY(timed(pr, "op_nonlinear", s, [&] {
            return op_launch(4, B, r->n_x, r->d_nbr27, r->d_soln_keep, u, f, r->dx, -aii * dt, uinf, s);
        }));
        LGF_TRY(timed(pr, "op_curl", s, [&] { return op_launch(0, B, r->n_x, r->d_nbr27, nullptr, f, g, r->dx, 1.0, nullptr, s); }));
        if (r->n_x > r->n_soln)
            LGF_CUDA_TRY(cudaMemsetAsync(g + (size_t)r->n_soln * 3 * B3, 0, (size_t)(r->n_x - r->n_soln) * 3 * B3 * sizeof(float), s));
        if (i < 3) {
            LGF_TRY(LC(z[i - 1], g, 1.0 / (aii * dt)));  // w^{i,i}
            if (i == 1) {
                LGF_TRY(H(1, w_in, q));  // q^2 = H^1 q^1, q^1 = w_k
            } else {
                LGF_TRY(H(i, q, spare));  // q^{i+1} = H^i q^i
                std::swap(q, spare);
            }
            for (int j = 1; j <= i; j++) {  // w^{i+1,j} = H^i w^{i,j}
                LGF_TRY(H(i, z[j - 1], spare));
                std::swap(z[j - 1], spare);
            }
            // stage value H^i r^i = q^{i+1} + dt sum_{j<=i} a~_ij w^{i+1,j}
            if (i == 1) LGF_TRY(LC(wi, q, 1.0, z[0], dt * r->at[1][1]));
            else LGF_TRY(LC(wi, q, 1.0, z[0], dt * r->at[2][1], z[1], dt * r->at[2][2]));
            wprev = wi;
        } else {
            LGF_TRY(LC(rv, q, 1.0, z[0], dt * r->at[3][1], z[1], dt * r->at[3][2], g, 1.0));  // r^3
            LGF_TRY(H(3, rv, w_out));
        }
    }
    return LGF_OK;
}
}  // namespace lgf

extern "C" {

lgf_status lgf_rk_step_vorticity(lgf_plan *p, const float *w_in, float *w_out, const double uinf[3], void *stream)
{
    clear_error();
    LGF_CHECK_ARG(p && w_in && w_out && uinf && w_in != w_out, "lgf_rk_step_vorticity: NULL or aliasing argument");
    LGF_CHECK_ARG(p->kind == LGF_PLAN_RK, "lgf_rk_step_vorticity: needs a plan from lgf_rk_plan");
    return rk_step_vorticity_launches(p, w_in, w_out, uinf, (cudaStream_t)stream);
}

lgf_status lgf_rk_refresh(lgf_plan *p, const float *u_in, float *u_out, void *stream)
{
    clear_error();
    LGF_CHECK_ARG(p && u_in && u_out, "lgf_rk_refresh: NULL argument");
    LGF_CHECK_ARG(p->kind == LGF_PLAN_RK, "lgf_rk_refresh: needs a plan from lgf_rk_plan");
    RkPlan *r = p->rk;
    cudaStream_t s = (cudaStream_t)stream;
    float *wx = r->work;  // w on D_xsoln (its first n_soln blocks: D_supp)
    Profiler &pr = p->prof;
    // w = M^xsoln C M^xsoln u; a = -M^xsoln L^{-1} M^supp w; u' = M^xsoln C^T M^xsoln a (eq. vel_refresh)
    LGF_TRY(timed(pr, "op_curl", s, [&] { return op_launch(0, r->B, r->n_x, r->d_nbr27, nullptr, u_in, wx, r->dx, 1.0, nullptr, s); }));
    return rk_vor2vel_supp(p, wx, u_out, s);
}

int lgf_rk_qmax(const lgf_plan *p, double eps)
{
    clear_error();
    if (!p || p->kind != LGF_PLAN_RK || !(eps > 0.0)) {
        set_error("lgf_rk_qmax: needs an RK plan and eps > 0");
        return -1;
    }
    // App. D: the integrating factors of q steps compose to E(q alpha) (alpha = dt / (dx^2 Re));
    // the relative error the D_xsoln mask causes at depth n_E = B (one buffer block) is the
    // kernel mass beyond n_E, sum_{n >= B} e^{-2 q alpha} I_n(2 q alpha)
    const RkPlan *r = p->rk;
    const int depth = r->B;
    const int nmax = depth + 400;
    std::vector<double> g(nmax + 1);
    int q = 0;
    while (q < 100000) {
        host_scaled_bessel(2.0 * (q + 1) * r->alpha, nmax, g.data());
        double tail = 0.0;  // sum_{n >= depth} g(n), smallest terms first
        for (int n = nmax; n >= depth; n--) tail += g[n];
        if (tail > eps) break;
        q++;
    }
    return q;
}

lgf_status lgf_rk_diagnostics(lgf_plan *p, const float *u, double out[9], void *stream)
{
    clear_error();
    LGF_CHECK_ARG(p && u && out, "lgf_rk_diagnostics: NULL argument");
    LGF_CHECK_ARG(p->kind == LGF_PLAN_RK, "lgf_rk_diagnostics: needs a plan from lgf_rk_plan");
    RkPlan *r = p->rk;
    cudaStream_t s = (cudaStream_t)stream;
    LGF_CUDA_TRY(cudaMemsetAsync(r->d_acc, 0, 15 * sizeof(double), s));
    LGF_TRY(diag_launch(r->B, r->n_soln, r->d_nbr27, r->d_coords, u, nullptr, r->dx, r->d_acc, s));
    double h[15];
    LGF_CUDA_TRY(cudaMemcpyAsync(h, r->d_acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    LGF_CUDA_TRY(cudaStreamSynchronize(s));
    const double dv = r->dx * r->dx * r->dx;
    const double I[3] = {h[0] * dv, h[1] * dv, h[2] * dv};
    const double ii = I[0] * I[0] + I[1] * I[1] + I[2] * I[2];
    for (int a = 0; a < 3; a++) out[a] = I[a];
    out[3] = h[3] * dv;
    out[4] = h[4] * dv;
    out[5] = h[5] * dv;
    for (int b = 0; b < 3; b++) {  // X_b = sum_a M_ab I_a / |I|^2
        double v = 0.0;
        for (int a = 0; a < 3; a++) v += h[6 + 3 * a + b] * dv * I[a];
        out[6 + b] = ii > 0.0 ? v / ii : 0.0;
    }
    return LGF_OK;
}

int lgf_rk_regrid_blocks(lgf_plan *p, const float *u, const double uinf[3], double eps_supp, int32_t *blocks_out,
                         int capacity, void *stream)
{
    clear_error();
    if (!p || !u || !uinf || p->kind != LGF_PLAN_RK || !(eps_supp > 0.0) || capacity < 0) {
        set_error("lgf_rk_regrid_blocks: bad argument");
        return -1;
    }
    RkPlan *r = p->rk;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t V = r->vec;
    float *w = r->work, *nl = r->work + V, *q = r->work + 8 * V;  // slot 0, slot 1, the d^ scalars
    auto ok = [](lgf_status st) { return st == LGF_OK; };
    // w = M C M u;  q = -M G^T M N~(M (u + u_inf)) (algorithm summary, step 1)
    if (!ok(op_launch(0, r->B, r->n_x, r->d_nbr27, nullptr, u, w, r->dx, 1.0, nullptr, s)) ||
        !ok(op_launch(4, r->B, r->n_x, r->d_nbr27, nullptr, u, nl, r->dx, 1.0, uinf, s)) ||
        !ok(op_launch(2, r->B, r->n_x, r->d_nbr27, nullptr, nl, q, r->dx, 1.0, nullptr, s)) ||
        !ok(block_max_launch(r->B, r->n_x, r->d_nbr27, w, q, r->d_mu, r->d_mu + r->n_x, s)))
        return -1;
    std::vector<float> h(2 * (size_t)r->n_x);
    if (cudaMemcpyAsync(h.data(), r->d_mu, h.size() * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("lgf_rk_regrid_blocks: copy failed");
        return -1;
    }
    float mg = 0.f, ng = 0.f;
    for (int b = 0; b < r->n_x; b++) {
        mg = std::max(mg, h[b]);
        ng = std::max(ng, h[r->n_x + b]);
    }
    int n = 0;
    for (int b = 0; b < r->n_x; b++) {
        // eq. weight_fun: W = max(mu / mu_global, nu / nu_global), kept where W > eps_supp
        const double W = std::max(mg > 0.f ? (double)h[b] / mg : 0.0, ng > 0.f ? (double)h[r->n_x + b] / ng : 0.0);
        if (W > eps_supp) {
            if (n < capacity) std::copy(r->xsoln.begin() + 3 * (size_t)b, r->xsoln.begin() + 3 * (size_t)b + 3,
                                        blocks_out + 3 * (size_t)n);
            n++;
        }
    }
    return n;
}

lgf_status lgf_rk_transfer(lgf_plan *from, const float *u_from, lgf_plan *to, float *u_to, void *stream)
{
    clear_error();
    LGF_CHECK_ARG(from && to && u_from && u_to && from->kind == LGF_PLAN_RK && to->kind == LGF_PLAN_RK,
                  "lgf_rk_transfer: needs two RK plans and buffers");
    RkPlan *a = from->rk, *b = to->rk;
    LGF_CHECK_ARG(a->B == b->B && a->dx == b->dx, "lgf_rk_transfer: plans differ in B or dx");
    cudaStream_t s = (cudaStream_t)stream;
    // index in `from`'s D_xsoln of every block of `to`'s D_supp (the vorticity copy of
    // the grid update; new D_supp blocks come from the old D_xsoln)
    std::unordered_map<int64_t, int> pos;
    for (int i = 0; i < a->n_x; i++) pos.emplace(pack3(a->xsoln[3 * i], a->xsoln[3 * i + 1], a->xsoln[3 * i + 2]), i);
    std::vector<int> idx(b->n_soln);
    for (int i = 0; i < b->n_soln; i++) {
        auto it = pos.find(pack3(b->xsoln[3 * i], b->xsoln[3 * i + 1], b->xsoln[3 * i + 2]));
        LGF_CHECK_ARG(it != pos.end(), "lgf_rk_transfer: D_supp block %d of the new plan is outside the old D_xsoln", i);
        idx[i] = it->second;
    }
    LGF_CUDA_TRY(cudaMemcpyAsync(b->d_tidx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    const int B3 = a->B * a->B * a->B;
    float *w_old = a->work;
    float *ws_new = b->work + 8 * b->vec + b->scal_x + b->scal_s;
    LGF_TRY(op_launch(0, a->B, a->n_x, a->d_nbr27, nullptr, u_from, w_old, a->dx, 1.0, nullptr, s));
    // the old mask edge's spurious vortex sheet must not enter the new D_supp
    LGF_TRY(zero_rim_launch(a->B, a->n_x, a->d_nbr27, w_old, s));
    LGF_TRY(gather_launch(w_old, ws_new, b->d_tidx, b->n_soln, 3 * B3, s));
    LGF_TRY(rk_vor2vel_supp(to, ws_new, u_to, s));
    // the host index array must outlive the copy
    LGF_CUDA_TRY(cudaStreamSynchronize(s));
    return LGF_OK;
}

lgf_status lgf_rk_run(lgf_plan *p, const float *u_in, float *u_out, int nsteps, const double uinf[3], int qmax,
                      void *stream)
{
    clear_error();
    LGF_CHECK_ARG(p && u_in && u_out && uinf && u_in != u_out, "lgf_rk_run: NULL or aliasing argument");
    LGF_CHECK_ARG(p->kind == LGF_PLAN_RK, "lgf_rk_run: needs a plan from lgf_rk_plan");
    LGF_CHECK_ARG(nsteps >= 1 && qmax >= 0, "lgf_rk_run: nsteps >= 1 and qmax >= 0 required");
    RkPlan *r = p->rk;
    float *tmp = r->work + 5 * r->vec;  // the vector slot the step leaves unused
    const float *cur = u_in;
    for (int k = 0; k < nsteps; k++) {
        float *nxt = ((nsteps - 1 - k) % 2 == 0) ? u_out : tmp;
        if (k > 0 && qmax > 0 && k % qmax == 0) LGF_TRY(lgf_rk_refresh(p, cur, const_cast<float *>(cur), stream));
        LGF_TRY(lgf_rk_step(p, cur, nxt, uinf, stream));
        cur = nxt;
    }
    return LGF_OK;
}

}  // extern "C"
