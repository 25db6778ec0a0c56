// C-ABI entry points of liblgf (declared in include/lgf.h): argument
// validation, plan analysis (bounding boxes, FFT sizes, block lookups),
// device allocation, and dispatch to the kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "plan.hpp"
#include "poisson_passes.hpp"

namespace lgf {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = '\0'; }

namespace {
struct TwTables {
    float2 *f = nullptr;
    double2 *d = nullptr;
};
std::mutex g_tw_mu;
std::map<int, TwTables> g_tw;

int current_device()
{
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) return -1;
    return d;
}

inline int64_t pack(int32_t x, int32_t y, int32_t z)
{
    const int64_t off = 1 << 20;
    return ((int64_t)(x + off) << 42) | ((int64_t)(y + off) << 21) | (int64_t)(z + off);
}

bool coords_ok(const int32_t *c, int n)
{
    for (int i = 0; i < 3 * n; i++)
        if (c[i] <= -(1 << 19) || c[i] >= (1 << 19)) return false;
    return true;
}

template <typename T>
lgf_status dalloc(T **p, size_t count, size_t &bytes)
{
    *p = nullptr;
    if (count == 0) return LGF_OK;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        *p = nullptr;
        return LGF_ERR_OOM;
    }
    bytes += count * sizeof(T);
    return LGF_OK;
}

template <typename T>
lgf_status upload(T *d, const std::vector<T> &h, cudaStream_t s)
{
    if (h.empty()) return LGF_OK;
    LGF_CUDA_TRY(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    LGF_CUDA_TRY(cudaStreamSynchronize(s));
    return LGF_OK;
}

void free_plan(lgf_plan *p)
{
    if (!p) return;
    for (auto &ps : p->solves) {
        cudaFree(ps.d_src_lut);
        cudaFree(ps.d_dst_lut);
        cudaFree(ps.d_dst_nbr);
        cudaFree(ps.d_dst2src);
        cudaFree(ps.d_stage_src);
        cudaFree(ps.d_stage_dst);
    }
    for (auto &sp : p->spectra) cudaFree(sp.d_Kh);
    cudaFree(p->d_wsA);
    cudaFree(p->d_wsB);
    cudaFree(p->d_wsA64);
    cudaFree(p->d_wsB64);
    for (auto &sp : p->spectra) cudaFree(sp.d_Kh64);
    for (auto e : p->unit_mark) cudaEventDestroy(e);
    for (auto w : p->lane_wsA) cudaFree(w);
    for (auto w : p->lane_wsB) cudaFree(w);
    for (auto st : p->lanes) cudaStreamDestroy(st);
    for (auto e : p->lane_done) cudaEventDestroy(e);
    if (p->fork) cudaEventDestroy(p->fork);
    cudaFree(p->d_acc);
    cudaFree(p->ifp.nbz);
    cudaFree(p->ifp.nby);
    cudaFree(p->ifp.nbx);
    cudaFree(p->ifp.y1);
    cudaFree(p->ifp.y2);
    for (auto &gr : p->groups)
        for (auto &gl : gr.pass) {
            cudaFree(gl.d_tasks);
            cudaFree(gl.d_cta);
        }
    for (auto *w : p->unit_wa) cudaFree(w);
    for (auto *w : p->unit_wb) cudaFree(w);
    if (p->graph) cudaGraphExecDestroy(p->graph);
    if (p->host_graph) cudaGraphExecDestroy(p->host_graph);
    if (p->rk) free_rk(p->rk);
    if (p->split) free_split(p->split);
    if (p->sub) free_plan(p->sub);
    delete p;
}

// neighbour table [n][27] of a block list (index of the block at offset
// (dx,dy,dz) in {-1,0,1}^3, -1 if absent), ordering (dz+1)*9 + (dy+1)*3 + (dx+1)
std::vector<int> neighbour_table(const int32_t *c, int n)
{
    std::unordered_map<int64_t, int> m;
    m.reserve(2 * n);
    for (int i = 0; i < n; i++) m[pack(c[3 * i], c[3 * i + 1], c[3 * i + 2])] = i;
    std::vector<int> out((size_t)n * 27, -1);
    for (int i = 0; i < n; i++)
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    auto it = m.find(pack(c[3 * i] + dx, c[3 * i + 1] + dy, c[3 * i + 2] + dz));
                    if (it != m.end()) out[(size_t)i * 27 + (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = it->second;
                }
    return out;
}

bool has_duplicates(const int32_t *c, int n)
{
    std::unordered_map<int64_t, int> m;
    m.reserve(2 * n);
    for (int i = 0; i < n; i++)
        if (!m.emplace(pack(c[3 * i], c[3 * i + 1], c[3 * i + 2]), i).second) return true;
    return false;
}

}  // namespace

lgf_status ensure_twiddles()
{
    const int dev = current_device();
    if (dev < 0) {
        set_error("no current CUDA device");
        return LGF_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_tw_mu);
    if (g_tw.count(dev)) return LGF_OK;
    // w_TW_MAX^j (j < TW_MAX), then w_TW_POW^j (j < TW_POW)
    const int total = TW_MAX + TW_POW;
    std::vector<float2> hf(total);
    std::vector<double2> hd(total);
    for (int j = 0; j < total; j++) {
        const double a = j < TW_MAX ? -2.0 * 3.14159265358979323846 * (double)j / (double)TW_MAX
                                    : -2.0 * 3.14159265358979323846 * (double)(j - TW_MAX) / (double)TW_POW;
        hd[j] = make_double2(std::cos(a), std::sin(a));
        hf[j] = make_float2((float)hd[j].x, (float)hd[j].y);
    }
    TwTables t;
    LGF_CUDA_TRY(cudaMalloc(&t.f, total * sizeof(float2)));
    LGF_CUDA_TRY(cudaMalloc(&t.d, total * sizeof(double2)));
    LGF_CUDA_TRY(cudaMemcpy(t.f, hf.data(), total * sizeof(float2), cudaMemcpyHostToDevice));
    LGF_CUDA_TRY(cudaMemcpy(t.d, hd.data(), total * sizeof(double2), cudaMemcpyHostToDevice));
    g_tw[dev] = t;
    return LGF_OK;
}

const float2 *twiddle_table_f32()
{
    std::lock_guard<std::mutex> lk(g_tw_mu);
    auto it = g_tw.find(current_device());
    return it == g_tw.end() ? nullptr : it->second.f;
}
const double2 *twiddle_table_f64()
{
    std::lock_guard<std::mutex> lk(g_tw_mu);
    auto it = g_tw.find(current_device());
    return it == g_tw.end() ? nullptr : it->second.d;
}


int Profiler::rec_of(const char *name)
{
    for (size_t i = 0; i < recs.size(); i++)
        if (recs[i].name == name) return (int)i;
    recs.push_back(Rec{name, 0, 0.0});
    return (int)recs.size() - 1;
}

cudaEvent_t Profiler::take()
{
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void Profiler::begin(cudaStream_t s)
{
    cur_a = take();
    if (cur_a) cudaEventRecord(cur_a, s);
}

void Profiler::end(const char *name, cudaStream_t s)
{
    cudaEvent_t b = take();
    if (!cur_a || !b) return;
    cudaEventRecord(b, s);
    pending.push_back(Pending{rec_of(name), cur_a, b});
    cur_a = nullptr;
}

lgf_status Profiler::collect()
{
    for (auto &p : pending) {
        LGF_CUDA_TRY(cudaEventSynchronize(p.b));
        float ms = 0.f;
        LGF_CUDA_TRY(cudaEventElapsedTime(&ms, p.a, p.b));
        recs[p.rec].launches += 1;
        recs[p.rec].ms += ms;
        pool.push_back(p.a);
        pool.push_back(p.b);
    }
    pending.clear();
    return LGF_OK;
}

void Profiler::clear()
{
    collect();
    recs.clear();
}

Profiler::~Profiler()
{
    for (auto &p : pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
}

}  // namespace lgf

using namespace lgf;

extern "C" {

const char *lgf_last_error(void) { return g_err; }

const char *lgf_version(void) { return "lgf 0.1 (sm_103a)"; }

int lgf_fft_length(int need) { return need <= 0 ? 16 : lgf::poisson_pick_n(need); }

lgf_status lgf_table_build(lgf_kernel kind, double alpha, int max_offset, void *stream, lgf_table **out)
{
    clear_error();
    LGF_CHECK_ARG(out != nullptr, "lgf_table_build: out is NULL");
    *out = nullptr;
    LGF_CHECK_ARG(kind == LGF_KERNEL_LAPLACE7 || kind == LGF_KERNEL_IFACTOR, "lgf_table_build: unknown kind %d", (int)kind);
    cudaStream_t s = (cudaStream_t)stream;
    const int dev = current_device();
    if (dev < 0) {
        set_error("lgf_table_build: no CUDA device");
        return LGF_ERR_CUDA;
    }
    lgf_table *t = new (std::nothrow) lgf_table();
    if (!t) {
        set_error("host allocation failed");
        return LGF_ERR_OOM;
    }
    t->kind = kind;
    t->device = dev;
    t->d_vals = nullptr;
    t->d_taps32 = nullptr;
    size_t bytes = 0;
    lgf_status st = LGF_OK;
    if (kind == LGF_KERNEL_LAPLACE7) {
        if (!(max_offset >= 1 && max_offset <= 1024)) {
            delete t;
            set_error("lgf_table_build: max_offset %d outside [1, 1024]", max_offset);
            return LGF_ERR_ARG;
        }
        t->K = max_offset;
        t->R = 0;
        t->alpha = 0.0;
        const int64_t K1 = max_offset + 1;
        t->n = K1 * (K1 + 1) * (K1 + 2) / 6;
        st = dalloc(&t->d_vals, (size_t)t->n, bytes);
        if (st == LGF_OK) st = build_lgf_octant(max_offset, t->d_vals, s);
    } else {
        if (!(alpha > 0.0 && alpha <= 50.0)) {
            delete t;
            set_error("lgf_table_build: alpha %g outside (0, 50]", alpha);
            return LGF_ERR_ARG;
        }
        t->alpha = alpha;
        t->K = 0;
        const int maxr = 64;
        st = dalloc(&t->d_vals, maxr + 1, bytes);
        int R = 0;
        if (st == LGF_OK) st = build_if_taps(alpha, 1e-14, t->d_vals, maxr, &R, s);
        if (st == LGF_OK && R >= maxr) {
            set_error("lgf_table_build: alpha %g needs more than %d integrating-factor taps", alpha, maxr);
            st = LGF_ERR_ARG;
        }
        if (st == LGF_OK) {
            t->R = R;
            t->n = R + 1;
            std::vector<double> h(R + 1);
            std::vector<float> hf(R + 1);
            if (cudaMemcpy(h.data(), t->d_vals, (R + 1) * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
                set_error("taps download failed");
                st = LGF_ERR_CUDA;
            } else {
                for (int i = 0; i <= R; i++) hf[i] = (float)h[i];
                t->h_taps32 = hf;
                st = dalloc(&t->d_taps32, R + 1, bytes);
                if (st == LGF_OK && cudaMemcpy(t->d_taps32, hf.data(), (R + 1) * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
                    set_error("taps upload failed");
                    st = LGF_ERR_CUDA;
                }
            }
        }
    }
    if (st != LGF_OK) {
        cudaFree(t->d_vals);
        cudaFree(t->d_taps32);
        delete t;
        return st;
    }
    *out = t;
    return LGF_OK;
}

lgf_status lgf_table_info(const lgf_table *t, int *kind, double *alpha, int *max_offset, int *radius)
{
    clear_error();
    LGF_CHECK_ARG(t != nullptr, "lgf_table_info: table is NULL");
    if (kind) *kind = t->kind;
    if (alpha) *alpha = t->alpha;
    if (max_offset) *max_offset = t->K;
    if (radius) *radius = t->R;
    return LGF_OK;
}

int64_t lgf_table_size(const lgf_table *t) { return t ? t->n : 0; }

lgf_status lgf_table_copy(const lgf_table *t, double *host_out, int64_t n)
{
    clear_error();
    LGF_CHECK_ARG(t != nullptr && host_out != nullptr, "lgf_table_copy: NULL argument");
    LGF_CHECK_ARG(n >= t->n, "lgf_table_copy: need %lld doubles, got %lld", (long long)t->n, (long long)n);
    LGF_CUDA_TRY(cudaMemcpy(host_out, t->d_vals, t->n * sizeof(double), cudaMemcpyDeviceToHost));
    return LGF_OK;
}

void lgf_table_destroy(lgf_table *t)
{
    if (!t) return;
    cudaFree(t->d_vals);
    cudaFree(t->d_taps32);
    delete t;
}

// A plan with at least this many units runs grouped: one launch per (pass, length).
constexpr int kGroupMinUnits = 8;

// Grouped execution: the units with the same FFT grid form a group, whose pass
// launches cover all its units through device task tables (thread blocks numbered
// unit after unit).  Groups are assigned to up to four worker streams, largest
// first; every unit gets its own workspaces.
static lgf_status plan_grouped(lgf_plan *p, cudaStream_t s)
{
    p->grouped = true;
    const int nu = (int)p->units.size();
    p->unit_wa.assign(nu, nullptr);
    p->unit_wb.assign(nu, nullptr);
    for (int i = 0; i < nu; i++) {
        LGF_TRY(dalloc(&p->unit_wa[i], p->units[i].elemsA, p->bytes));
        LGF_TRY(dalloc(&p->unit_wb[i], p->units[i].elemsB, p->bytes));
    }
    std::map<std::vector<int>, int> by_grid;
    std::vector<double> cost;
    for (int i = 0; i < nu; i++) {
        const Geom &g0 = p->solves[p->units[i].solve].g;
        const std::vector<int> key = {g0.N[0], g0.N[1], g0.N[2]};
        auto it = by_grid.find(key);
        if (it == by_grid.end()) {
            it = by_grid.emplace(key, (int)p->groups.size()).first;
            p->groups.emplace_back();
            cost.push_back(0.0);
        }
        p->groups[it->second].units.push_back(i);
        cost[it->second] += (double)(p->units[i].elemsA + p->units[i].elemsB);
    }
    const int ng = (int)p->groups.size();
    for (int gi = 0; gi < ng; gi++) {
        lgf_plan::Group &gr = p->groups[gi];
        for (int pass = 0; pass < 5; pass++) {
            std::vector<GroupTask<float>> tasks;
            std::vector<int> cta;
            for (int i : gr.units) {
                const auto &u = p->units[i];
                Geom g = p->solves[u.solve].g;
                g.c0 = u.c0;
                g.nc = 1;
                const int nt = poisson_tiles(pass, g);
                LGF_CHECK_ARG(nt >= 0, "grouped plan: unsupported FFT length %d", g.N[pass_axis(pass)]);
                GroupTask<float> t;
                t.g = g;
                t.wa = p->unit_wa[i];
                t.wb = p->unit_wb[i];
                t.solve = u.solve;
                t.first = (int)cta.size();
                cta.insert(cta.end(), nt, (int)tasks.size());
                tasks.push_back(t);
            }
            lgf_plan::GroupLaunch &L = gr.pass[pass];
            L.pass = pass;
            L.n = p->solves[p->units[gr.units[0]].solve].g.N[pass_axis(pass)];
            L.ncta = (int)cta.size();
            L.d_tasks = nullptr;
            L.d_cta = nullptr;
            GroupTask<float> *dt = nullptr;
            LGF_TRY(dalloc(&dt, tasks.size(), p->bytes));
            L.d_tasks = dt;
            LGF_TRY(upload(dt, tasks, s));
            LGF_TRY(dalloc(&L.d_cta, cta.size(), p->bytes));
            LGF_TRY(upload(L.d_cta, cta, s));
        }
    }
    // largest group first onto the least loaded stream
    const int nl = std::min(4, ng);
    std::vector<int> order(ng);
    for (int i = 0; i < ng; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(nl, 0.0);
    for (int gi : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        p->groups[gi].lane = k;
        load[k] += cost[gi];
    }
    p->lanes.assign(nl, nullptr);
    p->lane_done.assign(nl, nullptr);
    LGF_CUDA_TRY(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming));
    for (int k = 0; k < nl; k++) {
        LGF_CUDA_TRY(cudaStreamCreateWithFlags(&p->lanes[k], cudaStreamNonBlocking));
        LGF_CUDA_TRY(cudaEventCreateWithFlags(&p->lane_done[k], cudaEventDisableTiming));
    }
    return LGF_OK;
}

static lgf_status plan_poisson(lgf_plan *p, const lgf_table *t, const lgf_solve_desc *solves, int n_solves, cudaStream_t s)
{
    LGF_TRY(poisson_prepare());
    std::map<std::vector<int>, int> spec_index;
    size_t maxA = 0, maxB = 0;
    for (int i = 0; i < n_solves; i++) {
        const lgf_solve_desc &d = solves[i];
        LGF_CHECK_ARG(d.B == 8 || d.B == 16 || d.B == 32, "solve %d: B=%d not in {8,16,32}", i, d.B);
        LGF_CHECK_ARG(d.ncomp >= 1 && d.ncomp <= 3, "solve %d: ncomp=%d not in 1..3", i, d.ncomp);
        LGF_CHECK_ARG(d.n_src >= 1 && d.n_dst >= 1, "solve %d: empty block list", i);
        LGF_CHECK_ARG(d.src_blocks && d.dst_blocks, "solve %d: NULL block list", i);
        LGF_CHECK_ARG(d.dx > 0.0 && std::isfinite(d.dx) && std::isfinite(d.scale), "solve %d: bad dx/scale", i);
        LGF_CHECK_ARG(coords_ok(d.src_blocks, d.n_src) && coords_ok(d.dst_blocks, d.n_dst),
                      "solve %d: block coordinate out of range", i);
        LGF_CHECK_ARG(!has_duplicates(d.src_blocks, d.n_src), "solve %d: duplicate source block", i);
        LGF_CHECK_ARG(!has_duplicates(d.dst_blocks, d.n_dst), "solve %d: duplicate target block", i);
        PoissonSolve ps;
        Geom &g = ps.g;
        std::memset(&g, 0, sizeof(g));
        g.B = d.B;
        g.lB = d.B == 8 ? 3 : (d.B == 16 ? 4 : 5);
        g.ncomp = d.ncomp;
        g.c0 = 0;
        g.nc = d.ncomp;
        ps.nsrc = d.n_src;
        ps.ndst = d.n_dst;
        ps.dx = d.dx;
        ps.scale = d.scale;
        ps.src_coords.assign(d.src_blocks, d.src_blocks + 3 * d.n_src);
        ps.dst_coords.assign(d.dst_blocks, d.dst_blocks + 3 * d.n_dst);
        int smin[3], smax[3], tmin[3], tmax[3];
        for (int a = 0; a < 3; a++) {
            smin[a] = tmin[a] = 1 << 30;
            smax[a] = tmax[a] = -(1 << 30);
        }
        for (int b = 0; b < d.n_src; b++)
            for (int a = 0; a < 3; a++) {
                smin[a] = std::min(smin[a], d.src_blocks[3 * b + a]);
                smax[a] = std::max(smax[a], d.src_blocks[3 * b + a]);
            }
        for (int b = 0; b < d.n_dst; b++)
            for (int a = 0; a < 3; a++) {
                tmin[a] = std::min(tmin[a], d.dst_blocks[3 * b + a]);
                tmax[a] = std::max(tmax[a], d.dst_blocks[3 * b + a]);
            }
        for (int a = 0; a < 3; a++) {
            g.nbS[a] = smax[a] - smin[a] + 1;
            g.nbT[a] = tmax[a] - tmin[a] + 1;
            g.S0[a] = smin[a] * d.B;
            g.Es[a] = g.nbS[a] * d.B;
            g.T0[a] = tmin[a] * d.B;
            g.Et[a] = g.nbT[a] * d.B;
            const long lo = (long)g.T0[a] - (long)(g.S0[a] + g.Es[a] - 1);
            const long hi = (long)(g.T0[a] + g.Et[a] - 1) - (long)g.S0[a];
            const long maxabs = std::max(std::labs(lo), std::labs(hi));
            // exact embedding: N >= 2 maxabs + 2 (no two offsets share a wrapped
            // index); N >= 2 Es keeps every source sample in the lower half of
            // the line, which the forward transforms take as their zero pattern
            const long need = std::max<long>(2 * maxabs + 2, 2L * g.Es[a]);
            const int n = poisson_pick_n((int)std::min<long>(need, 1 << 20));
            LGF_CHECK_ARG(n > 0, "solve %d: source/target extent %ld along axis %d needs an FFT longer than 1024", i,
                          maxabs, a);
            g.N[a] = n;
        }
        g.KX = g.N[0] / 2 + 1;
        g.mul = (float)(d.scale * d.dx * d.dx / ((double)g.N[0] * g.N[1] * g.N[2]));
        // lookups
        std::vector<int> slut((size_t)g.nbS[0] * g.nbS[1] * g.nbS[2], -1), tlut((size_t)g.nbT[0] * g.nbT[1] * g.nbT[2], -1);
        for (int b = 0; b < d.n_src; b++) {
            const int x = d.src_blocks[3 * b] - smin[0], y = d.src_blocks[3 * b + 1] - smin[1], z = d.src_blocks[3 * b + 2] - smin[2];
            slut[((size_t)z * g.nbS[1] + y) * g.nbS[0] + x] = b;
        }
        for (int b = 0; b < d.n_dst; b++) {
            const int x = d.dst_blocks[3 * b] - tmin[0], y = d.dst_blocks[3 * b + 1] - tmin[1], z = d.dst_blocks[3 * b + 2] - tmin[2];
            tlut[((size_t)z * g.nbT[1] + y) * g.nbT[0] + x] = b;
        }
        std::vector<int> nbr = neighbour_table(d.dst_blocks, d.n_dst);
        std::vector<int> d2s(d.n_dst, -1);
        {
            std::unordered_map<int64_t, int> m;
            for (int b = 0; b < d.n_src; b++) m[pack(d.src_blocks[3 * b], d.src_blocks[3 * b + 1], d.src_blocks[3 * b + 2])] = b;
            for (int b = 0; b < d.n_dst; b++) {
                auto it = m.find(pack(d.dst_blocks[3 * b], d.dst_blocks[3 * b + 1], d.dst_blocks[3 * b + 2]));
                if (it != m.end()) d2s[b] = it->second;
            }
        }
        // device copies (pushed before the PoissonSolve is stored so cleanup sees them)
        p->solves.push_back(ps);
        PoissonSolve &q = p->solves.back();
        LGF_TRY(dalloc(&q.d_src_lut, slut.size(), p->bytes));
        LGF_TRY(dalloc(&q.d_dst_lut, tlut.size(), p->bytes));
        LGF_TRY(dalloc(&q.d_dst_nbr, nbr.size(), p->bytes));
        LGF_TRY(dalloc(&q.d_dst2src, d2s.size(), p->bytes));
        LGF_TRY(upload(q.d_src_lut, slut, s));
        LGF_TRY(upload(q.d_dst_lut, tlut, s));
        LGF_TRY(upload(q.d_dst_nbr, nbr, s));
        LGF_TRY(upload(q.d_dst2src, d2s, s));
        const size_t B3 = (size_t)d.B * d.B * d.B;
        LGF_TRY(dalloc(&q.d_stage_src, (size_t)d.n_src * d.ncomp * B3, p->bytes));
        LGF_TRY(dalloc(&q.d_stage_dst, (size_t)d.n_dst * d.ncomp * B3, p->bytes));
        q.g.src_lut = q.d_src_lut;
        q.g.dst_lut = q.d_dst_lut;
        const size_t KX = g.KX, nc = d.ncomp;
        q.elemsA = std::max(nc * g.Es[2] * g.Es[1] * KX, nc * g.Et[2] * (size_t)g.N[1] * KX);
        q.elemsB = std::max(nc * g.Es[2] * (size_t)g.N[1] * KX, nc * g.Et[2] * g.Et[1] * KX);
        maxA = std::max(maxA, q.elemsA);
        maxB = std::max(maxB, q.elemsB);
        std::vector<int> key = {g.N[0], g.N[1], g.N[2]};
        auto it = spec_index.find(key);
        if (it == spec_index.end()) {
            Spectrum sp;
            sp.N[0] = g.N[0];
            sp.N[1] = g.N[1];
            sp.N[2] = g.N[2];
            p->spectra.push_back(sp);
            Spectrum &spr = p->spectra.back();
            const size_t nK = (size_t)(g.N[0] / 2 + 1) * (g.N[1] / 2 + 1) * (g.N[2] / 2 + 1);
            LGF_TRY(dalloc(&spr.d_Kh, nK, p->bytes));
            if (p->precision == 1) LGF_TRY(dalloc(&spr.d_Kh64, nK, p->bytes));
            LGF_TRY(build_spectrum(t->d_vals, t->K, g.N, spr.d_Kh, spr.d_Kh64, s));
            it = spec_index.emplace(key, (int)p->spectra.size() - 1).first;
        }
        q.spec = it->second;
    }
    for (auto &q : p->solves) {
        q.g.Kh = p->spectra[q.spec].d_Kh;
        q.g.Kh64 = p->spectra[q.spec].d_Kh64;
        q.g.mul64 = q.scale * q.dx * q.dx / ((double)q.g.N[0] * q.g.N[1] * q.g.N[2]);
    }
    LGF_TRY(dalloc(&p->d_acc, 2, p->bytes));
    if (p->precision == 1) {
        for (auto &q : p->solves)
            LGF_CHECK_ARG(q.g.N[0] <= 512 && q.g.N[1] <= 512 && q.g.N[2] <= 512,
                          "FP64 plans are limited to FFT lengths <= 512 (need %d x %d x %d)", q.g.N[0], q.g.N[1], q.g.N[2]);
        LGF_TRY(dalloc(&p->d_wsA64, maxA, p->bytes));
        LGF_TRY(dalloc(&p->d_wsB64, maxB, p->bytes));
        return LGF_OK;
    }
    if (n_solves == 1 && p->solves[0].g.ncomp == 1) {
        LGF_TRY(dalloc(&p->d_wsA, maxA, p->bytes));
        LGF_TRY(dalloc(&p->d_wsB, maxB, p->bytes));
        p->wsA = maxA;
        p->wsB = maxB;
        return LGF_OK;
    }
    // Several independent units, one per (solve, component): each runs the five
    // passes on its own worker stream (up to 4), so the passes of different
    // units overlap (a memory-bound pass beside the compute-bound z pass).
    // Longest-first greedy assignment, the workspace size as the cost estimate.
    // (64 ragged solves: 2, 3, 4, 5, 6, 8, 12, 16 streams took 2.13, 1.93, 1.92,
    // 1.88, 1.97, 2.01, 2.09, 2.10 ms.)
    for (int i = 0; i < n_solves; i++) {
        const PoissonSolve &q = p->solves[i];
        for (int c = 0; c < q.g.ncomp; c++)
            p->units.push_back({i, c, 1, 0, q.elemsA / q.g.ncomp, q.elemsB / q.g.ncomp});
    }
    const int nu = (int)p->units.size();
    if (nu >= kGroupMinUnits && n_solves <= kGroupMaxSolves) return plan_grouped(p, s);
    const int nl = std::min(4, nu);
    std::vector<int> order(nu);
    for (int i = 0; i < nu; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        return p->units[a].elemsA + p->units[a].elemsB > p->units[b].elemsA + p->units[b].elemsB;
    });
    std::vector<double> load(nl, 0.0);
    std::vector<size_t> la(nl, 0), lb(nl, 0);
    for (int i : order) {
        lgf_plan::Unit &u = p->units[i];
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        u.lane = k;
        load[k] += (double)(u.elemsA + u.elemsB);
        la[k] = std::max(la[k], u.elemsA);
        lb[k] = std::max(lb[k], u.elemsB);
    }
    p->lanes.assign(nl, nullptr);
    p->lane_done.assign(nl, nullptr);
    p->lane_wsA.assign(nl, nullptr);
    p->lane_wsB.assign(nl, nullptr);
    LGF_CUDA_TRY(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming));
    p->unit_mark.assign(p->units.size(), nullptr);
    for (auto &e : p->unit_mark) LGF_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (int k = 0; k < nl; k++) {
        LGF_CUDA_TRY(cudaStreamCreateWithFlags(&p->lanes[k], cudaStreamNonBlocking));
        LGF_CUDA_TRY(cudaEventCreateWithFlags(&p->lane_done[k], cudaEventDisableTiming));
        LGF_TRY(dalloc(&p->lane_wsA[k], la[k], p->bytes));
        LGF_TRY(dalloc(&p->lane_wsB[k], lb[k], p->bytes));
    }
    return LGF_OK;
}

static lgf_status plan_ifactor(lgf_plan *p, const lgf_table *t, const lgf_solve_desc *solves, int n_solves, cudaStream_t s)
{
    LGF_CHECK_ARG(n_solves == 1, "integrating-factor plans take exactly one block set (got %d)", n_solves);
    const lgf_solve_desc &d = solves[0];
    LGF_CHECK_ARG(d.B == 8 || d.B == 16, "integrating factor: B=%d not in {8,16}", d.B);
    LGF_CHECK_ARG(d.ncomp >= 1 && d.ncomp <= 3, "ncomp=%d not in 1..3", d.ncomp);
    LGF_CHECK_ARG(d.n_src >= 1 && d.src_blocks, "empty block set");
    LGF_CHECK_ARG(coords_ok(d.src_blocks, d.n_src), "block coordinate out of range");
    LGF_CHECK_ARG(!has_duplicates(d.src_blocks, d.n_src), "duplicate block in the set");
    LGF_CHECK_ARG(t->R <= d.B && t->R <= 16,
                  "integrating-factor radius %d exceeds min(B=%d, 16) (alpha too large for this block size)", t->R, d.B);
    p->B = d.B;
    p->ncomp = d.ncomp;
    p->nblk = d.n_src;
    p->R = t->R;
    // block lists of the three passes (see ifactor.cu)
    const int n = d.n_src;
    const int32_t *c = d.src_blocks;
    std::unordered_map<int64_t, int> S, A1, Z1, A2, YZ;
    for (int i = 0; i < n; i++) S[pack(c[3 * i], c[3 * i + 1], c[3 * i + 2])] = i;
    auto add = [](std::unordered_map<int64_t, int> &m, int32_t x, int32_t y, int32_t z) { m.emplace(pack(x, y, z), 0); };
    for (int i = 0; i < n; i++) {
        const int32_t x = c[3 * i], y = c[3 * i + 1], z = c[3 * i + 2];
        for (int a = -1; a <= 1; a++) {
            add(Z1, x, y, z + a);
            add(A2, x + a, y, z);
            for (int b = -1; b <= 1; b++) {
                add(A1, x + a, y + b, z);
                add(YZ, x, y + a, z + b);
            }
        }
    }
    std::vector<int32_t> L1, L2;
    std::unordered_map<int64_t, int> L1i, L2i;
    for (auto &kv : A1)
        if (Z1.count(kv.first)) { L1i[kv.first] = 0; }
    for (auto &kv : A2)
        if (YZ.count(kv.first)) { L2i[kv.first] = 0; }
    auto unpack = [](int64_t k, int32_t &x, int32_t &y, int32_t &z) {
        const int64_t off = 1 << 20, m = (1 << 21) - 1;
        x = (int32_t)(((k >> 42) & m) - off);
        y = (int32_t)(((k >> 21) & m) - off);
        z = (int32_t)((k & m) - off);
    };
    // deterministic order: sort keys
    std::vector<int64_t> k1, k2;
    for (auto &kv : L1i) k1.push_back(kv.first);
    for (auto &kv : L2i) k2.push_back(kv.first);
    std::sort(k1.begin(), k1.end());
    std::sort(k2.begin(), k2.end());
    for (size_t i = 0; i < k1.size(); i++) L1i[k1[i]] = (int)i;
    for (size_t i = 0; i < k2.size(); i++) L2i[k2[i]] = (int)i;
    auto find = [](const std::unordered_map<int64_t, int> &m, int32_t x, int32_t y, int32_t z) {
        auto it = m.find(pack(x, y, z));
        return it == m.end() ? -1 : it->second;
    };
    std::vector<int> nbz(3 * k1.size()), nby(3 * k2.size()), nbx(3 * (size_t)n);
    for (size_t i = 0; i < k1.size(); i++) {
        int32_t x, y, z;
        unpack(k1[i], x, y, z);
        for (int a = -1; a <= 1; a++) nbz[3 * i + a + 1] = find(S, x, y, z + a);
    }
    for (size_t i = 0; i < k2.size(); i++) {
        int32_t x, y, z;
        unpack(k2[i], x, y, z);
        for (int a = -1; a <= 1; a++) nby[3 * i + a + 1] = find(L1i, x, y + a, z);
    }
    for (int i = 0; i < n; i++)
        for (int a = -1; a <= 1; a++) nbx[3 * i + a + 1] = find(L2i, c[3 * i] + a, c[3 * i + 1], c[3 * i + 2]);
    IfPlan &ip = p->ifp;
    ip.B = d.B;
    ip.R = t->R;
    ip.n0 = n;
    ip.n1 = (int)k1.size();
    ip.n2 = (int)k2.size();
    const size_t B3 = (size_t)d.B * d.B * d.B;
    LGF_TRY(dalloc(&ip.nbz, nbz.size(), p->bytes));
    LGF_TRY(dalloc(&ip.nby, nby.size(), p->bytes));
    LGF_TRY(dalloc(&ip.nbx, nbx.size(), p->bytes));
    LGF_TRY(upload(ip.nbz, nbz, s));
    LGF_TRY(upload(ip.nby, nby, s));
    LGF_TRY(upload(ip.nbx, nbx, s));
    LGF_TRY(dalloc(&ip.y1, (size_t)ip.n1 * d.ncomp * B3, p->bytes));
    LGF_TRY(dalloc(&ip.y2, (size_t)ip.n2 * d.ncomp * B3, p->bytes));
    return LGF_OK;
}

// A split plan keeps one PoissonSolve with the target neighbour tables of the FP64
// residual check, and host staging buffers for lgf_conv_execute_host.
static lgf_status plan_split_extras(lgf_plan *p, const lgf_solve_desc &d, cudaStream_t s)
{
    PoissonSolve ps;
    std::memset(&ps.g, 0, sizeof(ps.g));
    ps.g.B = d.B;
    ps.g.ncomp = d.ncomp;
    ps.g.nc = d.ncomp;
    ps.nsrc = d.n_src;
    ps.ndst = d.n_dst;
    ps.dx = d.dx;
    ps.scale = d.scale;
    ps.src_coords.assign(d.src_blocks, d.src_blocks + 3 * d.n_src);
    ps.dst_coords.assign(d.dst_blocks, d.dst_blocks + 3 * d.n_dst);
    std::vector<int> nbr = neighbour_table(d.dst_blocks, d.n_dst);
    std::vector<int> d2s(d.n_dst, -1);
    {
        std::unordered_map<int64_t, int> m;
        for (int b = 0; b < d.n_src; b++) m[pack(d.src_blocks[3 * b], d.src_blocks[3 * b + 1], d.src_blocks[3 * b + 2])] = b;
        for (int b = 0; b < d.n_dst; b++) {
            auto it = m.find(pack(d.dst_blocks[3 * b], d.dst_blocks[3 * b + 1], d.dst_blocks[3 * b + 2]));
            if (it != m.end()) d2s[b] = it->second;
        }
    }
    p->solves.push_back(ps);
    PoissonSolve &q = p->solves.back();
    LGF_TRY(dalloc(&q.d_dst_nbr, nbr.size(), p->bytes));
    LGF_TRY(dalloc(&q.d_dst2src, d2s.size(), p->bytes));
    LGF_TRY(upload(q.d_dst_nbr, nbr, s));
    LGF_TRY(upload(q.d_dst2src, d2s, s));
    LGF_TRY(dalloc(&p->d_acc, 2, p->bytes));
    const size_t B3 = (size_t)d.B * d.B * d.B;
    LGF_TRY(dalloc(&p->split->d_stage_src, (size_t)d.n_src * d.ncomp * B3, p->bytes));
    LGF_TRY(dalloc(&p->split->d_stage_dst, (size_t)d.n_dst * d.ncomp * B3, p->bytes));
    LGF_CUDA_TRY(cudaStreamSynchronize(s));
    return LGF_OK;
}

static lgf_status check_split_solve(const lgf_solve_desc &d)
{
    LGF_CHECK_ARG(d.ncomp >= 1 && d.ncomp <= 3 && d.n_src >= 1 && d.n_dst >= 1 && d.src_blocks && d.dst_blocks &&
                      d.dx > 0.0 && std::isfinite(d.dx) && std::isfinite(d.scale),
                  "lgf_conv_plan: bad solve description");
    LGF_CHECK_ARG(coords_ok(d.src_blocks, d.n_src) && coords_ok(d.dst_blocks, d.n_dst),
                  "lgf_conv_plan: block coordinate out of range");
    LGF_CHECK_ARG(!has_duplicates(d.src_blocks, d.n_src) && !has_duplicates(d.dst_blocks, d.n_dst),
                  "lgf_conv_plan: duplicate block");
    return LGF_OK;
}

// Mean device time of a few executions of plan q (after one untimed run) on scratch buffers.
static lgf_status time_plan(lgf_plan *q, const lgf_solve_desc &d, cudaStream_t s, double *ms)
{
    const size_t B3 = (size_t)d.B * d.B * d.B;
    float *x = nullptr, *y = nullptr;
    LGF_CUDA_TRY(cudaMalloc(&x, (size_t)d.n_src * d.ncomp * B3 * sizeof(float)));
    if (cudaMalloc(&y, (size_t)d.n_dst * d.ncomp * B3 * sizeof(float)) != cudaSuccess) {
        cudaFree(x);
        set_error("autotune scratch allocation failed");
        return LGF_ERR_OOM;
    }
    cudaEvent_t a = nullptr, b = nullptr;
    lgf_status st = LGF_OK;
    if (cudaMemsetAsync(x, 0, (size_t)d.n_src * d.ncomp * B3 * sizeof(float), s) != cudaSuccess ||
        cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        st = LGF_ERR_CUDA;
    const float *src[1] = {x};
    float *dst[1] = {y};
    if (st == LGF_OK) st = lgf_conv_execute(q, src, dst, s);
    const int reps = 3;
    if (st == LGF_OK) {
        cudaEventRecord(a, s);
        for (int r = 0; r < reps && st == LGF_OK; r++) st = lgf_conv_execute(q, src, dst, s);
        cudaEventRecord(b, s);
        float t = 0.f;
        if (st == LGF_OK && (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess))
            st = LGF_ERR_CUDA;
        *ms = t / reps;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(x);
    cudaFree(y);
    if (st == LGF_ERR_CUDA) set_error("autotune timing failed");
    return st;
}

// method 2: plan the whole-box and the split solve, time one of each, keep the faster
// as the plan's executing sub-plan.  A solve the split method does not take (B != 16)
// keeps the whole-box plan.
static lgf_status autotune_plan(lgf_plan *p, const lgf_table *t, const lgf_solve_desc *solves, const lgf_plan_opts *opts,
                                cudaStream_t s)
{
    lgf_plan_opts o = *opts;
    o.method = 0;
    lgf_plan *a = nullptr, *b = nullptr;
    LGF_TRY(lgf_conv_plan(t, solves, 1, &o, (void *)s, &a));
    p->auto_ms[0] = p->auto_ms[1] = -1.0;
    lgf_status st = time_plan(a, solves[0], s, &p->auto_ms[0]);
    if (st != LGF_OK) {
        lgf_plan_destroy(a);
        return st;
    }
    if (solves[0].B == 16) {
        o.method = 1;
        st = lgf_conv_plan(t, solves, 1, &o, (void *)s, &b);
        if (st == LGF_OK) st = time_plan(b, solves[0], s, &p->auto_ms[1]);
        if (st != LGF_OK) {  // the split plan does not fit (e.g. its coarse box): keep the whole box
            lgf_plan_destroy(b);
            b = nullptr;
            clear_error();
        }
    }
    if (b && p->auto_ms[1] < p->auto_ms[0]) {
        lgf_plan_destroy(a);
        p->sub = b;
    } else {
        lgf_plan_destroy(b);
        p->sub = a;
    }
    p->method = p->sub->method;
    p->bytes = p->sub->bytes;
    return LGF_OK;
}

lgf_status lgf_conv_plan(const lgf_table *t, const lgf_solve_desc *solves, int n_solves, const lgf_plan_opts *opts,
                         void *stream, lgf_plan **out)
{
    clear_error();
    LGF_CHECK_ARG(out != nullptr, "lgf_conv_plan: out is NULL");
    *out = nullptr;
    LGF_CHECK_ARG(t != nullptr && solves != nullptr && n_solves >= 1, "lgf_conv_plan: bad table/solves/n_solves");
    if (opts) {
        LGF_CHECK_ARG(opts->reserved[0] == 0, "lgf_conv_plan: reserved option fields must be zero");
        LGF_CHECK_ARG(opts->near_form >= 0 && opts->near_form <= 3, "lgf_conv_plan: near_form must be 0, 1, 2 or 3");
        LGF_CHECK_ARG(opts->precision == 0 || opts->precision == 1, "lgf_conv_plan: precision must be 0 or 1");
        LGF_CHECK_ARG(opts->method >= 0 && opts->method <= 2, "lgf_conv_plan: method must be 0, 1 or 2");
        LGF_CHECK_ARG(opts->far_precision == 0 || opts->far_precision == 1,
                      "lgf_conv_plan: far_precision must be 0 (FP32, CUDA cores) or 1 (tensor cores, TF32 split)");
        LGF_CHECK_ARG(opts->method == 0 || (opts->precision == 0 && t->kind == LGF_KERNEL_LAPLACE7 && n_solves == 1),
                      "lgf_conv_plan: methods 1 and 2 take one FP32 Poisson solve");
        LGF_CHECK_ARG(opts->split_alpha == 0.0 || (opts->split_alpha >= 1.0 && opts->split_alpha <= 64.0),
                      "lgf_conv_plan: split_alpha must be 0 or in [1, 64]");
    }
    const int dev = current_device();
    if (dev != t->device) {
        set_error("lgf_conv_plan: current device %d differs from the table's device %d", dev, t->device);
        return LGF_ERR_STATE;
    }
    LGF_TRY(ensure_twiddles());
    cudaStream_t s = (cudaStream_t)stream;
    lgf_plan *p = new (std::nothrow) lgf_plan();
    if (!p) {
        set_error("host allocation failed");
        return LGF_ERR_OOM;
    }
    p->kind = t->kind;
    p->device = dev;
    p->table = t;
    p->use_graph = opts ? opts->use_graph : 0;
    p->precision = opts ? opts->precision : 0;
    const int method = opts ? opts->method : 0;
    const double alpha = opts && opts->split_alpha > 0.0 ? opts->split_alpha : 20.0;
    lgf_status st;
    if (t->kind != LGF_KERNEL_LAPLACE7) {
        st = plan_ifactor(p, t, solves, n_solves, s);
    } else if (method == 1) {
        st = check_split_solve(solves[0]);
        p->method = 1;
        if (st == LGF_OK)
            st = plan_split(p, solves[0], alpha, opts ? opts->far_precision : 0, opts ? opts->near_form : 0, s);
        if (st == LGF_OK) st = plan_split_extras(p, solves[0], s);
    } else if (method == 2) {
        st = autotune_plan(p, t, solves, opts, s);
    } else {
        st = plan_poisson(p, t, solves, n_solves, s);
    }
    if (st != LGF_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return LGF_OK;
}

lgf_status lgf_plan_check(lgf_plan *p, void *stream)
{
    clear_error();
    LGF_CHECK_ARG(p != nullptr, "lgf_plan_check: NULL plan");
    if (p->sub) return lgf_plan_check(p->sub, stream);
    cudaStream_t s = (cudaStream_t)stream;
    if (p->split) return split_check(p, s);
    LGF_CUDA_TRY(cudaStreamSynchronize(s));
    return LGF_OK;
}

int lgf_plan_method(const lgf_plan *p, double *ms_whole_box, double *ms_split)
{
    if (!p) return -1;
    if (ms_whole_box) *ms_whole_box = p->auto_ms[0];
    if (ms_split) *ms_split = p->auto_ms[1];
    return p->method;
}

lgf_status lgf_plan_workspace_bytes(const lgf_plan *p, size_t *bytes)
{
    clear_error();
    LGF_CHECK_ARG(p && bytes, "lgf_plan_workspace_bytes: NULL argument");
    *bytes = p->bytes;
    return LGF_OK;
}

// Host buffers of lgf_conv_execute_host: each unit copies its own component
// slice in before its passes and out after them, on its own stream, so the
// copies of one unit overlap the passes of the others.
struct HostIO {
    const float *const *src;
    float *const *dst;
};

// components c0 .. c0+nc-1 of a [n][ncomp][B^3] block array (2-D copy: one row per block)
static lgf_status copy_slice(float *d, const float *h, const PoissonSolve &q, int n, int c0, int nc, bool to_device,
                             cudaStream_t s)
{
    const size_t B3 = (size_t)q.g.B * q.g.B * q.g.B, pitch = (size_t)q.g.ncomp * B3 * sizeof(float);
    const size_t off = (size_t)c0 * B3;
    if (to_device)
        LGF_CUDA_TRY(cudaMemcpy2DAsync(d + off, pitch, h + off, pitch, nc * B3 * sizeof(float), n,
                                       cudaMemcpyHostToDevice, s));
    else
        LGF_CUDA_TRY(cudaMemcpy2DAsync((float *)h + off, pitch, d + off, pitch, nc * B3 * sizeof(float), n,
                                       cudaMemcpyDeviceToHost, s));
    return LGF_OK;
}

static lgf_status run_poisson(lgf_plan *p, const float *const *src, float *const *dst, cudaStream_t s,
                              bool capturing = false, const HostIO *host = nullptr)
{
    Profiler *prof = capturing ? nullptr : &p->prof;
    auto unit_geom = [&](const lgf_plan::Unit &u) {
        Geom g = p->solves[u.solve].g;
        g.c0 = u.c0;
        g.nc = u.nc;
        return g;
    };
    // one unit on stream st: host copy in, five passes, host copy out
    // wait (optional): the unit (its copy in included) starts after that event
    auto run_unit = [&](const lgf_plan::Unit &u, cx<float> *wa, cx<float> *wb, cudaStream_t st, Profiler *pr,
                        cudaEvent_t wait = nullptr, cudaEvent_t mark = nullptr) -> lgf_status {
        const PoissonSolve &q = p->solves[u.solve];
        if (wait) LGF_CUDA_TRY(cudaStreamWaitEvent(st, wait, 0));
        if (host) LGF_TRY(copy_slice((float *)src[u.solve], host->src[u.solve], q, q.nsrc, u.c0, u.nc, true, st));
        LGF_TRY(poisson_launch(unit_geom(u), src[u.solve], dst[u.solve], wa, wb, st, pr, mark, mark ? 0 : -1));
        if (host) LGF_TRY(copy_slice(dst[u.solve], host->dst[u.solve], q, q.ndst, u.c0, u.nc, false, st));
        return LGF_OK;
    };
    if (p->grouped) {
        SolvePtrs<float> ptrs;
        for (size_t i = 0; i < p->solves.size(); i++) {
            ptrs.src[i] = src[i];
            ptrs.dst[i] = dst[i];
        }
        static const char *names[5] = {"x_fwd_gather_r2c", "y_fwd", "z_fwd_mul_inv", "y_inv", "x_inv_c2r_scatter"};
        // one group on stream st: its units' copies in, five grouped launches, copies out
        auto run_group = [&](const lgf_plan::Group &gr, cudaStream_t st, Profiler *pr) -> lgf_status {
            if (host)
                for (int i : gr.units) {
                    const auto &u = p->units[i];
                    const PoissonSolve &q = p->solves[u.solve];
                    LGF_TRY(copy_slice((float *)src[u.solve], host->src[u.solve], q, q.nsrc, u.c0, u.nc, true, st));
                }
            for (const auto &gl : gr.pass) {
                if (pr) pr->begin(st);
                LGF_TRY(poisson_launch_grouped(gl.pass, gl.n, (const GroupTask<float> *)gl.d_tasks, gl.d_cta, gl.ncta,
                                               ptrs, st));
                if (pr) pr->end(names[gl.pass], st);
            }
            if (host)
                for (int i : gr.units) {
                    const auto &u = p->units[i];
                    const PoissonSolve &q = p->solves[u.solve];
                    LGF_TRY(copy_slice(dst[u.solve], host->dst[u.solve], q, q.ndst, u.c0, u.nc, false, st));
                }
            return LGF_OK;
        };
        if (prof && prof->on) {
            for (const auto &gr : p->groups) LGF_TRY(run_group(gr, s, prof));
            return LGF_OK;
        }
        LGF_CUDA_TRY(cudaEventRecord(p->fork, s));
        for (size_t k = 0; k < p->lanes.size(); k++) LGF_CUDA_TRY(cudaStreamWaitEvent(p->lanes[k], p->fork, 0));
        for (const auto &gr : p->groups) LGF_TRY(run_group(gr, p->lanes[gr.lane], nullptr));
        for (size_t k = 0; k < p->lanes.size(); k++) {
            LGF_CUDA_TRY(cudaEventRecord(p->lane_done[k], p->lanes[k]));
            LGF_CUDA_TRY(cudaStreamWaitEvent(s, p->lane_done[k], 0));
        }
        return LGF_OK;
    }
    if (p->lanes.empty()) {
        for (size_t i = 0; i < p->solves.size(); i++)
            LGF_TRY(run_unit({(int)i, 0, p->solves[i].g.ncomp, 0, 0, 0}, p->d_wsA, p->d_wsB, s, prof));
        return LGF_OK;
    }
    if (prof && prof->on) {
        // per-pass event timing: the units run one after another on the
        // caller's stream, so that each pass is timed alone
        for (const auto &u : p->units) LGF_TRY(run_unit(u, p->lane_wsA[u.lane], p->lane_wsB[u.lane], s, prof));
        return LGF_OK;
    }
    // fork: every lane waits for the work queued so far on the caller's stream
    LGF_CUDA_TRY(cudaEventRecord(p->fork, s));
    for (size_t k = 0; k < p->lanes.size(); k++) LGF_CUDA_TRY(cudaStreamWaitEvent(p->lanes[k], p->fork, 0));
    // With host buffers the units start one pass apart: unit i (copy in, passes,
    // copy out) waits for unit i-1's first pass, so the units finish one after
    // another and each unit's copy out overlaps the passes of the others (device
    // buffers: all units start together, which is faster there).  Only when
    // every unit has a stream of its own.
    const bool stagger = host != nullptr && p->units.size() <= p->lanes.size();
    for (size_t i = 0; i < p->units.size(); i++) {
        const auto &u = p->units[i];
        LGF_TRY(run_unit(u, p->lane_wsA[u.lane], p->lane_wsB[u.lane], p->lanes[u.lane], nullptr,
                         stagger && i > 0 ? p->unit_mark[i - 1] : nullptr, stagger ? p->unit_mark[i] : nullptr));
    }
    // join: the caller's stream waits for every lane
    for (size_t k = 0; k < p->lanes.size(); k++) {
        LGF_CUDA_TRY(cudaEventRecord(p->lane_done[k], p->lanes[k]));
        LGF_CUDA_TRY(cudaStreamWaitEvent(s, p->lane_done[k], 0));
    }
    return LGF_OK;
}

lgf_status lgf_conv_execute_f64(lgf_plan *p, const double *const *src, double *const *dst, void *stream)
{
    clear_error();
    LGF_CHECK_ARG(p && src && dst, "lgf_conv_execute_f64: NULL argument");
    if (p->kind != LGF_KERNEL_LAPLACE7 || p->precision != 1) {
        set_error("lgf_conv_execute_f64: needs a Poisson plan built with precision = 1");
        return LGF_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    for (size_t i = 0; i < p->solves.size(); i++) {
        LGF_CHECK_ARG(src[i] && dst[i], "lgf_conv_execute_f64: NULL buffer for solve %zu", i);
        LGF_TRY(poisson_launch64(p->solves[i].g, src[i], dst[i], p->d_wsA64, p->d_wsB64, s, &p->prof));
    }
    return LGF_OK;
}

// FP32 execution of a whole-box or split plan (capturing: inside a stream capture)
static lgf_status run_fp32(lgf_plan *p, const float *const *src, float *const *dst, cudaStream_t s, bool capturing)
{
    if (p->split) return run_split(p, src[0], dst[0], s, capturing ? nullptr : &p->prof);
    return run_poisson(p, src, dst, s, capturing);
}

lgf_status lgf_conv_execute(lgf_plan *p, const float *const *src, float *const *dst, void *stream)
{
    clear_error();
    LGF_CHECK_ARG(p && src && dst, "lgf_conv_execute: NULL argument");
    if (p->kind != LGF_KERNEL_LAPLACE7) {
        set_error("lgf_conv_execute: plan is not a Poisson plan (use ifactor_apply)");
        return LGF_ERR_STATE;
    }
    if (p->precision != 0) {
        set_error("lgf_conv_execute: FP64 plan (use lgf_conv_execute_f64)");
        return LGF_ERR_STATE;
    }
    if (p->sub) return lgf_conv_execute(p->sub, src, dst, stream);
    const size_t nsol = p->split ? 1 : p->solves.size();
    for (size_t i = 0; i < nsol; i++)
        LGF_CHECK_ARG(src[i] && dst[i], "lgf_conv_execute: NULL buffer for solve %zu", i);
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->use_graph || p->prof.on) return run_fp32(p, src, dst, s, false);
    // graph path: one captured launch sequence per distinct set of buffers
    std::vector<const void *> key;
    for (size_t i = 0; i < nsol; i++) {
        key.push_back(src[i]);
        key.push_back(dst[i]);
    }
    if (!p->graph || key != p->graph_key) {
        if (p->graph) {
            cudaGraphExecDestroy(p->graph);
            p->graph = nullptr;
        }
        cudaStream_t cs;
        LGF_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t gr = nullptr;
        lgf_status st = LGF_OK;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            set_error("stream capture failed to start");
            st = LGF_ERR_CUDA;
        } else {
            st = run_fp32(p, src, dst, cs, true);
            cudaError_t e = cudaStreamEndCapture(cs, &gr);
            if (st == LGF_OK && e != cudaSuccess) {
                set_error("stream capture failed: %s", cudaGetErrorString(e));
                st = LGF_ERR_CUDA;
            }
            if (st == LGF_OK && cudaGraphInstantiate(&p->graph, gr, 0) != cudaSuccess) {
                set_error("graph instantiation failed");
                st = LGF_ERR_CUDA;
                p->graph = nullptr;
            }
        }
        if (gr) cudaGraphDestroy(gr);
        cudaStreamDestroy(cs);
        if (st != LGF_OK) return st;
        p->graph_key = key;
    }
    LGF_CUDA_TRY(cudaGraphLaunch(p->graph, s));
    return LGF_OK;
}

lgf_status lgf_conv_execute_host(lgf_plan *p, const float *const *src, float *const *dst, void *stream)
{
    clear_error();
    LGF_CHECK_ARG(p && src && dst, "lgf_conv_execute_host: NULL argument");
    if (p->kind != LGF_KERNEL_LAPLACE7 || p->precision != 0) {
        set_error("lgf_conv_execute_host: plan is not a Poisson plan");
        return LGF_ERR_STATE;
    }
    if (p->sub) return lgf_conv_execute_host(p->sub, src, dst, stream);
    cudaStream_t s = (cudaStream_t)stream;
    if (p->split) {
        SplitPlan *sp = p->split;
        LGF_CHECK_ARG(src[0] && dst[0], "lgf_conv_execute_host: NULL buffer");
        const size_t B3 = 16 * 16 * 16;
        const size_t ns = (size_t)sp->nsrc * sp->ncomp * B3, nd = (size_t)sp->ndst * sp->ncomp * B3;
        LGF_CUDA_TRY(cudaMemcpyAsync(sp->d_stage_src, src[0], ns * sizeof(float), cudaMemcpyHostToDevice, s));
        LGF_TRY(run_split(p, sp->d_stage_src, sp->d_stage_dst, s, &p->prof));
        LGF_CUDA_TRY(cudaMemcpyAsync(dst[0], sp->d_stage_dst, nd * sizeof(float), cudaMemcpyDeviceToHost, s));
        return split_check(p, s);
    }
    std::vector<const float *> ds(p->solves.size());
    std::vector<float *> dd(p->solves.size());
    for (size_t i = 0; i < p->solves.size(); i++) {
        const PoissonSolve &q = p->solves[i];
        LGF_CHECK_ARG(src[i] && dst[i], "lgf_conv_execute_host: NULL buffer for solve %zu", i);
        ds[i] = q.d_stage_src;
        dd[i] = q.d_stage_dst;
    }
    const HostIO host{src, dst};
    // page-locked host buffers (every one of them): the copies and passes are
    // captured once per set of host pointers and replayed as one graph
    bool pinned = p->use_graph && !p->prof.on;
    for (size_t i = 0; pinned && i < p->solves.size(); i++) {
        for (const void *h : {(const void *)src[i], (const void *)dst[i]}) {
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, h) != cudaSuccess || at.type != cudaMemoryTypeHost) {
                cudaGetLastError();  // a pageable pointer may leave an error behind: clear it
                pinned = false;
            }
        }
    }
    if (!pinned) {
        LGF_TRY(run_poisson(p, ds.data(), dd.data(), s, false, &host));
        LGF_CUDA_TRY(cudaStreamSynchronize(s));
        return LGF_OK;
    }
    std::vector<const void *> key;
    for (size_t i = 0; i < p->solves.size(); i++) {
        key.push_back(src[i]);
        key.push_back(dst[i]);
    }
    if (!p->host_graph || key != p->host_graph_key) {
        if (p->host_graph) {
            cudaGraphExecDestroy(p->host_graph);
            p->host_graph = nullptr;
        }
        cudaStream_t cs;
        LGF_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t gr = nullptr;
        lgf_status st = LGF_OK;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            set_error("stream capture failed to start");
            st = LGF_ERR_CUDA;
        } else {
            st = run_poisson(p, ds.data(), dd.data(), cs, true, &host);
            cudaError_t e = cudaStreamEndCapture(cs, &gr);
            if (st == LGF_OK && e != cudaSuccess) {
                set_error("stream capture failed: %s", cudaGetErrorString(e));
                st = LGF_ERR_CUDA;
            }
            if (st == LGF_OK && cudaGraphInstantiate(&p->host_graph, gr, 0) != cudaSuccess) {
                set_error("graph instantiation failed");
                st = LGF_ERR_CUDA;
                p->host_graph = nullptr;
            }
        }
        if (gr) cudaGraphDestroy(gr);
        cudaStreamDestroy(cs);
        if (st != LGF_OK) return st;
        p->host_graph_key = key;
    }
    LGF_CUDA_TRY(cudaGraphLaunch(p->host_graph, s));
    LGF_CUDA_TRY(cudaStreamSynchronize(s));
    return LGF_OK;
}

}  // extern "C"

namespace lgf {
lgf_status ifactor_apply_io(lgf_plan *p, const IfIO &io, float *y, cudaStream_t s)
{
    if (!p || p->kind != LGF_KERNEL_IFACTOR) {
        set_error("integrating factor: plan was not built from an integrating-factor table");
        return LGF_ERR_STATE;
    }
    LGF_CHECK_ARG(io.x0 && y && io.x0 != y && io.x1 != y, "integrating factor: NULL or aliasing argument");
    return ifactor_launch_ex(p->ifp, p->ncomp, p->table->h_taps32.data(), io, y, s, &p->prof);
}
}  // namespace lgf

extern "C" {

lgf_status ifactor_apply(lgf_plan *p, const float *x, float *y, void *stream)
{
    clear_error();
    LGF_CHECK_ARG(p && x && y, "ifactor_apply: NULL argument");
    LGF_CHECK_ARG(x != y, "ifactor_apply: x and y must not alias");
    if (p->kind != LGF_KERNEL_IFACTOR) {
        set_error("ifactor_apply: plan was not built from an integrating-factor table");
        return LGF_ERR_STATE;
    }
    return ifactor_launch(p->ifp, p->ncomp, p->table->h_taps32.data(), x, y, (cudaStream_t)stream, &p->prof);
}

lgf_status lgf_residual_fp64(lgf_plan *p, int solve, const float *src, const float *dst, double *rel_residual,
                             void *stream)
{
    clear_error();
    LGF_CHECK_ARG(p && src && dst && rel_residual, "lgf_residual_fp64: NULL argument");
    if (p->sub) return lgf_residual_fp64(p->sub, solve, src, dst, rel_residual, stream);
    if (p->kind != LGF_KERNEL_LAPLACE7) {
        set_error("lgf_residual_fp64: not a Poisson plan");
        return LGF_ERR_STATE;
    }
    LGF_CHECK_ARG(solve >= 0 && solve < (int)p->solves.size(), "lgf_residual_fp64: solve %d out of range", solve);
    cudaStream_t s = (cudaStream_t)stream;
    LGF_CUDA_TRY(cudaMemsetAsync(p->d_acc, 0, 2 * sizeof(double), s));
    LGF_TRY(residual_launch(p->solves[solve], src, dst, p->d_acc, s));
    double h[2];
    LGF_CUDA_TRY(cudaMemcpyAsync(h, p->d_acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    LGF_CUDA_TRY(cudaStreamSynchronize(s));
    *rel_residual = h[1] > 0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
    return LGF_OK;
}

lgf_status lgf_plan_set_profiling(lgf_plan *p, int enable)
{
    clear_error();
    LGF_CHECK_ARG(p != nullptr && enable >= 0 && enable <= 2, "lgf_plan_set_profiling: bad argument");
    if (p->sub) return lgf_plan_set_profiling(p->sub, enable);
    if (enable == 2) p->prof.clear();
    p->prof.on = enable != 0;
    if (p->rk) {  // an RK plan also times the kernels of its Poisson and IF sub-plans
        LGF_TRY(lgf_plan_set_profiling(p->rk->poisson, enable));
        LGF_TRY(lgf_plan_set_profiling(p->rk->poisson3, enable));
        for (int i = 0; i < 3; i++)
            if (p->rk->if_owned[i]) LGF_TRY(lgf_plan_set_profiling(p->rk->ifp[i], enable));
    }
    return LGF_OK;
}

// RK plans: fold the sub-plans' totals into the plan's own records
static lgf_status merge_sub_profiles(lgf_plan *p)
{
    LGF_TRY(p->prof.collect());
    if (!p->rk) return LGF_OK;
    std::vector<lgf_plan *> subs = {p->rk->poisson, p->rk->poisson3};
    for (int i = 0; i < 3; i++)
        if (p->rk->if_owned[i]) subs.push_back(p->rk->ifp[i]);
    for (lgf_plan *sub : subs) {
        LGF_TRY(sub->prof.collect());
        for (auto &r : sub->prof.recs) {
            const int k = p->prof.rec_of(r.name.c_str());
            p->prof.recs[k].launches += r.launches;
            p->prof.recs[k].ms += r.ms;
        }
        sub->prof.recs.clear();
    }
    return LGF_OK;
}

lgf_status lgf_plan_kernel_count(lgf_plan *p, int *count)
{
    clear_error();
    LGF_CHECK_ARG(p && count, "lgf_plan_kernel_count: NULL argument");
    if (p->sub) return lgf_plan_kernel_count(p->sub, count);
    LGF_TRY(merge_sub_profiles(p));
    *count = (int)p->prof.recs.size();
    return LGF_OK;
}

lgf_status lgf_plan_kernel_times(lgf_plan *p, int i, const char **name, long long *launches, double *total_ms)
{
    clear_error();
    LGF_CHECK_ARG(p != nullptr, "lgf_plan_kernel_times: NULL plan");
    if (p->sub) return lgf_plan_kernel_times(p->sub, i, name, launches, total_ms);
    LGF_TRY(merge_sub_profiles(p));
    LGF_CHECK_ARG(i >= 0 && i < (int)p->prof.recs.size(), "lgf_plan_kernel_times: index %d out of range", i);
    if (name) *name = p->prof.recs[i].name.c_str();
    if (launches) *launches = p->prof.recs[i].launches;
    if (total_ms) *total_ms = p->prof.recs[i].ms;
    return LGF_OK;
}

void lgf_plan_destroy(lgf_plan *p) { free_plan(p); }

}  // extern "C"
