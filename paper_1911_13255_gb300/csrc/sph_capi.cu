// C-ABI of the sphfsi library (include/sphfsi.h): contexts of one or more
// independent instances, set-up, the per-step launch sequence a1..a8 and its
// CUDA-graph replay, state I/O.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <utility>
#include <unordered_map>
#include <vector>

#include "sph_common.cuh"
#include "sph_learn.cuh"
#include "sphfsi.h"

using namespace sph;

namespace {

// host staging and bookkeeping of one instance
// Allocator of the large host staging arrays: resize leaves the elements
// uninitialised (every element is written before it is read), so that no
// single-threaded zero fill precedes the parallel loops that write them.
template <typename T>
struct DefaultInit : std::allocator<T> {
    template <typename U>
    struct rebind {
        using other = DefaultInit<U>;
    };
    DefaultInit() = default;
    template <typename U>
    DefaultInit(const DefaultInit<U> &) noexcept {}
    template <typename U, typename... Args>
    void construct(U *p, Args &&...args)
    {
        if constexpr (sizeof...(Args) == 0) ::new ((void *)p) U;
        else ::new ((void *)p) U(std::forward<Args>(args)...);
    }
};
template <typename T>
using hvec = std::vector<T, DefaultInit<T>>;

// Contiguous chunks of a set-up loop over n items for the host threads: at
// most 16, and at least min_per items each.
int host_chunks(int64_t n, int64_t min_per)
{
    unsigned nt = std::thread::hardware_concurrency();
    if (nt == 0) nt = 1;
    if (nt > 16) nt = 16;
    const int64_t by_size = min_per > 0 ? (n + min_per - 1) / min_per : n;
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nt, by_size));
}

// body(k, lo, hi) for chunk k of `chunks` contiguous chunks [lo, hi) of
// [0, n), each on its own host thread (chunk 0 on the calling thread; a
// thread that cannot be started runs its chunk here).  The set-up loops
// write disjoint outputs per item, so the result does not depend on the
// split.  Returns false when a chunk threw (out of host memory): no
// exception leaves a worker thread.
template <typename F>
bool host_parallel(int64_t n, int chunks, F &&body)
{
    std::vector<char> bad(chunks > 1 ? chunks : 1, 0);
    auto run = [&](int k, int64_t lo, int64_t hi) {
        try {
            body(k, lo, hi);
        } catch (...) {
            bad[k] = 1;
        }
    };
    if (chunks <= 1) {
        run(0, (int64_t)0, n);
        return !bad[0];
    }
    std::vector<std::thread> th;
    try {
        th.reserve(chunks - 1);
    } catch (...) {
    }
    for (int k = 1; k < chunks; k++) {
        const int64_t lo = n * k / chunks, hi = n * (k + 1) / chunks;
        try {
            th.emplace_back([&run, k, lo, hi] { run(k, lo, hi); });
        } catch (...) {
            run(k, lo, hi);
        }
    }
    run(0, (int64_t)0, n / chunks);
    for (auto &t : th) t.join();
    for (char b : bad)
        if (b) return false;
    return true;
}

struct InstHost {
    sphfsi_params prm{};
    sphfsi_inflow inflow{};
    int64_t nf = 0, nw = 0, ns = 0;
    hvec<double> f_r, f_v, f_p;
    bool f_has_p = false, f_added = false, w_added = false, s_added = false;
    double f_dp = 0, f_rho0 = 1, f_c0 = 1, f_eta = 0;
    hvec<double> w_r, w_n;
    double w_dp = 0;
    std::vector<double> s_r0, s_v0, s_n0;
    std::vector<uint8_t> s_cons;
    std::vector<int> s_order;   // device (locality) index -> original solid index
    double s_dp = 0, s_rho0 = 1, s_E = 1, s_nu = 0.3;
    Inst d{};                   // descriptor as uploaded
};

}  // namespace

struct sphfsi_ctx {
    cudaStream_t st = nullptr;
    int dim = 2;
    int B = 1;
    int sel = 0;
    bool finalized = false;
    int K_fixed = 0;
    std::vector<InstHost> ih;
    // device
    Fluid F{};
    Walls W{};
    Solid S{};
    Batch bt{};
    Inst *d_inst = nullptr;
    Ctl *ctl = nullptr;
    std::vector<std::pair<void *, size_t>> allocs;   // every device allocation (pointer, bytes)
    // graph replay
    cudaGraphExec_t gexec = nullptr;
    double graph_dt = 0.0;
    int graph_K = -1;
    int graph_prof = -1;
    int solid_path = 0;
    int last_status = 0;
    bool failed = false;   // a bounded wait gave up (seen at a sync): no steps until a checkpoint is restored
    bool runaway = false;  // a step ended non-finite or run away (seen at a sync): likewise
    // per-stage CUDA events (sphfsi_set_profiling), by index: 0 start, 2
    // binning, 1 neighbour rows, 3 reinit, 5 momentum, 6 continuity (main
    // stream); 4 branch start, 7 coupling force done, 8 sub-steps done (side
    // stream); 9 end of step
    static constexpr int kStages = 8;
    static constexpr int kEvents = 10;
    bool profiling = false;
    cudaEvent_t ev[kEvents] = {};
    int kernels_per_step = 0;
    int max_reach = 1;   // largest cell reach of the instances (sphfsi_params::cell_reach)
    // side stream for the solid branch, which runs beside momentum and continuity
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // asynchronous read of the solid positions: each device slot's output
    // row (original order), and the gathered rows
    int *d_orow = nullptr;
    double *d_spos = nullptr;
    // learned sub-stepper (sphfsi_set_learned)
    sphfsi_mpnn *mpnn = nullptr;
};

// ---------------------------------------------------------------------------
namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? SPHFSI_OK : SPHFSI_E_CUDA; }

template <typename T>
int dalloc(sphfsi_ctx *c, T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    void *q = nullptr;
    if (cudaMalloc(&q, sizeof(T) * count) != cudaSuccess) {
        cudaGetLastError();
        return SPHFSI_E_NOMEM;
    }
    cudaMemsetAsync(q, 0, sizeof(T) * count, c->st);
    c->allocs.push_back({q, sizeof(T) * count});
    *p = (T *)q;
    return SPHFSI_OK;
}

#define TRY(x)                                              \
    do {                                                    \
        int _rc = (x);                                      \
        if (_rc) return _rc < -7 ? SPHFSI_E_CUDA : _rc;     \
    } while (0)

// copy n elements from a user pointer (host or device) into a host vector;
// host memory (pinned or not) is copied by the host threads
template <typename T, typename A>
int fetch(std::vector<T, A> &dst, const T *src, size_t n)
{
    dst.resize(n);
    if (n == 0) return SPHFSI_OK;
    if (!src) return SPHFSI_E_INVAL;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, src) == cudaSuccess &&
        (at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered)) {
        T *d = dst.data();
        host_parallel((int64_t)n, host_chunks((int64_t)n, (int64_t)1 << 18), [&](int, int64_t lo, int64_t hi) {
            std::memcpy(d + lo, src + lo, sizeof(T) * (size_t)(hi - lo));
        });   // memcpy does not throw
        return SPHFSI_OK;
    }
    cudaGetLastError();   // a pointer the runtime does not know is not an error here
    return cuda_rc(cudaMemcpy(dst.data(), src, sizeof(T) * n, cudaMemcpyDefault));
}

// copy a host buffer out to a user pointer (host or device)
template <typename T>
int deliver(T *dst, const std::vector<T> &src)
{
    if (!dst || src.empty()) return SPHFSI_OK;
    return cuda_rc(cudaMemcpy(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyDefault));
}

template <typename T, typename A>
int upload(sphfsi_ctx *c, T *dst, const std::vector<T, A> &src)
{
    if (src.empty()) return SPHFSI_OK;
    return cuda_rc(cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, c->st));
}

template <typename T>
int download(sphfsi_ctx *c, std::vector<T> &dst, const T *src, size_t n)
{
    dst.resize(n);
    if (n == 0) return SPHFSI_OK;
    int rc = cuda_rc(cudaMemcpyAsync(dst.data(), src, sizeof(T) * n, cudaMemcpyDeviceToHost, c->st));
    if (rc) return rc;
    return cuda_rc(cudaStreamSynchronize(c->st));
}

double wendland_W(int dim, double r, double h)
{
    const double pi = 3.14159265358979323846;
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double a = 1.0 - 0.5 * q;
    double alpha = dim == 2 ? 7.0 / (4.0 * pi * h * h) : 21.0 / (16.0 * pi * h * h * h);
    return alpha * a * a * a * a * (1.0 + 2.0 * q);
}

// lattice number density at spacing dp (self included), reading R16
double lattice_sigma0(int dim, double dp, double h)
{
    int K = (int)std::ceil(2.0 * h / dp) + 1;
    double s = 0.0;
    for (int i = -K; i <= K; i++)
        for (int j = -K; j <= K; j++) {
            if (dim == 2) {
                s += wendland_W(2, std::sqrt((double)(i * i + j * j)) * dp, h);
            } else {
                for (int k = -K; k <= K; k++) s += wendland_W(3, std::sqrt((double)(i * i + j * j + k * k)) * dp, h);
            }
        }
    return s;
}

// stage boundary: an event record when profiling (captured as an event node
// inside a graph thanks to cudaEventRecordExternal)
int mark(sphfsi_ctx *c, int k, cudaStream_t st)
{
    if (!c->profiling) return SPHFSI_OK;
    return cuda_rc(cudaEventRecordWithFlags(c->ev[k], st, cudaEventRecordExternal));
}
int mark(sphfsi_ctx *c, int k) { return mark(c, k, c->st); }

int enqueue_step(sphfsi_ctx *c, double dt)
{
    cudaStream_t st = c->st;
    const int D = c->dim;
    TRY(mark(c, 0));
    // step control (dt_F, K, reinit flag per instance), a3 normal update,
    // a1 + a2: inflow, fluid first half drift; fluid (r^{n+1/2}) and solid
    // (r^n) binning, counting sort and FP32 records
    TRY(launch_bin_all(c->bt, c->F, c->S, D, 1, dt > 0.0 ? dt : 0.0, c->K_fixed, st));
    TRY(mark(c, 2));
    // neighbour rows of the pair loops (rebuild steps, when on)
    TRY(launch_pairlist(c->bt, c->F, c->W, c->S, D, st));
    TRY(mark(c, 1));
    // a3: density reinitialisation (no-op on other steps)
    TRY(launch_reinit(c->bt, c->F, c->W, c->S, D, st));
    TRY(mark(c, 3));
    // The solid branch (a5, then a7 + a8) depends only on the records written
    // so far, so it runs on the side stream while the main stream does a4
    // and a6; the two join before finish.
    if (c->S.n) {
        TRY(cuda_rc(cudaEventRecord(c->fork_ev, st)));
        TRY(cuda_rc(cudaStreamWaitEvent(c->side, c->fork_ev, 0)));
        TRY(mark(c, 4, c->side));
        TRY(launch_solid_fluid_force(c->bt, c->F, c->S, D, c->side));
        if (c->S.learned) {
            TRY(launch_learn_features(c->bt, c->S, mpnn_input(c->mpnn), D, c->side));
            TRY(mpnn_forward_async(c->mpnn));
            TRY(launch_learn_candidate(c->bt, c->S, mpnn_output(c->mpnn), D, c->side));
        }
        TRY(mark(c, 7, c->side));
        TRY(launch_solid_substeps(c->bt, c->S, c->ih[0].d.P, D, &c->solid_path, c->side));
        TRY(mark(c, 8, c->side));
        TRY(cuda_rc(cudaEventRecord(c->join_ev, c->side)));
    }
    TRY(launch_momentum(c->bt, c->F, c->W, c->S, D, st));
    TRY(mark(c, 5));
    TRY(launch_density(c->bt, c->F, c->W, c->S, D, st));
    TRY(mark(c, 6));
    if (c->S.n) TRY(cuda_rc(cudaStreamWaitEvent(st, c->join_ev, 0)));
    TRY(launch_finish(c->bt, c->S.learned, c->F.gbar, c->F, st));
    TRY(mark(c, 9));
    // kernels of this library per step (memsets excluded)
    c->kernels_per_step = 4 + bin_kernels(c->F) + (c->S.n ? 2 : 0) + (c->F.list && c->F.n ? 1 : 0) +
                          (c->S.learned ? 5 + mpnn_kernels_per_forward() : 0);
    return cuda_rc(cudaGetLastError());
}

// the next step rebuilds the held pair configuration (after a state change)
int request_rebuild(sphfsi_ctx *c)
{
    return cuda_rc(cudaMemsetAsync(c->F.held, 0xff, sizeof(int), c->st));
}

int check_ctx(sphfsi_ctx *c, bool need_final)
{
    if (!c) return SPHFSI_E_INVAL;
    if (need_final && !c->finalized) return SPHFSI_E_STATE;
    if (!need_final && c->finalized) return SPHFSI_E_STATE;
    return SPHFSI_OK;
}

void deinterleave(const std::vector<double> &src, int dim, int64_t n, std::vector<double> out[3])
{
    for (int k = 0; k < 3; k++) out[k].assign(n, 0.0);
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < dim; k++) out[k][i] = src[i * dim + k];
}

int check_params(const sphfsi_params *p)
{
    if (!p || (p->dim != 2 && p->dim != 3)) return SPHFSI_E_INVAL;
    if (p->periodic_x && !(p->Lx > 0.0)) return SPHFSI_E_INVAL;
    for (int k = 0; k < p->dim; k++)
        if (!(p->domain_hi[k] > p->domain_lo[k])) return SPHFSI_E_INVAL;
    return SPHFSI_OK;
}

// grid and constants of one instance (cells of edge >= 2 h_F)
int make_inst(const InstHost &h, int D, Inst &d)
{
    const double hF = 1.3 * h.f_dp;
    Grid &g = d.g;
    std::memset(&g, 0, sizeof(g));
    const int R = h.prm.cell_reach == 2 ? 2 : 1;   // cells of >= 2 h_F / R; neighbours within R cells
    if (h.prm.cell_reach < 0 || h.prm.cell_reach > 2) return SPHFSI_E_INVAL;
    g.reach = R;
    int64_t ncell = 1;
    for (int k = 0; k < 3; k++) {
        if (k >= D) {
            g.lo[k] = 0.0;
            g.cs[k] = 1.0;
            g.csf[k] = 1.0f;
            g.cslo[k] = 0.0f;
            g.nc[k] = 1;
            continue;
        }
        double lo = h.prm.domain_lo[k], L = h.prm.domain_hi[k] - lo;
        if (k == 0 && h.prm.periodic_x) {
            lo = h.prm.x_lo;
            L = h.prm.Lx;
        }
        int64_t n = (int64_t)std::floor(L / (2.0 * hF / R));
        if (n < 1) n = 1;
        if (k == 0 && h.prm.periodic_x && n < 2 * R + 1) return SPHFSI_E_INVAL;
        g.lo[k] = lo;
        g.nc[k] = (int)n;
        g.cs[k] = L / (double)n;
        g.csf[k] = (float)g.cs[k];
        g.cslo[k] = (float)(g.cs[k] - (double)g.csf[k]);
        ncell *= n;
        if (ncell > ((int64_t)1 << 28)) return SPHFSI_E_CAPACITY;
    }
    g.ncell = (int)ncell;
    g.periodic_x = h.prm.periodic_x;
    g.x_lo = h.prm.x_lo;
    g.Lx = h.prm.Lx;
    Phys &P = d.P;
    std::memset(&P, 0, sizeof(P));
    const double pi = 3.14159265358979323846;
    P.dim = D;
    for (int k = 0; k < 3; k++) P.g[k] = (float)h.prm.gravity[k];
    P.rho0 = (float)h.f_rho0;
    P.c0 = (float)h.f_c0;
    P.eta = (float)h.f_eta;
    P.hF = (float)hF;
    P.inv_hF = (float)(1.0 / hF);
    P.rc2F = (float)(4.0 * hF * hF);
    P.rc2F_d = 4.0 * hF * hF;
    double alpha = D == 2 ? 7.0 / (4.0 * pi * hF * hF) : 21.0 / (16.0 * pi * hF * hF * hF);
    P.WcF = (float)alpha;
    P.dWcF = (float)(-5.0 * alpha / hF);
    double VF = std::pow(h.f_dp, D);
    P.mF = (float)(h.f_rho0 * VF);
    P.p_coef = (float)(h.f_rho0 * h.f_c0 * h.f_c0 / 7.0);
    P.inv_p_coef = (float)(7.0 / (h.f_rho0 * h.f_c0 * h.f_c0));
    P.hreg = (float)(0.01 * hF);
    P.sigma0 = (float)lattice_sigma0(D, h.f_dp, hF);
    P.sigma0_d = lattice_sigma0(D, h.f_dp, hF);
    P.alphaF_d = alpha;
    P.ihF_hi = (float)(1.0 / hF);
    P.ihF_lo = (float)(1.0 / hF - (double)P.ihF_hi);
    double VW = h.w_dp > 0 ? std::pow(h.w_dp, D) : VF;
    double VS = h.s_dp > 0 ? std::pow(h.s_dp, D) : VF;
    P.VW = (float)VW;
    P.VS = (float)VS;
    P.VW_VF = (float)(VW / VF);
    P.VS_VF = (float)(VS / VF);
    P.VW_VF_d = VW / VF;
    P.VS_VF_d = VS / VF;
    P.free_surface = h.prm.free_surface;
    P.hF_d = hF;
    P.c0_d = h.f_c0;
    P.eta_d = h.f_eta;
    P.rho0_d = h.f_rho0;
    if (h.ns > 0) {
        double mu = h.s_E / (2.0 * (1.0 + h.s_nu));   // reading R10
        double lam = 2.0 * mu * h.s_nu / (1.0 - 2.0 * h.s_nu);
        P.rhoS = (float)h.s_rho0;
        P.mS = (float)(h.s_rho0 * VS);
        P.mu = (float)mu;
        P.lam = (float)lam;
        P.hS = (float)(1.3 * h.s_dp);
        P.hS_d = 1.3 * h.s_dp;
        P.cS_d = std::sqrt(h.s_E / (3.0 * (1.0 - 2.0 * h.s_nu)) / h.s_rho0);
    }
    P.inflow_on = h.inflow.on;
    P.inflow_profile = h.inflow.profile;
    P.in_w = h.inflow.width;
    P.in_y0 = h.inflow.y0;
    P.in_H = h.inflow.H;
    P.in_U = h.inflow.U;
    P.in_tramp = h.inflow.t_ramp;
    P.in_T = h.inflow.period;
    P.in_wo = h.inflow.womersley;
    P.in_z0 = h.inflow.z0;
    P.in_Hz = h.inflow.Hz;
    return SPHFSI_OK;
}

// Static reference neighbour list of every body (slots in device order,
// global): pairs a != b of one instance with |r0_a - r0_b|^2 < (2 h_S)^2 in
// FP64, computed as dx dx + dy dy (+ dz dz) without contraction, found
// through a cell grid of edge 2 h_S over the body; each row ascending.
int body_neighbours(sphfsi_ctx *c, std::vector<int> &ptr, std::vector<int> &idx)
{
    const int D = c->dim;
    ptr.assign(1, 0);
    idx.clear();
    for (const InstHost &h : c->ih) {
        const int n = (int)h.ns, s0 = h.d.s0;
        if (n == 0) continue;
        const double hS = 1.3 * h.s_dp, rc2 = 4.0 * hS * hS, edge = 2.0 * hS;
        double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int k = 0; k < D; k++) {
            lo[k] = hi[k] = h.s_r0[k];
            for (int a = 0; a < n; a++) {
                lo[k] = std::min(lo[k], h.s_r0[(size_t)a * D + k]);
                hi[k] = std::max(hi[k], h.s_r0[(size_t)a * D + k]);
            }
        }
        int nc[3] = {1, 1, 1};
        for (int k = 0; k < D; k++) nc[k] = (int)std::floor((hi[k] - lo[k]) / edge) + 1;
        auto cell = [&](int a, int k) {
            int q = (int)std::floor((h.s_r0[(size_t)a * D + k] - lo[k]) / edge);
            return q < 0 ? 0 : (q >= nc[k] ? nc[k] - 1 : q);
        };
        const size_t ncl = (size_t)nc[0] * nc[1] * nc[2];
        std::vector<int> start(ncl + 1, 0), items(n), cid(n);
        for (int a = 0; a < n; a++) {
            cid[a] = cell(a, 0) + nc[0] * (cell(a, 1) + nc[1] * (D == 3 ? cell(a, 2) : 0));
            start[cid[a] + 1]++;
        }
        for (size_t q = 0; q < ncl; q++) start[q + 1] += start[q];
        {
            std::vector<int> cur(start.begin(), start.end() - 1);
            for (int a = 0; a < n; a++) items[cur[cid[a]]++] = a;
        }
        // rows over the host threads, each chunk into its own lists, then
        // concatenated in particle order
        const int nch = host_chunks(n, 1024);
        std::vector<std::vector<int>> cidx(nch), clen(nch);
        const bool ok = host_parallel(n, nch, [&](int ch, int64_t lo_a, int64_t hi_a) {
            std::vector<int> row;
            for (int a = (int)lo_a; a < (int)hi_a; a++) {
                row.clear();
                const int cx = cell(a, 0), cy = cell(a, 1), cz = D == 3 ? cell(a, 2) : 0;
                for (int z = std::max(cz - 1, 0); z <= std::min(cz + 1, nc[2] - 1); z++)
                    for (int y = std::max(cy - 1, 0); y <= std::min(cy + 1, nc[1] - 1); y++)
                        for (int x = std::max(cx - 1, 0); x <= std::min(cx + 1, nc[0] - 1); x++) {
                            const int q = x + nc[0] * (y + nc[1] * z);
                            for (int t = start[q]; t < start[q + 1]; t++) {
                                const int b = items[t];
                                if (b == a) continue;
                                double r2 = 0.0;
                                for (int k = 0; k < D; k++) {
                                    const double d = h.s_r0[(size_t)a * D + k] - h.s_r0[(size_t)b * D + k];
                                    const double dd = d * d;
                                    r2 = r2 + dd;
                                }
                                if (r2 < rc2) row.push_back(s0 + b);
                            }
                        }
                std::sort(row.begin(), row.end());
                cidx[ch].insert(cidx[ch].end(), row.begin(), row.end());
                clen[ch].push_back((int)row.size());
            }
        });
        if (!ok) return SPHFSI_E_NOMEM;
        for (int ch = 0; ch < nch; ch++) {
            idx.insert(idx.end(), cidx[ch].begin(), cidx[ch].end());
            for (int len : clen[ch]) ptr.push_back(ptr.back() + len);
        }
    }
    return SPHFSI_OK;
}

// Locality order of a body on the device: lexicographic on the lattice index
// along the axes sorted by decreasing extent, so that a particle's neighbours
// sit within a few rows of it and mostly in the same CTA of the cluster
// sub-step kernels.  Permutes the staged arrays in place.
void locality_order(InstHost &h, int D)
{
    const int n = (int)h.ns;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int a = 0; a < n; a++)
        for (int k = 0; k < D; k++) {
            lo[k] = std::min(lo[k], h.s_r0[(size_t)a * D + k]);
            hi[k] = std::max(hi[k], h.s_r0[(size_t)a * D + k]);
        }
    int ax[3] = {0, 1, 2};
    std::sort(ax, ax + D, [&](int p, int q) { return hi[p] - lo[p] > hi[q] - lo[q]; });
    std::vector<std::array<long long, 4>> key(n);
    for (int a = 0; a < n; a++) {
        for (int k = 0; k < 3; k++)
            key[a][k] = k < D ? std::llround((h.s_r0[(size_t)a * D + ax[k]] - lo[ax[k]]) / h.s_dp) : 0;
        key[a][3] = a;
    }
    std::sort(key.begin(), key.end());
    h.s_order.resize(n);
    for (int a = 0; a < n; a++) h.s_order[a] = (int)key[a][3];
    auto perm_rows = [&](auto &v, int w) {
        auto t = v;
        for (int a = 0; a < n; a++)
            for (int j = 0; j < w; j++) t[(size_t)a * w + j] = v[(size_t)h.s_order[a] * w + j];
        v.swap(t);
    };
    perm_rows(h.s_r0, D);
    perm_rows(h.s_v0, D);
    perm_rows(h.s_n0, D);
    perm_rows(h.s_cons, 1);
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

const char *sphfsi_strerror(int code)
{
    switch (code) {
    case SPHFSI_OK: return "ok";
    case SPHFSI_E_INVAL: return "invalid argument";
    case SPHFSI_E_NOMEM: return "device allocation failed";
    case SPHFSI_E_CUDA: return "CUDA runtime error";
    case SPHFSI_E_STATE: return "call out of order";
    case SPHFSI_E_UNSTABLE: return "run-away (non-finite) state detected on the device";
    case SPHFSI_E_TIMEOUT: return "bounded device wait timed out";
    case SPHFSI_E_CAPACITY: return "problem exceeds a device limit";
    default: return "unknown error";
    }
}

int sphfsi_create_batch(sphfsi_ctx **out, int32_t n, const sphfsi_params *p, void *cuda_stream)
{
    if (!out || !p || n < 1 || n > (1 << 20)) return SPHFSI_E_INVAL;
    *out = nullptr;
    for (int b = 0; b < n; b++) {
        TRY(check_params(p + b));
        if (p[b].dim != p[0].dim) return SPHFSI_E_INVAL;
    }
    sphfsi_ctx *c = new (std::nothrow) sphfsi_ctx();
    if (!c) return SPHFSI_E_NOMEM;
    c->ih.resize(n);
    for (int b = 0; b < n; b++) c->ih[b].prm = p[b];
    c->B = n;
    c->dim = p[0].dim;
    c->st = (cudaStream_t)cuda_stream;
    *out = c;
    return SPHFSI_OK;
}

int sphfsi_create(sphfsi_ctx **out, const sphfsi_params *p, void *cuda_stream)
{
    return sphfsi_create_batch(out, 1, p, cuda_stream);
}

int sphfsi_select(sphfsi_ctx *c, int32_t inst)
{
    if (!c || inst < 0 || inst >= c->B) return SPHFSI_E_INVAL;
    c->sel = inst;
    return SPHFSI_OK;
}

int sphfsi_add_fluid(sphfsi_ctx *c, int64_t n, const double *r, const double *v, const double *p_init, double dp,
                     double rho0, double c0, double eta)
{
    TRY(check_ctx(c, false));
    InstHost &h = c->ih[c->sel];
    if (h.f_added || n < 0 || n > (int64_t)1 << 30 || !(dp > 0) || !(rho0 > 0) || !(c0 > 0) || eta < 0)
        return SPHFSI_E_INVAL;
    if (n > 0 && (!r || !v)) return SPHFSI_E_INVAL;
    TRY(fetch(h.f_r, r, (size_t)n * c->dim));
    TRY(fetch(h.f_v, v, (size_t)n * c->dim));
    h.f_has_p = p_init != nullptr;
    if (p_init) TRY(fetch(h.f_p, p_init, (size_t)n));
    h.nf = n;
    h.f_dp = dp;
    h.f_rho0 = rho0;
    h.f_c0 = c0;
    h.f_eta = eta;
    h.f_added = true;
    return SPHFSI_OK;
}

int sphfsi_set_walls(sphfsi_ctx *c, int64_t n, const double *r, const double *nrm, double dp)
{
    TRY(check_ctx(c, false));
    InstHost &h = c->ih[c->sel];
    if (h.w_added || n < 0 || n > (int64_t)1 << 30 || !(dp > 0)) return SPHFSI_E_INVAL;
    if (n > 0 && (!r || !nrm)) return SPHFSI_E_INVAL;
    TRY(fetch(h.w_r, r, (size_t)n * c->dim));
    TRY(fetch(h.w_n, nrm, (size_t)n * c->dim));
    h.nw = n;
    h.w_dp = dp;
    h.w_added = true;
    return SPHFSI_OK;
}

int sphfsi_add_solid(sphfsi_ctx *c, int64_t n, const double *r0, const double *v0, const double *n0,
                     const uint8_t *constrained, double dp, double rho0, double E, double nu)
{
    TRY(check_ctx(c, false));
    InstHost &h = c->ih[c->sel];
    if (h.s_added || n < 0 || n > (int64_t)1 << 26 || !(dp > 0) || !(rho0 > 0) || !(E > 0) || !(nu > -1.0) ||
        !(nu < 0.5))
        return SPHFSI_E_INVAL;
    if (n > 0 && (!r0 || !v0 || !n0 || !constrained)) return SPHFSI_E_INVAL;
    TRY(fetch(h.s_r0, r0, (size_t)n * c->dim));
    TRY(fetch(h.s_v0, v0, (size_t)n * c->dim));
    TRY(fetch(h.s_n0, n0, (size_t)n * c->dim));
    TRY(fetch(h.s_cons, constrained, (size_t)n));
    h.ns = n;
    h.s_dp = dp;
    h.s_rho0 = rho0;
    h.s_E = E;
    h.s_nu = nu;
    h.s_added = true;
    return SPHFSI_OK;
}

int sphfsi_set_inflow(sphfsi_ctx *c, const sphfsi_inflow *f)
{
    TRY(check_ctx(c, false));
    if (!f || (f->on && (!(f->width > 0) || f->profile < 0 || f->profile > 3 ||
                         (f->profile != 1 && !(f->H > 0)) ||
                         (f->profile == 2 && (!(f->period > 0) || !(f->womersley > 0))) ||
                         (f->profile == 3 && (!(f->Hz > 0) || !std::isfinite(f->z0))))))
        return SPHFSI_E_INVAL;
    c->ih[c->sel].inflow = *f;
    return SPHFSI_OK;
}

// Halo maps of the 2-D cluster kernel's push form.  A body's particles are
// split into CTAs of kSolidCta in device (locality) order.  For every static
// neighbour entry q of particle a: the slot in CTA(a) where the neighbour's
// stress and velocity are found (its own slot when it lives in CTA(a), else a
// halo slot kSolidCta + h, h in order of first use); for every particle:
// the (CTA, halo slot) copies other CTAs hold of it, which it writes after
// each update.  push_ok = 0 when a halo or a push list exceeds kHaloMax or
// kPushMax (the kernel then reads neighbours across the cluster instead).
int halo_maps(sphfsi_ctx *c, const std::vector<int> &ptr, const std::vector<int> &nbi)
{
    Solid &S = c->S;
    const int64_t ns = S.n;
    std::vector<int> slot(nbi.size(), 0);
    std::vector<std::vector<int2>> pushes(ns);
    std::vector<int> halo_n(c->ih.size() * 16, 0);
    bool ok = true;
    // one-barrier form: per (instance, CTA) its halo particles with their
    // entries' velocity slots, and every particle's velocity copies
    std::vector<int> h1_ptr(c->ih.size() * 16 + 1, 0), h1_part, h1_eptr(1, 0), h1_vslot;
    std::vector<std::vector<int2>> push2(ns);
    bool one_ok = true;
    for (size_t bi = 0; bi < c->ih.size(); bi++) {
        auto &h = c->ih[bi];
        const int s0 = h.d.s0, n = h.d.ns;
        const int ctas = (n + kSolidCta - 1) / kSolidCta;
        std::vector<std::vector<int>> halo_of(ctas);                    // local particle per halo slot
        std::vector<std::unordered_map<int, int>> where(ctas);          // local particle -> halo slot
        for (int la = 0; la < n; la++) {
            const int r = la / kSolidCta;
            for (int q = ptr[s0 + la]; q < ptr[s0 + la + 1]; q++) {
                const int lb = nbi[q] - s0;
                if (lb / kSolidCta == r) {
                    slot[q] = lb % kSolidCta;
                    continue;
                }
                auto it = where[r].find(lb);
                if (it == where[r].end()) {
                    const int hs = kSolidCta + (int)halo_of[r].size();
                    it = where[r].emplace(lb, hs).first;
                    halo_of[r].push_back(lb);
                }
                slot[q] = it->second;
            }
        }
        for (int r = 0; r < ctas; r++) {
            if ((int)halo_of[r].size() > kHaloMax || r >= 16) ok = false;
            else halo_n[bi * 16 + r] = (int)halo_of[r].size();
            for (size_t k = 0; k < halo_of[r].size(); k++)
                pushes[s0 + halo_of[r][k]].push_back(make_int2(r, kSolidCta + (int)k));
        }
        // the velocity copies of CTA r: its halo in the same slots, then the
        // other CTAs' neighbours of its halo particles, in order of first use
        for (int r = 0; r < ctas && r < 16; r++) {
            std::vector<int> vh = halo_of[r];
            std::unordered_map<int, int> at = where[r];
            if ((int)halo_of[r].size() > kSolidCta) one_ok = false;
            for (int lb : halo_of[r]) {
                h1_part.push_back(s0 + lb);
                for (int q = ptr[s0 + lb]; q < ptr[s0 + lb + 1]; q++) {
                    const int lc = nbi[q] - s0;
                    if (lc / kSolidCta == r) {
                        h1_vslot.push_back(lc % kSolidCta);
                        continue;
                    }
                    auto it = at.find(lc);
                    if (it == at.end()) {
                        it = at.emplace(lc, kSolidCta + (int)vh.size()).first;
                        vh.push_back(lc);
                    }
                    h1_vslot.push_back(it->second);
                }
                h1_eptr.push_back((int)h1_vslot.size());
            }
            h1_ptr[bi * 16 + r + 1] = (int)h1_part.size();
            if ((int)vh.size() > kHaloMax) one_ok = false;
            for (size_t k = 0; k < vh.size(); k++) push2[s0 + vh[k]].push_back(make_int2(r, kSolidCta + (int)k));
        }
        for (int r = ctas; r < 16; r++) h1_ptr[bi * 16 + r + 1] = (int)h1_part.size();
        if (ctas > 16) one_ok = false;
    }
    std::vector<int> pptr(ns + 1, 0);
    std::vector<int2> pl;
    for (int64_t a = 0; a < ns; a++) {
        if ((int)pushes[a].size() > kPushMax) ok = false;
        pptr[a + 1] = pptr[a] + (int)pushes[a].size();
        pl.insert(pl.end(), pushes[a].begin(), pushes[a].end());
    }
    if (pl.empty()) pl.push_back(make_int2(0, 0));
    std::vector<int> p2ptr(ns + 1, 0);
    std::vector<int2> p2;
    for (int64_t a = 0; a < ns; a++) {
        if ((int)push2[a].size() > kPushMax) one_ok = false;
        p2ptr[a + 1] = p2ptr[a] + (int)push2[a].size();
        p2.insert(p2.end(), push2[a].begin(), push2[a].end());
    }
    if (p2.empty()) p2.push_back(make_int2(0, 0));
    if (h1_part.empty()) h1_part.push_back(0);
    if (h1_vslot.empty()) h1_vslot.push_back(0);
    TRY(dalloc(c, &S.h1_ptr, h1_ptr.size()));
    TRY(upload(c, S.h1_ptr, h1_ptr));
    TRY(dalloc(c, &S.h1_part, h1_part.size()));
    TRY(upload(c, S.h1_part, h1_part));
    TRY(dalloc(c, &S.h1_eptr, h1_eptr.size()));
    TRY(upload(c, S.h1_eptr, h1_eptr));
    TRY(dalloc(c, &S.h1_vslot, h1_vslot.size()));
    TRY(upload(c, S.h1_vslot, h1_vslot));
    TRY(dalloc(c, &S.push2_ptr, p2ptr.size()));
    TRY(upload(c, S.push2_ptr, p2ptr));
    TRY(dalloc(c, &S.push2, p2.size()));
    TRY(upload(c, S.push2, p2));
    S.one_ok = one_ok && ok ? 1 : 0;
    TRY(dalloc(c, &S.nb_slot, slot.size()));
    TRY(upload(c, S.nb_slot, slot));
    TRY(dalloc(c, &S.push_ptr, pptr.size()));
    TRY(upload(c, S.push_ptr, pptr));
    TRY(dalloc(c, &S.push, pl.size()));
    TRY(upload(c, S.push, pl));
    TRY(dalloc(c, &S.halo_n, halo_n.size()));
    TRY(upload(c, S.halo_n, halo_n));
    S.push_ok = ok ? 1 : 0;
    return SPHFSI_OK;
}

int sphfsi_finalize(sphfsi_ctx *c)
{
    TRY(check_ctx(c, false));
    const int D = c->dim, B = c->B;
    // ---- per-instance descriptors and offsets
    int64_t nf = 0, nw = 0, ns = 0, ncell = 0;
    int max_ns = 0;
    for (int b = 0; b < B; b++) {
        InstHost &h = c->ih[b];
        if (!h.f_added) return SPHFSI_E_STATE;
        TRY(make_inst(h, D, h.d));
        c->max_reach = std::max(c->max_reach, h.d.g.reach);
        h.d.f0 = (int)nf;
        h.d.nf = (int)h.nf;
        h.d.w0 = (int)nw;
        h.d.nw = (int)h.nw;
        h.d.s0 = (int)ns;
        h.d.ns = (int)h.ns;
        h.d.c0 = (int)ncell;
        nf += h.nf;
        nw += h.nw;
        ns += h.ns;
        ncell += h.d.g.ncell;
        max_ns = std::max(max_ns, (int)h.ns);
        if (nf > ((int64_t)1 << 30) || nw > ((int64_t)1 << 30) || ns > ((int64_t)1 << 28) ||
            ncell > ((int64_t)1 << 29))
            return SPHFSI_E_CAPACITY;
        if (h.ns > 0) locality_order(h, D);
    }
    TRY(dalloc(c, &c->ctl, B));
    TRY(dalloc(c, &c->d_inst, B));
    // ---- fluid
    Fluid &F = c->F;
    F.n = (int)nf;
    // small problems are latency-bound: 8 lanes per target and direct pair
    // evaluation (dam break: 0.105 -> 0.102 ms per step); large 2-D problems
    // are issue-bound: 4 lanes and compacted pairs; 3-D: 8 lanes below 200 000
    // fluid particles, else 4, direct pairs
    const bool small = nf + ns < 262144;
    F.lanes = D == 2 ? (small ? 8 : 4) : (nf < 200000 ? 8 : 4);
    F.block = 128;
    F.compact = D == 2 && !small ? 1 : 0;
    F.tile = 0;
    // records from the cell groups for small problems (one launch fewer),
    // one thread per slot for large ones (no idle lanes)
    F.split_records = small ? 0 : 1;
    // the cooperative single-kernel binning (records form 2) measured slower
    // than the four kernels with programmatic launches (dam break: binning
    // 35.4 vs 31.2 us): off by default
    F.bin_fused = 0;
    // neighbour cells a row at a time where latency, not issue, bounds the loops
    // (rows and tiles are built for cells of >= 2 h_F)
    F.rows = small && c->max_reach == 1 ? 1 : 0;
    F.reach = c->max_reach;
    // tiles: T cells of a grid row per block (16 in 2-D, 4 in 3-D); the
    // staging area holds about three times the mean neighbourhood
    {
        const int T = D == 2 ? 16 : 4;
        std::vector<int4> tiles;
        for (int b = 0; b < B; b++) {
            const Grid &g = c->ih[b].d.g;
            for (int z = 0; z < g.nc[2]; z++)
                for (int y = 0; y < g.nc[1]; y++)
                    for (int x = 0; x < g.nc[0]; x += T)
                        tiles.push_back(make_int4(b, c->ih[b].d.c0 + x + g.nc[0] * (y + g.nc[1] * z),
                                                  std::min(T, g.nc[0] - x), 0));
        }
        F.ntiles = (int)tiles.size();
        F.tile_cap = D == 2 ? 1024 : 2048;
        TRY(dalloc(c, &F.tiles, tiles.size()));
        TRY(upload(c, F.tiles, tiles));
    }
    for (int k = 0; k < 2; k++) {
        FluidState &S = F.s[k];
        TRY(dalloc(c, &S.x, nf));
        TRY(dalloc(c, &S.y, nf));
        TRY(dalloc(c, &S.z, D == 3 ? nf : 1));
        TRY(dalloc(c, &S.vx, nf));
        TRY(dalloc(c, &S.vy, nf));
        TRY(dalloc(c, &S.vz, D == 3 ? nf : 1));
        TRY(dalloc(c, &S.drho, nf));
        TRY(dalloc(c, &S.rhodot, nf));
        TRY(dalloc(c, &S.id, nf));
        if (D == 2) S.z = nullptr, S.vz = nullptr;
    }
    TRY(dalloc(c, &F.inst, nf));
    TRY(dalloc(c, &F.P4, nf));
    TRY(dalloc(c, &F.V4, nf));
    TRY(dalloc(c, &F.W4, nf));
    TRY(dalloc(c, &F.L4, nf));
    TRY(dalloc(c, &F.dvdt, (size_t)nf * D));
    TRY(dalloc(c, &F.key, nf));
    TRY(dalloc(c, &F.perm, nf));
    TRY(dalloc(c, &F.sperm, nf));
    TRY(dalloc(c, &F.cell_of, nf));
    TRY(dalloc(c, &F.cstart, (size_t)ncell + 1));
    TRY(dalloc(c, &F.ccount, ncell));
    TRY(dalloc(c, &F.live, 2 * (size_t)ncell));
    TRY(dalloc(c, &F.nlive, 1));
    {
        // tiles of the histogram scan, segment by segment (fluid of every
        // instance, then solid)
        std::vector<int2> tiles;
        const int sets = ns > 0 ? 2 : 1, tc = scan_tile_cells();
        for (int set = 0; set < sets; set++)
            for (int b = 0; b < B; b++) {
                const int nt = (c->ih[b].d.g.ncell + tc - 1) / tc;
                for (int k = 0; k < nt; k++) tiles.push_back(make_int2(set * B + b, k));
            }
        F.nscan_tiles = (int)tiles.size();
        TRY(dalloc(c, &F.scan_tiles, tiles.size()));
        TRY(upload(c, F.scan_tiles, tiles));
        TRY(dalloc(c, &F.scan_status, tiles.size()));
        TRY(dalloc(c, &F.scan_ctl, 2));
    }
    TRY(dalloc(c, &F.bsum, 4096));
    TRY(dalloc(c, &F.gbar, 2));
    // neighbour rows (tuned): about 20 (2-D) or 80 (3-D) neighbours per fluid
    // particle on a lattice, wall neighbours included.  On by default for
    // large 3-D problems (3-D duct, 3M fluid: momentum 6.2 -> 2.4 ms,
    // continuity 4.9 -> 1.65 ms for a 2.4 ms row build); off for 2-D, where
    // the row build costs more than it saves (dam break 0.100 -> 0.107 ms)
    F.list = D == 3 && !small ? 1 : 0;
    if (F.list) F.compact = 0;
    F.list_lanes = D == 2 ? 8 : 1;
    F.list_cap = D == 2 ? 64 : 128;
    TRY(dalloc(c, &F.nbl, (size_t)nf * F.list_cap));
    TRY(dalloc(c, &F.nbc, nf));
    // held pair configuration: off (rebuilt every step); the first step builds it
    F.held_n = 1;
    TRY(dalloc(c, &F.held, 3));
    TRY(upload(c, F.held, std::vector<int>{1, 0, 0}));
    // ---- walls
    Walls &W = c->W;
    W.n = (int)nw;
    TRY(dalloc(c, &W.inst, nw));
    TRY(dalloc(c, &W.x, nw));
    TRY(dalloc(c, &W.y, nw));
    TRY(dalloc(c, &W.z, D == 3 ? nw : 1));
    TRY(dalloc(c, &W.nx, nw));
    TRY(dalloc(c, &W.ny, nw));
    TRY(dalloc(c, &W.nz, D == 3 ? nw : 1));
    if (D == 2) W.z = nullptr, W.nz = nullptr;
    TRY(dalloc(c, &W.A4, nw));
    TRY(dalloc(c, &W.N4, nw));
    TRY(dalloc(c, &W.L4, nw));
    TRY(dalloc(c, &W.key, nw));
    TRY(dalloc(c, &W.perm, nw));
    TRY(dalloc(c, &W.cell_of, nw));
    TRY(dalloc(c, &W.cstart, (size_t)ncell + 1));
    TRY(dalloc(c, &W.ccount, ncell));
    // ---- solid
    Solid &S = c->S;
    S.n = (int)ns;
    S.max_ns = max_ns;
    TRY(dalloc(c, &S.inst, ns));
    TRY(dalloc(c, &S.x, ns));
    TRY(dalloc(c, &S.y, ns));
    TRY(dalloc(c, &S.z, D == 3 ? ns : 1));
    TRY(dalloc(c, &S.x0, ns));
    TRY(dalloc(c, &S.y0, ns));
    TRY(dalloc(c, &S.z0, D == 3 ? ns : 1));
    TRY(dalloc(c, &S.xs, ns));
    TRY(dalloc(c, &S.ys, ns));
    TRY(dalloc(c, &S.zs, D == 3 ? ns : 1));
    if (D == 2) S.z = S.z0 = S.zs = nullptr;
    TRY(dalloc(c, &S.v4, ns));
    TRY(dalloc(c, &S.H, (size_t)9 * ns));
    TRY(dalloc(c, &S.Hd, (size_t)9 * ns));
    TRY(dalloc(c, &S.B0, (size_t)9 * ns));
    TRY(dalloc(c, &S.Q4, (size_t)(D == 2 ? 1 : 3) * ns));
    TRY(dalloc(c, &S.n0, (size_t)3 * ns));
    TRY(dalloc(c, &S.nrm, (size_t)3 * ns));
    TRY(dalloc(c, &S.cons, ns));
    TRY(dalloc(c, &S.vbar, (size_t)3 * ns));
    TRY(dalloc(c, &S.abar, (size_t)3 * ns));
    TRY(dalloc(c, &S.asum, (size_t)3 * ns));
    TRY(dalloc(c, &S.fF, (size_t)3 * ns));
    TRY(dalloc(c, &S.nb_ptr, (size_t)ns + 1));
    TRY(dalloc(c, &S.A4, ns));
    TRY(dalloc(c, &S.VB4, ns));
    TRY(dalloc(c, &S.AB4, ns));
    TRY(dalloc(c, &S.N4, ns));
    TRY(dalloc(c, &S.L4, ns));
    TRY(dalloc(c, &S.key, ns));
    TRY(dalloc(c, &S.perm, ns));
    TRY(dalloc(c, &S.sperm, ns));
    TRY(dalloc(c, &S.cell_of, ns));
    TRY(dalloc(c, &S.cstart, (size_t)ncell + 1));
    TRY(dalloc(c, &S.ccount, ncell));
    TRY(dalloc(c, &S.bar, 2));
    TRY(dalloc(c, &S.queue, 1));

    // ---- concatenated host copies and upload
    {
        // fluid and walls: per-item loops over the host threads (every
        // element written once)
        hvec<double> fx(nf), fy(nf), fz(D == 3 ? nf : 0);
        hvec<float> fvx(nf), fvy(nf), fvz(D == 3 ? nf : 0), fdr(nf);
        hvec<int> fid(nf), finst(nf);
        hvec<double> wx(nw), wy(nw), wz(D == 3 ? nw : 0);
        hvec<float> wnx(nw), wny(nw), wnz(D == 3 ? nw : 0);
        hvec<int> winst(nw);
        std::vector<double> sx(ns), sy(ns), sz(D == 3 ? ns : 0), svbar(3 * (size_t)ns, 0.0);
        std::vector<float4> sv4(ns);
        std::vector<float> sn0(3 * (size_t)ns, 0.0f);
        std::vector<uint8_t> scons(ns);
        std::vector<int> sinst(ns);
        std::vector<Ctl> hctl(B);
        std::vector<Inst> hinst(B);
        for (int b = 0; b < B; b++) {
            InstHost &h = c->ih[b];
            const int f0 = h.d.f0, w0 = h.d.w0, s0 = h.d.s0;
            double vmax = 0.0;
            const int fch = host_chunks(h.nf, (int64_t)1 << 15);
            std::vector<double> cmax(fch, 0.0);
            std::vector<char> cbad(fch, 0);
            const bool fok = host_parallel(h.nf, fch, [&](int k, int64_t lo, int64_t hi) {
                double m = 0.0;
                for (int64_t i = lo; i < hi; i++) {
                    fx[f0 + i] = h.f_r[i * D];
                    fy[f0 + i] = h.f_r[i * D + 1];
                    if (D == 3) fz[f0 + i] = h.f_r[i * D + 2];
                    fvx[f0 + i] = (float)h.f_v[i * D];
                    fvy[f0 + i] = (float)h.f_v[i * D + 1];
                    if (D == 3) fvz[f0 + i] = (float)h.f_v[i * D + 2];
                    double v2 = 0.0;
                    for (int d = 0; d < D; d++) {
                        double vk = (double)(float)h.f_v[i * D + d];
                        v2 += vk * vk;
                    }
                    m = std::max(m, std::sqrt(v2));
                    fdr[f0 + i] = 0.0f;
                    if (h.f_has_p) {
                        // inverse of Eq. eqeos: rho - rho0 = rho0 expm1(log1p(7 p / (rho0 c0^2)) / 7)
                        double x = 7.0 * h.f_p[i] / (h.f_rho0 * h.f_c0 * h.f_c0);
                        if (!(x > -1.0)) cbad[k] = 1;
                        else fdr[f0 + i] = (float)(h.f_rho0 * std::expm1(std::log1p(x) / 7.0));
                    }
                    fid[f0 + i] = (int)i;
                    finst[f0 + i] = b;
                }
                cmax[k] = m;
            });
            if (!fok) return SPHFSI_E_NOMEM;
            for (int k = 0; k < fch; k++) {
                if (cbad[k]) return SPHFSI_E_INVAL;
                vmax = std::max(vmax, cmax[k]);
            }
            host_parallel(h.nw, host_chunks(h.nw, (int64_t)1 << 15), [&](int, int64_t lo, int64_t hi) {
                for (int64_t q = lo; q < hi; q++) {
                    wx[w0 + q] = h.w_r[q * D];
                    wy[w0 + q] = h.w_r[q * D + 1];
                    if (D == 3) wz[w0 + q] = h.w_r[q * D + 2];
                    wnx[w0 + q] = (float)h.w_n[q * D];
                    wny[w0 + q] = (float)h.w_n[q * D + 1];
                    if (D == 3) wnz[w0 + q] = (float)h.w_n[q * D + 2];
                    winst[w0 + q] = b;
                }
            });
            double vs = 0.0;
            for (int64_t a = 0; a < h.ns; a++) {
                sx[s0 + a] = h.s_r0[a * D];
                sy[s0 + a] = h.s_r0[a * D + 1];
                if (D == 3) sz[s0 + a] = h.s_r0[a * D + 2];
                double vv[3] = {0, 0, 0}, v2 = 0.0;
                for (int k = 0; k < D; k++) {
                    vv[k] = h.s_cons[a] ? 0.0 : h.s_v0[a * D + k];
                    sn0[3 * (s0 + a) + k] = (float)h.s_n0[a * D + k];
                    svbar[3 * (s0 + a) + k] = vv[k];
                    v2 += vv[k] * vv[k];
                }
                vs = std::max(vs, std::sqrt(v2));
                sv4[s0 + a] = make_float4((float)vv[0], (float)vv[1], (float)vv[2], 0.0f);
                scons[s0 + a] = h.s_cons[a];
                sinst[s0 + a] = b;
            }
            Ctl &ct = hctl[b];
            std::memset(&ct, 0, sizeof(ct));
            // the first step's dt_F and K come from the initial velocities
            ct.prev_vmaxF = (float)vmax;
            ct.prev_vmaxS = (float)vs;
            ct.n_reinit = h.prm.n_reinit;
            hinst[b] = h.d;
        }
        FluidState &S0 = F.s[0];
        TRY(upload(c, S0.x, fx));
        TRY(upload(c, S0.y, fy));
        if (D == 3) TRY(upload(c, S0.z, fz));
        TRY(upload(c, S0.vx, fvx));
        TRY(upload(c, S0.vy, fvy));
        if (D == 3) TRY(upload(c, S0.vz, fvz));
        TRY(upload(c, S0.drho, fdr));
        TRY(upload(c, S0.id, fid));
        TRY(upload(c, F.inst, finst));
        TRY(upload(c, W.x, wx));
        TRY(upload(c, W.y, wy));
        if (D == 3) TRY(upload(c, W.z, wz));
        TRY(upload(c, W.nx, wnx));
        TRY(upload(c, W.ny, wny));
        if (D == 3) TRY(upload(c, W.nz, wnz));
        TRY(upload(c, W.inst, winst));
        TRY(upload(c, S.x0, sx));
        TRY(upload(c, S.y0, sy));
        TRY(upload(c, S.x, sx));
        TRY(upload(c, S.y, sy));
        if (D == 3) {
            TRY(upload(c, S.z0, sz));
            TRY(upload(c, S.z, sz));
        }
        TRY(upload(c, S.v4, sv4));
        TRY(upload(c, S.n0, sn0));
        TRY(upload(c, S.nrm, sn0));
        TRY(upload(c, S.cons, scons));
        TRY(upload(c, S.vbar, svbar));
        TRY(upload(c, S.inst, sinst));
        std::vector<int> orow(ns);
        for (const InstHost &h : c->ih)
            for (int64_t a = 0; a < h.ns; a++) orow[h.d.s0 + a] = (int)(h.d.s0 + h.s_order[a]);
        TRY(dalloc(c, &c->d_orow, ns));
        TRY(upload(c, c->d_orow, orow));
        TRY(dalloc(c, &c->d_spos, (size_t)ns * D));
        TRY(upload(c, c->ctl, hctl));
        TRY(upload(c, c->d_inst, hinst));
    }
    c->bt.I = c->d_inst;
    c->bt.ctl = c->ctl;
    c->bt.B = B;
    c->bt.ncell = (int)ncell;
    c->bt.spin = kSpinLimit;
    TRY(dalloc(c, &c->bt.fail, 1));
    // ---- walls binned once; solid static neighbour list and B0
    TRY(launch_wall_bin(c->bt, W, D, c->st));
    if (ns > 0) {
        std::vector<int> ptr, nbi;
        TRY(body_neighbours(c, ptr, nbi));
        S.max_nb = 0;
        for (int64_t a = 0; a < ns; a++) S.max_nb = std::max(S.max_nb, ptr[a + 1] - ptr[a]);
        S.nnz = ptr[ns];
        int *d_nbi = nullptr;
        TRY(dalloc(c, &d_nbi, nbi.size()));
        TRY(upload(c, d_nbi, nbi));
        std::vector<Inst> hinst(B);
        for (int b = 0; b < B; b++) {
            InstHost &h = c->ih[b];
            h.d.nnz = ptr[h.d.s0 + h.d.ns] - ptr[h.d.s0];
            hinst[b] = h.d;
        }
        TRY(upload(c, S.nb_ptr, ptr));
        TRY(upload(c, c->d_inst, hinst));
        TRY(dalloc(c, &S.nb, S.nnz));
        TRY(launch_solid_setup_fill(c->bt, S, d_nbi, D, c->st));
        if (D == 2) TRY(halo_maps(c, ptr, nbi));
    }
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    for (int k = 0; k < sphfsi_ctx::kEvents; k++) TRY(cuda_rc(cudaEventCreate(&c->ev[k])));
    // the solid branch (coupling force, sub-steps) is the longer branch of a
    // step for small and medium problems: its stream gets the highest priority
    // so that its blocks are scheduled ahead of queued fluid blocks
    {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        TRY(cuda_rc(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi)));
    }
    TRY(cuda_rc(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming)));
    TRY(cuda_rc(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming)));
    c->finalized = true;
    // release the host staging copies that are not needed any more
    for (auto &h : c->ih) {
        hvec<double>().swap(h.f_r);
        hvec<double>().swap(h.f_v);
        hvec<double>().swap(h.f_p);
        hvec<double>().swap(h.w_r);
        hvec<double>().swap(h.w_n);
        h.s_r0.clear(); h.s_v0.clear(); h.s_n0.clear();
    }
    return SPHFSI_OK;
}

int sphfsi_set_substeps(sphfsi_ctx *c, int32_t K)
{
    if (!c || K < 0) return SPHFSI_E_INVAL;
    c->K_fixed = K;
    return SPHFSI_OK;
}

int sphfsi_set_time_stepping(sphfsi_ctx *c, int32_t mode)
{
    if (!c || mode < 0 || mode > 2) return SPHFSI_E_INVAL;
    c->K_fixed = -mode;   // 0 keeps the kappa sub-steps
    return SPHFSI_OK;
}

int sphfsi_set_advection_cadence(sphfsi_ctx *c, int32_t n)
{
    TRY(check_ctx(c, true));
    if (n < 0) return SPHFSI_E_INVAL;
    c->F.held_n = n;   // 0: automatic (the advection criterion)
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return request_rebuild(c);
}

int sphfsi_step(sphfsi_ctx *c, double dt_F)
{
    TRY(check_ctx(c, true));
    if (std::isnan(dt_F)) return SPHFSI_E_INVAL;
    if (c->failed) return SPHFSI_E_TIMEOUT;
    if (c->runaway) return SPHFSI_E_UNSTABLE;
    return enqueue_step(c, dt_F);
}

int sphfsi_set_wait_limit(sphfsi_ctx *c, int64_t iterations)
{
    TRY(check_ctx(c, true));
    if (iterations < 0) return SPHFSI_E_INVAL;
    c->bt.spin = iterations == 0 ? kSpinLimit : (long long)iterations;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return SPHFSI_OK;
}

int sphfsi_run(sphfsi_ctx *c, int64_t nsteps, double dt_F)
{
    TRY(check_ctx(c, true));
    if (nsteps < 0 || std::isnan(dt_F)) return SPHFSI_E_INVAL;
    if (c->failed) return SPHFSI_E_TIMEOUT;
    if (c->runaway) return SPHFSI_E_UNSTABLE;
    if (nsteps == 0) return SPHFSI_OK;
    if (c->st == nullptr) {
        // the legacy default stream cannot be captured: plain launches
        for (int64_t i = 0; i < nsteps; i++) TRY(enqueue_step(c, dt_F));
        return SPHFSI_OK;
    }
    double dtk = dt_F > 0.0 ? dt_F : 0.0;
    if (!c->gexec || c->graph_dt != dtk || c->graph_K != c->K_fixed || c->graph_prof != (int)c->profiling) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        cudaGraph_t gr;
        TRY(cuda_rc(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal)));
        int rc = enqueue_step(c, dtk);
        cudaError_t e = cudaStreamEndCapture(c->st, &gr);
        if (rc) return rc;
        TRY(cuda_rc(e));
        e = cudaGraphInstantiate(&c->gexec, gr, 0);
        cudaGraphDestroy(gr);
        TRY(cuda_rc(e));
        c->graph_dt = dtk;
        c->graph_K = c->K_fixed;
        c->graph_prof = (int)c->profiling;
    }
    for (int64_t i = 0; i < nsteps; i++) TRY(cuda_rc(cudaGraphLaunch(c->gexec, c->st)));
    return SPHFSI_OK;
}

int sphfsi_sync(sphfsi_ctx *c)
{
    if (!c) return SPHFSI_E_INVAL;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    if (!c->finalized) return SPHFSI_OK;
    std::vector<Ctl> h;
    TRY(download(c, h, c->ctl, c->B));
    int status = 0;
    for (const Ctl &x : h) status |= x.status;
    c->last_status = status;
    if (status & ST_TIMEOUT) {
        c->failed = true;
        return SPHFSI_E_TIMEOUT;
    }
    if (status & ST_NONFINITE) {
        c->runaway = true;
        return SPHFSI_E_UNSTABLE;
    }
    return SPHFSI_OK;
}

int sphfsi_get_fluid(sphfsi_ctx *c, double *r, float *v, double *rho, float *drho_dt, float *dvdt)
{
    TRY(check_ctx(c, true));
    const int D = c->dim;
    const InstHost &h = c->ih[c->sel];
    const int64_t n = h.nf, f0 = h.d.f0;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    const FluidState &S = c->F.s[0];
    std::vector<int> id;
    TRY(download(c, id, S.id + f0, n));
    if (r) {
        std::vector<double> x, y, z, out(n * D);
        TRY(download(c, x, S.x + f0, n));
        TRY(download(c, y, S.y + f0, n));
        if (D == 3) TRY(download(c, z, S.z + f0, n));
        for (int64_t k = 0; k < n; k++) {
            out[(size_t)id[k] * D] = x[k];
            out[(size_t)id[k] * D + 1] = y[k];
            if (D == 3) out[(size_t)id[k] * D + 2] = z[k];
        }
        TRY(deliver(r, out));
    }
    if (v) {
        std::vector<float> x, y, z, out(n * D);
        TRY(download(c, x, S.vx + f0, n));
        TRY(download(c, y, S.vy + f0, n));
        if (D == 3) TRY(download(c, z, S.vz + f0, n));
        for (int64_t k = 0; k < n; k++) {
            out[(size_t)id[k] * D] = x[k];
            out[(size_t)id[k] * D + 1] = y[k];
            if (D == 3) out[(size_t)id[k] * D + 2] = z[k];
        }
        TRY(deliver(v, out));
    }
    if (rho) {
        std::vector<float> d;
        std::vector<double> out(n);
        TRY(download(c, d, S.drho + f0, n));
        for (int64_t k = 0; k < n; k++) out[id[k]] = h.f_rho0 + (double)d[k];
        TRY(deliver(rho, out));
    }
    if (drho_dt) {
        std::vector<float> d, out(n);
        TRY(download(c, d, S.rhodot + f0, n));
        for (int64_t k = 0; k < n; k++) out[id[k]] = d[k];
        TRY(deliver(drho_dt, out));
    }
    if (dvdt) {
        std::vector<float> d, out(n * D);
        TRY(download(c, d, c->F.dvdt + (size_t)f0 * D, (size_t)n * D));
        for (int64_t k = 0; k < n; k++)
            for (int q = 0; q < D; q++) out[(size_t)id[k] * D + q] = d[(size_t)k * D + q];
        TRY(deliver(dvdt, out));
    }
    return SPHFSI_OK;
}

int sphfsi_get_solid(sphfsi_ctx *c, double *r, float *v, double *F, double *vbar, double *abar, float *fF, float *nrm)
{
    TRY(check_ctx(c, true));
    const int D = c->dim;
    const InstHost &h = c->ih[c->sel];
    const int64_t n = h.ns, s0 = h.d.s0;
    const Solid &S = c->S;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    if (n == 0) return SPHFSI_OK;
    const std::vector<int> &ord = h.s_order;   // device index -> original index
    if (r) {
        std::vector<double> x, y, z, out(n * D);
        TRY(download(c, x, S.x + s0, n));
        TRY(download(c, y, S.y + s0, n));
        if (D == 3) TRY(download(c, z, S.z + s0, n));
        for (int64_t a = 0; a < n; a++) {
            size_t o = (size_t)ord[a] * D;
            out[o] = x[a];
            out[o + 1] = y[a];
            if (D == 3) out[o + 2] = z[a];
        }
        TRY(deliver(r, out));
    }
    if (v) {
        std::vector<float4> hv;
        TRY(download(c, hv, S.v4 + s0, n));
        std::vector<float> out(n * D);
        for (int64_t a = 0; a < n; a++) {
            size_t o = (size_t)ord[a] * D;
            out[o] = hv[a].x;
            out[o + 1] = hv[a].y;
            if (D == 3) out[o + 2] = hv[a].z;
        }
        TRY(deliver(v, out));
    }
    if (F) {
        std::vector<float> hh;
        std::vector<double> out(n * D * D);
        TRY(download(c, hh, S.H + 9 * s0, (size_t)9 * n));
        for (int64_t a = 0; a < n; a++)
            for (int i = 0; i < D * D; i++)
                out[(size_t)ord[a] * D * D + i] = (double)hh[9 * a + i] + ((i % (D + 1)) == 0 ? 1.0 : 0.0);
        TRY(deliver(F, out));
    }
    auto vec3 = [&](const auto *src, auto *dst, auto zero) -> int {
        using T = decltype(zero);
        if (!dst) return SPHFSI_OK;
        std::vector<T> hv, out(n * D);
        int rc = download(c, hv, src + 3 * s0, (size_t)3 * n);
        if (rc) return rc;
        for (int64_t a = 0; a < n; a++)
            for (int k = 0; k < D; k++) out[(size_t)ord[a] * D + k] = hv[3 * a + k];
        return deliver(dst, out);
    };
    TRY(vec3(S.vbar, vbar, 0.0));
    TRY(vec3(S.abar, abar, 0.0));
    TRY(vec3(S.fF, fF, 0.0f));
    TRY(vec3(S.nrm, nrm, 0.0f));
    return SPHFSI_OK;
}

// solid positions in original order (row orow[a] of out) for the
// asynchronous read
__global__ void k_gather_solid_positions(const double *x, const double *y, const double *z, const int *orow,
                                         int n, int D, double *out)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const size_t o = (size_t)orow[a] * D;
    out[o] = x[a];
    out[o + 1] = y[a];
    if (D == 3) out[o + 2] = z[a];
}

int sphfsi_get_solid_positions_async(sphfsi_ctx *c, double *r)
{
    TRY(check_ctx(c, true));
    if (!r) return SPHFSI_E_INVAL;
    const int64_t n = c->S.n;
    if (n == 0) return SPHFSI_OK;
    k_gather_solid_positions<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>(c->S.x, c->S.y, c->S.z, c->d_orow,
                                                                          (int)n, c->dim, c->d_spos);
    TRY(cuda_rc(cudaGetLastError()));
    return cuda_rc(cudaMemcpyAsync(r, c->d_spos, sizeof(double) * (size_t)n * c->dim, cudaMemcpyDefault, c->st));
}

int sphfsi_get_solid_positions_all(sphfsi_ctx *c, double *r)
{
    TRY(check_ctx(c, true));
    if (!r) return SPHFSI_E_INVAL;
    const int D = c->dim;
    const Solid &S = c->S;
    const int64_t n = S.n;
    if (n == 0) return SPHFSI_OK;
    std::vector<double> xyz[3];
    TRY(download(c, xyz[0], S.x, n));
    TRY(download(c, xyz[1], S.y, n));
    if (D == 3) TRY(download(c, xyz[2], S.z, n));
    std::vector<double> out((size_t)n * D);
    for (const InstHost &h : c->ih) {
        const int64_t s0 = h.d.s0;
        for (int64_t a = 0; a < h.ns; a++) {
            const size_t o = (size_t)(s0 + h.s_order[a]) * D;
            for (int k = 0; k < D; k++) out[o + k] = xyz[k][s0 + a];
        }
    }
    return deliver(r, out);
}

int sphfsi_set_fluid_state(sphfsi_ctx *c, const double *r, const double *v, const double *rho, const double *drho_dt)
{
    TRY(check_ctx(c, true));
    TRY(request_rebuild(c));
    const int D = c->dim;
    const InstHost &h = c->ih[c->sel];
    const int64_t n = h.nf, f0 = h.d.f0;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    FluidState &S = c->F.s[0];
    // the instance's slots are rewritten in original order (id = index)
    std::vector<int> cur_id;
    TRY(download(c, cur_id, S.id + f0, n));
    std::vector<int> inv(n);
    for (int64_t k = 0; k < n; k++) inv[cur_id[k]] = (int)k;
    auto reorder = [&](auto *dev, auto &out) -> int {
        using V = typename std::remove_reference<decltype(out)>::type;
        V hv;
        int rc = download(c, hv, dev + f0, n);
        if (rc) return rc;
        out.resize(n);
        for (int64_t i = 0; i < n; i++) out[i] = hv[inv[i]];
        return SPHFSI_OK;
    };
    std::vector<double> x, y, z;
    std::vector<float> vx, vy, vz, dr, rd;
    TRY(reorder(S.x, x));
    TRY(reorder(S.y, y));
    if (D == 3) TRY(reorder(S.z, z));
    TRY(reorder(S.vx, vx));
    TRY(reorder(S.vy, vy));
    if (D == 3) TRY(reorder(S.vz, vz));
    TRY(reorder(S.drho, dr));
    TRY(reorder(S.rhodot, rd));
    std::vector<double> in;
    if (r) {
        TRY(fetch(in, r, (size_t)n * D));
        for (int64_t i = 0; i < n; i++) {
            x[i] = in[i * D];
            y[i] = in[i * D + 1];
            if (D == 3) z[i] = in[i * D + 2];
        }
    }
    if (v) {
        TRY(fetch(in, v, (size_t)n * D));
        for (int64_t i = 0; i < n; i++) {
            vx[i] = (float)in[i * D];
            vy[i] = (float)in[i * D + 1];
            if (D == 3) vz[i] = (float)in[i * D + 2];
        }
    }
    if (rho) {
        TRY(fetch(in, rho, (size_t)n));
        for (int64_t i = 0; i < n; i++) dr[i] = (float)(in[i] - h.f_rho0);
    }
    if (drho_dt) {
        TRY(fetch(in, drho_dt, (size_t)n));
        for (int64_t i = 0; i < n; i++) rd[i] = (float)in[i];
    }
    std::vector<int> id(n);
    for (int64_t i = 0; i < n; i++) id[i] = (int)i;
    auto put = [&](auto *dev, const auto &hv) -> int {
        if (hv.empty()) return SPHFSI_OK;
        return cuda_rc(cudaMemcpyAsync(dev + f0, hv.data(), sizeof(hv[0]) * hv.size(), cudaMemcpyHostToDevice, c->st));
    };
    TRY(put(S.x, x));
    TRY(put(S.y, y));
    if (D == 3) TRY(put(S.z, z));
    TRY(put(S.vx, vx));
    TRY(put(S.vy, vy));
    if (D == 3) TRY(put(S.vz, vz));
    TRY(put(S.drho, dr));
    TRY(put(S.rhodot, rd));
    TRY(put(S.id, id));
    return cuda_rc(cudaStreamSynchronize(c->st));
}

int sphfsi_set_solid_state(sphfsi_ctx *c, const double *r, const double *v, const double *F, const double *vbar,
                           const double *abar, const double *nrm)
{
    TRY(check_ctx(c, true));
    TRY(request_rebuild(c));
    const int D = c->dim;
    const InstHost &h = c->ih[c->sel];
    const int64_t n = h.ns, s0 = h.d.s0;
    Solid &S = c->S;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    if (n == 0) return SPHFSI_OK;
    std::vector<double> in;
    // rows arrive in original order; the device keeps its locality order
    auto to_dev = [&](int w) {
        std::vector<double> t(in.size());
        for (int64_t a = 0; a < n; a++)
            for (int j = 0; j < w; j++) t[(size_t)a * w + j] = in[(size_t)h.s_order[a] * w + j];
        in.swap(t);
    };
    auto put = [&](auto *dev, const auto &hv) -> int {
        if (hv.empty()) return SPHFSI_OK;
        return cuda_rc(cudaMemcpyAsync(dev, hv.data(), sizeof(hv[0]) * hv.size(), cudaMemcpyHostToDevice, c->st));
    };
    if (r) {
        TRY(fetch(in, r, (size_t)n * D));
        to_dev(D);
        std::vector<double> xyz[3];
        deinterleave(in, D, n, xyz);
        TRY(put(S.x + s0, xyz[0]));
        TRY(put(S.y + s0, xyz[1]));
        if (D == 3) TRY(put(S.z + s0, xyz[2]));
    }
    if (v) {
        TRY(fetch(in, v, (size_t)n * D));
        to_dev(D);
        std::vector<float4> hv(n);
        for (int64_t a = 0; a < n; a++)
            hv[a] = make_float4((float)in[a * D], (float)in[a * D + 1], D == 3 ? (float)in[a * D + 2] : 0.0f, 0.0f);
        TRY(put(S.v4 + s0, hv));
    }
    if (F) {
        TRY(fetch(in, F, (size_t)n * D * D));
        to_dev(D * D);
        std::vector<float> hv(9 * (size_t)n, 0.0f);
        for (int64_t a = 0; a < n; a++)
            for (int i = 0; i < D * D; i++) hv[9 * a + i] = (float)(in[a * D * D + i] - ((i % (D + 1)) == 0 ? 1.0 : 0.0));
        TRY(put(S.H + 9 * s0, hv));
    }
    auto put3 = [&](const double *src, auto *dev, auto zero) -> int {
        using T = decltype(zero);
        if (!src) return SPHFSI_OK;
        int rc = fetch(in, src, (size_t)n * D);
        if (rc) return rc;
        to_dev(D);
        std::vector<T> hv(3 * (size_t)n, (T)0);
        for (int64_t a = 0; a < n; a++)
            for (int k = 0; k < D; k++) hv[3 * a + k] = (T)in[a * D + k];
        return put(dev + 3 * s0, hv);
    };
    TRY(put3(vbar, S.vbar, 0.0));
    TRY(put3(abar, S.abar, 0.0));
    TRY(put3(nrm, S.nrm, 0.0f));
    return cuda_rc(cudaStreamSynchronize(c->st));
}

int sphfsi_set_time(sphfsi_ctx *c, double t, int64_t step)
{
    TRY(check_ctx(c, true));
    TRY(request_rebuild(c));
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    Ctl hc;
    Ctl *dc = c->ctl + c->sel;
    TRY(cuda_rc(cudaMemcpy(&hc, dc, sizeof(Ctl), cudaMemcpyDeviceToHost)));
    hc.t = t;
    hc.step = step;
    return cuda_rc(cudaMemcpy(dc, &hc, sizeof(Ctl), cudaMemcpyHostToDevice));
}

// Time-step criteria of the selected instance at its current state (the
// maxima of the last finished step, or the initial velocities before the
// first): Eqs. dt-relax (acoustic), the advection/viscous limit, and Eq.
// dts-advection (solid).
int sphfsi_suggest_dt(sphfsi_ctx *c, double *dt_ac, double *dt_ad, double *dt_S)
{
    TRY(check_ctx(c, true));
    if (!dt_ac || !dt_ad || !dt_S) return SPHFSI_E_INVAL;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    Ctl hc;
    TRY(cuda_rc(cudaMemcpy(&hc, c->ctl + c->sel, sizeof(Ctl), cudaMemcpyDeviceToHost)));
    const Phys &P = c->ih[c->sel].d.P;
    const double vF = hc.prev_vmaxF, vS = hc.prev_vmaxS, aS = hc.prev_amaxS;
    *dt_ac = 0.6 * P.hF_d / (P.c0_d + vF);
    const double nu = P.eta_d / P.rho0_d;
    const double a1 = vF > 0.0 ? P.hF_d / vF : 1e300, a2 = nu > 0.0 ? P.hF_d * P.hF_d / nu : 1e300;
    *dt_ad = 0.25 * (a1 < a2 ? a1 : a2);
    if (c->ih[c->sel].ns > 0) {
        const double b1 = P.hS_d / (P.cS_d + vS), b2 = aS > 0.0 ? std::sqrt(P.hS_d / aS) : 1e300;
        *dt_S = 0.6 * (b1 < b2 ? b1 : b2);
    } else {
        *dt_S = 1e300;
    }
    return SPHFSI_OK;
}

// Checkpoint blob: a header, then every device allocation of the context in
// allocation order, each preceded by its size.
namespace {
constexpr uint64_t kStateMagic = 0x3130305354534853ull;   // "SHSTS001"
}

int sphfsi_state_size(sphfsi_ctx *c, int64_t *bytes)
{
    TRY(check_ctx(c, true));
    if (!bytes) return SPHFSI_E_INVAL;
    uint64_t n = 3 * sizeof(uint64_t);
    for (auto &a : c->allocs) n += sizeof(uint64_t) + a.second;
    *bytes = (int64_t)n;
    return SPHFSI_OK;
}

int sphfsi_get_state(sphfsi_ctx *c, void *blob, int64_t bytes)
{
    int64_t need = 0;
    TRY(sphfsi_state_size(c, &need));
    if (!blob || bytes < need) return SPHFSI_E_INVAL;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    if (c->side) TRY(cuda_rc(cudaStreamSynchronize(c->side)));
    uint8_t *p = (uint8_t *)blob;
    const uint64_t head[3] = {kStateMagic, (uint64_t)c->allocs.size(), (uint64_t)need};
    std::memcpy(p, head, sizeof(head));
    p += sizeof(head);
    for (auto &a : c->allocs) {
        const uint64_t sz = a.second;
        std::memcpy(p, &sz, sizeof(sz));
        p += sizeof(sz);
        TRY(cuda_rc(cudaMemcpy(p, a.first, a.second, cudaMemcpyDeviceToHost)));
        p += a.second;
    }
    return SPHFSI_OK;
}

int sphfsi_set_state(sphfsi_ctx *c, const void *blob, int64_t bytes)
{
    int64_t need = 0;
    TRY(sphfsi_state_size(c, &need));
    if (!blob || bytes != need) return SPHFSI_E_INVAL;
    const uint8_t *p = (const uint8_t *)blob;
    uint64_t head[3];
    std::memcpy(head, p, sizeof(head));
    if (head[0] != kStateMagic || head[1] != (uint64_t)c->allocs.size() || head[2] != (uint64_t)need)
        return SPHFSI_E_INVAL;
    p += sizeof(head);
    // check every size first, so that a mismatched blob leaves the state untouched
    const uint8_t *q = p;
    for (auto &a : c->allocs) {
        uint64_t sz;
        std::memcpy(&sz, q, sizeof(sz));
        if (sz != a.second) return SPHFSI_E_INVAL;
        q += sizeof(sz) + sz;
    }
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    if (c->side) TRY(cuda_rc(cudaStreamSynchronize(c->side)));
    for (auto &a : c->allocs) {
        p += sizeof(uint64_t);
        TRY(cuda_rc(cudaMemcpy(a.first, p, a.second, cudaMemcpyHostToDevice)));
        p += a.second;
    }
    // steps are allowed again unless the checkpoint itself was taken after a
    // scan that gave up or a step that ran away
    int fail = 0;
    TRY(cuda_rc(cudaMemcpy(&fail, c->bt.fail, sizeof(int), cudaMemcpyDeviceToHost)));
    c->failed = fail == kFailWait;
    c->runaway = fail == kFailRunaway;
    c->last_status = 0;
    return SPHFSI_OK;
}

int sphfsi_get_info(sphfsi_ctx *c, sphfsi_info *out)
{
    if (!c || !out) return SPHFSI_E_INVAL;
    std::memset(out, 0, sizeof(*out));
    const InstHost &h = c->ih[c->sel];
    out->n_fluid = h.nf;
    out->n_solid = h.ns;
    out->n_wall = h.nw;
    if (!c->finalized) return SPHFSI_OK;
    out->n_cells = h.d.g.ncell;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    Ctl hc;
    TRY(cuda_rc(cudaMemcpy(&hc, c->ctl + c->sel, sizeof(Ctl), cudaMemcpyDeviceToHost)));
    out->step = hc.step;
    out->t = hc.t;
    out->last_dt = hc.last_dt;
    out->last_K = hc.last_K;
    out->status = hc.status;
    out->pairs_ff = (int64_t)hc.n_ff;
    out->pairs_fw = (int64_t)hc.n_fw;
    out->pairs_fs = (int64_t)hc.n_fs;
    out->pairs_sf = (int64_t)hc.n_sf;
    out->pairs_ss = (int64_t)h.d.nnz;
    out->pairs_total = (int64_t)hc.pairs_total;
    // maxima of the last step (the finish kernel moves them to prev_*)
    out->vmax_f = hc.prev_vmaxF;
    out->vmax_s = hc.prev_vmaxS;
    out->amax_s = hc.prev_amaxS;
    for (int k = 0; k < 3; k++) {
        out->mom_fs_fluid[k] = hc.mom_fluid[k];
        out->mom_fs_solid[k] = hc.mom_solid[k];
    }
    out->solid_path = c->solid_path;
    out->kernels_per_step = c->kernels_per_step;
    out->learned_accepted = hc.l_acc;
    out->learned_rejected = hc.l_rej;
    out->learned_residual = hc.l_res;
    return SPHFSI_OK;
}

int sphfsi_pairs_total(sphfsi_ctx *c, int64_t *total)
{
    TRY(check_ctx(c, true));
    if (!total) return SPHFSI_E_INVAL;
    std::vector<Ctl> h;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    TRY(download(c, h, c->ctl, c->B));
    int64_t s = 0;
    for (const Ctl &x : h) s += (int64_t)x.pairs_total;
    *total = s;
    return SPHFSI_OK;
}

int sphfsi_debug_neighbors(sphfsi_ctx *c, int which, int64_t *ptr, int64_t *idx, int64_t *nnz)
{
    TRY(check_ctx(c, true));
    if (which < 0 || which > 3 || !nnz) return SPHFSI_E_INVAL;
    if (c->F.held_n != 1) return SPHFSI_E_STATE;   // binning here would replace the held configuration
    const InstHost &h = c->ih[c->sel];
    const int64_t nrows = which == 3 ? h.ns : h.nf;
    // bin the current positions (no drift) and build the solid records
    TRY(launch_bin_all(c->bt, c->F, c->S, c->dim, 0, 0.0, 0, c->st));
    int *counts = nullptr, *offs = nullptr, *out = nullptr;
    if (cudaMalloc(&counts, sizeof(int) * (nrows + 1)) != cudaSuccess) return SPHFSI_E_NOMEM;
    int rc = launch_debug_pairs(c->bt, c->F, c->W, c->S, c->dim, c->sel, which, counts, nullptr, nullptr, c->st);
    // solid rows (which 3) and solid columns (which 2) come in the device's
    // locality order; rows and columns are reported in original order
    std::vector<int> hc_dev, hc(nrows, 0);
    if (!rc) rc = download(c, hc_dev, counts, nrows);
    for (int64_t i = 0; i < nrows && !rc; i++) hc[which == 3 ? h.s_order[i] : i] = hc_dev[i];
    std::vector<int64_t> p(nrows + 1, 0);
    for (int64_t i = 0; i < nrows && !rc; i++) p[i + 1] = p[i] + hc[i];
    *nnz = p[nrows];
    if (!rc && ptr) std::memcpy(ptr, p.data(), sizeof(int64_t) * (nrows + 1));
    if (!rc && idx && p[nrows] > 0) {
        std::vector<int> po(nrows);
        for (int64_t i = 0; i < nrows; i++) po[i] = (int)p[which == 3 ? h.s_order[i] : i];
        if (cudaMalloc(&offs, sizeof(int) * nrows) != cudaSuccess || cudaMalloc(&out, sizeof(int) * p[nrows]) != cudaSuccess)
            rc = SPHFSI_E_NOMEM;
        if (!rc) rc = upload(c, offs, po);
        if (!rc) rc = launch_debug_pairs(c->bt, c->F, c->W, c->S, c->dim, c->sel, which, counts, offs, out, c->st);
        std::vector<int> hv;
        if (!rc) rc = download(c, hv, out, (size_t)p[nrows]);
        if (!rc) {
            if (which == 2)
                for (auto &col : hv) col = h.s_order[col];
            for (int64_t i = 0; i < nrows; i++) {
                std::sort(hv.begin() + p[i], hv.begin() + p[i + 1]);
                for (int64_t q = p[i]; q < p[i + 1]; q++) idx[q] = hv[q];
            }
        }
    }
    cudaFree(counts);
    if (offs) cudaFree(offs);
    if (out) cudaFree(out);
    return rc;
}

int sphfsi_set_solid_path(sphfsi_ctx *c, int path)
{
    TRY(check_ctx(c, true));
    if (path < 0 || path > 2) return SPHFSI_E_INVAL;
    if (path == 2 && c->B != 1) return SPHFSI_E_INVAL;
    c->S.force_grid_path = path == 2 ? 1 : 0;
    c->S.force_lane_path = path == 1 ? 1 : 0;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return SPHFSI_OK;
}

static bool valid_lanes(int dim, int L)
{
    return dim == 2 ? (L == 2 || L == 4 || L == 8) : (L == 4 || L == 8 || L == 16);
}

int sphfsi_set_tuning(sphfsi_ctx *c, const sphfsi_tuning *t)
{
    TRY(check_ctx(c, true));
    if (!t || !valid_lanes(c->dim, t->lanes) || (t->block != 64 && t->block != 128 && t->block != 256) ||
        t->solid_variant < 0 || t->solid_variant > 5 || t->compact < 0 || t->compact > 1 || t->tile < 0 ||
        t->tile > 1 || t->records < 0 || t->records > 2 || t->rows < 0 || t->rows > 1 || (t->rows && t->tile) ||
        (c->max_reach > 1 && (t->rows || t->tile)) || t->list < 0 || t->list > 1 ||
        (t->list && (t->tile || c->max_reach > 1)) ||
        (t->list_lanes != 0 && t->list_lanes != 1 && t->list_lanes != 8 && t->list_lanes != 16 &&
         t->list_lanes != 32))
        return SPHFSI_E_INVAL;
    c->F.lanes = t->lanes;
    c->F.block = t->block;
    c->F.compact = t->compact;
    c->F.tile = t->tile;
    c->F.split_records = t->records == 1 ? 1 : 0;
    c->F.bin_fused = t->records == 2 ? 1 : 0;
    c->F.rows = t->rows;
    c->F.list = t->list;
    if (t->list_lanes) c->F.list_lanes = t->list_lanes;
    c->S.force_lane_path = t->solid_variant;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return SPHFSI_OK;
}

int sphfsi_get_tuning(sphfsi_ctx *c, sphfsi_tuning *t)
{
    TRY(check_ctx(c, true));
    if (!t) return SPHFSI_E_INVAL;
    t->lanes = c->F.lanes;
    t->block = c->F.block;
    t->solid_variant = c->S.force_lane_path;
    t->compact = c->F.compact;
    t->tile = c->F.tile;
    t->records = c->F.bin_fused ? 2 : c->F.split_records;
    t->rows = c->F.rows;
    t->list = c->F.list;
    t->list_lanes = c->F.list_lanes;
    t->step_ms = 0.0f;
    return SPHFSI_OK;
}

int sphfsi_autotune(sphfsi_ctx *c, double dt_F, int32_t steps, sphfsi_tuning *best)
{
    TRY(check_ctx(c, true));
    if (!best || steps < 1 || steps > 10000 || std::isnan(dt_F) || c->st == nullptr) return SPHFSI_E_INVAL;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    // snapshot of every device allocation, restored before each trial and at the end
    size_t total = 0;
    for (auto &a : c->allocs) total += (a.second + 255) & ~(size_t)255;
    char *snap = nullptr;
    if (cudaMalloc(&snap, total) != cudaSuccess) {
        cudaGetLastError();
        return SPHFSI_E_NOMEM;
    }
    auto copy_all = [&](bool save) -> int {
        size_t off = 0;
        for (auto &a : c->allocs) {
            void *dst = save ? (void *)(snap + off) : a.first;
            const void *src = save ? a.first : (const void *)(snap + off);
            if (cudaMemcpyAsync(dst, src, a.second, cudaMemcpyDeviceToDevice, c->st) != cudaSuccess) return SPHFSI_E_CUDA;
            off += (a.second + 255) & ~(size_t)255;
        }
        return cuda_rc(cudaStreamSynchronize(c->st));
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sphfsi_tuning cur{}, keep{};
    sphfsi_get_tuning(c, &keep);
    int rc = copy_all(true);
    if (!rc) rc = cuda_rc(cudaEventCreate(&e0));
    if (!rc) rc = cuda_rc(cudaEventCreate(&e1));
    auto trial = [&](const sphfsi_tuning &t, float *ms) -> int {
        int r = copy_all(false);
        if (!r) r = sphfsi_set_tuning(c, &t);
        if (!r) r = sphfsi_run(c, steps, dt_F);   // capture + warm-up
        if (!r) r = cuda_rc(cudaEventRecord(e0, c->st));
        if (!r) r = sphfsi_run(c, steps, dt_F);
        if (!r) r = cuda_rc(cudaEventRecord(e1, c->st));
        if (!r) r = sphfsi_sync(c);
        if (!r) r = cuda_rc(cudaEventElapsedTime(ms, e0, e1));
        if (!r) *ms /= (float)steps;
        return r;
    };
    best->step_ms = 0.0f;
    if (!rc) {
        // coordinate search: lanes, pair form, tiles, rows, block size, records form, 2-D solid variant
        cur = keep;
        cur.solid_variant = 0;
        const int lanes2[3] = {2, 4, 8}, lanes3[3] = {4, 8, 16}, blocks[3] = {64, 128, 256};
        float tbest = 0.0f;
        bool have = false;
        auto consider = [&](const sphfsi_tuning &t) -> int {
            float ms = 0.0f;
            int r = trial(t, &ms);
            if (r) return r;
            if (!have || ms < tbest) {
                have = true;
                tbest = ms;
                *best = t;
                best->step_ms = ms;
            }
            return SPHFSI_OK;
        };
        for (int k = 0; k < 3 && !rc; k++) {
            cur.lanes = c->dim == 2 ? lanes2[k] : lanes3[k];
            cur.block = 128;
            rc = consider(cur);
        }
        cur = *best;
        if (!rc) {
            cur.compact = 1 - cur.compact;
            rc = consider(cur);
        }
        cur = *best;
        if (!rc && c->max_reach == 1) {
            cur.list = 1 - cur.list;
            if (cur.list) cur.tile = 0;
            rc = consider(cur);
        }
        cur = *best;
        for (int k = 0; k < 3 && !rc && cur.list; k++) {
            const int ll[3] = {1, 8, 32};
            if (ll[k] == best->list_lanes) continue;
            cur.list_lanes = ll[k];
            rc = consider(cur);
        }
        cur = *best;
        if (!rc && c->max_reach == 1 && !cur.list) {
            cur.tile = 1 - cur.tile;
            if (cur.tile) cur.rows = 0;
            rc = consider(cur);
        }
        cur = *best;
        if (!rc && !cur.tile && !cur.list && c->max_reach == 1) {
            cur.rows = 1 - cur.rows;
            rc = consider(cur);
        }
        cur = *best;
        for (int k = 0; k < 3 && !rc; k++) {
            if (blocks[k] == 128) continue;
            cur.block = blocks[k];
            rc = consider(cur);
        }
        cur = *best;
        for (int r = 0; r < 3 && !rc; r++) {
            if (r == best->records) continue;
            cur.records = r;
            rc = consider(cur);
        }
        cur = *best;
        if (!rc && c->dim == 2 && c->S.n && !c->S.force_grid_path) {
            for (int v = 0; v < 6 && !rc; v++) {
                if (v == best->solid_variant) continue;
                cur.solid_variant = v;
                rc = consider(cur);
            }
        }
    }
    int rc2 = copy_all(false);
    if (!rc) rc = rc2;
    if (!rc) rc = sphfsi_set_tuning(c, best);
    else sphfsi_set_tuning(c, &keep);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(snap);
    return rc;
}

// Graph of the bodies for the network: the static reference neighbour
// list, w_ab = V0 W(|r0_a - r0_b|, h_S) in FP64 and g_ab = h_S V0 grad0_a W_ab
// (the list's FP32 entries).  inst < 0: every instance, device order, global
// slots; else that instance in its original order with local indices.
static int body_graph(sphfsi_ctx *c, int inst, std::vector<int64_t> &ptr, std::vector<int64_t> &idx,
                      std::vector<double> &w, std::vector<double> &g)
{
    const int D = c->dim;
    const Solid &S = c->S;
    std::vector<int> hp;
    std::vector<float4> hnb;
    std::vector<double> X[3];
    TRY(download(c, hp, S.nb_ptr, (size_t)S.n + 1));
    TRY(download(c, hnb, S.nb, (size_t)S.nnz));
    TRY(download(c, X[0], S.x0, S.n));
    TRY(download(c, X[1], S.y0, S.n));
    if (D == 3) TRY(download(c, X[2], S.z0, S.n));
    const double pi = 3.14159265358979323846;
    ptr.assign(1, 0);
    idx.clear();
    w.clear();
    g.clear();
    for (int b = 0; b < c->B; b++) {
        if (inst >= 0 && b != inst) continue;
        const InstHost &h = c->ih[b];
        const int s0 = h.d.s0;
        const double hS = h.d.P.hS_d, V0 = std::pow(h.s_dp, D);
        const double alpha = D == 2 ? 7.0 / (4.0 * pi * hS * hS) : 21.0 / (16.0 * pi * hS * hS * hS);
        std::vector<int> inv(h.ns);
        for (int64_t a = 0; a < h.ns; a++) inv[h.s_order[a]] = (int)a;
        for (int64_t r = 0; r < h.ns; r++) {
            // row r: device slot (device order) or the slot of original particle r
            const int a = s0 + (inst >= 0 ? inv[r] : (int)r);
            for (int q = hp[a]; q < hp[a + 1]; q++) {
                int bb;
                std::memcpy(&bb, &hnb[q].w, sizeof(int));
                double d2 = 0.0;
                for (int k = 0; k < D; k++) d2 += (X[k][a] - X[k][bb]) * (X[k][a] - X[k][bb]);
                const double qq = std::sqrt(d2) / hS, t = 1.0 - 0.5 * qq;
                idx.push_back(inst >= 0 ? h.s_order[bb - s0] : bb);
                w.push_back(V0 * alpha * t * t * t * t * (1.0 + 2.0 * qq));
                const float e[3] = {hnb[q].x, hnb[q].y, hnb[q].z};
                for (int k = 0; k < D; k++) g.push_back(hS * (double)e[k]);
            }
            ptr.push_back((int64_t)idx.size());
        }
    }
    // rows in original order: sort each row's columns ascending
    if (inst >= 0) {
        const size_t n = ptr.size() - 1;
        for (size_t r = 0; r < n; r++) {
            std::vector<size_t> o(ptr[r + 1] - ptr[r]);
            for (size_t k = 0; k < o.size(); k++) o[k] = ptr[r] + k;
            std::sort(o.begin(), o.end(), [&](size_t p, size_t q) { return idx[p] < idx[q]; });
            std::vector<int64_t> i2;
            std::vector<double> w2, g2;
            for (size_t p : o) {
                i2.push_back(idx[p]);
                w2.push_back(w[p]);
                for (int k = 0; k < D; k++) g2.push_back(g[p * D + k]);
            }
            std::copy(i2.begin(), i2.end(), idx.begin() + ptr[r]);
            std::copy(w2.begin(), w2.end(), w.begin() + ptr[r]);
            std::copy(g2.begin(), g2.end(), g.begin() + ptr[r] * D);
        }
    }
    return SPHFSI_OK;
}

int sphfsi_solid_graph(sphfsi_ctx *c, int64_t *ptr, int64_t *idx, double *w, double *g)
{
    TRY(check_ctx(c, true));
    std::vector<int64_t> p, i;
    std::vector<double> wv, gv;
    TRY(body_graph(c, c->sel, p, i, wv, gv));
    if (ptr) std::memcpy(ptr, p.data(), sizeof(int64_t) * p.size());
    if (idx && !i.empty()) std::memcpy(idx, i.data(), sizeof(int64_t) * i.size());
    if (w && !wv.empty()) std::memcpy(w, wv.data(), sizeof(double) * wv.size());
    if (g && !gv.empty()) std::memcpy(g, gv.data(), sizeof(double) * gv.size());
    return SPHFSI_OK;
}

int sphfsi_set_learned(sphfsi_ctx *c, const float *theta, const double *scales, double tol)
{
    TRY(check_ctx(c, true));
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (tol < 0.0) {
        c->S.learned = 0;
        return SPHFSI_OK;
    }
    if (!theta || !scales || c->S.n == 0 || std::isnan(tol)) return SPHFSI_E_INVAL;
    for (int k = 0; k < 7; k++)
        if (!(scales[k] > 0.0)) return SPHFSI_E_INVAL;
    Solid &S = c->S;
    if (!c->mpnn) {
        std::vector<int64_t> p, i;
        std::vector<double> wv, gv;
        TRY(body_graph(c, -1, p, i, wv, gv));
        TRY(sphfsi_mpnn_create(&c->mpnn, c->dim, S.n, (int64_t)i.size(), p.data(), i.data(), wv.data(), gv.data(), 1,
                               c->side));
        const int n = S.n, D = c->dim;
        TRY(dalloc(c, &S.lx, n));
        TRY(dalloc(c, &S.ly, n));
        TRY(dalloc(c, &S.lz, D == 3 ? n : 1));
        TRY(dalloc(c, &S.mx, n));
        TRY(dalloc(c, &S.my, n));
        TRY(dalloc(c, &S.mz, D == 3 ? n : 1));
        TRY(dalloc(c, &S.lv4, n));
        TRY(dalloc(c, &S.lH, (size_t)9 * n));
        TRY(dalloc(c, &S.lQ, (size_t)(D == 2 ? 1 : 3) * n));
        TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    }
    TRY(sphfsi_mpnn_set_params(c->mpnn, theta));
    S.l_su = (float)scales[0];
    S.l_sv = (float)scales[1];
    S.l_sf = (float)scales[2];
    S.l_st = (float)scales[3];
    S.l_sdu = (float)scales[4];
    S.l_sdv = (float)scales[5];
    S.l_sH = (float)scales[6];
    S.l_tol = tol > 3.0e38 ? 3.0e38f : (float)tol;
    S.learned = 1;
    return SPHFSI_OK;
}

int sphfsi_get_learned_features(sphfsi_ctx *c, float *x)
{
    TRY(check_ctx(c, true));
    if (!x) return SPHFSI_E_INVAL;
    if (!c->mpnn) return SPHFSI_E_STATE;
    constexpr int kFin = 64;
    std::vector<float> all;
    TRY(download(c, all, mpnn_input(c->mpnn), (size_t)c->S.n * kFin));
    const InstHost &h = c->ih[c->sel];
    std::vector<float> out((size_t)h.ns * kFin);
    // device row s0 + k holds original particle s_order[k]
    for (int64_t k = 0; k < h.ns; k++)
        std::memcpy(&out[(size_t)h.s_order[k] * kFin], &all[(size_t)(h.d.s0 + k) * kFin], sizeof(float) * kFin);
    return deliver(x, out);
}

int sphfsi_set_profiling(sphfsi_ctx *c, int on)
{
    TRY(check_ctx(c, true));
    c->profiling = on != 0;
    return SPHFSI_OK;
}

int sphfsi_stage_times(sphfsi_ctx *c, float *ms, int n)
{
    TRY(check_ctx(c, true));
    if (!ms || n < sphfsi_ctx::kStages) return SPHFSI_E_INVAL;
    if (!c->profiling) return SPHFSI_E_STATE;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    auto el = [&](int a, int b, float *o) { return cuda_rc(cudaEventElapsedTime(o, c->ev[a], c->ev[b])); };
    // events: 0 start, 2 binning, 3 reinit, 5 momentum, 6 continuity (main
    // stream); 4 branch start, 7 coupling force done, 8 sub-steps done (side
    // stream); 9 end of step
    TRY(el(0, 2, &ms[0]));
    TRY(el(2, 1, &ms[7]));
    TRY(el(1, 3, &ms[1]));
    TRY(el(3, 5, &ms[2]));
    TRY(el(5, 6, &ms[4]));
    if (c->S.n) {
        float fin_a = 0.f, fin_b = 0.f;
        TRY(el(4, 7, &ms[3]));
        TRY(el(7, 8, &ms[5]));
        TRY(el(6, 9, &fin_a));
        TRY(el(8, 9, &fin_b));
        ms[6] = fin_a < fin_b ? fin_a : fin_b;
    } else {
        ms[3] = ms[5] = 0.0f;
        TRY(el(6, 9, &ms[6]));
    }
    return sphfsi_ctx::kStages;
}

int sphfsi_step_time(sphfsi_ctx *c, float *ms)
{
    TRY(check_ctx(c, true));
    if (!ms) return SPHFSI_E_INVAL;
    if (!c->profiling) return SPHFSI_E_STATE;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    return cuda_rc(cudaEventElapsedTime(ms, c->ev[0], c->ev[9]));
}

void sphfsi_destroy(sphfsi_ctx *c)
{
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    if (c->side) cudaStreamSynchronize(c->side);
    if (c->mpnn) sphfsi_mpnn_destroy(c->mpnn);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    for (int k = 0; k < sphfsi_ctx::kEvents; k++)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->side) cudaStreamDestroy(c->side);
    for (auto &a : c->allocs) cudaFree(a.first);
    delete c;
}

}  // extern "C"
