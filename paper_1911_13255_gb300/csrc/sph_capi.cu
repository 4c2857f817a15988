// C-ABI of the sphfsi library (include/sphfsi.h): context, set-up, the
// per-step launch sequence a1..a8 and its CUDA-graph replay, state I/O.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "sph_common.cuh"
#include "sphfsi.h"

using namespace sph;

struct sphfsi_ctx {
    sphfsi_params prm;
    sphfsi_inflow inflow;
    cudaStream_t st;
    int dim;
    bool finalized = false;
    int K_fixed = 0;
    // host staging until finalize
    int64_t nf = 0, nw = 0, ns = 0;
    std::vector<double> f_r, f_v, f_p;
    bool f_has_p = false, f_added = false, w_added = false, s_added = false;
    double f_dp = 0, f_rho0 = 1, f_c0 = 1, f_eta = 0;
    std::vector<double> w_r, w_n;
    double w_dp = 0;
    std::vector<double> s_r0, s_v0, s_n0;
    std::vector<uint8_t> s_cons;
    std::vector<int> s_order;   // device (locality) index -> original solid index
    double s_dp = 0, s_rho0 = 1, s_E = 1, s_nu = 0.3;
    // device
    Grid g{};
    Phys P{};
    Fluid F{};
    Walls W{};
    Solid S{};
    Ctl *ctl = nullptr;
    std::vector<void *> allocs;
    // graph replay
    cudaGraphExec_t gexec = nullptr;
    double graph_dt = 0.0;
    int graph_K = -1;
    int solid_path = 0;
    unsigned long long ss_pairs = 0;
    int last_status = 0;
    // per-stage CUDA events (sphfsi_set_profiling): start, solid binned,
    // fluid sorted, reinit, momentum, solid-side force, continuity (main
    // stream), solid sub-steps begin/end (side stream), end of step
    static constexpr int kStages = 8;
    static constexpr int kEvents = 10;
    bool profiling = false;
    int graph_prof = -1;
    cudaEvent_t ev[kEvents] = {};
    int kernels_per_step = 0;
    // side stream for the solid sub-steps, which run concurrently with the
    // continuity kernel (both need only the coupling force and the records)
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
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
    c->allocs.push_back(q);
    *p = (T *)q;
    return SPHFSI_OK;
}

#define TRY(x)                         \
    do {                               \
        int _rc = (x);                 \
        if (_rc) return _rc < -7 ? SPHFSI_E_CUDA : _rc; \
    } while (0)

// copy n elements from a user pointer (host or device) into a host vector
template <typename T>
int fetch(std::vector<T> &dst, const T *src, size_t n)
{
    dst.resize(n);
    if (n == 0) return SPHFSI_OK;
    if (!src) return SPHFSI_E_INVAL;
    return cuda_rc(cudaMemcpy(dst.data(), src, sizeof(T) * n, cudaMemcpyDefault));
}

// copy a host buffer out to a user pointer (host or device)
template <typename T>
int deliver(T *dst, const std::vector<T> &src)
{
    if (!dst || src.empty()) return SPHFSI_OK;
    return cuda_rc(cudaMemcpy(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyDefault));
}

template <typename T>
int upload(sphfsi_ctx *c, T *dst, const std::vector<T> &src)
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

__global__ void k_set_step(Ctl *ctl, double dt_fixed, int K_fixed)
{
    ctl->dt_fixed = dt_fixed;
    ctl->K_fixed = K_fixed;
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
    TRY(mark(c, 0));
    // dt_F, K, reinit flag; a3 normal update before the solid records are built
    TRY(launch_control_normals(c->ctl, c->P, c->S, dt > 0.0 ? dt : 0.0, c->K_fixed, st));
    TRY(mark(c, 1));
    // a1 + a2: inflow, fluid first half drift; fluid (r^{n+1/2}) and solid
    // (r^n) binning, counting sort and FP32 records
    TRY(launch_bin_all(c->F, c->S, c->g, c->P, c->ctl, 1, st));
    TRY(mark(c, 2));
    // a3: density reinitialisation (no-op on other steps)
    TRY(launch_reinit(c->F, c->W, c->S, c->g, c->P, c->ctl, st));
    TRY(mark(c, 3));
    // The solid branch (a5 then a7 + a8) reads only the records written so
    // far, so it runs on the side stream while the main stream does a4 and
    // a6; the two join before finish.
    if (c->S.n) {
        TRY(cuda_rc(cudaEventRecord(c->fork_ev, st)));
        TRY(cuda_rc(cudaStreamWaitEvent(c->side, c->fork_ev, 0)));
        TRY(mark(c, 4, c->side));
        TRY(launch_solid_fluid_force(c->F, c->S, c->g, c->P, c->ctl, c->side));
        TRY(mark(c, 7, c->side));
        TRY(launch_solid_substeps(c->S, c->P, c->ctl, &c->solid_path, c->side));
        TRY(mark(c, 8, c->side));
        TRY(cuda_rc(cudaEventRecord(c->join_ev, c->side)));
    }
    TRY(launch_momentum(c->F, c->W, c->S, c->g, c->P, c->ctl, st));
    TRY(mark(c, 5));
    TRY(launch_density(c->F, c->W, c->S, c->g, c->P, c->ctl, st));
    TRY(mark(c, 6));
    if (c->S.n) TRY(cuda_rc(cudaStreamWaitEvent(st, c->join_ev, 0)));
    TRY(launch_finish(c->ctl, c->ss_pairs, st));
    TRY(mark(c, 9));
    // kernels of this library per step (memsets excluded)
    c->kernels_per_step = 10 + (c->S.n ? 2 : 0);
    return cuda_rc(cudaGetLastError());
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
    case SPHFSI_E_UNSTABLE: return "non-finite state detected on the device";
    case SPHFSI_E_TIMEOUT: return "bounded device wait timed out";
    case SPHFSI_E_CAPACITY: return "problem exceeds a device limit";
    default: return "unknown error";
    }
}

int sphfsi_create(sphfsi_ctx **out, const sphfsi_params *p, void *cuda_stream)
{
    if (!out || !p) return SPHFSI_E_INVAL;
    *out = nullptr;
    if (p->dim != 2 && p->dim != 3) return SPHFSI_E_INVAL;
    if (p->periodic_x && !(p->Lx > 0.0)) return SPHFSI_E_INVAL;
    for (int k = 0; k < p->dim; k++)
        if (!(p->domain_hi[k] > p->domain_lo[k])) return SPHFSI_E_INVAL;
    sphfsi_ctx *c = new (std::nothrow) sphfsi_ctx();
    if (!c) return SPHFSI_E_NOMEM;
    c->prm = *p;
    c->dim = p->dim;
    c->st = (cudaStream_t)cuda_stream;
    std::memset(&c->inflow, 0, sizeof(c->inflow));
    *out = c;
    return SPHFSI_OK;
}

int sphfsi_add_fluid(sphfsi_ctx *c, int64_t n, const double *r, const double *v, const double *p_init, double dp,
                     double rho0, double c0, double eta)
{
    TRY(check_ctx(c, false));
    if (c->f_added || n < 0 || n > (int64_t)1 << 30 || !(dp > 0) || !(rho0 > 0) || !(c0 > 0) || eta < 0)
        return SPHFSI_E_INVAL;
    if (n > 0 && (!r || !v)) return SPHFSI_E_INVAL;
    TRY(fetch(c->f_r, r, (size_t)n * c->dim));
    TRY(fetch(c->f_v, v, (size_t)n * c->dim));
    c->f_has_p = p_init != nullptr;
    if (p_init) TRY(fetch(c->f_p, p_init, (size_t)n));
    c->nf = n;
    c->f_dp = dp;
    c->f_rho0 = rho0;
    c->f_c0 = c0;
    c->f_eta = eta;
    c->f_added = true;
    return SPHFSI_OK;
}

int sphfsi_set_walls(sphfsi_ctx *c, int64_t n, const double *r, const double *nrm, double dp)
{
    TRY(check_ctx(c, false));
    if (c->w_added || n < 0 || n > (int64_t)1 << 30 || !(dp > 0)) return SPHFSI_E_INVAL;
    if (n > 0 && (!r || !nrm)) return SPHFSI_E_INVAL;
    TRY(fetch(c->w_r, r, (size_t)n * c->dim));
    TRY(fetch(c->w_n, nrm, (size_t)n * c->dim));
    c->nw = n;
    c->w_dp = dp;
    c->w_added = true;
    return SPHFSI_OK;
}

int sphfsi_add_solid(sphfsi_ctx *c, int64_t n, const double *r0, const double *v0, const double *n0,
                     const uint8_t *constrained, double dp, double rho0, double E, double nu)
{
    TRY(check_ctx(c, false));
    if (c->s_added || n < 0 || n > (int64_t)1 << 26 || !(dp > 0) || !(rho0 > 0) || !(E > 0) || !(nu > -1.0) ||
        !(nu < 0.5))
        return SPHFSI_E_INVAL;
    if (n > 0 && (!r0 || !v0 || !n0 || !constrained)) return SPHFSI_E_INVAL;
    TRY(fetch(c->s_r0, r0, (size_t)n * c->dim));
    TRY(fetch(c->s_v0, v0, (size_t)n * c->dim));
    TRY(fetch(c->s_n0, n0, (size_t)n * c->dim));
    TRY(fetch(c->s_cons, constrained, (size_t)n));
    c->ns = n;
    c->s_dp = dp;
    c->s_rho0 = rho0;
    c->s_E = E;
    c->s_nu = nu;
    c->s_added = true;
    return SPHFSI_OK;
}

int sphfsi_set_inflow(sphfsi_ctx *c, const sphfsi_inflow *f)
{
    TRY(check_ctx(c, false));
    if (!f || (f->on && (!(f->width > 0) || (f->profile == 0 && !(f->H > 0))))) return SPHFSI_E_INVAL;
    c->inflow = *f;
    return SPHFSI_OK;
}

int sphfsi_finalize(sphfsi_ctx *c)
{
    TRY(check_ctx(c, false));
    if (!c->f_added) return SPHFSI_E_STATE;
    const int D = c->dim;
    const double hF = 1.3 * c->f_dp;
    // ---- grid: cells of edge >= 2 h_F
    Grid &g = c->g;
    std::memset(&g, 0, sizeof(g));
    int64_t ncell = 1;
    for (int k = 0; k < 3; k++) {
        if (k >= D) {
            g.lo[k] = 0.0;
            g.cs[k] = 1.0;
            g.csf[k] = 1.0f;
            g.nc[k] = 1;
            continue;
        }
        double lo = c->prm.domain_lo[k], L = c->prm.domain_hi[k] - lo;
        if (k == 0 && c->prm.periodic_x) {
            lo = c->prm.x_lo;
            L = c->prm.Lx;
        }
        int64_t n = (int64_t)std::floor(L / (2.0 * hF));
        if (n < 1) n = 1;
        if (k == 0 && c->prm.periodic_x && n < 3) return SPHFSI_E_INVAL;
        g.lo[k] = lo;
        g.nc[k] = (int)n;
        g.cs[k] = L / (double)n;
        g.csf[k] = (float)g.cs[k];
        ncell *= n;
        if (ncell > ((int64_t)1 << 28)) return SPHFSI_E_CAPACITY;
    }
    g.ncell = (int)ncell;
    g.periodic_x = c->prm.periodic_x;
    g.x_lo = c->prm.x_lo;
    g.Lx = c->prm.Lx;
    // ---- physical constants
    Phys &P = c->P;
    std::memset(&P, 0, sizeof(P));
    const double pi = 3.14159265358979323846;
    P.dim = D;
    for (int k = 0; k < 3; k++) P.g[k] = (float)c->prm.gravity[k];
    P.rho0 = (float)c->f_rho0;
    P.c0 = (float)c->f_c0;
    P.eta = (float)c->f_eta;
    P.hF = (float)hF;
    P.inv_hF = (float)(1.0 / hF);
    P.rc2F = (float)(4.0 * hF * hF);
    P.rc2F_d = 4.0 * hF * hF;
    double alpha = D == 2 ? 7.0 / (4.0 * pi * hF * hF) : 21.0 / (16.0 * pi * hF * hF * hF);
    P.WcF = (float)alpha;
    P.dWcF = (float)(-5.0 * alpha / hF);
    double VF = std::pow(c->f_dp, D);
    P.mF = (float)(c->f_rho0 * VF);
    P.p_coef = (float)(c->f_rho0 * c->f_c0 * c->f_c0 / 7.0);
    P.inv_p_coef = (float)(7.0 / (c->f_rho0 * c->f_c0 * c->f_c0));
    P.hreg = (float)(0.01 * hF);
    P.sigma0 = (float)lattice_sigma0(D, c->f_dp, hF);
    P.sigma0_d = lattice_sigma0(D, c->f_dp, hF);
    P.alphaF_d = alpha;
    double VW = c->w_dp > 0 ? std::pow(c->w_dp, D) : VF;
    double VS = c->s_dp > 0 ? std::pow(c->s_dp, D) : VF;
    P.VW = (float)VW;
    P.VS = (float)VS;
    P.VW_VF = (float)(VW / VF);
    P.VS_VF = (float)(VS / VF);
    P.VW_VF_d = VW / VF;
    P.VS_VF_d = VS / VF;
    P.free_surface = c->prm.free_surface;
    P.hF_d = hF;
    P.c0_d = c->f_c0;
    P.eta_d = c->f_eta;
    P.rho0_d = c->f_rho0;
    if (c->ns > 0) {
        double mu = c->s_E / (2.0 * (1.0 + c->s_nu));            // reading R10
        double lam = 2.0 * mu * c->s_nu / (1.0 - 2.0 * c->s_nu);
        P.rhoS = (float)c->s_rho0;
        P.mS = (float)(c->s_rho0 * VS);
        P.mu = (float)mu;
        P.lam = (float)lam;
        P.hS = (float)(1.3 * c->s_dp);
        P.hS_d = 1.3 * c->s_dp;
        P.cS_d = std::sqrt(c->s_E / (3.0 * (1.0 - 2.0 * c->s_nu)) / c->s_rho0);
    }
    P.inflow_on = c->inflow.on;
    P.inflow_profile = c->inflow.profile;
    P.in_w = c->inflow.width;
    P.in_y0 = c->inflow.y0;
    P.in_H = c->inflow.H;
    P.in_U = c->inflow.U;
    P.in_tramp = c->inflow.t_ramp;

    // ---- control block
    TRY(dalloc(c, &c->ctl, 1));
    // ---- fluid
    Fluid &F = c->F;
    F.n = (int)c->nf;
    for (int b = 0; b < 2; b++) {
        FluidState &S = F.s[b];
        TRY(dalloc(c, &S.x, F.n));
        TRY(dalloc(c, &S.y, F.n));
        TRY(dalloc(c, &S.z, D == 3 ? F.n : 1));
        TRY(dalloc(c, &S.vx, F.n));
        TRY(dalloc(c, &S.vy, F.n));
        TRY(dalloc(c, &S.vz, D == 3 ? F.n : 1));
        TRY(dalloc(c, &S.drho, F.n));
        TRY(dalloc(c, &S.rhodot, F.n));
        TRY(dalloc(c, &S.id, F.n));
        if (D == 2) S.z = nullptr, S.vz = nullptr;
    }
    TRY(dalloc(c, &F.P4, F.n));
    TRY(dalloc(c, &F.V4, F.n));
    TRY(dalloc(c, &F.W4, F.n));
    TRY(dalloc(c, &F.dvdt, (size_t)F.n * D));
    TRY(dalloc(c, &F.key, F.n));
    TRY(dalloc(c, &F.perm, F.n));
    TRY(dalloc(c, &F.cell_of, F.n));
    TRY(dalloc(c, &F.cstart, (size_t)g.ncell + 1));
    TRY(dalloc(c, &F.ccount, g.ncell));
    {
        std::vector<double> xyz[3];
        deinterleave(c->f_r, D, c->nf, xyz);
        std::vector<float> v[3];
        for (int k = 0; k < 3; k++) v[k].assign(c->nf, 0.0f);
        std::vector<float> drho(c->nf, 0.0f);
        std::vector<int> id(c->nf);
        double vmax = 0.0;
        for (int64_t i = 0; i < c->nf; i++) {
            double v2 = 0.0;
            for (int k = 0; k < D; k++) {
                v[k][i] = (float)c->f_v[i * D + k];
                v2 += (double)v[k][i] * (double)v[k][i];
            }
            vmax = std::max(vmax, std::sqrt(v2));
            if (c->f_has_p) {
                // inverse of Eq. eqeos: rho - rho0 = rho0 expm1(log1p(7 p / (rho0 c0^2)) / 7)
                double x = 7.0 * c->f_p[i] / (c->f_rho0 * c->f_c0 * c->f_c0);
                if (!(x > -1.0)) return SPHFSI_E_INVAL;
                drho[i] = (float)(c->f_rho0 * std::expm1(std::log1p(x) / 7.0));
            }
            id[i] = (int)i;
        }
        FluidState &S = F.s[0];
        TRY(upload(c, S.x, xyz[0]));
        TRY(upload(c, S.y, xyz[1]));
        if (D == 3) TRY(upload(c, S.z, xyz[2]));
        TRY(upload(c, S.vx, v[0]));
        TRY(upload(c, S.vy, v[1]));
        if (D == 3) TRY(upload(c, S.vz, v[2]));
        TRY(upload(c, S.drho, drho));
        TRY(upload(c, S.id, id));
        Ctl h{};
        h.vmaxF = 0;
        float vmf = (float)vmax;
        std::memcpy(&h.vmaxF, &vmf, 4);
        h.n_reinit = c->prm.n_reinit;
        // solid maxima at rest
        if (c->ns > 0) {
            double vs = 0.0;
            for (int64_t a = 0; a < c->ns; a++) {
                if (c->s_cons[a]) continue;
                double v2 = 0.0;
                for (int k = 0; k < D; k++) v2 += c->s_v0[a * D + k] * c->s_v0[a * D + k];
                vs = std::max(vs, std::sqrt(v2));
            }
            float vsf = (float)vs;
            std::memcpy(&h.vmaxS, &vsf, 4);
        }
        TRY(cuda_rc(cudaMemcpyAsync(c->ctl, &h, sizeof(h), cudaMemcpyHostToDevice, c->st)));
        TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    }
    // ---- walls
    Walls &W = c->W;
    W.n = (int)c->nw;
    {
        TRY(dalloc(c, &W.x, W.n));
        TRY(dalloc(c, &W.y, W.n));
        TRY(dalloc(c, &W.z, D == 3 ? W.n : 1));
        TRY(dalloc(c, &W.nx, W.n));
        TRY(dalloc(c, &W.ny, W.n));
        TRY(dalloc(c, &W.nz, D == 3 ? W.n : 1));
        if (D == 2) W.z = nullptr, W.nz = nullptr;
        TRY(dalloc(c, &W.A4, W.n));
        TRY(dalloc(c, &W.N4, W.n));
        TRY(dalloc(c, &W.key, W.n));
        TRY(dalloc(c, &W.perm, W.n));
        TRY(dalloc(c, &W.cell_of, W.n));
        TRY(dalloc(c, &W.cstart, (size_t)g.ncell + 1));
        TRY(dalloc(c, &W.ccount, g.ncell));
        std::vector<double> xyz[3], nn[3];
        deinterleave(c->w_r, D, c->nw, xyz);
        deinterleave(c->w_n, D, c->nw, nn);
        std::vector<float> nf[3];
        for (int k = 0; k < 3; k++) nf[k].assign(nn[k].begin(), nn[k].end());
        TRY(upload(c, W.x, xyz[0]));
        TRY(upload(c, W.y, xyz[1]));
        if (D == 3) TRY(upload(c, W.z, xyz[2]));
        TRY(upload(c, W.nx, nf[0]));
        TRY(upload(c, W.ny, nf[1]));
        if (D == 3) TRY(upload(c, W.nz, nf[2]));
        TRY(launch_wall_bin(W, g, c->st));
    }
    // ---- solid
    Solid &S = c->S;
    S.n = (int)c->ns;
    {
        int n = S.n;
        TRY(dalloc(c, &S.x, n));
        TRY(dalloc(c, &S.y, n));
        TRY(dalloc(c, &S.z, D == 3 ? n : 1));
        TRY(dalloc(c, &S.x0, n));
        TRY(dalloc(c, &S.y0, n));
        TRY(dalloc(c, &S.z0, D == 3 ? n : 1));
        TRY(dalloc(c, &S.xs, n));
        TRY(dalloc(c, &S.ys, n));
        TRY(dalloc(c, &S.zs, D == 3 ? n : 1));
        if (D == 2) S.z = S.z0 = S.zs = nullptr;
        TRY(dalloc(c, &S.v4, n));
        TRY(dalloc(c, &S.H, (size_t)9 * n));
        TRY(dalloc(c, &S.Hd, (size_t)9 * n));
        TRY(dalloc(c, &S.B0, (size_t)9 * n));
        TRY(dalloc(c, &S.Q4, (size_t)(D == 2 ? 1 : 3) * n));
        TRY(dalloc(c, &S.n0, (size_t)3 * n));
        TRY(dalloc(c, &S.nrm, (size_t)3 * n));
        TRY(dalloc(c, &S.cons, n));
        TRY(dalloc(c, &S.vbar, (size_t)3 * n));
        TRY(dalloc(c, &S.abar, (size_t)3 * n));
        TRY(dalloc(c, &S.asum, (size_t)3 * n));
        TRY(dalloc(c, &S.fF, (size_t)3 * n));
        TRY(dalloc(c, &S.nb_ptr, (size_t)n + 1));
        TRY(dalloc(c, &S.A4, n));
        TRY(dalloc(c, &S.VB4, n));
        TRY(dalloc(c, &S.AB4, n));
        TRY(dalloc(c, &S.N4, n));
        TRY(dalloc(c, &S.key, n));
        TRY(dalloc(c, &S.perm, n));
        TRY(dalloc(c, &S.cell_of, n));
        TRY(dalloc(c, &S.cstart, (size_t)g.ncell + 1));
        TRY(dalloc(c, &S.ccount, g.ncell));
        TRY(dalloc(c, &S.bar, 2));
        if (n > 0) {
            // Locality order of the body on the device: lexicographic on the
            // lattice index along the axes sorted by decreasing extent, so
            // that a particle's neighbours sit within a few rows of it and
            // mostly in the same CTA of the cluster-resident sub-step kernel.
            {
                double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
                for (int a = 0; a < n; a++)
                    for (int k = 0; k < D; k++) {
                        lo[k] = std::min(lo[k], c->s_r0[(size_t)a * D + k]);
                        hi[k] = std::max(hi[k], c->s_r0[(size_t)a * D + k]);
                    }
                int ax[3] = {0, 1, 2};
                std::sort(ax, ax + D, [&](int p, int q) { return hi[p] - lo[p] > hi[q] - lo[q]; });
                std::vector<std::array<long long, 4>> key(n);
                for (int a = 0; a < n; a++) {
                    for (int k = 0; k < 3; k++)
                        key[a][k] = k < D ? std::llround((c->s_r0[(size_t)a * D + ax[k]] - lo[ax[k]]) / c->s_dp) : 0;
                    key[a][3] = a;
                }
                std::sort(key.begin(), key.end());
                c->s_order.resize(n);
                for (int a = 0; a < n; a++) c->s_order[a] = (int)key[a][3];
                auto perm_rows = [&](auto &v, int w) {
                    auto t = v;
                    for (int a = 0; a < n; a++)
                        for (int j = 0; j < w; j++) t[(size_t)a * w + j] = v[(size_t)c->s_order[a] * w + j];
                    v.swap(t);
                };
                perm_rows(c->s_r0, D);
                perm_rows(c->s_v0, D);
                perm_rows(c->s_n0, D);
                perm_rows(c->s_cons, 1);
            }
            std::vector<double> xyz[3];
            deinterleave(c->s_r0, D, c->ns, xyz);
            std::vector<float4> v4(n);
            std::vector<float> n0(3 * (size_t)n, 0.0f);
            std::vector<double> vbar(3 * (size_t)n, 0.0);
            for (int a = 0; a < n; a++) {
                double vv[3] = {0, 0, 0};
                for (int k = 0; k < D; k++) {
                    vv[k] = c->s_cons[a] ? 0.0 : c->s_v0[(size_t)a * D + k];
                    n0[3 * a + k] = (float)c->s_n0[(size_t)a * D + k];
                    vbar[3 * a + k] = vv[k];
                }
                v4[a] = make_float4((float)vv[0], (float)vv[1], (float)vv[2], 0.0f);
            }
            TRY(upload(c, S.x0, xyz[0]));
            TRY(upload(c, S.y0, xyz[1]));
            TRY(upload(c, S.x, xyz[0]));
            TRY(upload(c, S.y, xyz[1]));
            if (D == 3) {
                TRY(upload(c, S.z0, xyz[2]));
                TRY(upload(c, S.z, xyz[2]));
            }
            TRY(upload(c, S.v4, v4));
            TRY(upload(c, S.n0, n0));
            TRY(upload(c, S.nrm, n0));
            TRY(upload(c, S.cons, c->s_cons));
            TRY(upload(c, S.vbar, vbar));
            // static reference neighbour list: counts, host scan, fill
            int *counts = nullptr;
            TRY(dalloc(c, &counts, n));
            TRY(launch_solid_setup_count(S, P, counts, c->st));
            std::vector<int> hc;
            TRY(download(c, hc, counts, n));
            std::vector<int> ptr(n + 1, 0);
            S.max_nb = 0;
            for (int a = 0; a < n; a++) {
                ptr[a + 1] = ptr[a] + hc[a];
                S.max_nb = std::max(S.max_nb, hc[a]);
            }
            S.nnz = ptr[n];
            TRY(upload(c, S.nb_ptr, ptr));
            TRY(dalloc(c, &S.nb, S.nnz));
            TRY(launch_solid_setup_fill(S, P, c->st));
            c->ss_pairs = (unsigned long long)S.nnz;
        }
    }
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    for (int k = 0; k < sphfsi_ctx::kEvents; k++) TRY(cuda_rc(cudaEventCreate(&c->ev[k])));
    TRY(cuda_rc(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking)));
    TRY(cuda_rc(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming)));
    TRY(cuda_rc(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming)));
    c->finalized = true;
    // release the host staging copies
    c->f_r.clear(); c->f_v.clear(); c->f_p.clear();
    c->w_r.clear(); c->w_n.clear();
    return SPHFSI_OK;
}

int sphfsi_set_substeps(sphfsi_ctx *c, int32_t K)
{
    if (!c || K < 0) return SPHFSI_E_INVAL;
    c->K_fixed = K;
    return SPHFSI_OK;
}

int sphfsi_step(sphfsi_ctx *c, double dt_F)
{
    TRY(check_ctx(c, true));
    if (std::isnan(dt_F)) return SPHFSI_E_INVAL;
    return enqueue_step(c, dt_F);
}

int sphfsi_run(sphfsi_ctx *c, int64_t nsteps, double dt_F)
{
    TRY(check_ctx(c, true));
    if (nsteps < 0 || std::isnan(dt_F)) return SPHFSI_E_INVAL;
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
    int status = 0;
    TRY(cuda_rc(cudaMemcpy(&status, &c->ctl->status, sizeof(int), cudaMemcpyDeviceToHost)));
    c->last_status = status;
    if (status & ST_TIMEOUT) return SPHFSI_E_TIMEOUT;
    if (status & ST_NONFINITE) return SPHFSI_E_UNSTABLE;
    return SPHFSI_OK;
}

int sphfsi_get_fluid(sphfsi_ctx *c, double *r, float *v, double *rho, float *drho_dt, float *dvdt)
{
    TRY(check_ctx(c, true));
    const int D = c->dim;
    const int64_t n = c->nf;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    const FluidState &S = c->F.s[0];
    std::vector<int> id;
    TRY(download(c, id, S.id, n));
    if (r) {
        std::vector<double> x, y, z, out(n * D);
        TRY(download(c, x, S.x, n));
        TRY(download(c, y, S.y, n));
        if (D == 3) TRY(download(c, z, S.z, n));
        for (int64_t k = 0; k < n; k++) {
            out[(size_t)id[k] * D] = x[k];
            out[(size_t)id[k] * D + 1] = y[k];
            if (D == 3) out[(size_t)id[k] * D + 2] = z[k];
        }
        TRY(deliver(r, out));
    }
    if (v) {
        std::vector<float> x, y, z, out(n * D);
        TRY(download(c, x, S.vx, n));
        TRY(download(c, y, S.vy, n));
        if (D == 3) TRY(download(c, z, S.vz, n));
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
        TRY(download(c, d, S.drho, n));
        for (int64_t k = 0; k < n; k++) out[id[k]] = c->f_rho0 + (double)d[k];
        TRY(deliver(rho, out));
    }
    if (drho_dt) {
        std::vector<float> d, out(n);
        TRY(download(c, d, S.rhodot, n));
        for (int64_t k = 0; k < n; k++) out[id[k]] = d[k];
        TRY(deliver(drho_dt, out));
    }
    if (dvdt) {
        std::vector<float> d, out(n * D);
        TRY(download(c, d, c->F.dvdt, (size_t)n * D));
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
    const int64_t n = c->ns;
    const Solid &S = c->S;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    if (n == 0) return SPHFSI_OK;
    const std::vector<int> &ord = c->s_order;   // device index -> original index
    if (r) {
        std::vector<double> x, y, z, out(n * D);
        TRY(download(c, x, S.x, n));
        TRY(download(c, y, S.y, n));
        if (D == 3) TRY(download(c, z, S.z, n));
        for (int64_t a = 0; a < n; a++) {
            size_t o = (size_t)ord[a] * D;
            out[o] = x[a];
            out[o + 1] = y[a];
            if (D == 3) out[o + 2] = z[a];
        }
        TRY(deliver(r, out));
    }
    if (v) {
        std::vector<float4> h;
        TRY(download(c, h, S.v4, n));
        std::vector<float> out(n * D);
        for (int64_t a = 0; a < n; a++) {
            size_t o = (size_t)ord[a] * D;
            out[o] = h[a].x;
            out[o + 1] = h[a].y;
            if (D == 3) out[o + 2] = h[a].z;
        }
        TRY(deliver(v, out));
    }
    if (F) {
        std::vector<float> h;
        std::vector<double> out(n * D * D);
        TRY(download(c, h, S.H, (size_t)9 * n));
        for (int64_t a = 0; a < n; a++)
            for (int i = 0; i < D * D; i++)
                out[(size_t)ord[a] * D * D + i] = (double)h[9 * a + i] + ((i % (D + 1)) == 0 ? 1.0 : 0.0);
        TRY(deliver(F, out));
    }
    auto vec3 = [&](const auto *src, auto *dst, auto zero) -> int {
        using T = decltype(zero);
        if (!dst) return SPHFSI_OK;
        std::vector<T> h, out(n * D);
        int rc = download(c, h, src, (size_t)3 * n);
        if (rc) return rc;
        for (int64_t a = 0; a < n; a++)
            for (int k = 0; k < D; k++) out[(size_t)ord[a] * D + k] = h[3 * a + k];
        return deliver(dst, out);
    };
    TRY(vec3(S.vbar, vbar, 0.0));
    TRY(vec3(S.abar, abar, 0.0));
    TRY(vec3(S.fF, fF, 0.0f));
    TRY(vec3(S.nrm, nrm, 0.0f));
    return SPHFSI_OK;
}

int sphfsi_set_fluid_state(sphfsi_ctx *c, const double *r, const double *v, const double *rho, const double *drho_dt)
{
    TRY(check_ctx(c, true));
    const int D = c->dim;
    const int64_t n = c->nf;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    FluidState &S = c->F.s[0];
    // the state is written in original order (storage order = id = identity)
    std::vector<int> cur_id;
    TRY(download(c, cur_id, S.id, n));
    std::vector<int> inv(n);
    for (int64_t k = 0; k < n; k++) inv[cur_id[k]] = (int)k;
    auto reorder_f = [&](const float *dev, std::vector<float> &out) -> int {
        std::vector<float> h;
        int rc = download(c, h, dev, n);
        if (rc) return rc;
        out.resize(n);
        for (int64_t i = 0; i < n; i++) out[i] = h[inv[i]];
        return SPHFSI_OK;
    };
    auto reorder_d = [&](const double *dev, std::vector<double> &out) -> int {
        std::vector<double> h;
        int rc = download(c, h, dev, n);
        if (rc) return rc;
        out.resize(n);
        for (int64_t i = 0; i < n; i++) out[i] = h[inv[i]];
        return SPHFSI_OK;
    };
    std::vector<double> x, y, z;
    std::vector<float> vx, vy, vz, dr, rd;
    TRY(reorder_d(S.x, x));
    TRY(reorder_d(S.y, y));
    if (D == 3) TRY(reorder_d(S.z, z));
    TRY(reorder_f(S.vx, vx));
    TRY(reorder_f(S.vy, vy));
    if (D == 3) TRY(reorder_f(S.vz, vz));
    TRY(reorder_f(S.drho, dr));
    TRY(reorder_f(S.rhodot, rd));
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
        for (int64_t i = 0; i < n; i++) dr[i] = (float)(in[i] - c->f_rho0);
    }
    if (drho_dt) {
        TRY(fetch(in, drho_dt, (size_t)n));
        for (int64_t i = 0; i < n; i++) rd[i] = (float)in[i];
    }
    std::vector<int> id(n);
    for (int64_t i = 0; i < n; i++) id[i] = (int)i;
    TRY(upload(c, S.x, x));
    TRY(upload(c, S.y, y));
    if (D == 3) TRY(upload(c, S.z, z));
    TRY(upload(c, S.vx, vx));
    TRY(upload(c, S.vy, vy));
    if (D == 3) TRY(upload(c, S.vz, vz));
    TRY(upload(c, S.drho, dr));
    TRY(upload(c, S.rhodot, rd));
    TRY(upload(c, S.id, id));
    return cuda_rc(cudaStreamSynchronize(c->st));
}

int sphfsi_set_solid_state(sphfsi_ctx *c, const double *r, const double *v, const double *F, const double *vbar,
                           const double *abar, const double *nrm)
{
    TRY(check_ctx(c, true));
    const int D = c->dim;
    const int64_t n = c->ns;
    Solid &S = c->S;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    if (n == 0) return SPHFSI_OK;
    std::vector<double> in;
    // rows arrive in original order; the device keeps its locality order
    auto to_dev = [&](int w) {
        std::vector<double> t(in.size());
        for (int64_t a = 0; a < n; a++)
            for (int j = 0; j < w; j++) t[(size_t)a * w + j] = in[(size_t)c->s_order[a] * w + j];
        in.swap(t);
    };
    if (r) {
        TRY(fetch(in, r, (size_t)n * D));
        to_dev(D);
        std::vector<double> xyz[3];
        deinterleave(in, D, n, xyz);
        TRY(upload(c, S.x, xyz[0]));
        TRY(upload(c, S.y, xyz[1]));
        if (D == 3) TRY(upload(c, S.z, xyz[2]));
    }
    if (v) {
        TRY(fetch(in, v, (size_t)n * D));
        to_dev(D);
        std::vector<float4> h(n);
        for (int64_t a = 0; a < n; a++)
            h[a] = make_float4((float)in[a * D], (float)in[a * D + 1], D == 3 ? (float)in[a * D + 2] : 0.0f, 0.0f);
        TRY(upload(c, S.v4, h));
    }
    if (F) {
        TRY(fetch(in, F, (size_t)n * D * D));
        to_dev(D * D);
        std::vector<float> h(9 * (size_t)n, 0.0f);
        for (int64_t a = 0; a < n; a++)
            for (int i = 0; i < D * D; i++) h[9 * a + i] = (float)(in[a * D * D + i] - ((i % (D + 1)) == 0 ? 1.0 : 0.0));
        TRY(upload(c, S.H, h));
    }
    auto put3 = [&](const double *src, auto *dev, auto zero) -> int {
        using T = decltype(zero);
        if (!src) return SPHFSI_OK;
        int rc = fetch(in, src, (size_t)n * D);
        if (rc) return rc;
        to_dev(D);
        std::vector<T> h(3 * (size_t)n, (T)0);
        for (int64_t a = 0; a < n; a++)
            for (int k = 0; k < D; k++) h[3 * a + k] = (T)in[a * D + k];
        return upload(c, dev, h);
    };
    TRY(put3(vbar, S.vbar, 0.0));
    TRY(put3(abar, S.abar, 0.0));
    TRY(put3(nrm, S.nrm, 0.0f));
    return cuda_rc(cudaStreamSynchronize(c->st));
}

int sphfsi_set_time(sphfsi_ctx *c, double t, int64_t step)
{
    TRY(check_ctx(c, true));
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    Ctl h;
    TRY(cuda_rc(cudaMemcpy(&h, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost)));
    h.t = t;
    h.step = step;
    return cuda_rc(cudaMemcpy(c->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice));
}

int sphfsi_get_info(sphfsi_ctx *c, sphfsi_info *out)
{
    if (!c || !out) return SPHFSI_E_INVAL;
    std::memset(out, 0, sizeof(*out));
    out->n_fluid = c->nf;
    out->n_solid = c->ns;
    out->n_wall = c->nw;
    if (!c->finalized) return SPHFSI_OK;
    out->n_cells = c->g.ncell;
    TRY(cuda_rc(cudaStreamSynchronize(c->st)));
    Ctl h;
    TRY(cuda_rc(cudaMemcpy(&h, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost)));
    out->step = h.step;
    out->t = h.t;
    out->last_dt = h.last_dt;
    out->last_K = h.last_K;
    out->status = h.status;
    out->pairs_ff = (int64_t)h.n_ff;
    out->pairs_fw = (int64_t)h.n_fw;
    out->pairs_fs = (int64_t)h.n_fs;
    out->pairs_sf = (int64_t)h.n_sf;
    out->pairs_ss = (int64_t)c->S.nnz;
    out->pairs_total = (int64_t)h.pairs_total;
    float f;
    std::memcpy(&f, &h.vmaxF, 4);
    out->vmax_f = f;
    std::memcpy(&f, &h.vmaxS, 4);
    out->vmax_s = f;
    std::memcpy(&f, &h.amaxS, 4);
    out->amax_s = f;
    for (int k = 0; k < 3; k++) {
        out->mom_fs_fluid[k] = h.mom_fluid[k];
        out->mom_fs_solid[k] = h.mom_solid[k];
    }
    out->solid_path = c->solid_path;
    out->kernels_per_step = c->kernels_per_step;
    return SPHFSI_OK;
}

int sphfsi_debug_neighbors(sphfsi_ctx *c, int which, int64_t *ptr, int64_t *idx, int64_t *nnz)
{
    TRY(check_ctx(c, true));
    if (which < 0 || which > 3 || !nnz) return SPHFSI_E_INVAL;
    int64_t nrows = which == 3 ? c->ns : c->nf;
    // bin the current positions (no drift) and build the solid records
    TRY(launch_bin_all(c->F, c->S, c->g, c->P, c->ctl, 0, c->st));
    int *counts = nullptr, *offs = nullptr, *out = nullptr;
    if (cudaMalloc(&counts, sizeof(int) * (nrows + 1)) != cudaSuccess) return SPHFSI_E_NOMEM;
    int rc = launch_debug_pairs(c->F, c->W, c->S, c->g, c->P, which, counts, nullptr, nullptr, c->st);
    // solid rows (which 3) and solid columns (which 2) come in the device's
    // locality order; rows and columns are reported in original order
    std::vector<int> hc_dev, hc(nrows, 0);
    if (!rc) rc = download(c, hc_dev, counts, nrows);
    for (int64_t i = 0; i < nrows && !rc; i++) hc[which == 3 ? c->s_order[i] : i] = hc_dev[i];
    std::vector<int64_t> p(nrows + 1, 0);
    for (int64_t i = 0; i < nrows && !rc; i++) p[i + 1] = p[i] + hc[i];
    *nnz = p[nrows];
    if (!rc && ptr) std::memcpy(ptr, p.data(), sizeof(int64_t) * (nrows + 1));
    if (!rc && idx && p[nrows] > 0) {
        std::vector<int> po(nrows);
        for (int64_t i = 0; i < nrows; i++) po[i] = (int)p[which == 3 ? c->s_order[i] : i];
        if (cudaMalloc(&offs, sizeof(int) * nrows) != cudaSuccess || cudaMalloc(&out, sizeof(int) * p[nrows]) != cudaSuccess)
            rc = SPHFSI_E_NOMEM;
        if (!rc) rc = upload(c, offs, po);
        if (!rc) rc = launch_debug_pairs(c->F, c->W, c->S, c->g, c->P, which, counts, offs, out, c->st);
        std::vector<int> h;
        if (!rc) rc = download(c, h, out, (size_t)p[nrows]);
        if (!rc) {
            if (which == 2)
                for (auto &col : h) col = c->s_order[col];
            for (int64_t i = 0; i < nrows; i++) {
                std::sort(h.begin() + p[i], h.begin() + p[i + 1]);
                for (int64_t q = p[i]; q < p[i + 1]; q++) idx[q] = h[q];
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
    c->S.force_grid_path = path == 2 ? 1 : 0;
    c->S.force_lane_path = path == 1 ? 1 : 0;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return SPHFSI_OK;
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
    auto el = [&](int a, int b, float *out) { return cuda_rc(cudaEventElapsedTime(out, c->ev[a], c->ev[b])); };
    // events: 0 start, 1 control, 2 binning, 3 reinit, 5 momentum, 6 continuity
    // (main stream); 4 branch start, 7 coupling force done, 8 sub-steps done
    // (side stream); 9 end of step
    TRY(el(0, 1, &ms[0]));
    TRY(el(1, 2, &ms[1]));
    TRY(el(2, 3, &ms[2]));
    TRY(el(3, 5, &ms[3]));
    TRY(el(5, 6, &ms[5]));
    if (c->S.n) {
        float fin_a = 0.f, fin_b = 0.f;
        TRY(el(4, 7, &ms[4]));                                 // coupling force (side stream)
        TRY(el(7, 8, &ms[6]));                                 // solid sub-steps (side stream)
        TRY(el(6, 9, &fin_a));
        TRY(el(8, 9, &fin_b));
        ms[7] = fin_a < fin_b ? fin_a : fin_b;                 // finish, after the join
    } else {
        ms[4] = ms[6] = 0.0f;
        TRY(el(6, 9, &ms[7]));
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
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->side) cudaStreamSynchronize(c->side);
    for (int k = 0; k < sphfsi_ctx::kEvents; k++)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->side) cudaStreamDestroy(c->side);
    for (void *p : c->allocs) cudaFree(p);
    delete c;
}

}  // extern "C"
