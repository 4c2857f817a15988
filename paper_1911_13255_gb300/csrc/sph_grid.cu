// Cell-linked-list neighbour build (Alg. 1, "particle-neighbour list"; the
// paper rebuilds it per advection step, this library every coarse step):
// a counting sort of particles by the linear index of their cell, cells of
// edge >= 2 h_F (or >= h_F, Grid::reach = 2).  The sort is a single-digit
// radix sort whose digit is the global cell index: histogram (atomics),
// exclusive scan per instance, scatter, then a per-cell ranking by particle
// id so the order is deterministic and depends on the current state only;
// the ranking kernel gathers the fluid state into cell order and emits the
// FP32 records the pair loops read.  The binning kernel also does the step
// control; the finish kernel ends a step.
#include "sph_common.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// Step control, done by the binning kernel of a step: dt_F, K and the
// reinitialisation flag of the step from the instance's maxima of the
// previous step (which the finish kernel moves to prev_*), so that every
// thread can evaluate it and the leader thread of the instance stores it.
// ---------------------------------------------------------------------------
// Solid step (Eq. dts-advection) from the solid's maxima
__device__ __forceinline__ double solid_dt(const Phys &P, double vS, double aS)
{
    const double b1 = P.hS_d / (P.cS_d + vS);
    const double b2 = aS > 0.0 ? sqrt(P.hS_d / aS) : 1e300;
    return 0.6 * (b1 < b2 ? b1 : b2);
}

// dt_F of the step.  K_fixed < 0 selects a single time step for fluid and
// solid (K = 1), the baselines the paper compares multiple time steps with:
// -1 the single-step criterion of Section 2.2 (|v|max over both phases,
// |dv/dt|max over the solid, h^2/nu with nu = eta/rho0, each phase's own h),
// -2 the smaller of the acoustic fluid step and the solid step (Section 3.2).
__device__ __forceinline__ double step_dt(const Inst &In, const Ctl *ctl, double dt_fixed, int K_fixed)
{
    const Phys &P = In.P;
    if (dt_fixed > 0.0) return dt_fixed;
    const double vF = ctl->prev_vmaxF;
    const double ac = 0.6 * P.hF_d / (P.c0_d + vF);   // Eq. dt-relax
    if (K_fixed >= 0) return ac;
    const double vS = ctl->prev_vmaxS, aS = ctl->prev_amaxS;
    if (K_fixed == -2) {
        const double ds = In.ns > 0 ? solid_dt(P, vS, aS) : 1e300;
        return ac < ds ? ac : ds;
    }
    const double v = vF > vS ? vF : vS;
    const double nu = P.eta_d / P.rho0_d;
    double fl = P.hF_d / (P.c0_d + v);
    if (nu > 0.0 && P.hF_d * P.hF_d / nu < fl) fl = P.hF_d * P.hF_d / nu;
    const double so = In.ns > 0 ? solid_dt(P, v, aS) : 1e300;
    return 0.25 * fl < so ? 0.25 * fl : so;
}

__device__ __forceinline__ bool step_reinit(const Ctl *ctl)
{
    return ctl->n_reinit > 0 && (ctl->step % ctl->n_reinit) == 0;
}

__device__ void step_control(const Inst &In, Ctl *ctl, double dt_fixed, int K_fixed)
{
    const Phys &P = In.P;
    const double dt = step_dt(In, ctl, dt_fixed, K_fixed);
    int K = 1;
    if (K_fixed > 0) {
        K = K_fixed;
    } else if (K_fixed == 0 && In.ns > 0) {
        const double dts = solid_dt(P, ctl->prev_vmaxS, ctl->prev_amaxS);
        double k = floor(dt / dts) + 1.0;          // kappa = [dt_F / dt_S] + 1
        // a solid step a million times shorter than the fluid step (or a
        // non-finite one): the state has run away; one sub-step, and the
        // finish kernel stops the context
        if (!(k <= 1e6)) {
            k = 1.0;
            ctl->status |= ST_NONFINITE;
        }
        K = (int)k;
    }
    ctl->dt_fixed = dt_fixed;
    ctl->K_fixed = K_fixed;
    ctl->dt = dt;
    ctl->K = K;
    ctl->dts = dt / (double)K;
    ctl->reinit = step_reinit(ctl) ? 1 : 0;
    ctl->n_ff = ctl->n_fw = ctl->n_fs = ctl->n_sf = 0ull;
    for (int k = 0; k < 3; k++) ctl->mom_fluid[k] = ctl->mom_solid[k] = 0.0;
    ctl->learned_ok = 0;
    ctl->lnum = ctl->lden = 0.0;
}

// normal update n = normalize(F^-T n0), F^-T = cof(F) / det F (Alg. 1, on
// reinitialisation steps)
template <int D>
__device__ void update_normal(const Solid &s, int a)
{
    const float *Hm = s.H + 9 * a;
    float F[9];
    for (int i = 0; i < 9; i++) F[i] = Hm[i];
    const float *n0 = s.n0 + 3 * a;
    float n[3], det;
    if (D == 2) {
        F[0] += 1.0f;
        F[3] += 1.0f;
        n[0] = F[3] * n0[0] - F[2] * n0[1];
        n[1] = -F[1] * n0[0] + F[0] * n0[1];
        n[2] = 0.0f;
        det = F[0] * F[3] - F[1] * F[2];
    } else {
        F[0] += 1.0f;
        F[4] += 1.0f;
        F[8] += 1.0f;
        float c00 = F[4] * F[8] - F[5] * F[7], c01 = F[5] * F[6] - F[3] * F[8], c02 = F[3] * F[7] - F[4] * F[6];
        float c10 = F[2] * F[7] - F[1] * F[8], c11 = F[0] * F[8] - F[2] * F[6], c12 = F[1] * F[6] - F[0] * F[7];
        float c20 = F[1] * F[5] - F[2] * F[4], c21 = F[2] * F[3] - F[0] * F[5], c22 = F[0] * F[4] - F[1] * F[3];
        n[0] = c00 * n0[0] + c01 * n0[1] + c02 * n0[2];
        n[1] = c10 * n0[0] + c11 * n0[1] + c12 * n0[2];
        n[2] = c20 * n0[0] + c21 * n0[1] + c22 * n0[2];
        det = F[0] * c00 + F[1] * c01 + F[2] * c02;
    }
    float inv = (det < 0.0f ? -1.0f : 1.0f) * rsqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    s.nrm[3 * a] = n[0] * inv;
    s.nrm[3 * a + 1] = n[1] * inv;
    s.nrm[3 * a + 2] = n[2] * inv;
}

// The advection criterion of Eq. dtf-advection, 0.25 min(h_F / |v|max,
// h_F^2 / nu), nu = eta / rho0 (the printed eta read as the kinematic
// viscosity, as in the single-step criterion); a zero speed or viscosity
// drops its term.
__device__ __forceinline__ double advection_dt(const Phys &P, double vmax)
{
    const double nu = P.eta_d / P.rho0_d;
    const double a1 = vmax > 0.0 ? P.hF_d / vmax : 1e300;
    const double a2 = nu > 0.0 ? P.hF_d * P.hF_d / nu : 1e300;
    return 0.25 * (a1 < a2 ? a1 : a2);
}

// finish: time, step, pair counters, non-finite check, maxima for the next
// step's control (one thread per instance)
__global__ void k_finish(Batch bt, int learned, unsigned *gbar, Fluid f)
{
    pdl_enter();
    if (step_failed(bt)) return;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0 && gbar) gbar[0] = 0u;   // the fused binning's barrier, even after a time-out
    if (b == 0 && f.held) {
        // before instance 0's step index advances (below, same thread)
        const bool rb = rebuild_step(bt, f);
        f.held[1] = rb ? 1 : 0;
        f.held[0] = 0;
        if (f.held_n == 0) {
            // Algorithm 1 (reading F3): an advection step lasts while the
            // acoustic steps taken in it sum to at most dt_ad, the advection
            // criterion (Eq. dtf-advection) at the maxima each step started
            // from (its minimum over the advection step, so that one that
            // starts at rest still ends); instance 0 decides for the context.
            // This thread is instance 0's own, and prev_vmaxF is still the
            // maximum this step's control used.
            Ctl *c0 = bt.ctl;
            const double ad = advection_dt(bt.I[0].P, c0->prev_vmaxF);
            c0->t_ad = rb ? ad : fmin(c0->t_ad, ad);
            c0->t_acc = (rb ? 0.0 : c0->t_acc) + c0->dt;
            f.held[2] = c0->t_acc > c0->t_ad ? 1 : 0;
        }
    }
    if (b >= bt.B) return;
    Ctl *ctl = bt.ctl + b;
    float vF = __uint_as_float(ctl->vmaxF), vS = __uint_as_float(ctl->vmaxS), aS = __uint_as_float(ctl->amaxS);
    // non-finite maxima, or a fluid particle faster than the artificial sound
    // speed (the weakly-compressible model holds for |v| << c0): the state
    // has run away, and the context's later steps do nothing
    if (!(vF <= 3.0e38f) || !(vS <= 3.0e38f) || !(aS <= 3.0e38f) || vF > bt.I[b].P.c0)
        ctl->status |= ST_NONFINITE;
    if (ctl->status & ST_NONFINITE) atomicCAS(bt.fail, 0, kFailRunaway);
    // the maxima of this step set the next step's dt_F and K
    ctl->prev_vmaxF = vF;
    ctl->prev_vmaxS = vS;
    ctl->prev_amaxS = aS;
    ctl->vmaxF = ctl->vmaxS = ctl->amaxS = 0u;
    unsigned long long fl = ctl->n_ff + ctl->n_fw + ctl->n_fs;
    const unsigned long long nnz = (unsigned long long)bt.I[b].nnz;
    unsigned long long p = 2ull * fl + ctl->n_sf + (ctl->reinit ? fl : 0ull);
    // learned step: F at the mid and end positions and one force loop (3
    // solid pair loops); the sub-steps (2 K + 1) only when it was rejected
    if (learned && bt.I[b].ns > 0) {
        p += 3ull * nnz;
        if (ctl->learned_ok) ctl->l_acc += 1;
        else ctl->l_rej += 1;
    }
    if (!ctl->learned_ok) p += (unsigned long long)(2 * ctl->K + 1) * nnz;
    ctl->pairs_total += p;
    ctl->last_dt = ctl->dt;
    ctl->last_K = ctl->K;
    ctl->t += ctl->dt;
    ctl->step += 1;
}

int launch_finish(const Batch &bt, int learned, unsigned *gbar, const Fluid &f, cudaStream_t st)
{
    launch_k(k_finish, (bt.B + kBlock - 1) / kBlock, kBlock, 0, st, bt, learned, gbar, f);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// fluid: inflow buffer, first half drift (Eq. verlet-first-half), cell key;
// solid: cell key at the start-of-step position
// ---------------------------------------------------------------------------
__device__ __forceinline__ double inflow_u(const Phys &P, double y, double z, double t)
{
    double U = P.in_U;
    if (P.in_tramp > 0.0 && t < P.in_tramp) U = 0.5 * U * (1.0 - cos(3.14159265358979323846 * t / P.in_tramp));
    if (P.inflow_profile == 1) return U;
    double yy = y - P.in_y0, H = P.in_H;
    yy = yy < 0.0 ? 0.0 : (yy > H ? H : yy);
    if (P.inflow_profile == 2) {
        // Womersley channel flow under dp/dx = -A cos(w t) (Appendix A), U = A / rho:
        // with b = Wo / sqrt(2), s = 2 y / H - 1, f1,2 = b (1 +- s), g = cosh 2b + cos 2b,
        // u = U / (w g) [(sinh f1 sin f2 + sinh f2 sin f1) cos wt + (g - cosh f1 cos f2 - cosh f2 cos f1) sin wt]
        const double w = 2.0 * 3.14159265358979323846 / P.in_T, b = P.in_wo * 0.70710678118654752440;
        const double sy = 2.0 * (yy - 0.5 * H) / H;
        const double f1 = b * (1.0 + sy), f2 = b * (1.0 - sy);
        const double g = cosh(2.0 * b) + cos(2.0 * b);
        const double c = sinh(f1) * sin(f2) + sinh(f2) * sin(f1);
        const double q = g - cosh(f1) * cos(f2) - cosh(f2) * cos(f1);
        return U / (w * g) * (c * cos(w * t) + q * sin(w * t));
    }
    if (P.inflow_profile == 3) {
        // a 3-D duct: the channel profile across y times the one across z
        // (zero on the four walls, mean U over the cross-section)
        double zz = z - P.in_z0;
        const double Hz = P.in_Hz;
        zz = zz < 0.0 ? 0.0 : (zz > Hz ? Hz : zz);
        return U * (6.0 * yy * (H - yy) / (H * H)) * (6.0 * zz * (Hz - zz) / (Hz * Hz));
    }
    return 6.0 * U * yy * (H - yy) / (H * H);
}

template <int D>
__device__ __forceinline__ int global_key(const Inst &In, double x, double y, double z)
{
    const Grid &g = In.g;
    int cx = cell_coord(x, g.lo[0], g.cs[0], g.nc[0]);
    int cy = cell_coord(y, g.lo[1], g.cs[1], g.nc[1]);
    int cz = D == 3 ? cell_coord(z, g.lo[2], g.cs[2], g.nc[2]) : 0;
    return In.c0 + cx + g.nc[0] * (cy + g.nc[1] * cz);
}

// With step = 1 (a coarse step) the kernel also does the step control: one
// leader thread per instance (after the particles' threads) stores dt_F, K
// and the reinitialisation flag and clears the step's counters; the fluid
// threads evaluate the same dt_F themselves, the solid threads update their
// normals on reinitialisation steps.  Thread 0 clears the list of non-empty
// cells that the scatter fills.
template <int D>
__device__ __forceinline__ void bin_one(const Batch &bt, const Fluid &f, const Solid &s, int t, int step,
                                        double dt_fixed, int K_fixed)
{
    // held configuration: no keys or histograms between rebuilds (the slots,
    // cell lists and record positions of the last rebuild stay)
    const bool rebuild = rebuild_step(bt, f);
    if (t < f.n) {
        const int i = t;
        const int b = f.inst[i];
        const Inst &In = bt.I[b];
        FluidState S = f.s[0];
        double x = S.x[i], y = S.y[i], z = D == 3 ? S.z[i] : 0.0;
        if (step) {
            const Phys &P = In.P;
            const Grid &g = In.g;
            const Ctl *ctl = bt.ctl + b;
            const double dt = step_dt(In, ctl, dt_fixed, K_fixed), tm = ctl->t;
            float vx = S.vx[i], vy = S.vy[i], vz = D == 3 ? S.vz[i] : 0.0f;
            if (P.inflow_on && x >= g.x_lo && x < g.x_lo + P.in_w) {   // inflow buffer (reading R18)
                vx = (float)inflow_u(P, y, z, tm);
                vy = 0.0f;
                vz = 0.0f;
                S.vx[i] = vx;
                S.vy[i] = vy;
                if (D == 3) S.vz[i] = vz;
            }
            double h = 0.5 * dt;   // first half drift (Eq. verlet-first-half)
            S.drho[i] = S.drho[i] + (float)h * S.rhodot[i];
            x = x + h * (double)vx;
            y = y + h * (double)vy;
            if (D == 3) z = z + h * (double)vz;
            if (g.periodic_x) {
                if (x >= g.x_lo + g.Lx) x -= g.Lx;
                else if (x < g.x_lo) x += g.Lx;
            }
            S.x[i] = x;
            S.y[i] = y;
            if (D == 3) S.z[i] = z;
        }
        if (!rebuild) return;
        int key = global_key<D>(In, x, y, z);
        f.key[i] = key;
        atomicAdd(&f.ccount[key], 1);
    } else if (t < f.n + s.n) {
        const int a = t - f.n;
        const int b = s.inst[a];
        if (step && step_reinit(bt.ctl + b)) update_normal<D>(s, a);
        if (!rebuild) return;
        int key = global_key<D>(bt.I[b], s.x[a], s.y[a], D == 3 ? s.z[a] : 0.0);
        s.key[a] = key;
        atomicAdd(&s.ccount[key], 1);
    } else if (step && t < f.n + s.n + bt.B) {
        const int b = t - f.n - s.n;
        step_control(bt.I[b], bt.ctl + b, dt_fixed, K_fixed);
    }
}

template <int D>
__global__ void k_bin_all(Batch bt, Fluid f, Solid s, int step, double dt_fixed, int K_fixed)
{
    pdl_enter();
    if (step_failed(bt)) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        *f.nlive = 0;
        f.scan_ctl[0] = 0u;    // the scan's tickets
        f.scan_ctl[1] += 1u;   // and its epoch: this binning's tile states
    }
    bin_one<D>(bt, f, s, t, step, dt_fixed, K_fixed);
}

// ---------------------------------------------------------------------------
// exclusive scan of the cell histograms, one block per (instance, set):
// set 0 fluid, 1 solid, 2 walls; the cells of instance b are [c0, c0+ncell)
// and its slots start at f0 / s0 / w0.  A tile is 24 rows of 32 cells per
// warp (24 576 cells per block of 1024 threads): the rows are loaded
// coalesced and all at once, scanned with warp shuffles, then offset by the
// scanned warp totals.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanRows = 24;
constexpr int kTile = kScanRows * kScanThreads;

// returns base + the sum of the counts (to every thread); count may alias
// count_in: each thread writes only the cells it has read
__device__ int scan_cells(const int *count_in, int *count, int *start, int n, int base)
{
    __shared__ int warp_off[32];
    __shared__ int tile_sum;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int carry = base;
    for (int b0 = 0; b0 < n; b0 += kTile) {
        const int w0 = b0 + w * 32 * kScanRows;
        int ex[kScanRows];
        int run = 0;
        if (w0 < n) {   // warp-uniform: a warp past the end has nothing to scan
#pragma unroll
            for (int r = 0; r < kScanRows; r++) {
                const int i = w0 + r * 32 + lane;
                ex[r] = i < n ? count_in[i] : 0;
            }
#pragma unroll
            for (int r = 0; r < kScanRows; r++) {
                const int v = ex[r];
                int x = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += u;
                }
                ex[r] = run + x - v;
                run += __shfl_sync(0xffffffffu, x, 31);
            }
        }
        if (lane == 0) warp_off[w] = run;
        __syncthreads();
        if (w == 0) {
            const int x = warp_off[lane];
            int xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= o) xi += u;
            }
            warp_off[lane] = xi - x;
            if (lane == 31) tile_sum = xi;
        }
        __syncthreads();
        const int off = carry + warp_off[w];
        if (w0 < n) {
#pragma unroll
            for (int r = 0; r < kScanRows; r++) {
                const int i = w0 + r * 32 + lane;
                if (i < n) {
                    start[i] = off + ex[r];
                    count[i] = 0;   // the histogram becomes the scatter cursor
                }
            }
        }
        carry += tile_sum;
        __syncthreads();   // warp_off and tile_sum are rewritten by the next tile
    }
    return carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_seg(Batch bt, int *fcount, int *fstart, int nf, int *scount,
                                                           int *sstart, int ns, int *wcount, int *wstart, int nw,
                                                           int set0)
{
    pdl_enter();
    const int b = blockIdx.x % bt.B, set = set0 + blockIdx.x / bt.B;
    const Inst &In = bt.I[b];
    int *count = set == 0 ? fcount : (set == 1 ? scount : wcount);
    int *start = set == 0 ? fstart : (set == 1 ? sstart : wstart);
    const int base = set == 0 ? In.f0 : (set == 1 ? In.s0 : In.w0);
    scan_cells(count + In.c0, count + In.c0, start + In.c0, In.g.ncell, base);
    if (b == bt.B - 1 && threadIdx.x == 0) start[bt.ncell] = set == 0 ? nf : (set == 1 ? ns : nw);
}

// ---------------------------------------------------------------------------
// Exclusive scan of the cell histograms over many blocks: every (instance,
// set) segment is cut into tiles of kScanTile cells, and tiles take tickets
// in segment order, so a tile only waits for tiles that started before it.
// Each block scans its tile (8 consecutive cells per thread), publishes the
// tile's sum, then adds the sums published by the tiles before it in its
// segment, back to the first that has published its inclusive prefix
// (decoupled look-back), and publishes its own inclusive prefix.  A tile's
// state word holds the binning's epoch (bits 34..63), a flag (1 sum, 2
// inclusive prefix) and the value, so no reset is needed between steps.
// Waits are bounded: on a time-out the status bit is set.
// ---------------------------------------------------------------------------
constexpr int kScanLbThreads = 256, kScanLbPer = 8, kScanTile = kScanLbThreads * kScanLbPer;

__device__ __forceinline__ unsigned long long scan_word(unsigned epoch, unsigned flag, int value)
{
    return ((unsigned long long)(epoch & 0x3fffffffu) << 34) | ((unsigned long long)flag << 32) | (unsigned)value;
}

__global__ void __launch_bounds__(kScanLbThreads) k_scan_lb(Batch bt, Fluid f, Solid s)
{
    pdl_enter();
    if (!rebuild_step(bt, f)) return;   // held configuration: cell starts stay
    __shared__ int s_tile, s_pre, s_warp[kScanLbThreads / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) s_tile = (int)atomicAdd(&f.scan_ctl[0], 1u);
    __syncthreads();
    const int T = s_tile;
    if (T >= f.nscan_tiles) return;
    const unsigned epoch = f.scan_ctl[1];
    const int2 tk = f.scan_tiles[T];
    const int set = tk.x / bt.B, b = tk.x % bt.B;
    const Inst &In = bt.I[b];
    int *count = (set == 0 ? f.ccount : s.ccount) + In.c0;
    int *start = (set == 0 ? f.cstart : s.cstart) + In.c0;
    const int base = set == 0 ? In.f0 : In.s0;
    const int n = In.g.ncell;
    // this thread's cells c0 .. c0 + 7 of the tile
    const int c0 = tk.y * kScanTile + t * kScanLbPer;
    int v[kScanLbPer], run = 0;
#pragma unroll
    for (int j = 0; j < kScanLbPer; j++) {
        v[j] = c0 + j < n ? count[c0 + j] : 0;
        run += v[j];
    }
    int x = run;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    int woff = 0, tile_sum = 0;
#pragma unroll
    for (int k = 0; k < kScanLbThreads / 32; k++) {
        woff += k < w ? s_warp[k] : 0;
        tile_sum += s_warp[k];
    }
    if (t == 0) {
        int pre = 0;
        if (tk.y == 0) {
            __threadfence();
            atomicExch(&f.scan_status[T], scan_word(epoch, 2u, tile_sum));
        } else {
            __threadfence();
            atomicExch(&f.scan_status[T], scan_word(epoch, 1u, tile_sum));
            for (int j = T - 1;;) {
                const unsigned long long wd = atomicAdd(&f.scan_status[j], 0ull);
                const unsigned fl = (unsigned)(wd >> 32) & 3u;
                if ((unsigned)(wd >> 34) != (epoch & 0x3fffffffu) || fl == 0u) {
                    long long it = 0;
                    unsigned long long w2 = wd;
                    while (((unsigned)(w2 >> 34) != (epoch & 0x3fffffffu) || ((unsigned)(w2 >> 32) & 3u) == 0u) &&
                           ++it < bt.spin)
                        w2 = atomicAdd(&f.scan_status[j], 0ull);
                    if (it >= bt.spin) {
                        // this tile's prefix is unknown: the step's cell starts are invalid
                        atomicOr(&bt.ctl[b].status, ST_TIMEOUT);
                        atomicExch(bt.fail, kFailWait);
                        break;
                    }
                    continue;
                }
                pre += (int)(unsigned)wd;
                if (fl == 2u) break;
                --j;
            }
            __threadfence();
            atomicExch(&f.scan_status[T], scan_word(epoch, 2u, pre + tile_sum));
        }
        s_pre = pre;
    }
    __syncthreads();
    int st = base + s_pre + woff + x - run;
#pragma unroll
    for (int j = 0; j < kScanLbPer; j++) {
        if (c0 + j < n) {
            start[c0 + j] = st;
            count[c0 + j] = 0;   // the histogram becomes the scatter cursor
        }
        st += v[j];
    }
    // the end of the last instance's slots
    if (b == bt.B - 1 && t == 0 && c0 <= n && n <= tk.y * kScanTile + kScanTile)
        (set == 0 ? f.cstart : s.cstart)[bt.ncell] = set == 0 ? f.n : s.n;
}

// Scatter into the cells' slot ranges (arbitrary order inside a cell); with
// list_cells the particle that opens a cell appends it to the list of
// non-empty cells (fluid cell c as c, solid cell c as ncell + c), one atomic
// per warp (on one counter: for small problems only).
// (called by all 32 lanes of a warp together)
__device__ __forceinline__ void scatter_one(const Fluid &f, const Solid &s, int t, int ncell, int list_cells)
{
    int opened = -1;
    if (t < f.n) {
        const int k = f.key[t];
        const int q = atomicAdd(&f.ccount[k], 1);
        f.perm[f.cstart[k] + q] = t;
        if (q == 0) opened = k;
    } else if (t < f.n + s.n) {
        const int a = t - f.n;
        const int k = s.key[a];
        const int q = atomicAdd(&s.ccount[k], 1);
        s.perm[s.cstart[k] + q] = a;
        if (q == 0) opened = ncell + k;
    }
    if (!list_cells) return;
    const unsigned m = __ballot_sync(0xffffffffu, opened >= 0);
    if (m == 0u) return;
    const int lane = threadIdx.x & 31, lead = __ffs(m) - 1;
    int base = 0;
    if (lane == lead) base = atomicAdd(f.nlive, __popc(m));
    base = __shfl_sync(0xffffffffu, base, lead);
    if (opened >= 0) f.live[base + __popc(m & ((1u << lane) - 1u))] = opened;
}

__global__ void k_scatter2(Batch bt, Fluid f, Solid s, int ncell, int list_cells)
{
    pdl_enter();
    if (step_failed(bt)) return;
    if (!rebuild_step(bt, f)) return;
    scatter_one(f, s, blockIdx.x * blockDim.x + threadIdx.x, ncell, list_cells);
}

// per-cell insertion sort by slot (walls, binned once), and the cursor reset
// for the next binning
__device__ __forceinline__ void sort_cell(int a, int b, int *perm, const int *id)
{
    for (int i = a + 1; i < b; i++) {
        int v = perm[i];
        int kv = id ? id[v] : v;
        int j = i - 1;
        while (j >= a) {
            int u = perm[j];
            int ku = id ? id[u] : u;
            if (ku <= kv) break;
            perm[j + 1] = u;
            j--;
        }
        perm[j + 1] = v;
    }
}

// Position relative to the origin of its cell, rounded to FP32; with lo,
// also the rounding remainder (FP64 offset - FP32 offset, rounded to FP32),
// so that hi + lo carries the FP64 offset to about 2^-48 of the cell edge.
template <int D>
__device__ __forceinline__ float4 rel_pos(const Inst &In, int gkey, double x, double y, double z,
                                          float4 *lo = nullptr)
{
    const Grid &g = In.g;
    int key = gkey - In.c0;
    int cx = key % g.nc[0], cy = (key / g.nc[0]) % g.nc[1], cz = D == 3 ? key / (g.nc[0] * g.nc[1]) : 0;
    double dx = x - (g.lo[0] + (double)cx * g.cs[0]);
    double dy = y - (g.lo[1] + (double)cy * g.cs[1]);
    double dz = D == 3 ? z - (g.lo[2] + (double)cz * g.cs[2]) : 0.0;
    float xr = (float)dx, yr = (float)dy, zr = (float)dz;
    if (lo) *lo = make_float4((float)(dx - (double)xr), (float)(dy - (double)yr), (float)(dz - (double)zr), 0.0f);
    return make_float4(xr, yr, zr, 0.0f);
}

// Record of fluid slot k (cell order) from storage slot src: the sorted
// copy of the state in s[1] and the FP32 records the pair loops read.  The
// source is read first (fluid_src) and written later (fluid_put), so that the
// ranking kernel can issue the reads before ranking.  An instance's slots
// are the same range in storage and in cell order, so src's instance is k's.
struct FluidSrc {
    double x, y, z;
    float vx, vy, vz, dr, rd;
    int id, key, b;
};

template <int D>
__device__ __forceinline__ FluidSrc fluid_src(const Fluid &f, int src)
{
    const FluidState A = f.s[0];
    FluidSrc v;
    v.x = A.x[src];
    v.y = A.y[src];
    v.z = D == 3 ? A.z[src] : 0.0;
    v.vx = A.vx[src];
    v.vy = A.vy[src];
    v.vz = D == 3 ? A.vz[src] : 0.0f;
    v.dr = A.drho[src];
    v.rd = A.rhodot[src];
    v.id = A.id[src];
    v.key = f.key[src];
    v.b = f.inst[src];
    return v;
}

template <int D>
__device__ __forceinline__ void fluid_put(const Batch &bt, const Fluid &f, int k, const FluidSrc &v)
{
    const FluidState B = f.s[1];
    const Inst &In = bt.I[v.b];
    B.x[k] = v.x;
    B.y[k] = v.y;
    B.vx[k] = v.vx;
    B.vy[k] = v.vy;
    if (D == 3) {
        B.z[k] = v.z;
        B.vz[k] = v.vz;
    }
    B.drho[k] = v.dr;
    B.rhodot[k] = v.rd;
    B.id[k] = v.id;
    f.cell_of[k] = v.key;
    // the double-float remainders serve the reinitialisation; with a held
    // configuration a later step of the advection step may reinitialise
    const bool reinit = bt.ctl[v.b].reinit || held_on(f);
    float4 lo;
    float4 r = rel_pos<D>(In, v.key, v.x, v.y, v.z, reinit ? &lo : nullptr);
    if (reinit) f.L4[k] = lo;
    r.w = eos_p(v.dr, In.P);
    f.P4[k] = r;
    f.V4[k] = make_float4(v.vx, v.vy, v.vz, v.dr);
}

template <int D>
__device__ __forceinline__ void fluid_record(const Batch &bt, const Fluid &f, int k, int src)
{
    fluid_put<D>(bt, f, k, fluid_src<D>(f, src));
}

// Record of solid slot k of the fluid grid from solid particle a (N4.w
// carries a).
template <int D>
__device__ __forceinline__ void solid_record(const Batch &bt, const Solid &s, int k, int a, bool held)
{
    int key = s.key[a];
    s.cell_of[k] = key;
    const int b = s.inst[a];
    const bool reinit = bt.ctl[b].reinit || held;
    float4 lo;
    s.A4[k] = rel_pos<D>(bt.I[b], key, s.x[a], s.y[a], D == 3 ? s.z[a] : 0.0, reinit ? &lo : nullptr);
    if (reinit) s.L4[k] = lo;
    s.VB4[k] = make_float4((float)s.vbar[3 * a], (float)s.vbar[3 * a + 1], (float)s.vbar[3 * a + 2], 0.0f);
    s.AB4[k] = make_float4((float)s.abar[3 * a], (float)s.abar[3 * a + 1], (float)s.abar[3 * a + 2], 0.0f);
    s.N4[k] = make_float4(s.nrm[3 * a], s.nrm[3 * a + 1], s.nrm[3 * a + 2], __int_as_float(a));
}

// Canonical order inside every cell (the scatter's atomics leave it
// arbitrary) and the records, in one pass over the non-empty cells (listed)
// or over all cells (fluid, then solid): a group
// of G lanes per cell ranks the cell's entries by key (fluid: original id,
// solid: particle index; keys are unique in a cell, so an entry's place is
// the number of smaller keys) and writes entry e's record to slot
// start + rank(e).  Entries and keys are compared G at a time through
// shuffles, so a cell of any size is ranked by the same group (quadratic in
// its size; about 7 fluid entries per cell in 2-D, 18 in 3-D).  The perm
// array is only read, so ranking and writing need no ordering.  Every loop
// bound is uniform over the warp (the largest cell of its groups), as the
// shuffles require.  G = 16 in 2-D, 32 in 3-D.  REC = false only ranks
// (sperm[start + rank(e)] = e) and k_records_sorted writes the records with
// one thread per slot (Fluid::split_records): one launch more, but no idle
// lanes while writing, which pays for large batches.
// One cell per group of G lanes (valid: this group has cell e); every lane
// of the warp calls it together.  A fluid entry's source state is read
// before the ranking, so those loads overlap the shuffles.
template <int D, int G, bool REC>
__device__ __forceinline__ void rank_cell(const Batch &bt, const Fluid &f, const Solid &s, bool valid, int e,
                                          int lane)
{
    const bool fl = e < bt.ncell;
    const int c = fl ? e : e - bt.ncell;
    const int *cs = fl ? f.cstart : s.cstart;
    const int *perm = fl ? f.perm : s.perm;
    int a = 0, n = 0;
    if (valid) {
        a = cs[c];
        n = cs[c + 1] - a;
        if (lane == 0) (fl ? f.ccount : s.ccount)[c] = 0;   // cursor reset for the next binning
    }
    const int nmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)n);
    for (int m0 = 0; m0 < nmax; m0 += G) {
        const bool mine = m0 + lane < n;
        const int v = mine ? perm[a + m0 + lane] : 0;
        FluidSrc src{};
        int kv = 0x7fffffff;
        if (mine) {
            if (fl) {
                if (REC) src = fluid_src<D>(f, v);
                else src.id = f.s[0].id[v];
                kv = src.id;
            } else {
                kv = v;
            }
        }
        int rank = 0;
        for (int c0 = 0; c0 < nmax; c0 += G) {
            int ko = kv;
            if (c0 != m0) {
                const bool has = c0 + lane < n;
                const int u = has ? perm[a + c0 + lane] : 0;
                ko = has ? (fl ? f.s[0].id[u] : u) : 0x7fffffff;
            }
            const int lim = nmax - c0 < G ? nmax - c0 : G;
            for (int q = 0; q < lim; q++) rank += __shfl_sync(0xffffffffu, ko, q, G) < kv ? 1 : 0;
        }
        if (mine) {
            if (!REC) (fl ? f.sperm : s.sperm)[a + rank] = v;
            else if (fl) fluid_put<D>(bt, f, a + rank, src);
            else solid_record<D>(bt, s, a + rank, v, held_on(f));
        }
    }
}

template <int D, int G, bool REC>
__global__ void __launch_bounds__(256) k_cell_records(Batch bt, Fluid f, Solid s, int listed, int ncells)
{
    pdl_enter();
    if (step_failed(bt)) return;
    if (!rebuild_step(bt, f)) return;   // held configuration: k_held_records refreshes the records
    const int nlive = listed ? *f.nlive : ncells;
    const int lane = threadIdx.x % G;
    const int per_grid = gridDim.x * (blockDim.x / G);
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) / G;; w += per_grid) {
        const bool valid = w < nlive;
        if (!__any_sync(0xffffffffu, valid)) break;
        rank_cell<D, G, REC>(bt, f, s, valid, valid ? (listed ? f.live[w] : w) : 0, lane);
    }
}

template <int D>
__global__ void k_records_sorted(Batch bt, Fluid f, Solid s)
{
    pdl_enter();
    if (step_failed(bt)) return;
    if (!rebuild_step(bt, f)) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < f.n) fluid_record<D>(bt, f, t, f.sperm[t]);
    else if (t < f.n + s.n) solid_record<D>(bt, s, t - f.n, s.sperm[t - f.n], held_on(f));
}

// Held configuration, steps between rebuilds: every slot keeps its particle
// and its record keeps the position of the last rebuild (the pair geometry);
// the mid-step copy of the state and the records' pressure, velocity and
// density (fluid) and time-averaged velocity, acceleration and normal (solid
// records) are refreshed in place.
template <int D>
__global__ void k_held_records(Batch bt, Fluid f, Solid s)
{
    pdl_enter();
    if (step_failed(bt)) return;
    if (rebuild_step(bt, f)) return;   // the binning wrote every record
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < f.n) {
        const FluidState A = f.s[0], B = f.s[1];
        const Phys &P = bt.I[f.inst[t]].P;
        const float vx = A.vx[t], vy = A.vy[t], vz = D == 3 ? A.vz[t] : 0.0f, dr = A.drho[t];
        B.x[t] = A.x[t];
        B.y[t] = A.y[t];
        B.vx[t] = vx;
        B.vy[t] = vy;
        if (D == 3) {
            B.z[t] = A.z[t];
            B.vz[t] = vz;
        }
        B.drho[t] = dr;
        B.rhodot[t] = A.rhodot[t];
        B.id[t] = A.id[t];
        f.P4[t].w = eos_p(dr, P);
        f.V4[t] = make_float4(vx, vy, vz, dr);
    } else if (t < f.n + s.n) {
        const int k = t - f.n;
        const float4 n4 = s.N4[k];
        const int a = __float_as_int(n4.w);
        s.VB4[k] = make_float4((float)s.vbar[3 * a], (float)s.vbar[3 * a + 1], (float)s.vbar[3 * a + 2], 0.0f);
        s.AB4[k] = make_float4((float)s.abar[3 * a], (float)s.abar[3 * a + 1], (float)s.abar[3 * a + 2], 0.0f);
        s.N4[k] = make_float4(s.nrm[3 * a], s.nrm[3 * a + 1], s.nrm[3 * a + 2], n4.w);
    }
}

constexpr int kRecordBlocksPerSM = 64;
constexpr bool kScanLookBack = true;   // the many-block scan; false: one block per segment

// ---------------------------------------------------------------------------
// Binning as one cooperative kernel (Fluid::bin_fused, small problems, where
// the four kernels above cost more in launch gaps and tails than in work):
// the same four phases, each a grid-stride loop, separated by grid barriers
// (all blocks are resident: cooperative launch).  The scan is two-level:
// every block sums its range of the concatenated histograms [fluid | solid],
// then scans its range from the sum of the preceding blocks' totals.  One
// exclusive scan over all instances' cells gives every instance's starts,
// because instance b's cells and slots both follow those of instance b - 1
// (the solid half is offset back by the fluid total).
// ---------------------------------------------------------------------------
constexpr int kBinFusedThreads = 512, kBinFusedMaxBlocks = 4096;

// sum over the block (every thread calls it; every thread gets the sum)
__device__ __forceinline__ int block_sum(int v, int *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    int t = lane < nw ? red[lane] : 0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// inclusive scan over the block in thread order; *total gets the block sum
__device__ __forceinline__ int block_scan(int v, int *red, int *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    __syncthreads();
    if (lane == 31) red[w] = x;
    __syncthreads();
    int y = lane < nw ? red[lane] : 0, yi = y;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, yi, o);
        if (lane >= o) yi += u;
    }
    *total = __shfl_sync(0xffffffffu, yi, 31);
    return x + (__shfl_sync(0xffffffffu, yi, w) - __shfl_sync(0xffffffffu, y, w));
}

template <int D, int G>
__global__ void __launch_bounds__(kBinFusedThreads, 1)
    k_bin_fused(Batch bt, Fluid f, Solid s, int step, double dt_fixed, int K_fixed)
{
    pdl_enter();
    if (step_failed(bt)) return;
    __shared__ int red[32];
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    int *status = &bt.ctl[0].status;
    const int np = f.n + s.n;
    // (1) step control, drift, cell keys, histograms
    if (gt == 0) *f.nlive = 0;
    for (int t = gt; t < np + (step ? bt.B : 0); t += gs) bin_one<D>(bt, f, s, t, step, dt_fixed, K_fixed);
    if (!grid_barrier(f.gbar, status, bt.spin, bt.fail)) return;
    // (2) exclusive scan of [fluid counts | solid counts]
    const int ncell = bt.ncell, L = (s.n ? 2 : 1) * ncell;
    const int chunk = (L + gridDim.x - 1) / gridDim.x;
    const int i0 = min(L, (int)blockIdx.x * chunk), i1 = min(L, i0 + chunk);
    auto count_at = [&](int i) { return i < ncell ? f.ccount[i] : s.ccount[i - ncell]; };
    int part = 0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) part += count_at(i);
    part = block_sum(part, red);
    if (threadIdx.x == 0) f.bsum[blockIdx.x] = part;
    if (!grid_barrier(f.gbar, status, bt.spin, bt.fail)) return;
    int off = 0;
    for (int j = threadIdx.x; j < (int)blockIdx.x; j += blockDim.x) off += f.bsum[j];
    off = block_sum(off, red);
    for (int b0 = i0; b0 < i1; b0 += blockDim.x) {
        const int i = b0 + threadIdx.x;
        const int v = i < i1 ? count_at(i) : 0;
        int tot;
        const int incl = block_scan(v, red, &tot);
        if (i < i1) {
            const int st = off + incl - v;
            if (i < ncell) {
                f.cstart[i] = st;
                f.ccount[i] = 0;   // the histogram becomes the scatter cursor
            } else {
                s.cstart[i - ncell] = st - f.n;
                s.ccount[i - ncell] = 0;
            }
        }
        off += tot;
    }
    if (gt == 0) {
        f.cstart[ncell] = f.n;
        if (s.n) s.cstart[ncell] = s.n;
    }
    if (!grid_barrier(f.gbar, status, bt.spin, bt.fail)) return;
    // (3) scatter and the list of non-empty cells (whole warps per call)
    for (int t = gt; t < ((np + 31) & ~31); t += gs) scatter_one(f, s, t, ncell, 1);
    if (!grid_barrier(f.gbar, status, bt.spin, bt.fail)) return;
    // (4) canonical order and records of the non-empty cells
    const int nlive = *f.nlive;
    const int lane = threadIdx.x % G;
    const int per_grid = gridDim.x * (blockDim.x / G);
    for (int w = gt / G;; w += per_grid) {
        const bool valid = w < nlive;
        if (!__any_sync(0xffffffffu, valid)) break;
        rank_cell<D, G, true>(bt, f, s, valid, valid ? f.live[w] : 0, lane);
    }
}

// grid of the fused binning kernel: one block per SM (0: it cannot run)
template <typename K>
static int bin_fused_blocks(K kern, int dim)
{
    static int cached_d[2] = {-1, -1};
    int &cached = cached_d[dim == 2 ? 0 : 1];
    if (cached < 0) {
        int dev = 0, nsm = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kBinFusedThreads, 0) != cudaSuccess) {
            cudaGetLastError();
            per = 0;
        }
        cached = per >= 1 ? (nsm < kBinFusedMaxBlocks ? nsm : kBinFusedMaxBlocks) : 0;
    }
    return cached;
}

template <typename K>
static int launch_bin_fused(K kern, int nb, cudaStream_t st, const Batch &bt, const Fluid &f, const Solid &s, int step,
                            double dt_fixed, int K_fixed)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(kBinFusedThreads);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, bt, f, s, step, dt_fixed, K_fixed) == cudaSuccess ? 0 : -3;
}

// kernels launch_bin_all launches in a step with particles
int bin_kernels(const Fluid &f)
{
    if (held_on(f)) return (f.split_records ? 5 : 4) + 1;
    return f.bin_fused ? 1 : (f.split_records ? 5 : 4);
}

int scan_tile_cells() { return kScanTile; }

int launch_bin_all(const Batch &bt, Fluid &f, Solid &s, int dim, int step, double dt_fixed, int K_fixed,
                   cudaStream_t st)
{
    const int np = f.n + s.n;
    const int nt = np + (step ? bt.B : 0);
    if (nt == 0) return 0;
    if (f.bin_fused && np > 0 && !held_on(f)) {
        auto kern = dim == 2 ? k_bin_fused<2, 16> : k_bin_fused<3, 32>;
        const int nb = bin_fused_blocks(kern, dim);
        if (nb > 0) return launch_bin_fused(kern, nb, st, bt, f, s, step, dt_fixed, K_fixed);
    }
    const unsigned nbt = (unsigned)((nt + kBlock - 1) / kBlock);
    if (dim == 2) launch_k(k_bin_all<2>, nbt, kBlock, 0, st, bt, f, s, step, dt_fixed, K_fixed);
    else launch_k(k_bin_all<3>, nbt, kBlock, 0, st, bt, f, s, step, dt_fixed, K_fixed);
    if (np == 0) return cudaGetLastError() == cudaSuccess ? 0 : -3;
    if (kScanLookBack)
        launch_k(k_scan_lb, (unsigned)f.nscan_tiles, kScanLbThreads, 0, st, bt, f, s);
    else
        launch_k(k_scan_seg, bt.B * (s.n ? 2 : 1), kScanThreads, 0, st, bt, f.ccount, f.cstart, f.n, s.ccount,
                 s.cstart, s.n, (int *)nullptr, (int *)nullptr, 0, 0);
    // records from the cell groups: over the listed non-empty cells; ranks
    // only (large problems): over all cells, no list (its counter would
    // serialise one atomic per warp)
    const bool split = f.split_records != 0;
    launch_k(k_scatter2, (np + kBlock - 1) / kBlock, kBlock, 0, st, bt, f, s, bt.ncell, split ? 0 : 1);
    const long long cells_all = (long long)(s.n ? 2 : 1) * bt.ncell;
    const long long cells = split ? cells_all : (cells_all < np ? cells_all : np);
    const long long cap = (long long)kRecordBlocksPerSM * 152;
    const unsigned nbr = (unsigned)((np + kBlock - 1) / kBlock);
    const int G = dim == 2 ? 16 : 32;
    const long long nb = (cells * G + kBlock - 1) / kBlock;
    const unsigned grid = (unsigned)(split || nb < cap ? nb : cap);   // all cells: one group each
    const int listed = split ? 0 : 1, ncells = (int)cells_all;
    if (dim == 2) {
        if (split) {
            launch_k(k_cell_records<2, 16, false>, grid, kBlock, 0, st, bt, f, s, listed, ncells);
            launch_k(k_records_sorted<2>, nbr, kBlock, 0, st, bt, f, s);
        } else {
            launch_k(k_cell_records<2, 16, true>, grid, kBlock, 0, st, bt, f, s, listed, ncells);
        }
    } else {
        if (split) {
            launch_k(k_cell_records<3, 32, false>, grid, kBlock, 0, st, bt, f, s, listed, ncells);
            launch_k(k_records_sorted<3>, nbr, kBlock, 0, st, bt, f, s);
        } else {
            launch_k(k_cell_records<3, 32, true>, grid, kBlock, 0, st, bt, f, s, listed, ncells);
        }
    }
    if (held_on(f)) {
        if (dim == 2) launch_k(k_held_records<2>, nbr, kBlock, 0, st, bt, f, s);
        else launch_k(k_held_records<3>, nbr, kBlock, 0, st, bt, f, s);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// static walls: binned once
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_wall_key(Batch bt, Walls w)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= w.n) return;
    int key = global_key<D>(bt.I[w.inst[q]], w.x[q], w.y[q], D == 3 ? w.z[q] : 0.0);
    w.key[q] = key;
    atomicAdd(&w.ccount[key], 1);
}

__global__ void k_wall_scatter(Walls w)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= w.n) return;
    int k = w.key[q];
    w.perm[w.cstart[k] + atomicAdd(&w.ccount[k], 1)] = q;
}

__global__ void k_wall_cellsort(Walls w, int ncell)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    w.ccount[c] = 0;
    sort_cell(w.cstart[c], w.cstart[c + 1], w.perm, nullptr);
}

template <int D>
__global__ void k_wall_records(Batch bt, Walls w)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= w.n) return;
    int q = w.perm[k];
    int key = w.key[q];
    w.cell_of[k] = key;
    float4 lo;
    w.A4[k] = rel_pos<D>(bt.I[w.inst[q]], key, w.x[q], w.y[q], D == 3 ? w.z[q] : 0.0, &lo);
    w.L4[k] = lo;
    w.N4[k] = make_float4(w.nx[q], w.ny[q], D == 3 ? w.nz[q] : 0.0f, 0.0f);
}

int launch_wall_bin(const Batch &bt, Walls &w, int dim, cudaStream_t st)
{
    if (w.n == 0) {
        cudaMemsetAsync(w.cstart, 0, sizeof(int) * (bt.ncell + 1), st);
        return cudaGetLastError() == cudaSuccess ? 0 : -3;
    }
    int nb = (w.n + kBlock - 1) / kBlock;
    if (dim == 2) k_wall_key<2><<<nb, kBlock, 0, st>>>(bt, w);
    else k_wall_key<3><<<nb, kBlock, 0, st>>>(bt, w);
    k_scan_seg<<<bt.B, kScanThreads, 0, st>>>(bt, nullptr, nullptr, 0, nullptr, nullptr, 0, w.ccount, w.cstart, w.n, 2);
    k_wall_scatter<<<nb, kBlock, 0, st>>>(w);
    k_wall_cellsort<<<(bt.ncell + kBlock - 1) / kBlock, kBlock, 0, st>>>(w, bt.ncell);
    if (dim == 2) k_wall_records<2><<<nb, kBlock, 0, st>>>(bt, w);
    else k_wall_records<3><<<nb, kBlock, 0, st>>>(bt, w);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// generic single-block scan and scatter (the allocation-free entry point)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kScanThreads) k_scan(int *count, int *start, int n)
{
    int total = scan_cells(count, count, start, n, 0);
    if (threadIdx.x == 0) start[n] = total;
}

int launch_scan(int *ccount, int *cstart, int ncell, cudaStream_t st)
{
    k_scan<<<1, kScanThreads, 0, st>>>(ccount, cstart, ncell);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

__global__ void k_scatter(const int *__restrict__ key, const int *__restrict__ cstart, int *cursor, int *perm, int n)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int k = key[s];
    perm[cstart[k] + atomicAdd(&cursor[k], 1)] = s;
}

int launch_scatter(const int *key, const int *cstart, int *ccount, int *perm, int n, cudaStream_t st)
{
    if (n == 0) return 0;
    k_scatter<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(key, cstart, ccount, perm, n);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace sph
