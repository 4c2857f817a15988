// Cell-linked-list neighbour build (Alg. 1, "particle-neighbour list"; the
// paper rebuilds it per advection step, this library every coarse step):
// a counting sort of particles by the linear index of their cell, cells of
// edge >= 2 h_F.  The sort is a single-digit radix sort whose digit is the
// cell index: histogram (atomics), exclusive scan, scatter, then a per-cell
// insertion sort by particle id so the order is deterministic and depends
// on the current state only.  The reorder kernel gathers the fluid state
// into cell order and emits the FP32 records the pair loops read.
#include "sph_common.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// control / finish (one thread each)
// ---------------------------------------------------------------------------
__global__ void k_control(Ctl *ctl, Phys P, int has_solid)
{
    // previous step's maxima drive the automatic time steps (Section 3.2)
    float vF = __uint_as_float(ctl->vmaxF), vS = __uint_as_float(ctl->vmaxS), aS = __uint_as_float(ctl->amaxS);
    ctl->prev_vmaxF = vF;
    ctl->prev_vmaxS = vS;
    ctl->prev_amaxS = aS;
    ctl->vmaxF = ctl->vmaxS = ctl->amaxS = 0u;
    double dt = ctl->dt_fixed > 0.0 ? ctl->dt_fixed : 0.6 * P.hF_d / (P.c0_d + (double)vF);  // Eq. dt-relax
    int K = 1;
    if (ctl->K_fixed > 0) {
        K = ctl->K_fixed;
    } else if (has_solid) {
        double b1 = P.hS_d / (P.cS_d + (double)vS);
        double b2 = aS > 0.0f ? sqrt(P.hS_d / (double)aS) : 1e300;
        double dts = 0.6 * (b1 < b2 ? b1 : b2);      // Eq. dts-advection
        double k = floor(dt / dts) + 1.0;             // kappa = [dt_F / dt_S] + 1
        K = k > 1e6 ? 1000000 : (int)k;
    }
    ctl->dt = dt;
    ctl->K = K;
    ctl->dts = dt / (double)K;
    ctl->reinit = (ctl->n_reinit > 0 && (ctl->step % ctl->n_reinit) == 0) ? 1 : 0;
    ctl->n_ff = ctl->n_fw = ctl->n_fs = ctl->n_sf = 0ull;
    for (int k = 0; k < 3; k++) ctl->mom_fluid[k] = ctl->mom_solid[k] = 0.0;
}

__global__ void k_finish(Ctl *ctl, unsigned long long ss_pairs_per_step)
{
    float vF = __uint_as_float(ctl->vmaxF), vS = __uint_as_float(ctl->vmaxS), aS = __uint_as_float(ctl->amaxS);
    if (!(vF <= 3.0e38f) || !(vS <= 3.0e38f) || !(aS <= 3.0e38f)) ctl->status |= ST_NONFINITE;
    unsigned long long fl = ctl->n_ff + ctl->n_fw + ctl->n_fs;
    unsigned long long p = 2ull * fl + ctl->n_sf + (ctl->reinit ? fl : 0ull) +
                           (unsigned long long)(2 * ctl->K + 1) * ss_pairs_per_step;
    ctl->pairs_total += p;
    ctl->last_dt = ctl->dt;
    ctl->last_K = ctl->K;
    ctl->t += ctl->dt;
    ctl->step += 1;
}

int launch_control(Ctl *ctl, const Phys &P, int has_solid, cudaStream_t st)
{
    k_control<<<1, 1, 0, st>>>(ctl, P, has_solid);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// fluid: inflow buffer, first half drift (Eq. verlet-first-half), cell key
// ---------------------------------------------------------------------------
__device__ __forceinline__ double inflow_u(const Phys &P, double y, double t)
{
    double U = P.in_U;
    if (P.in_tramp > 0.0 && t < P.in_tramp) U = 0.5 * U * (1.0 - cos(3.14159265358979323846 * t / P.in_tramp));
    if (P.inflow_profile == 1) return U;
    double yy = y - P.in_y0, H = P.in_H;
    yy = yy < 0.0 ? 0.0 : (yy > H ? H : yy);
    return 6.0 * U * yy * (H - yy) / (H * H);
}

template <int D>
__global__ void k_fluid_drift_bin(Fluid f, Grid g, Phys P, const Ctl *__restrict__ ctl, int do_drift)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= f.n) return;
    // s[0] holds the state (cell order of the previous step); the reorder
    // writes the cell-ordered mid-step copy to s[1]; the density kernel
    // writes the end-of-step state back to s[0]
    FluidState S = f.s[0];
    double x = S.x[s], y = S.y[s], z = D == 3 ? S.z[s] : 0.0;
    if (do_drift) {
        double dt = ctl->dt, t = ctl->t;
        float vx = S.vx[s], vy = S.vy[s], vz = D == 3 ? S.vz[s] : 0.0f;
        if (P.inflow_on && x >= g.x_lo && x < g.x_lo + P.in_w) {
            vx = (float)inflow_u(P, y, t);
            vy = 0.0f;
            vz = 0.0f;
            S.vx[s] = vx;
            S.vy[s] = vy;
            if (D == 3) S.vz[s] = vz;
        }
        double h = 0.5 * dt;
        S.drho[s] = S.drho[s] + (float)h * S.rhodot[s];
        x = x + h * (double)vx;
        y = y + h * (double)vy;
        if (D == 3) z = z + h * (double)vz;
        if (g.periodic_x) {
            if (x >= g.x_lo + g.Lx) x -= g.Lx;
            else if (x < g.x_lo) x += g.Lx;
        }
        S.x[s] = x;
        S.y[s] = y;
        if (D == 3) S.z[s] = z;
    }
    int cx = cell_coord(x, g.lo[0], g.cs[0], g.nc[0]);
    int cy = cell_coord(y, g.lo[1], g.cs[1], g.nc[1]);
    int cz = D == 3 ? cell_coord(z, g.lo[2], g.cs[2], g.nc[2]) : 0;
    int key = cx + g.nc[0] * (cy + g.nc[1] * cz);
    f.key[s] = key;
    atomicAdd(&f.ccount[key], 1);
}

int launch_fluid_drift_bin(const Fluid &f, const Grid &g, const Phys &P, Ctl *ctl, int do_drift, cudaStream_t st)
{
    if (f.n == 0) return 0;
    int nb = (f.n + kBlock - 1) / kBlock;
    if (P.dim == 2) k_fluid_drift_bin<2><<<nb, kBlock, 0, st>>>(f, g, P, ctl, do_drift);
    else k_fluid_drift_bin<3><<<nb, kBlock, 0, st>>>(f, g, P, ctl, do_drift);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// exclusive scan of the cell histogram (one block); resets nothing: the
// histogram becomes the scatter cursor after being zeroed here.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;

// One pass: thread t owns the contiguous chunk [t*per, (t+1)*per) (served
// from L1/L2), a block-wide scan of the chunk sums gives each chunk's base.
__global__ void __launch_bounds__(kScanThreads) k_scan(int *count, int *start, int n)
{
    __shared__ int warp_tot[32];
    const int t = threadIdx.x;
    const int per = (n + kScanThreads - 1) / kScanThreads;
    const int b0 = min(n, t * per), b1 = min(n, b0 + per);
    int loc = 0;
    for (int i = b0; i < b1; i++) loc += count[i];
    const int lane = t & 31, w = t >> 5;
    int incl = loc;
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = warp_tot[lane];
        int xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += u;
        }
        warp_tot[lane] = xi - x;  // exclusive warp offsets
    }
    __syncthreads();
    int run = warp_tot[w] + incl - loc;
    for (int i = b0; i < b1; i++) {
        int v = count[i];
        start[i] = run;
        count[i] = 0;   // the histogram becomes the scatter cursor
        run += v;
    }
    if (t == kScanThreads - 1) start[n] = run;
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

// per-cell insertion sort of the slots by particle id (id == nullptr: by the
// storage index itself); zeroes the cursor for the next binning
__global__ void k_cellsort(const int *__restrict__ cstart, int *perm, const int *__restrict__ id, int *cursor,
                           int ncell)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    cursor[c] = 0;
    int a = cstart[c], b = cstart[c + 1];
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

static int cellsort(const int *cstart, int *perm, const int *id, int *cursor, int ncell, cudaStream_t st)
{
    k_cellsort<<<(ncell + kBlock - 1) / kBlock, kBlock, 0, st>>>(cstart, perm, id, cursor, ncell);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// fluid reorder into cell order + FP32 records
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_fluid_reorder(Fluid f, Grid g, Phys P)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= f.n) return;
    FluidState A = f.s[0], B = f.s[1];
    int s = f.perm[k];
    double x = A.x[s], y = A.y[s], z = D == 3 ? A.z[s] : 0.0;
    float vx = A.vx[s], vy = A.vy[s], vz = D == 3 ? A.vz[s] : 0.0f;
    float dr = A.drho[s];
    B.x[k] = x;
    B.y[k] = y;
    B.vx[k] = vx;
    B.vy[k] = vy;
    if (D == 3) {
        B.z[k] = z;
        B.vz[k] = vz;
    }
    B.drho[k] = dr;
    B.rhodot[k] = A.rhodot[s];
    B.id[k] = A.id[s];
    int key = f.key[s];
    f.cell_of[k] = key;
    int cx = key % g.nc[0];
    int cy = (key / g.nc[0]) % g.nc[1];
    int cz = D == 3 ? key / (g.nc[0] * g.nc[1]) : 0;
    float xr = (float)(x - (g.lo[0] + (double)cx * g.cs[0]));
    float yr = (float)(y - (g.lo[1] + (double)cy * g.cs[1]));
    float zr = D == 3 ? (float)(z - (g.lo[2] + (double)cz * g.cs[2])) : 0.0f;
    f.P4[k] = make_float4(xr, yr, zr, eos_p(dr, P));
    f.V4[k] = make_float4(vx, vy, vz, dr);
}

int launch_fluid_reorder(Fluid &f, const Grid &g, const Phys &P, cudaStream_t st)
{
    if (f.n == 0) return 0;
    int rc;
    if ((rc = launch_scan(f.ccount, f.cstart, g.ncell, st))) return rc;
    if ((rc = launch_scatter(f.key, f.cstart, f.ccount, f.perm, f.n, st))) return rc;
    if ((rc = cellsort(f.cstart, f.perm, f.s[0].id, f.ccount, g.ncell, st))) return rc;
    int nb = (f.n + kBlock - 1) / kBlock;
    if (P.dim == 2) k_fluid_reorder<2><<<nb, kBlock, 0, st>>>(f, g, P);
    else k_fluid_reorder<3><<<nb, kBlock, 0, st>>>(f, g, P);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// static walls: binned once
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_wall_key(Walls w, Grid g)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= w.n) return;
    int cx = cell_coord(w.x[s], g.lo[0], g.cs[0], g.nc[0]);
    int cy = cell_coord(w.y[s], g.lo[1], g.cs[1], g.nc[1]);
    int cz = D == 3 ? cell_coord(w.z[s], g.lo[2], g.cs[2], g.nc[2]) : 0;
    int key = cx + g.nc[0] * (cy + g.nc[1] * cz);
    w.key[s] = key;
    atomicAdd(&w.ccount[key], 1);
}

template <int D>
__global__ void k_wall_records(Walls w, Grid g)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= w.n) return;
    int s = w.perm[k];
    int key = w.key[s];
    w.cell_of[k] = key;
    int cx = key % g.nc[0];
    int cy = (key / g.nc[0]) % g.nc[1];
    int cz = D == 3 ? key / (g.nc[0] * g.nc[1]) : 0;
    float xr = (float)(w.x[s] - (g.lo[0] + (double)cx * g.cs[0]));
    float yr = (float)(w.y[s] - (g.lo[1] + (double)cy * g.cs[1]));
    float zr = D == 3 ? (float)(w.z[s] - (g.lo[2] + (double)cz * g.cs[2])) : 0.0f;
    w.A4[k] = make_float4(xr, yr, zr, 0.0f);
    w.N4[k] = make_float4(w.nx[s], w.ny[s], D == 3 ? w.nz[s] : 0.0f, 0.0f);
}

int launch_wall_bin(Walls &w, const Grid &g, cudaStream_t st)
{
    if (w.n == 0) {
        cudaMemsetAsync(w.cstart, 0, sizeof(int) * (g.ncell + 1), st);
        return cudaGetLastError() == cudaSuccess ? 0 : -3;
    }
    int nb = (w.n + kBlock - 1) / kBlock;
    int D = w.z ? 3 : 2;
    if (D == 2) k_wall_key<2><<<nb, kBlock, 0, st>>>(w, g);
    else k_wall_key<3><<<nb, kBlock, 0, st>>>(w, g);
    int rc;
    if ((rc = launch_scan(w.ccount, w.cstart, g.ncell, st))) return rc;
    if ((rc = launch_scatter(w.key, w.cstart, w.ccount, w.perm, w.n, st))) return rc;
    if ((rc = cellsort(w.cstart, w.perm, nullptr, w.ccount, g.ncell, st))) return rc;
    if (D == 2) k_wall_records<2><<<nb, kBlock, 0, st>>>(w, g);
    else k_wall_records<3><<<nb, kBlock, 0, st>>>(w, g);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// solid particles in the fluid grid (at the start-of-step positions)
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_solid_key(Solid s, Grid g)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= s.n) return;
    int cx = cell_coord(s.x[a], g.lo[0], g.cs[0], g.nc[0]);
    int cy = cell_coord(s.y[a], g.lo[1], g.cs[1], g.nc[1]);
    int cz = D == 3 ? cell_coord(s.z[a], g.lo[2], g.cs[2], g.nc[2]) : 0;
    int key = cx + g.nc[0] * (cy + g.nc[1] * cz);
    s.key[a] = key;
    atomicAdd(&s.ccount[key], 1);
}

template <int D>
__global__ void k_solid_records(Solid s, Grid g)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.n) return;
    int a = s.perm[k];
    int key = s.key[a];
    s.cell_of[k] = key;
    int cx = key % g.nc[0];
    int cy = (key / g.nc[0]) % g.nc[1];
    int cz = D == 3 ? key / (g.nc[0] * g.nc[1]) : 0;
    float xr = (float)(s.x[a] - (g.lo[0] + (double)cx * g.cs[0]));
    float yr = (float)(s.y[a] - (g.lo[1] + (double)cy * g.cs[1]));
    float zr = D == 3 ? (float)(s.z[a] - (g.lo[2] + (double)cz * g.cs[2])) : 0.0f;
    s.A4[k] = make_float4(xr, yr, zr, 0.0f);
    s.VB4[k] = make_float4((float)s.vbar[3 * a], (float)s.vbar[3 * a + 1], (float)s.vbar[3 * a + 2], 0.0f);
    s.AB4[k] = make_float4((float)s.abar[3 * a], (float)s.abar[3 * a + 1], (float)s.abar[3 * a + 2], 0.0f);
    s.N4[k] = make_float4(s.nrm[3 * a], s.nrm[3 * a + 1], s.nrm[3 * a + 2], __int_as_float(a));
}

int launch_solid_bin(Solid &s, const Grid &g, const Phys &P, Ctl *ctl, cudaStream_t st)
{
    (void)ctl;
    if (s.n == 0) return 0;
    int nb = (s.n + kBlock - 1) / kBlock;
    if (P.dim == 2) k_solid_key<2><<<nb, kBlock, 0, st>>>(s, g);
    else k_solid_key<3><<<nb, kBlock, 0, st>>>(s, g);
    int rc;
    if ((rc = launch_scan(s.ccount, s.cstart, g.ncell, st))) return rc;
    if ((rc = launch_scatter(s.key, s.cstart, s.ccount, s.perm, s.n, st))) return rc;
    if ((rc = cellsort(s.cstart, s.perm, nullptr, s.ccount, g.ncell, st))) return rc;
    if (P.dim == 2) k_solid_records<2><<<nb, kBlock, 0, st>>>(s, g);
    else k_solid_records<3><<<nb, kBlock, 0, st>>>(s, g);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// normal update n = normalize(F^-T n0) at the reinitialisation cadence (Alg. 1)
template <int D>
__global__ void k_solid_normals(Solid s, const Ctl *__restrict__ ctl)
{
    if (!ctl->reinit) return;
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= s.n) return;
    const float *Hm = s.H + 9 * a;
    float F[9];
    for (int i = 0; i < 9; i++) F[i] = Hm[i];
    if (D == 2) {
        F[0] += 1.0f;
        F[3] += 1.0f;
    } else {
        F[0] += 1.0f;
        F[4] += 1.0f;
        F[8] += 1.0f;
    }
    const float *n0 = s.n0 + 3 * a;
    float n[3];
    if (D == 2) {
        // F^-T = (1/J) [[F11, -F10], [-F01, F00]]; the 1/J drops in the normalisation
        n[0] = F[3] * n0[0] - F[2] * n0[1];
        n[1] = -F[1] * n0[0] + F[0] * n0[1];
        n[2] = 0.0f;
    } else {
        // cofactor matrix of F = J F^-T
        float c00 = F[4] * F[8] - F[5] * F[7], c01 = F[5] * F[6] - F[3] * F[8], c02 = F[3] * F[7] - F[4] * F[6];
        float c10 = F[2] * F[7] - F[1] * F[8], c11 = F[0] * F[8] - F[2] * F[6], c12 = F[1] * F[6] - F[0] * F[7];
        float c20 = F[1] * F[5] - F[2] * F[4], c21 = F[2] * F[3] - F[0] * F[5], c22 = F[0] * F[4] - F[1] * F[3];
        n[0] = c00 * n0[0] + c01 * n0[1] + c02 * n0[2];
        n[1] = c10 * n0[0] + c11 * n0[1] + c12 * n0[2];
        n[2] = c20 * n0[0] + c21 * n0[1] + c22 * n0[2];
    }
    float det = D == 2 ? F[0] * F[3] - F[1] * F[2]
                       : F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                             F[2] * (F[3] * F[7] - F[4] * F[6]);
    float sgn = det < 0.0f ? -1.0f : 1.0f;
    float inv = sgn * rsqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    s.nrm[3 * a] = n[0] * inv;
    s.nrm[3 * a + 1] = n[1] * inv;
    s.nrm[3 * a + 2] = n[2] * inv;
}

int launch_solid_normals(Solid &s, const Phys &P, Ctl *ctl, cudaStream_t st)
{
    if (s.n == 0) return 0;
    int nb = (s.n + kBlock - 1) / kBlock;
    if (P.dim == 2) k_solid_normals<2><<<nb, kBlock, 0, st>>>(s, ctl);
    else k_solid_normals<3><<<nb, kBlock, 0, st>>>(s, ctl);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// Merged per-step binning of the fluid (after its first half drift) and of
// the solid (at its start-of-step position): five kernels for both sets.
// ---------------------------------------------------------------------------

// control (thread 0 of block 0) + normal update on reinit steps (every
// solid particle); the reinit decision is recomputed from the step index,
// which no thread of this kernel modifies
template <int D>
__global__ void k_control_normals(Ctl *ctl, Phys P, Solid s, int has_solid, double dt_fixed, int K_fixed)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->dt_fixed = dt_fixed;
        ctl->K_fixed = K_fixed;
        float vF = __uint_as_float(ctl->vmaxF), vS = __uint_as_float(ctl->vmaxS), aS = __uint_as_float(ctl->amaxS);
        ctl->prev_vmaxF = vF;
        ctl->prev_vmaxS = vS;
        ctl->prev_amaxS = aS;
        ctl->vmaxF = ctl->vmaxS = ctl->amaxS = 0u;
        double dt = dt_fixed > 0.0 ? dt_fixed : 0.6 * P.hF_d / (P.c0_d + (double)vF);   // Eq. dt-relax
        int K = 1;
        if (K_fixed > 0) {
            K = K_fixed;
        } else if (has_solid) {
            double b1 = P.hS_d / (P.cS_d + (double)vS);
            double b2 = aS > 0.0f ? sqrt(P.hS_d / (double)aS) : 1e300;
            double dts = 0.6 * (b1 < b2 ? b1 : b2);   // Eq. dts-advection
            double k = floor(dt / dts) + 1.0;          // kappa = [dt_F / dt_S] + 1
            K = k > 1e6 ? 1000000 : (int)k;
        }
        ctl->dt = dt;
        ctl->K = K;
        ctl->dts = dt / (double)K;
        ctl->reinit = (ctl->n_reinit > 0 && (ctl->step % ctl->n_reinit) == 0) ? 1 : 0;
        ctl->n_ff = ctl->n_fw = ctl->n_fs = ctl->n_sf = 0ull;
        for (int k = 0; k < 3; k++) ctl->mom_fluid[k] = ctl->mom_solid[k] = 0.0;
    }
    const bool reinit = ctl->n_reinit > 0 && (ctl->step % ctl->n_reinit) == 0;
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (!reinit || a >= s.n) return;
    // n = normalize(F^-T n0), F^-T = cof(F) / det F
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

int launch_control_normals(Ctl *ctl, const Phys &P, const Solid &s, double dt_fixed, int K_fixed, cudaStream_t st)
{
    int nb = s.n > 0 ? (s.n + kBlock - 1) / kBlock : 1;
    if (P.dim == 2) k_control_normals<2><<<nb, kBlock, 0, st>>>(ctl, P, s, s.n > 0, dt_fixed, K_fixed);
    else k_control_normals<3><<<nb, kBlock, 0, st>>>(ctl, P, s, s.n > 0, dt_fixed, K_fixed);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

template <int D>
__global__ void k_bin_all(Fluid f, Solid s, Grid g, Phys P, const Ctl *__restrict__ ctl, int do_drift)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < f.n) {
        const int i = t;
        FluidState S = f.s[0];
        double x = S.x[i], y = S.y[i], z = D == 3 ? S.z[i] : 0.0;
        if (do_drift) {
            double dt = ctl->dt, tm = ctl->t;
            float vx = S.vx[i], vy = S.vy[i], vz = D == 3 ? S.vz[i] : 0.0f;
            if (P.inflow_on && x >= g.x_lo && x < g.x_lo + P.in_w) {   // inflow buffer (reading R18)
                vx = (float)inflow_u(P, y, tm);
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
        int key = cell_coord(x, g.lo[0], g.cs[0], g.nc[0]) +
                  g.nc[0] * (cell_coord(y, g.lo[1], g.cs[1], g.nc[1]) +
                             g.nc[1] * (D == 3 ? cell_coord(z, g.lo[2], g.cs[2], g.nc[2]) : 0));
        f.key[i] = key;
        atomicAdd(&f.ccount[key], 1);
    } else if (t < f.n + s.n) {
        const int a = t - f.n;
        int key = cell_coord(s.x[a], g.lo[0], g.cs[0], g.nc[0]) +
                  g.nc[0] * (cell_coord(s.y[a], g.lo[1], g.cs[1], g.nc[1]) +
                             g.nc[1] * (D == 3 ? cell_coord(s.z[a], g.lo[2], g.cs[2], g.nc[2]) : 0));
        s.key[a] = key;
        atomicAdd(&s.ccount[key], 1);
    }
}

// exclusive scan of one or two histograms (block b scans pair b): tiles of
// 8192 cells loaded and stored coalesced through shared memory
constexpr int kTile = 8 * kScanThreads;
__global__ void __launch_bounds__(kScanThreads) k_scan2(int *countA, int *startA, int *countB, int *startB, int n)
{
    __shared__ int sm[kTile];
    __shared__ int warp_tot[32];
    __shared__ int carry;
    int *count = blockIdx.x == 0 ? countA : countB;
    int *start = blockIdx.x == 0 ? startA : startB;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) carry = 0;
    for (int base = 0; base < n; base += kTile) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            int i = base + j * kScanThreads + t;
            sm[j * kScanThreads + t] = i < n ? count[i] : 0;
        }
        __syncthreads();
        int v[8], loc = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            v[j] = sm[t * 8 + j];
            loc += v[j];
        }
        int incl = loc;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) warp_tot[w] = incl;
        __syncthreads();
        if (w == 0) {
            int x = warp_tot[lane], xi = x;
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= o) xi += u;
            }
            warp_tot[lane] = xi - x;
        }
        __syncthreads();
        int run = carry + warp_tot[w] + incl - loc;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            sm[t * 8 + j] = run;
            run += v[j];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 8; j++) {
            int i = base + j * kScanThreads + t;
            if (i < n) {
                start[i] = sm[j * kScanThreads + t];
                count[i] = 0;   // the histogram becomes the scatter cursor
            }
        }
        if (t == kScanThreads - 1) carry = run;
        __syncthreads();
    }
    if (t == 0) start[n] = carry;
}

__global__ void k_scatter2(Fluid f, Solid s)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < f.n) {
        int k = f.key[t];
        f.perm[f.cstart[k] + atomicAdd(&f.ccount[k], 1)] = t;
    } else if (t < f.n + s.n) {
        int a = t - f.n;
        int k = s.key[a];
        s.perm[s.cstart[k] + atomicAdd(&s.ccount[k], 1)] = a;
    }
}

// per-cell insertion sort by particle id (fluid) or index (solid), and the
// cursor reset for the next binning
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

__global__ void k_cellsort2(Fluid f, Solid s, int ncell)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ncell) {
        f.ccount[t] = 0;
        sort_cell(f.cstart[t], f.cstart[t + 1], f.perm, f.s[0].id);
    } else if (s.n && t < 2 * ncell) {
        int c = t - ncell;
        s.ccount[c] = 0;
        sort_cell(s.cstart[c], s.cstart[c + 1], s.perm, nullptr);
    }
}

template <int D>
__global__ void k_records_all(Fluid f, Solid s, Grid g, Phys P)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < f.n) {
        const int k = t;
        FluidState A = f.s[0], B = f.s[1];
        int src = f.perm[k];
        double x = A.x[src], y = A.y[src], z = D == 3 ? A.z[src] : 0.0;
        float vx = A.vx[src], vy = A.vy[src], vz = D == 3 ? A.vz[src] : 0.0f;
        float dr = A.drho[src];
        B.x[k] = x;
        B.y[k] = y;
        B.vx[k] = vx;
        B.vy[k] = vy;
        if (D == 3) {
            B.z[k] = z;
            B.vz[k] = vz;
        }
        B.drho[k] = dr;
        B.rhodot[k] = A.rhodot[src];
        B.id[k] = A.id[src];
        int key = f.key[src];
        f.cell_of[k] = key;
        int cx = key % g.nc[0], cy = (key / g.nc[0]) % g.nc[1], cz = D == 3 ? key / (g.nc[0] * g.nc[1]) : 0;
        float xr = (float)(x - (g.lo[0] + (double)cx * g.cs[0]));
        float yr = (float)(y - (g.lo[1] + (double)cy * g.cs[1]));
        float zr = D == 3 ? (float)(z - (g.lo[2] + (double)cz * g.cs[2])) : 0.0f;
        f.P4[k] = make_float4(xr, yr, zr, eos_p(dr, P));
        f.V4[k] = make_float4(vx, vy, vz, dr);
    } else if (t < f.n + s.n) {
        const int k = t - f.n;
        int a = s.perm[k];
        int key = s.key[a];
        s.cell_of[k] = key;
        int cx = key % g.nc[0], cy = (key / g.nc[0]) % g.nc[1], cz = D == 3 ? key / (g.nc[0] * g.nc[1]) : 0;
        float xr = (float)(s.x[a] - (g.lo[0] + (double)cx * g.cs[0]));
        float yr = (float)(s.y[a] - (g.lo[1] + (double)cy * g.cs[1]));
        float zr = D == 3 ? (float)(s.z[a] - (g.lo[2] + (double)cz * g.cs[2])) : 0.0f;
        s.A4[k] = make_float4(xr, yr, zr, 0.0f);
        s.VB4[k] = make_float4((float)s.vbar[3 * a], (float)s.vbar[3 * a + 1], (float)s.vbar[3 * a + 2], 0.0f);
        s.AB4[k] = make_float4((float)s.abar[3 * a], (float)s.abar[3 * a + 1], (float)s.abar[3 * a + 2], 0.0f);
        s.N4[k] = make_float4(s.nrm[3 * a], s.nrm[3 * a + 1], s.nrm[3 * a + 2], __int_as_float(a));
    }
}

int launch_bin_all(Fluid &f, Solid &s, const Grid &g, const Phys &P, Ctl *ctl, int do_drift, cudaStream_t st)
{
    const int nt = f.n + s.n;
    if (nt == 0) return 0;
    const int nb = (nt + kBlock - 1) / kBlock;
    if (P.dim == 2) k_bin_all<2><<<nb, kBlock, 0, st>>>(f, s, g, P, ctl, do_drift);
    else k_bin_all<3><<<nb, kBlock, 0, st>>>(f, s, g, P, ctl, do_drift);
    k_scan2<<<s.n ? 2 : 1, kScanThreads, 0, st>>>(f.ccount, f.cstart, s.ccount, s.cstart, g.ncell);
    k_scatter2<<<nb, kBlock, 0, st>>>(f, s);
    k_cellsort2<<<((s.n ? 2 : 1) * g.ncell + kBlock - 1) / kBlock, kBlock, 0, st>>>(f, s, g.ncell);
    if (P.dim == 2) k_records_all<2><<<nb, kBlock, 0, st>>>(f, s, g, P);
    else k_records_all<3><<<nb, kBlock, 0, st>>>(f, s, g, P);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_finish(Ctl *ctl, unsigned long long ss, cudaStream_t st)
{
    k_finish<<<1, 1, 0, st>>>(ctl, ss);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace sph
