// Cell-linked-list neighbour build (Alg. 1, "particle-neighbour list"; the
// paper rebuilds it per advection step, this library every coarse step):
// a counting sort of particles by the linear index of their cell, cells of
// edge >= 2 h_F.  The sort is a single-digit radix sort whose digit is the
// global cell index: histogram (atomics), exclusive scan per instance,
// scatter, then a per-cell insertion sort by particle id so the order is
// deterministic and depends on the current state only.  The records kernel
// gathers the fluid state into cell order and emits the FP32 records the
// pair loops read.  Also: the per-step control kernel and the finish kernel.
#include "sph_common.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// control (one thread per instance) + normal update on reinit steps (one
// thread per solid particle); the reinit decision is recomputed from the
// instance's step index, which no thread of this kernel modifies
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_control_normals(Batch bt, Solid s, double dt_fixed, int K_fixed)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < bt.B) {
        const Phys &P = bt.I[t].P;
        Ctl *ctl = bt.ctl + t;
        const int has_solid = bt.I[t].ns > 0;
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
        ctl->learned_ok = 0;
        ctl->lnum = ctl->lden = 0.0;
    }
    if (t >= s.n) return;
    const int a = t;
    const Ctl *cb = bt.ctl + s.inst[a];
    if (!(cb->n_reinit > 0 && (cb->step % cb->n_reinit) == 0)) return;
    // n = normalize(F^-T n0), F^-T = cof(F) / det F   (Alg. 1, normal update)
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

int launch_control_normals(const Batch &bt, const Solid &s, double dt_fixed, int K_fixed, int dim, cudaStream_t st)
{
    int nt = s.n > bt.B ? s.n : bt.B;
    int nb = (nt + kBlock - 1) / kBlock;
    if (dim == 2) k_control_normals<2><<<nb, kBlock, 0, st>>>(bt, s, dt_fixed, K_fixed);
    else k_control_normals<3><<<nb, kBlock, 0, st>>>(bt, s, dt_fixed, K_fixed);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// finish: time, step, pair counters, non-finite check (one thread per instance)
__global__ void k_finish(Batch bt, int learned)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= bt.B) return;
    Ctl *ctl = bt.ctl + b;
    float vF = __uint_as_float(ctl->vmaxF), vS = __uint_as_float(ctl->vmaxS), aS = __uint_as_float(ctl->amaxS);
    if (!(vF <= 3.0e38f) || !(vS <= 3.0e38f) || !(aS <= 3.0e38f)) ctl->status |= ST_NONFINITE;
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

int launch_finish(const Batch &bt, int learned, cudaStream_t st)
{
    k_finish<<<(bt.B + kBlock - 1) / kBlock, kBlock, 0, st>>>(bt, learned);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// fluid: inflow buffer, first half drift (Eq. verlet-first-half), cell key;
// solid: cell key at the start-of-step position
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
__device__ __forceinline__ int global_key(const Inst &In, double x, double y, double z)
{
    const Grid &g = In.g;
    int cx = cell_coord(x, g.lo[0], g.cs[0], g.nc[0]);
    int cy = cell_coord(y, g.lo[1], g.cs[1], g.nc[1]);
    int cz = D == 3 ? cell_coord(z, g.lo[2], g.cs[2], g.nc[2]) : 0;
    return In.c0 + cx + g.nc[0] * (cy + g.nc[1] * cz);
}

template <int D>
__global__ void k_bin_all(Batch bt, Fluid f, Solid s, int do_drift)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < f.n) {
        const int i = t;
        const int b = f.inst[i];
        const Inst &In = bt.I[b];
        FluidState S = f.s[0];
        double x = S.x[i], y = S.y[i], z = D == 3 ? S.z[i] : 0.0;
        if (do_drift) {
            const Phys &P = In.P;
            const Grid &g = In.g;
            const Ctl *ctl = bt.ctl + b;
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
        int key = global_key<D>(In, x, y, z);
        f.key[i] = key;
        atomicAdd(&f.ccount[key], 1);
    } else if (t < f.n + s.n) {
        const int a = t - f.n;
        int key = global_key<D>(bt.I[s.inst[a]], s.x[a], s.y[a], D == 3 ? s.z[a] : 0.0);
        s.key[a] = key;
        atomicAdd(&s.ccount[key], 1);
    }
}

// ---------------------------------------------------------------------------
// exclusive scan of the cell histograms, one block per (instance, set):
// set 0 fluid, 1 solid, 2 walls; the cells of instance b are [c0, c0+ncell)
// and its slots start at f0 / s0 / w0.  Tiles of 8192 cells are loaded and
// stored coalesced through shared memory.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kTile = 8 * kScanThreads;

// returns base + the sum of the counts (to every thread)
__device__ int scan_cells(const int *count_in, int *count, int *start, int n, int base)
{
    __shared__ int sm[kTile];
    __shared__ int warp_tot[32];
    __shared__ int carry;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) carry = base;
    __syncthreads();
    for (int b0 = 0; b0 < n; b0 += kTile) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            int i = b0 + j * kScanThreads + t;
            sm[j * kScanThreads + t] = i < n ? count_in[i] : 0;
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
            int i = b0 + j * kScanThreads + t;
            if (i < n) {
                start[i] = sm[j * kScanThreads + t];
                count[i] = 0;   // the histogram becomes the scatter cursor
            }
        }
        if (t == kScanThreads - 1) carry = run;
        __syncthreads();
    }
    return carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_seg(Batch bt, int *fcount, int *fstart, int nf, int *scount,
                                                           int *sstart, int ns, int *wcount, int *wstart, int nw,
                                                           int set0)
{
    const int b = blockIdx.x % bt.B, set = set0 + blockIdx.x / bt.B;
    const Inst &In = bt.I[b];
    int *count = set == 0 ? fcount : (set == 1 ? scount : wcount);
    int *start = set == 0 ? fstart : (set == 1 ? sstart : wstart);
    const int base = set == 0 ? In.f0 : (set == 1 ? In.s0 : In.w0);
    scan_cells(count + In.c0, count + In.c0, start + In.c0, In.g.ncell, base);
    if (b == bt.B - 1 && threadIdx.x == 0) start[bt.ncell] = set == 0 ? nf : (set == 1 ? ns : nw);
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

// per-cell insertion sort by particle id (fluid) or slot (solid, walls), and
// the cursor reset for the next binning
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

// Canonical order inside every cell (the scatter's atomics leave it
// arbitrary): fluid entries by original id, solid entries by slot.  Keys are
// unique in a cell, so an entry's place is the number of smaller keys.
// Pass 1: a group of G lanes per cell (fluid cells, then solid cells); cells
// of up to G entries are ranked in registers with shuffles, larger ones are
// listed for pass 2, where blocks rank them in shared memory.  G = 16 in 2-D
// (about 7 fluid particles per cell), 32 in 3-D (about 18).
constexpr int kBigCellCap = 4096;

template <int G>
__global__ void k_cellsort_group(Fluid f, Solid s, int ncell, int *big, int *nbig)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int w = (int)(t / G), lane = threadIdx.x % G;
    const int total = (s.n ? 2 : 1) * ncell;
    const bool valid = w < total;
    const bool fl = w < ncell;
    const int c = fl ? w : w - ncell;
    int *perm = fl ? f.perm : s.perm;
    const int *id = fl ? f.s[0].id : nullptr;
    int a = 0, n = 0;
    if (valid) {
        const int *cs = fl ? f.cstart : s.cstart;
        if (lane == 0) (fl ? f.ccount : s.ccount)[c] = 0;
        a = cs[c];
        n = cs[c + 1] - a;
        if (n > G) {
            if (lane == 0) big[atomicAdd(nbig, 1)] = w;
            n = 0;
        }
    }
    // every lane of the warp runs the shuffle loop up to the warp's largest cell
    const int nmax = __reduce_max_sync(0xffffffffu, (unsigned)n);
    if (nmax <= 1) return;
    const bool mine = lane < n;
    const int v = mine ? perm[a + lane] : 0;
    const int kv = mine ? (id ? id[v] : v) : 0x7fffffff;
    int rank = 0;
    for (int k = 0; k < nmax; k++) {
        const int kk = __shfl_sync(0xffffffffu, kv, k, G);
        rank += (k < n && kk < kv) ? 1 : 0;
    }
    __syncwarp();
    if (mine && n > 1) perm[a + rank] = v;
}

__global__ void __launch_bounds__(256) k_cellsort_big(Fluid f, Solid s, int ncell, const int *big, const int *nbig)
{
    __shared__ int keys[kBigCellCap], vals[kBigCellCap];
    const int nb = *nbig;
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        const int w = big[t];
        const bool fl = w < ncell;
        const int c = fl ? w : w - ncell;
        int *perm = fl ? f.perm : s.perm;
        const int *id = fl ? f.s[0].id : nullptr;
        const int *cs = fl ? f.cstart : s.cstart;
        const int a = cs[c], n = cs[c + 1] - a;
        if (n > kBigCellCap) {   // beyond the shared-memory stage: one thread, in place
            if (threadIdx.x == 0) sort_cell(a, a + n, perm, id);
            __syncthreads();
            continue;
        }
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int v = perm[a + k];
            vals[k] = v;
            keys[k] = id ? id[v] : v;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int kv = keys[k];
            int r = 0;
            for (int m = 0; m < n; m++) r += keys[m] < kv;
            perm[a + r] = vals[k];
        }
        __syncthreads();
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

template <int D>
__global__ void k_records_all(Batch bt, Fluid f, Solid s)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < f.n) {
        const int k = t;
        FluidState A = f.s[0], B = f.s[1];
        int src = f.perm[k];
        const Inst &In = bt.I[f.inst[k]];
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
        const bool reinit = bt.ctl[f.inst[k]].reinit;
        float4 lo;
        float4 r = rel_pos<D>(In, key, x, y, z, reinit ? &lo : nullptr);
        if (reinit) f.L4[k] = lo;
        r.w = eos_p(dr, In.P);
        f.P4[k] = r;
        f.V4[k] = make_float4(vx, vy, vz, dr);
    } else if (t < f.n + s.n) {
        const int k = t - f.n;
        int a = s.perm[k];
        int key = s.key[a];
        s.cell_of[k] = key;
        const int b = s.inst[a];
        const bool reinit = bt.ctl[b].reinit;
        float4 lo;
        s.A4[k] = rel_pos<D>(bt.I[b], key, s.x[a], s.y[a], D == 3 ? s.z[a] : 0.0, reinit ? &lo : nullptr);
        if (reinit) s.L4[k] = lo;
        s.VB4[k] = make_float4((float)s.vbar[3 * a], (float)s.vbar[3 * a + 1], (float)s.vbar[3 * a + 2], 0.0f);
        s.AB4[k] = make_float4((float)s.abar[3 * a], (float)s.abar[3 * a + 1], (float)s.abar[3 * a + 2], 0.0f);
        s.N4[k] = make_float4(s.nrm[3 * a], s.nrm[3 * a + 1], s.nrm[3 * a + 2], __int_as_float(a));
    }
}

int launch_bin_all(const Batch &bt, Fluid &f, Solid &s, int dim, int do_drift, cudaStream_t st)
{
    const int nt = f.n + s.n;
    if (nt == 0) return 0;
    const int nb = (nt + kBlock - 1) / kBlock;
    if (dim == 2) k_bin_all<2><<<nb, kBlock, 0, st>>>(bt, f, s, do_drift);
    else k_bin_all<3><<<nb, kBlock, 0, st>>>(bt, f, s, do_drift);
    k_scan_seg<<<bt.B * (s.n ? 2 : 1), kScanThreads, 0, st>>>(bt, f.ccount, f.cstart, f.n, s.ccount, s.cstart, s.n,
                                                               nullptr, nullptr, 0, 0);
    k_scatter2<<<nb, kBlock, 0, st>>>(f, s);
    cudaMemsetAsync(f.nbig, 0, sizeof(int), st);
    const long long groups = (long long)(s.n ? 2 : 1) * bt.ncell;
    if (dim == 2)
        k_cellsort_group<16><<<(unsigned)((groups * 16 + kBlock - 1) / kBlock), kBlock, 0, st>>>(f, s, bt.ncell, f.big,
                                                                                                f.nbig);
    else
        k_cellsort_group<32><<<(unsigned)((groups * 32 + kBlock - 1) / kBlock), kBlock, 0, st>>>(f, s, bt.ncell, f.big,
                                                                                                f.nbig);
    k_cellsort_big<<<2 * 152, 256, 0, st>>>(f, s, bt.ncell, f.big, f.nbig);
    if (dim == 2) k_records_all<2><<<nb, kBlock, 0, st>>>(bt, f, s);
    else k_records_all<3><<<nb, kBlock, 0, st>>>(bt, f, s);
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
