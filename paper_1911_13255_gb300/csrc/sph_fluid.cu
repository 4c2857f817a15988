// Fluid pair loops at h_F (Section 3.1): momentum (Eq. fluid-model-mr-mom)
// with the low-dissipation Riemann pressure and the viscous term, the
// fluid-solid ghost forces (Eqs. fs-force-mr-sp, fs-force-mr-sv with the
// time-averaged solid state of Eq. fs-coupling-mr), their solid-side
// counterparts (Eqs. F:p, F:v), continuity (Eq. fluid-model-mr-con) and the
// density reinitialisation of Alg. 1.
//
// L consecutive threads share one target particle (cell order): each visits
// the 3^d cells around the target and takes every L-th candidate of each
// cell; the partial sums are combined with warp shuffles.  Consecutive
// targets share their neighbour cells, so the records (two float4 per
// particle) are served from L1/L2.  Pair geometry is FP32 on cell-relative
// coordinates: r_ij = (x_i - x_cell_i) - (x_j - x_cell_j) - dcell * edge.
#include "sph_common.cuh"

namespace sph {

// lanes per target particle
template <int D> struct Lanes { static constexpr int L = D == 2 ? 4 : 8; };

// Visit the 3^d neighbour cells of (cx, cy, cz).  fn(cell, ox, oy, oz)
// receives the offset o = -(dcell) * edge to add to (rel_i - rel_j).
template <int D, typename Fn>
__device__ __forceinline__ void for_each_cell(const Grid &g, int cx, int cy, int cz, Fn &&fn)
{
    const int z0 = D == 3 ? -1 : 0, z1 = D == 3 ? 1 : 0;
#pragma unroll 1
    for (int dz = z0; dz <= z1; dz++) {
        int z = cz + dz;
        if (z < 0 || z >= g.nc[2]) continue;
#pragma unroll 1
        for (int dy = -1; dy <= 1; dy++) {
            int y = cy + dy;
            if (y < 0 || y >= g.nc[1]) continue;
#pragma unroll 1
            for (int dx = -1; dx <= 1; dx++) {
                int x = cx + dx;
                if (x < 0 || x >= g.nc[0]) {
                    if (!g.periodic_x) continue;
                    x = x < 0 ? x + g.nc[0] : x - g.nc[0];
                }
                int c = x + g.nc[0] * (y + g.nc[1] * z);
                fn(c, -(float)dx * g.csf[0], -(float)dy * g.csf[1], -(float)dz * g.csf[2]);
            }
        }
    }
}

template <int L>
__device__ __forceinline__ float group_sum(float v)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int L>
__device__ __forceinline__ double group_sum_d(double v)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// p_i - p_j of Eq. eqeos without cancellation: with a = 1 + drho_i / rho0 and
// b = 1 + drho_j / rho0, p_i - p_j = (rho0 c^2 / 7) (a^7 - b^7)
//                                  = (rho0 c^2 / 7) (a - b) sum_k a^k b^(6-k)
__device__ __forceinline__ float eos_dp(float drho_i, float drho_j, const Phys &P)
{
    float inv = 1.0f / P.rho0;
    float a = 1.0f + drho_i * inv, b = 1.0f + drho_j * inv;
    float s = a + b;
    s = a * a + b * s;
    s = a * a * a + b * s;
    s = a * a * a * a + b * s;
    float a2 = a * a;
    s = a2 * a2 * a + b * s;
    s = a2 * a2 * a2 + b * s;
    return P.p_coef * ((drho_i - drho_j) * inv) * s;
}

__device__ __forceinline__ void cell_xyz(int key, const Grid &g, int &cx, int &cy, int &cz)
{
    cx = key % g.nc[0];
    cy = (key / g.nc[0]) % g.nc[1];
    cz = key / (g.nc[0] * g.nc[1]);
}

// Fluid-solid (or fluid-wall) pair: force on the fluid particle divided by
// its volume V_i, i.e. V_a [-2 p_bar dW/r d + 4 eta (v_i - v~_a) dW / (r + 0.01 h_F)]
// (Eqs. fs-force-mr-sp, fs-force-mr-sv with v_i - v^d_a = 2 (v_i - v~_a),
// reading R6: p^d = p_i + rho_i max(0, -(g - a~).n) max(0, r_ia.n), rho^d from
// the inverse EoS).  Identical arithmetic on the fluid and the solid side,
// so each pair's term is bitwise antisymmetric.
template <int D>
__device__ __forceinline__ void fs_pair_force(const float d[3], float r2, const float vi[3], float rhoi, float pi,
                                              const float4 &vb, const float4 &ab, const float4 &n, float Va,
                                              const Phys &P, float out[3])
{
    float r = sqrtf(r2);
    float invr = 1.0f / r;
    float dW = dW_F(r, P);
    float gn = (P.g[0] - ab.x) * n.x + (P.g[1] - ab.y) * n.y;
    float dn = d[0] * n.x + d[1] * n.y;
    if (D == 3) {
        gn += (P.g[2] - ab.z) * n.z;
        dn += d[2] * n.z;
    }
    float pd = pi + rhoi * fmaxf(0.0f, -gn) * fmaxf(0.0f, dn);
    float rhod = eos_rho(pd, P);
    float pbar = (pi * rhod + pd * rhoi) / (rhoi + rhod);
    float sp = -2.0f * pbar * dW * invr;
    float sv = 4.0f * P.eta * dW / (r + P.hreg);
    out[0] = Va * (sp * d[0] + sv * (vi[0] - vb.x));
    out[1] = Va * (sp * d[1] + sv * (vi[1] - vb.y));
    out[2] = D == 3 ? Va * (sp * d[2] + sv * (vi[2] - vb.z)) : 0.0f;
}

// Continuity contribution of a fluid-solid/wall pair (reading R7): the
// Riemann interface velocity between (v_i, p_i, rho_i) and the ghost
// (v^d, p^d, rho^d); only its normal part enters.
template <int D>
__device__ __forceinline__ float fs_pair_drho(const float d[3], float r2, const float vi[3], float rhoi, float pi,
                                              const float4 &vb, const float4 &ab, const float4 &n, float Va,
                                              const Phys &P)
{
    float r = sqrtf(r2);
    float invr = 1.0f / r;
    float dW = dW_F(r, P);
    float gn = (P.g[0] - ab.x) * n.x + (P.g[1] - ab.y) * n.y;
    float dn = d[0] * n.x + d[1] * n.y;
    float UL = -(vi[0] * d[0] + vi[1] * d[1]) * invr;
    float Ub = -(vb.x * d[0] + vb.y * d[1]) * invr;
    if (D == 3) {
        gn += (P.g[2] - ab.z) * n.z;
        dn += d[2] * n.z;
        UL -= vi[2] * d[2] * invr;
        Ub -= vb.z * d[2] * invr;
    }
    float dpg = rhoi * fmaxf(0.0f, -gn) * fmaxf(0.0f, dn);   // p^d - p_i
    float pd = pi + dpg;
    float rhod = eos_rho(pd, P);
    float rb = 0.5f * (rhoi + rhod);
    float diff = (UL - Ub) + dpg / (2.0f * rb * P.c0);
    return Va * (-dW) * diff;   // times 2 rho_i by the caller
}

template <int D>
__device__ __forceinline__ float rel_d(const float4 &Pi, const float4 &Pj, float ox, float oy, float oz, float d[3])
{
    d[0] = (Pi.x - Pj.x) + ox;
    d[1] = (Pi.y - Pj.y) + oy;
    d[2] = D == 3 ? (Pi.z - Pj.z) + oz : 0.0f;
    return d[0] * d[0] + d[1] * d[1] + (D == 3 ? d[2] * d[2] : 0.0f);
}

template <int D>
static inline int grid_blocks(int n)
{
    long long t = (long long)n * Lanes<D>::L;
    return (int)((t + kBlock - 1) / kBlock);
}

// ---------------------------------------------------------------------------
// a4: equation of state + momentum + kick
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kBlock) k_momentum(Fluid f, Walls w, Solid s, Grid g, Phys P, Ctl *ctl)
{
    constexpr int L = Lanes<D>::L;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / L, lane = t % L;
    const bool act = i < f.n;
    unsigned nff = 0, nfw = 0, nfs = 0;
    float acc[3] = {0.f, 0.f, 0.f}, afs[3] = {0.f, 0.f, 0.f};
    float4 Pi = make_float4(0.f, 0.f, 0.f, 0.f), Vi = Pi;
    if (act) {
        Pi = f.P4[i];
        Vi = f.V4[i];
        const float vi[3] = {Vi.x, Vi.y, Vi.z};
        const float rhoi = P.rho0 + Vi.w, pi = Pi.w;
        int cx, cy, cz;
        cell_xyz(f.cell_of[i], g, cx, cy, cz);
        const float c0 = P.c0, eta2 = 2.0f * P.eta;
        for_each_cell<D>(g, cx, cy, cz, [&](int c, float ox, float oy, float oz) {
            // fluid neighbours: Riemann pressure + viscous (Eq. fluid-model-mr-mom, reading R4)
            const int j1 = f.cstart[c + 1];
            for (int j = f.cstart[c] + lane; j < j1; j += L) {
                if (j == i) continue;
                const float4 Pj = f.P4[j];
                float d[3];
                float r2 = rel_d<D>(Pi, Pj, ox, oy, oz, d);
                if (r2 >= P.rc2F) continue;
                nff++;
                const float4 Vj = f.V4[j];
                const float rhoj = P.rho0 + Vj.w;
                float r = sqrtf(r2), invr = 1.0f / r;
                float dW = dW_F(r, P);
                // U = v.e with e = -d / r (from i to j)
                float UL = -(vi[0] * d[0] + vi[1] * d[1] + (D == 3 ? vi[2] * d[2] : 0.0f)) * invr;
                float UR = -(Vj.x * d[0] + Vj.y * d[1] + (D == 3 ? Vj.z * d[2] : 0.0f)) * invr;
                float rb = 0.5f * (rhoi + rhoj);
                float beta = fminf(3.0f * fmaxf(UL - UR, 0.0f), c0);
                float Ps = 0.5f * (pi + Pj.w) + 0.5f * rb * beta * (UL - UR);
                float sc = (P.mF / rhoj) * dW * invr;
                acc[0] += sc * (-2.0f * Ps * d[0] + eta2 * (vi[0] - Vj.x));
                acc[1] += sc * (-2.0f * Ps * d[1] + eta2 * (vi[1] - Vj.y));
                if (D == 3) acc[2] += sc * (-2.0f * Ps * d[2] + eta2 * (vi[2] - Vj.z));
            }
            // walls: v~ = a~ = 0
            const int a1 = w.cstart[c + 1];
            for (int a = w.cstart[c] + lane; a < a1; a += L) {
                float d[3];
                float r2 = rel_d<D>(Pi, w.A4[a], ox, oy, oz, d);
                if (r2 >= P.rc2F) continue;
                nfw++;
                const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                float o[3];
                fs_pair_force<D>(d, r2, vi, rhoi, pi, z4, z4, w.N4[a], P.VW, P, o);
                acc[0] += o[0];
                acc[1] += o[1];
                acc[2] += o[2];
            }
            // solid particles at their start-of-step positions with v~, a~
            if (s.n) {
                const int b1 = s.cstart[c + 1];
                for (int b = s.cstart[c] + lane; b < b1; b += L) {
                    float d[3];
                    float r2 = rel_d<D>(Pi, s.A4[b], ox, oy, oz, d);
                    if (r2 >= P.rc2F) continue;
                    nfs++;
                    float o[3];
                    fs_pair_force<D>(d, r2, vi, rhoi, pi, s.VB4[b], s.AB4[b], s.N4[b], P.VS, P, o);
                    afs[0] += o[0];
                    afs[1] += o[1];
                    afs[2] += o[2];
                }
            }
        });
    }
    for (int k = 0; k < D; k++) {
        acc[k] = group_sum<L>(acc[k]);
        afs[k] = group_sum<L>(afs[k]);
    }
    float vmax2 = 0.0f;
    double mfs[3] = {0.0, 0.0, 0.0};
    if (act && lane == 0) {
        const float rhoi = P.rho0 + Vi.w;
        const float vi[3] = {Vi.x, Vi.y, Vi.z};
        float inv_rho = 1.0f / rhoi;
        float a[3], vn[3] = {0.f, 0.f, 0.f};
        double dt = ctl->dt;
        for (int k = 0; k < D; k++) {
            a[k] = (acc[k] + afs[k]) * inv_rho + P.g[k];
            vn[k] = vi[k] + (float)dt * a[k];
            f.dvdt[(size_t)i * D + k] = a[k];
        }
        f.W4[i] = make_float4(vn[0], vn[1], vn[2], Vi.w);
        vmax2 = vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2];
        float Vi_ = P.mF / rhoi;   // force = V_i * afs (same V_i as the solid side)
        for (int k = 0; k < D; k++) mfs[k] = (double)(Vi_ * afs[k]);
    }
    // warp reductions, one atomic per warp
    unsigned tff = warp_sum_u(nff), tfw = warp_sum_u(nfw), tfs = warp_sum_u(nfs);
    float vm = warp_max(vmax2);
    for (int k = 0; k < D; k++) mfs[k] = warp_sum_d(mfs[k]);
    if ((threadIdx.x & 31) == 0) {
        if (tff) atomicAdd(&ctl->n_ff, (unsigned long long)tff);
        if (tfw) atomicAdd(&ctl->n_fw, (unsigned long long)tfw);
        if (tfs) {
            atomicAdd(&ctl->n_fs, (unsigned long long)tfs);
            for (int k = 0; k < D; k++) atomicAdd(&ctl->mom_fluid[k], mfs[k]);
        }
        atomic_max_pos(&ctl->vmaxF, sqrtf(vm));
    }
}

int launch_momentum(const Fluid &f, const Walls &w, const Solid &s, const Grid &g, const Phys &P, Ctl *ctl,
                    cudaStream_t st)
{
    if (f.n == 0) return 0;
    if (P.dim == 2) k_momentum<2><<<grid_blocks<2>(f.n), kBlock, 0, st>>>(f, w, s, g, P, ctl);
    else k_momentum<3><<<grid_blocks<3>(f.n), kBlock, 0, st>>>(f, w, s, g, P, ctl);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// a5: fluid force on each solid particle, f_a^F = -sum_i V_i (pair term),
// the same pair expression and inputs as a4 (fluid at r^{n+1/2}, v^n)
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kBlock) k_solid_fluid_force(Fluid f, Solid s, Grid g, Phys P, Ctl *ctl)
{
    constexpr int L = Lanes<D>::L;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = t / L, lane = t % L;
    const bool act = k < s.n;
    unsigned nsf = 0;
    float fa[3] = {0.f, 0.f, 0.f};
    int a = 0;
    if (act) {
        const float4 A = s.A4[k], VB = s.VB4[k], AB = s.AB4[k], N = s.N4[k];
        a = __float_as_int(N.w);
        int cx, cy, cz;
        cell_xyz(s.cell_of[k], g, cx, cy, cz);
        for_each_cell<D>(g, cx, cy, cz, [&](int c, float ox, float oy, float oz) {
            const int j1 = f.cstart[c + 1];
            for (int j = f.cstart[c] + lane; j < j1; j += L) {
                const float4 Pj = f.P4[j];
                // the fluid side sees this pair with the opposite cell offset
                float d[3] = {(Pj.x - A.x) - ox, (Pj.y - A.y) - oy, D == 3 ? (Pj.z - A.z) - oz : 0.0f};
                float r2 = d[0] * d[0] + d[1] * d[1] + (D == 3 ? d[2] * d[2] : 0.0f);
                if (r2 >= P.rc2F) continue;
                nsf++;
                const float4 Vj = f.V4[j];
                const float vj[3] = {Vj.x, Vj.y, Vj.z};
                const float rhoj = P.rho0 + Vj.w;
                float o[3];
                fs_pair_force<D>(d, r2, vj, rhoj, Pj.w, VB, AB, N, P.VS, P, o);
                float Vf = P.mF / rhoj;
                fa[0] -= Vf * o[0];
                fa[1] -= Vf * o[1];
                fa[2] -= Vf * o[2];
            }
        });
    }
    for (int q = 0; q < D; q++) fa[q] = group_sum<L>(fa[q]);
    double ms[3] = {0.0, 0.0, 0.0};
    if (act && lane == 0) {
        for (int q = 0; q < 3; q++) s.fF[3 * a + q] = q < D ? fa[q] : 0.0f;
        for (int q = 0; q < D; q++) ms[q] = (double)fa[q];
    }
    unsigned tt = warp_sum_u(nsf);
    for (int q = 0; q < D; q++) ms[q] = warp_sum_d(ms[q]);
    if ((threadIdx.x & 31) == 0 && tt) {
        atomicAdd(&ctl->n_sf, (unsigned long long)tt);
        for (int q = 0; q < D; q++) atomicAdd(&ctl->mom_solid[q], ms[q]);
    }
}

int launch_solid_fluid_force(const Fluid &f, const Solid &s, const Grid &g, const Phys &P, Ctl *ctl,
                             cudaStream_t st)
{
    if (s.n == 0 || f.n == 0) {
        if (s.n) cudaMemsetAsync(s.fF, 0, sizeof(float) * 3 * s.n, st);
        return cudaGetLastError() == cudaSuccess ? 0 : -3;
    }
    if (P.dim == 2) k_solid_fluid_force<2><<<grid_blocks<2>(s.n), kBlock, 0, st>>>(f, s, g, P, ctl);
    else k_solid_fluid_force<3><<<grid_blocks<3>(s.n), kBlock, 0, st>>>(f, s, g, P, ctl);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// a6: continuity at (r^{n+1/2}, rho^{n+1/2}, v^{n+1}) + second half drift;
// writes the end-of-step state to s[0] in cell order
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kBlock) k_density(Fluid f, Walls w, Solid s, Grid g, Phys P, Ctl *ctl)
{
    constexpr int L = Lanes<D>::L;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / L, lane = t % L;
    const bool act = i < f.n;
    float rate = 0.0f;
    float4 Pi = make_float4(0.f, 0.f, 0.f, 0.f), Wi = Pi;
    if (act) {
        Pi = f.P4[i];
        Wi = f.W4[i];
        const float vi[3] = {Wi.x, Wi.y, Wi.z};
        const float drhoi = Wi.w, rhoi = P.rho0 + Wi.w, pi = Pi.w;
        int cx, cy, cz;
        cell_xyz(f.cell_of[i], g, cx, cy, cz);
        const float inv2c0 = 0.5f / P.c0;
        for_each_cell<D>(g, cx, cy, cz, [&](int c, float ox, float oy, float oz) {
            const int j1 = f.cstart[c + 1];
            for (int j = f.cstart[c] + lane; j < j1; j += L) {
                if (j == i) continue;
                const float4 Pj = f.P4[j];
                float d[3];
                float r2 = rel_d<D>(Pi, Pj, ox, oy, oz, d);
                if (r2 >= P.rc2F) continue;
                const float4 Wj = f.W4[j];
                const float rhoj = P.rho0 + Wj.w;
                float r = sqrtf(r2), invr = 1.0f / r;
                float dW = dW_F(r, P);
                float UL = -(vi[0] * d[0] + vi[1] * d[1] + (D == 3 ? vi[2] * d[2] : 0.0f)) * invr;
                float UR = -(Wj.x * d[0] + Wj.y * d[1] + (D == 3 ? Wj.z * d[2] : 0.0f)) * invr;
                float rb = 0.5f * (rhoi + rhoj);
                // (v_i - v~_ij).grad_i W = -dW (U_L - U*), U* = (U_L + U_R)/2 + (p_i - p_j) / (2 rho c0)
                float diff = 0.5f * (UL - UR) - eos_dp(drhoi, Wj.w, P) * inv2c0 / rb;
                rate += (P.mF / rhoj) * (-dW) * diff;
            }
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            const int a1 = w.cstart[c + 1];
            for (int a = w.cstart[c] + lane; a < a1; a += L) {
                float d[3];
                float r2 = rel_d<D>(Pi, w.A4[a], ox, oy, oz, d);
                if (r2 >= P.rc2F) continue;
                rate += fs_pair_drho<D>(d, r2, vi, rhoi, pi, z4, z4, w.N4[a], P.VW, P);
            }
            if (s.n) {
                const int b1 = s.cstart[c + 1];
                for (int b = s.cstart[c] + lane; b < b1; b += L) {
                    float d[3];
                    float r2 = rel_d<D>(Pi, s.A4[b], ox, oy, oz, d);
                    if (r2 >= P.rc2F) continue;
                    rate += fs_pair_drho<D>(d, r2, vi, rhoi, pi, s.VB4[b], s.AB4[b], s.N4[b], P.VS, P);
                }
            }
        });
    }
    rate = group_sum<L>(rate);
    if (!act || lane != 0) return;
    const float vi[3] = {Wi.x, Wi.y, Wi.z};
    const float rhoi = P.rho0 + Wi.w;
    float rhodot = 2.0f * rhoi * rate;
    // second half drift (Eq. verlet-first-final) and the new state
    const FluidState M = f.s[1], S = f.s[0];
    double h = 0.5 * ctl->dt;
    double x = M.x[i] + h * (double)vi[0];
    double y = M.y[i] + h * (double)vi[1];
    if (g.periodic_x) {
        if (x >= g.x_lo + g.Lx) x -= g.Lx;
        else if (x < g.x_lo) x += g.Lx;
    }
    S.x[i] = x;
    S.y[i] = y;
    S.vx[i] = vi[0];
    S.vy[i] = vi[1];
    if (D == 3) {
        S.z[i] = M.z[i] + h * (double)vi[2];
        S.vz[i] = vi[2];
    }
    S.drho[i] = M.drho[i] + (float)h * rhodot;
    S.rhodot[i] = rhodot;
    S.id[i] = M.id[i];
}

int launch_density(const Fluid &f, const Walls &w, const Solid &s, const Grid &g, const Phys &P, Ctl *ctl,
                   cudaStream_t st)
{
    if (f.n == 0) return 0;
    if (P.dim == 2) k_density<2><<<grid_blocks<2>(f.n), kBlock, 0, st>>>(f, w, s, g, P, ctl);
    else k_density<3><<<grid_blocks<3>(f.n), kBlock, 0, st>>>(f, w, s, g, P, ctl);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// a3: density reinitialisation rho = rho0 sigma / sigma0 (reading R16).
// rho0 (sigma - sigma0) / sigma0 cancels about three digits, so each kernel
// value is evaluated in FP64 from the FP64 positions (the FP32 records only
// screen out candidates well outside the support) and summed in FP64.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ double W_fp64_shape(double dx, double dy, double dz, const Grid &g, double rc2,
                                               double inv_h)
{
    if (g.periodic_x) {
        if (dx > 0.5 * g.Lx) dx -= g.Lx;
        else if (dx < -0.5 * g.Lx) dx += g.Lx;
    }
    double r2 = dx * dx + dy * dy + (D == 3 ? dz * dz : 0.0);
    if (!(r2 < rc2)) return 0.0;
    // FP64 square root from the FP32 one and one Newton step (relative error ~1e-14)
    float rf = sqrtf((float)r2);
    double r = rf > 0.0f ? (double)rf + (r2 - (double)rf * (double)rf) * (double)(0.5f / rf) : 0.0;
    double q = r * inv_h, a = 1.0 - 0.5 * q, a2 = a * a;
    return a2 * a2 * (1.0 + 2.0 * q);   // times alpha_d by the caller
}

template <int D>
__global__ void __launch_bounds__(kBlock) k_reinit(Fluid f, Walls w, Solid s, Grid g, Phys P, const Ctl *ctl)
{
    if (!ctl->reinit) return;
    constexpr int L = Lanes<D>::L;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / L, lane = t % L;
    const bool act = i < f.n;
    const FluidState M = f.s[1];
    const double inv_h = 1.0 / P.hF_d, rc2 = P.rc2F_d;
    const float screen = P.rc2F * 1.0001f;
    double sF = 0.0, sW = 0.0, sS = 0.0;
    if (act) {
        const float4 Pi = f.P4[i];
        const double xi = M.x[i], yi = M.y[i], zi = D == 3 ? M.z[i] : 0.0;
        int cx, cy, cz;
        cell_xyz(f.cell_of[i], g, cx, cy, cz);
        for_each_cell<D>(g, cx, cy, cz, [&](int c, float ox, float oy, float oz) {
            const int j1 = f.cstart[c + 1];
            for (int j = f.cstart[c] + lane; j < j1; j += L) {
                if (j == i) continue;
                float d[3];
                if (rel_d<D>(Pi, f.P4[j], ox, oy, oz, d) >= screen) continue;
                sF += W_fp64_shape<D>(xi - M.x[j], yi - M.y[j], D == 3 ? zi - M.z[j] : 0.0, g, rc2, inv_h);
            }
            const int a1 = w.cstart[c + 1];
            for (int q = w.cstart[c] + lane; q < a1; q += L) {
                float d[3];
                if (rel_d<D>(Pi, w.A4[q], ox, oy, oz, d) >= screen) continue;
                int a = w.perm[q];
                sW += W_fp64_shape<D>(xi - w.x[a], yi - w.y[a], D == 3 ? zi - w.z[a] : 0.0, g, rc2, inv_h);
            }
            if (s.n) {
                const int b1 = s.cstart[c + 1];
                for (int q = s.cstart[c] + lane; q < b1; q += L) {
                    float d[3];
                    if (rel_d<D>(Pi, s.A4[q], ox, oy, oz, d) >= screen) continue;
                    int a = s.perm[q];
                    sS += W_fp64_shape<D>(xi - s.x[a], yi - s.y[a], D == 3 ? zi - s.z[a] : 0.0, g, rc2, inv_h);
                }
            }
        });
    }
    sF = group_sum_d<L>(sF);
    sW = group_sum_d<L>(sW);
    sS = group_sum_d<L>(sS);
    if (!act || lane != 0) return;
    double sigma = P.alphaF_d * (1.0 + sF + P.VW_VF_d * sW + P.VS_VF_d * sS);
    double dr = P.rho0_d * ((sigma - P.sigma0_d) / P.sigma0_d);
    if (P.free_surface && dr < 0.0) dr = 0.0;
    float drho = (float)dr;
    M.drho[i] = drho;
    f.P4[i].w = eos_p(drho, P);
    f.V4[i].w = drho;
}

int launch_reinit(const Fluid &f, const Walls &w, const Solid &s, const Grid &g, const Phys &P, Ctl *ctl,
                  cudaStream_t st)
{
    if (f.n == 0) return 0;
    if (P.dim == 2) k_reinit<2><<<grid_blocks<2>(f.n), kBlock, 0, st>>>(f, w, s, g, P, ctl);
    else k_reinit<3><<<grid_blocks<3>(f.n), kBlock, 0, st>>>(f, w, s, g, P, ctl);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// Neighbour sets with the FP64 in-support test (debug entry point).  Rows are
// fluid particles (which 0..2, cell-ordered mid-step copy s[1]) or solid
// particles (which 3); counts/fill two-phase; ids in original order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double r2_fp64(double dx, double dy, double dz, int D)
{
    double r2 = __dmul_rn(dx, dx);
    r2 = __dadd_rn(r2, __dmul_rn(dy, dy));
    if (D == 3) r2 = __dadd_rn(r2, __dmul_rn(dz, dz));
    return r2;
}

template <int D>
__global__ void k_debug_pairs(Fluid f, Walls w, Solid s, Grid g, Phys P, int which, int *counts,
                              const int *offs, int *out)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int nrows = which == 3 ? s.n : f.n;
    if (k >= nrows) return;
    double xi, yi, zi;
    int row, key;
    const FluidState M = f.s[1];
    if (which == 3) {
        int a = s.perm[k];
        xi = s.x[a];
        yi = s.y[a];
        zi = D == 3 ? s.z[a] : 0.0;
        row = a;
        key = s.cell_of[k];
    } else {
        xi = M.x[k];
        yi = M.y[k];
        zi = D == 3 ? M.z[k] : 0.0;
        row = M.id[k];
        key = f.cell_of[k];
    }
    int cx, cy, cz;
    cell_xyz(key, g, cx, cy, cz);
    int cnt = 0;
    int base = out ? offs[row] : 0;
    for_each_cell<D>(g, cx, cy, cz, [&](int c, float, float, float) {
        int j0, j1;
        if (which == 0 || which == 3) {
            j0 = f.cstart[c];
            j1 = f.cstart[c + 1];
        } else if (which == 1) {
            j0 = w.cstart[c];
            j1 = w.cstart[c + 1];
        } else {
            j0 = s.cstart[c];
            j1 = s.cstart[c + 1];
        }
        for (int j = j0; j < j1; j++) {
            double xj, yj, zj;
            int col;
            if (which == 0 || which == 3) {
                if (which == 0 && j == k) continue;
                xj = M.x[j];
                yj = M.y[j];
                zj = D == 3 ? M.z[j] : 0.0;
                col = M.id[j];
            } else if (which == 1) {
                int a = w.perm[j];
                xj = w.x[a];
                yj = w.y[a];
                zj = D == 3 ? w.z[a] : 0.0;
                col = a;
            } else {
                int a = s.perm[j];
                xj = s.x[a];
                yj = s.y[a];
                zj = D == 3 ? s.z[a] : 0.0;
                col = a;
            }
            double dx = xi - xj;
            if (g.periodic_x) {
                if (dx > 0.5 * g.Lx) dx -= g.Lx;
                else if (dx < -0.5 * g.Lx) dx += g.Lx;
            }
            if (r2_fp64(dx, yi - yj, zi - zj, D) < P.rc2F_d) {
                if (out) out[base + cnt] = col;
                cnt++;
            }
        }
    });
    if (!out) counts[row] = cnt;
}

int launch_debug_pairs(const Fluid &f, const Walls &w, const Solid &s, const Grid &g, const Phys &P, int which,
                       int *counts, int *offs, int *out, cudaStream_t st)
{
    int nrows = which == 3 ? s.n : f.n;
    if (nrows == 0) return 0;
    int nb = (nrows + kBlock - 1) / kBlock;
    if (P.dim == 2) k_debug_pairs<2><<<nb, kBlock, 0, st>>>(f, w, s, g, P, which, counts, offs, out);
    else k_debug_pairs<3><<<nb, kBlock, 0, st>>>(f, w, s, g, P, which, counts, offs, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace sph
