// Fluid pair loops at h_F (Section 3.1), part 2: continuity (Eq.
// fluid-model-mr-con) with the second half drift, and the density
// reinitialisation of Alg. 1.  Shared loop machinery: sph_pairs.cuh.
#include <type_traits>

#include "sph_common.cuh"
#include "sph_pairs.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// a6: continuity at (r^{n+1/2}, rho^{n+1/2}, v^{n+1}) + second half drift;
// writes the end-of-step state to s[0] in cell order
// ---------------------------------------------------------------------------
template <int D, int L, bool CP, int FORM>
__device__ __forceinline__ void density_one(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int i,
                                                 bool act_, int lane, uint32_t *list, int stride, const TileSrc *ts)
{
    const bool act = act_;
    const int b = act ? f.inst[i] : 0;
    const Inst &In = bt.I[b];
    const Grid &g = In.g;
    const Phys &P = In.P;
    float rate = 0.0f;
    float4 Pi = make_float4(0.f, 0.f, 0.f, 0.f), Wi = Pi;
    if (act) {
        Pi = f.P4[i];
        Wi = f.W4[i];
        const float vi[3] = {Wi.x, Wi.y, Wi.z};
        const float drhoi = Wi.w, rhoi = P.rho0 + Wi.w, pi = Pi.w;
        int cx, cy, cz;
        cell_xyz(f.cell_of[i], In, cx, cy, cz);
        const float inv2c0 = 0.5f / P.c0;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        auto wall_pair = [&](int a, float ox, float oy, float oz) {
            float d[3];
            float r2 = rel_d<D>(Pi, w.A4[a], ox, oy, oz, d);
            if (r2 >= P.rc2F) return;
            rate += fs_pair_drho<D>(d, r2, vi, rhoi, pi, z4, z4, w.N4[a], P.VW, P);
        };
        auto solid_pair = [&](int b, float ox, float oy, float oz) {
            float d[3];
            float r2 = rel_d<D>(Pi, s.A4[b], ox, oy, oz, d);
            if (r2 >= P.rc2F) return;
            rate += fs_pair_drho<D>(d, r2, vi, rhoi, pi, s.VB4[b], s.AB4[b], s.N4[b], P.VS, P);
        };
        fluid_pairs<D, L, CP, FORM>(f, w, s, g, In.c0, cx, cy, cz, i, lane, Pi, P.rc2F, list, stride, ts,
                                [&](int j) { return f.W4[j]; },
                                [&](int, const float4 &, const float4 &Wj, const float *d, float r2, float, float,
                                    float) {
                if (r2 == 0.0f) return;   // a clumped pair: no direction, dW(0) = 0
                const float rhoj = P.rho0 + Wj.w;
                // one reciprocal square root for 1/r and r (r2 > 0 here)
                const float invr = rsqrtf(r2), r = r2 * invr;
                float dW = dW_F(r, P);
                float UL = -(vi[0] * d[0] + vi[1] * d[1] + (D == 3 ? vi[2] * d[2] : 0.0f)) * invr;
                float UR = -(Wj.x * d[0] + Wj.y * d[1] + (D == 3 ? Wj.z * d[2] : 0.0f)) * invr;
                float rb = 0.5f * (rhoi + rhoj);
                // (v_i - v~_ij).grad_i W = -dW (U_L - U*), U* = (U_L + U_R)/2 + (p_i - p_j) / (2 rho c0)
                float diff = 0.5f * (UL - UR) - eos_dp(drhoi, Wj.w, P) * inv2c0 / rb;
                rate += __fdividef(P.mF, rhoj) * (-dW) * diff;
            }, wall_pair, solid_pair);
    }
    rate = group_sum<L>(rate);
    if (!act || lane != 0) return;
    const float vi[3] = {Wi.x, Wi.y, Wi.z};
    const float rhoi = P.rho0 + Wi.w;
    float rhodot = 2.0f * rhoi * rate;
    // second half drift (Eq. verlet-first-final) and the new state
    const FluidState M = f.s[1], S = f.s[0];
    double h = 0.5 * bt.ctl[b].dt;
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

template <int D, int L, bool CP, bool TILE, int FORM>
__global__ void __launch_bounds__(kMaxBlock) k_density(Batch bt, Fluid f, Walls w, Solid s)
{
    pdl_enter();
    if (step_failed(bt)) return;   // the step's cell starts are not valid
    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint32_t *const list = (uint32_t *)s_dyn + threadIdx.x;
    const int stride = blockDim.x;
    if constexpr (!TILE) {
        const int t = blockIdx.x * blockDim.x + threadIdx.x;
        density_one<D, L, CP, FORM>(bt, f, w, s, t / L, t / L < f.n, t % L, list, stride, nullptr);
    } else {
        tile_loop<D, L>(bt, f, f.W4, s_dyn + (CP ? (size_t)kListBytes * blockDim.x : 0),
                        [&](int i, bool act, const TileSrc *ts) {
                            density_one<D, L, CP, FORM>(bt, f, w, s, i, act, (int)threadIdx.x % L, list, stride, ts);
                        });
    }
}

int launch_density(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int dim, cudaStream_t st)
{
    if (f.n == 0) return 0;
    if (f.n >= kMaxPairTargets) return -7;
    SPH_LAUNCH_PAIRS(k_density, f.n, bt, f, w, s);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// Density reinitialisation (Alg. 1, every n_reinit steps): rho = rho0 sigma /
// sigma0 with the number density sigma = sum_j W_ij V_j / V_i, self term
// included (reading R16).  rho - rho0 = rho0 (sigma - sigma0) / sigma0 loses
// three to four digits to cancellation, so each W_ij must be good to far
// better than FP32.  FP64 arithmetic is a small fraction of the FP32 rate on
// this GPU; the pair terms are therefore evaluated in double-float
// arithmetic (an unevaluated sum hi + lo of two FP32 numbers, about 44
// significant bits, built from the error-free transformations TwoSum
// (Knuth), FastTwoSum (Dekker) and TwoProduct with one FMA), starting from
// cell-relative positions carried as hi + lo pairs.  Per-particle sums are
// finished in FP64.
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_sqr(ff a)
{
    const float p = __fmul_rn(a.hi, a.hi);
    const float e = fmaf(2.0f * a.hi, a.lo, fmaf(a.hi, a.hi, -p));
    return ff_fast_two_sum(p, e);
}
// (xi + li) - (xj + lj) + (o + ol)
__device__ __forceinline__ ff ff_delta(float xi, float li, float xj, float lj, float o, float ol)
{
    const ff t = ff_two_sum(xi, -xj);
    const ff u = ff_two_sum(t.hi, o);
    return ff_fast_two_sum(u.hi, __fadd_rn(__fadd_rn(t.lo, u.lo), __fadd_rn(__fsub_rn(li, lj), ol)));
}
// cell offset o = -dcell * edge as hi + lo (o is 0, +-csf or +-2 csf)
__device__ __forceinline__ float off_lo(float o, float csf, float cslo)
{
    // o = -dcell csf exactly, |dcell| <= 2; the remainder scales the same way
    const float m = fabsf(o) > 1.5f * csf ? 2.0f : 1.0f;
    return o == 0.0f ? 0.0f : (o > 0.0f ? m * cslo : -m * cslo);
}

// Wendland C2 shape (1 - q/2)^4 (1 + 2q) of the pair, q = |r_ij| / h_F, in
// double-float; 0 outside the support.
template <int D>
__device__ __forceinline__ ff W_ff_shape(const float4 &Pi, const float4 &Li, const float4 &Pj, const float4 &Lj,
                                         float ox, float oy, float oz, const Grid &g, const Phys &P)
{
    const ff dx = ff_delta(Pi.x, Li.x, Pj.x, Lj.x, ox, off_lo(ox, g.csf[0], g.cslo[0]));
    const ff dy = ff_delta(Pi.y, Li.y, Pj.y, Lj.y, oy, off_lo(oy, g.csf[1], g.cslo[1]));
    ff r2 = ff_add(ff_sqr(dx), ff_sqr(dy));
    if (D == 3) r2 = ff_add(r2, ff_sqr(ff_delta(Pi.z, Li.z, Pj.z, Lj.z, oz, off_lo(oz, g.csf[2], g.cslo[2]))));
    if (!(r2.hi > 0.0f)) return {1.0f, 0.0f};
    // r = sqrt(r2): FP32 root s plus one Newton correction (r2 - s^2) / (2 s)
    const float s = sqrtf(r2.hi);
    const float p = __fmul_rn(s, s);
    const float res = __fadd_rn(__fsub_rn(__fsub_rn(r2.hi, p), fmaf(s, s, -p)), r2.lo);
    const ff r = ff_fast_two_sum(s, __fmul_rn(res, __fmul_rn(0.5f, __frcp_rn(s))));
    const ff q = ff_mul(r, ff{P.ihF_hi, P.ihF_lo});
    if (q.hi >= 2.0f) return {0.0f, 0.0f};
    const ff a = {1.0f, 0.0f};
    const ff ha = ff_add(a, ff{-0.5f * q.hi, -0.5f * q.lo});       // 1 - q/2
    const ff bq = ff_add(a, ff{2.0f * q.hi, 2.0f * q.lo});         // 1 + 2q
    const ff a2 = ff_sqr(ha);
    return ff_mul(ff_sqr(a2), bq);
}

template <int D, int L, bool CP, int FORM>
__device__ __forceinline__ void reinit_one(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int i,
                                                 bool act_, int lane, uint32_t *list, int stride, const TileSrc *ts)
{
    const int b = act_ ? f.inst[i] : 0;
    // the L lanes of a particle share its instance, so this is group-uniform
    const bool act = act_ && bt.ctl[b].reinit;
    const Inst &In = bt.I[b];
    const Grid &g = In.g;
    const Phys &P = In.P;
    const float screen = P.rc2F * 1.0001f;
    ff sF = {0.0f, 0.0f}, sW = {0.0f, 0.0f}, sS = {0.0f, 0.0f};
    if (act) {
        const float4 Pi = f.P4[i], Li = f.L4[i];
        int cx, cy, cz;
        cell_xyz(f.cell_of[i], In, cx, cy, cz);
        auto wall_pair = [&](int q, float ox, float oy, float oz) {
            float d[3];
            const float4 Aq = w.A4[q];
            if (rel_d<D>(Pi, Aq, ox, oy, oz, d) >= screen) return;
            sW = ff_add(sW, W_ff_shape<D>(Pi, Li, Aq, w.L4[q], ox, oy, oz, g, P));
        };
        auto solid_pair = [&](int q, float ox, float oy, float oz) {
            float d[3];
            const float4 Aq = s.A4[q];
            if (rel_d<D>(Pi, Aq, ox, oy, oz, d) >= screen) return;
            sS = ff_add(sS, W_ff_shape<D>(Pi, Li, Aq, s.L4[q], ox, oy, oz, g, P));
        };
        // the screen passes pairs up to 1.0001 (2 h)^2; W_ff_shape returns 0 beyond the support
        fluid_pairs<D, L, CP, FORM>(f, w, s, g, In.c0, cx, cy, cz, i, lane, Pi, screen, list, stride, ts,
                                [&](int j) { return f.L4[j]; },
                                [&](int, const float4 &Pj, const float4 &Lj, const float *, float, float ox, float oy,
                                    float oz) {
                sF = ff_add(sF, W_ff_shape<D>(Pi, Li, Pj, Lj, ox, oy, oz, g, P));
            }, wall_pair, solid_pair);
    }
    const double dF = group_sum_d<L>((double)sF.hi + (double)sF.lo);
    const double dW = group_sum_d<L>((double)sW.hi + (double)sW.lo);
    const double dS = group_sum_d<L>((double)sS.hi + (double)sS.lo);
    if (!act || lane != 0) return;
    double sigma = P.alphaF_d * (1.0 + dF + P.VW_VF_d * dW + P.VS_VF_d * dS);
    double dr = P.rho0_d * ((sigma - P.sigma0_d) / P.sigma0_d);
    if (P.free_surface && dr < 0.0) dr = 0.0;
    float drho = (float)dr;
    f.s[1].drho[i] = drho;
    f.P4[i].w = eos_p(drho, P);
    f.V4[i].w = drho;
}

template <int D, int L, bool CP, bool TILE, int FORM>
__global__ void __launch_bounds__(kMaxBlock) k_reinit(Batch bt, Fluid f, Walls w, Solid s)
{
    pdl_enter();
    if (step_failed(bt)) return;   // the step's cell starts are not valid
    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint32_t *const list = (uint32_t *)s_dyn + threadIdx.x;
    const int stride = blockDim.x;
    if constexpr (!TILE) {
        const int t = blockIdx.x * blockDim.x + threadIdx.x;
        reinit_one<D, L, CP, FORM>(bt, f, w, s, t / L, t / L < f.n, t % L, list, stride, nullptr);
    } else {
        if (!bt.ctl[f.tiles[blockIdx.x].x].reinit) return;   // not a reinitialisation step of this instance
        tile_loop<D, L>(bt, f, f.L4, s_dyn + (CP ? (size_t)kListBytes * blockDim.x : 0),
                        [&](int i, bool act, const TileSrc *ts) {
                            reinit_one<D, L, CP, FORM>(bt, f, w, s, i, act, (int)threadIdx.x % L, list, stride, ts);
                        });
    }
}

int launch_reinit(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int dim, cudaStream_t st)
{
    if (f.n == 0) return 0;
    if (f.n >= kMaxPairTargets) return -7;
    SPH_LAUNCH_PAIRS(k_reinit, f.n, bt, f, w, s);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace sph
