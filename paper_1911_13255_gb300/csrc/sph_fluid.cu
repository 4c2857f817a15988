// Fluid pair loops at h_F (Section 3.1), part 1: momentum (Eq.
// fluid-model-mr-mom) with the low-dissipation Riemann pressure and the
// viscous term, the fluid-solid ghost forces (Eqs. fs-force-mr-sp,
// fs-force-mr-sv with the time-averaged solid state of Eq. fs-coupling-mr),
// their solid-side counterparts (Eqs. F:p, F:v), and the FP64 neighbour-set
// debug kernel.  Shared loop machinery: sph_pairs.cuh.
#include <type_traits>

#include "sph_common.cuh"
#include "sph_pairs.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// a4: equation of state + momentum + kick
// ---------------------------------------------------------------------------
template <int D, int L, bool CP, int FORM>
__device__ __forceinline__ void momentum_one(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int i,
                                                 bool act_, int lane, uint32_t *list, int stride, const TileSrc *ts)
{
    const bool act = act_;
    const int b = act ? f.inst[i] : 0;
    const Inst &In = bt.I[b];
    const Grid &g = In.g;
    const Phys &P = In.P;
    unsigned nff = 0, nfw = 0, nfs = 0;
    float acc[3] = {0.f, 0.f, 0.f}, afs[3] = {0.f, 0.f, 0.f};
    float4 Pi = make_float4(0.f, 0.f, 0.f, 0.f), Vi = Pi;
    if (act) {
        Pi = f.P4[i];
        Vi = f.V4[i];
        const float vi[3] = {Vi.x, Vi.y, Vi.z};
        const float rhoi = P.rho0 + Vi.w, pi = Pi.w;
        int cx, cy, cz;
        cell_xyz(f.cell_of[i], In, cx, cy, cz);
        const float c0 = P.c0, eta2 = 2.0f * P.eta;
        // walls (v~ = a~ = 0) and solid particles at their start-of-step
        // positions with v~, a~
        auto wall_pair = [&](int a, float ox, float oy, float oz) {
            float d[3];
            float r2 = rel_d<D>(Pi, w.A4[a], ox, oy, oz, d);
            if (r2 >= P.rc2F) return;
            nfw++;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            float o[3];
            fs_pair_force<D>(d, r2, vi, rhoi, pi, z4, z4, w.N4[a], P.VW, P, o);
            acc[0] += o[0];
            acc[1] += o[1];
            acc[2] += o[2];
        };
        auto solid_pair = [&](int b, float ox, float oy, float oz) {
            float d[3];
            float r2 = rel_d<D>(Pi, s.A4[b], ox, oy, oz, d);
            if (r2 >= P.rc2F) return;
            nfs++;
            float o[3];
            fs_pair_force<D>(d, r2, vi, rhoi, pi, s.VB4[b], s.AB4[b], s.N4[b], P.VS, P, o);
            afs[0] += o[0];
            afs[1] += o[1];
            afs[2] += o[2];
        };
        // fluid neighbours: Riemann pressure + viscous (Eq. fluid-model-mr-mom, reading R4)
        nff = fluid_pairs<D, L, CP, FORM>(f, w, s, g, In.c0, cx, cy, cz, i, lane, Pi, P.rc2F, list, stride, ts,
                                      [&](int j) { return f.V4[j]; },
                                      [&](int, const float4 &Pj, const float4 &Vj, const float *d, float r2, float,
                                          float, float) {
                // two particles at one FP32 position (a clumped pair): the
                // direction is undefined and the pair's terms vanish with r
                if (r2 == 0.0f) return;
                const float rhoj = P.rho0 + Vj.w;
                // one reciprocal square root for 1/r and r (r2 > 0 here)
                const float invr = rsqrtf(r2), r = r2 * invr;
                float dW = dW_F(r, P);
                // U = v.e with e = -d / r (from i to j)
                float UL = -(vi[0] * d[0] + vi[1] * d[1] + (D == 3 ? vi[2] * d[2] : 0.0f)) * invr;
                float UR = -(Vj.x * d[0] + Vj.y * d[1] + (D == 3 ? Vj.z * d[2] : 0.0f)) * invr;
                float rb = 0.5f * (rhoi + rhoj);
                float beta = fminf(3.0f * fmaxf(UL - UR, 0.0f), c0);
                float Ps = 0.5f * (pi + Pj.w) + 0.5f * rb * beta * (UL - UR);
                float sc = __fdividef(P.mF, rhoj) * dW * invr;   // V_j dW / r
                acc[0] += sc * (-2.0f * Ps * d[0] + eta2 * (vi[0] - Vj.x));
                acc[1] += sc * (-2.0f * Ps * d[1] + eta2 * (vi[1] - Vj.y));
                if (D == 3) acc[2] += sc * (-2.0f * Ps * d[2] + eta2 * (vi[2] - Vj.z));
            }, wall_pair, solid_pair);
    }
    for (int k = 0; k < D; k++) {
        acc[k] = group_sum<L>(acc[k]);
        afs[k] = group_sum<L>(afs[k]);
    }
    Counts cnt = {nff, nfw, nfs, 0u, 0.0f, {0.0, 0.0, 0.0}};
    if (act && lane == 0) {
        const float rhoi = P.rho0 + Vi.w;
        const float vi[3] = {Vi.x, Vi.y, Vi.z};
        float inv_rho = 1.0f / rhoi;
        float a[3], vn[3] = {0.f, 0.f, 0.f};
        double dt = bt.ctl[b].dt;
        for (int k = 0; k < D; k++) {
            a[k] = (acc[k] + afs[k]) * inv_rho + P.g[k];
            vn[k] = vi[k] + (float)dt * a[k];
            f.dvdt[(size_t)i * D + k] = a[k];
        }
        f.W4[i] = make_float4(vn[0], vn[1], vn[2], Vi.w);
        cnt.vmax = sqrtf(vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]);
        float Vi_ = P.mF / rhoi;   // force = V_i * afs (same V_i as the solid side)
        for (int k = 0; k < D; k++) cnt.mom[k] = (double)(Vi_ * afs[k]);
    }
    flush_counts<D>(bt, b, act, cnt, true);
}

template <int D, int L, bool CP, bool TILE, int FORM>
__global__ void __launch_bounds__(kMaxBlock) k_momentum(Batch bt, Fluid f, Walls w, Solid s)
{
    pdl_enter();
    if (step_failed(bt)) return;   // the step's cell starts are not valid
    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint32_t *const list = (uint32_t *)s_dyn + threadIdx.x;
    const int stride = blockDim.x;
    if constexpr (!TILE) {
        const int t = blockIdx.x * blockDim.x + threadIdx.x;
        momentum_one<D, L, CP, FORM>(bt, f, w, s, t / L, t / L < f.n, t % L, list, stride, nullptr);
    } else {
        tile_loop<D, L>(bt, f, f.V4, s_dyn + (CP ? (size_t)kListBytes * blockDim.x : 0),
                        [&](int i, bool act, const TileSrc *ts) {
                            momentum_one<D, L, CP, FORM>(bt, f, w, s, i, act, (int)threadIdx.x % L, list, stride, ts);
                        });
    }
}

int launch_momentum(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int dim, cudaStream_t st)
{
    if (f.n == 0) return 0;
    if (f.n >= kMaxPairTargets) return -7;
    SPH_LAUNCH_PAIRS(k_momentum, f.n, bt, f, w, s);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// a2 (neighbour rows): each fluid target's in-support fluid neighbours (from
// the front of its row) and in-support wall neighbours (from the back),
// over the 3^(d-1) rows of three cells around its cell (a row's cells are
// consecutive in the cell-sorted records, so its candidates are one flat
// range), with the pair loops' own FP32 test on the records, and whether a
// neighbour cell holds solid particles.  L lanes per target test 2 L
// candidates a round (both loads issued first); the in-support ones get their
// places by ballots over the L lanes, so a row lists its entries in the
// candidate order whatever L is.  Entries that do not fit are dropped and the
// row is marked overflowed (its target then takes the cell form; every
// write stays inside the row).  Runs on rebuild steps.
// ---------------------------------------------------------------------------
template <int D, int L>
__global__ void __launch_bounds__(kMaxBlock) k_pairlist(Batch bt, Fluid f, Walls w, Solid s)
{
    pdl_enter();
    if (step_failed(bt)) return;   // the step's cell starts are not valid
    if (!rebuild_step(bt, f)) return;   // held configuration: the rows stay
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / L, lane = t % L;
    if (i >= f.n) return;   // the L lanes of a target leave together
    const int wl = threadIdx.x & 31;
    const unsigned gmask = L == 32 ? 0xffffffffu : ((1u << L) - 1u) << (wl & ~(L - 1));
    const unsigned below = (1u << wl) - 1u;
    const Inst &In = bt.I[f.inst[i]];
    const Grid &g = In.g;
    const float rc2 = In.P.rc2F;
    const float4 Pi = f.P4[i];
    int cx, cy, cz;
    cell_xyz(f.cell_of[i], In, cx, cy, cz);
    uint32_t *row = f.nbl + (size_t)i * f.list_cap;
    const int cap = f.list_cap;
    int nF = 0, nW = 0;
    bool solid = false;
    // every loop bound below is the same for the L lanes of the target
    for_each_row<D>(g, In.c0, cx, cy, cz, [&](const int c[3], float oy, float oz, int code0) {
        const Row3 rf = row_of(f.cstart, c);
        const Row3 rw = row_of(w.cstart, c);
        if (s.n) solid = solid || row_of(s.cstart, c).n > 0;
        for (int qb = 0; qb < rf.n; qb += 2 * L) {
            const int q0 = qb + lane, q1 = q0 + L;
            int k0 = 0, k1 = 0;
            const int j0 = q0 < rf.n ? row_slot(rf, q0, k0) : -1;
            const int j1 = q1 < rf.n ? row_slot(rf, q1, k1) : -1;
            const float4 P0 = j0 >= 0 ? f.P4[j0] : Pi;
            const float4 P1 = j1 >= 0 ? f.P4[j1] : Pi;
            float d[3];
            const bool in0 = j0 >= 0 && j0 != i && rel_d<D>(Pi, P0, row_ox(k0, g), oy, oz, d) < rc2;
            const bool in1 = j1 >= 0 && j1 != i && rel_d<D>(Pi, P1, row_ox(k1, g), oy, oz, d) < rc2;
            const unsigned m0 = __ballot_sync(gmask, in0) & gmask;
            const unsigned m1 = __ballot_sync(gmask, in1) & gmask;
            const int n0 = __popc(m0);
            if (in0) {
                const int q = nF + __popc(m0 & below);
                if (q < cap) row[q] = ((uint32_t)j0 << kCodeBits) | row_code(code0 + k0);
            }
            if (in1) {
                const int q = nF + n0 + __popc(m1 & below);
                if (q < cap) row[q] = ((uint32_t)j1 << kCodeBits) | row_code(code0 + k1);
            }
            nF += n0 + __popc(m1);
        }
        for (int qb = 0; qb < rw.n; qb += L) {
            const int q0 = qb + lane;
            int k0 = 0;
            const int a = q0 < rw.n ? row_slot(rw, q0, k0) : -1;
            float d[3];
            const bool in = a >= 0 && rel_d<D>(Pi, w.A4[a], row_ox(k0, g), oy, oz, d) < rc2;
            const unsigned m = __ballot_sync(gmask, in) & gmask;
            if (in) {
                const int q = cap - 1 - (nW + __popc(m & below));
                if (q >= 0) row[q] = ((uint32_t)a << kCodeBits) | row_code(code0 + k0);
            }
            nW += __popc(m);
        }
    });
    if (lane == 0)
        f.nbc[i] = (nF + nW > cap || nF > (int)kListCountMask || nW > (int)kListCountMask)
                       ? kListOver
                       : ((uint32_t)nF | ((uint32_t)nW << 11) | (solid ? kListSolid : 0u));
}

// The same rows built per cell, one lane per particle of the cell: each lane
// appends to its own row, so the entries come in the same order as above
// (fluid by cell, then slot, from the front; walls likewise from the back).
// The rows of the targets [t0, t1) of one non-empty cell, G lanes of a
// group per round (this thread is lane `lane` of its group): every
// candidate of the 3^d neighbour cells is loaded once for the group and each
// lane tests its own target against it.  No warp-wide operation, so the two
// half-warps of a warp may run two cells side by side.
template <int D>
__device__ __forceinline__ void cell_rows(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int cell,
                                          int t0, int t1, int lane, int G)
{
    const Inst &In = bt.I[f.inst[t0]];
    const Grid &g = In.g;
    const float rc2 = In.P.rc2F;
    const int cap = f.list_cap;
    int cx, cy, cz;
    cell_xyz(cell, In, cx, cy, cz);
    for (int tb = t0; tb < t1; tb += G) {
        const int i = tb + lane;
        const bool act = i < t1;
        const float4 Pi = f.P4[act ? i : t0];
        uint32_t *row = f.nbl + (size_t)(act ? i : t0) * cap;
        int nF = 0, nW = 0;
        bool solid = false;
        for_each_cell<D, 1>(g, In.c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int code) {
            const uint32_t rc = row_code(code);
            const int j1 = f.cstart[c + 1];
#pragma unroll 4
            for (int j = f.cstart[c]; j < j1; j++) {
                float d[3];
                const bool in = rel_d<D>(Pi, f.P4[j], ox, oy, oz, d) < rc2 && j != i && act;
                if (in) {
                    if (nF < cap) row[nF] = ((uint32_t)j << kCodeBits) | rc;
                    nF++;
                }
            }
            const int a1 = w.cstart[c + 1];
            for (int a = w.cstart[c]; a < a1; a++) {
                float d[3];
                const bool in = rel_d<D>(Pi, w.A4[a], ox, oy, oz, d) < rc2 && act;
                if (in) {
                    if (nW < cap) row[cap - 1 - nW] = ((uint32_t)a << kCodeBits) | rc;
                    nW++;
                }
            }
            if (s.n && s.cstart[c + 1] > s.cstart[c]) solid = true;
        });
        if (act)
            f.nbc[i] = (nF + nW > cap || nF > (int)kListCountMask || nW > (int)kListCountMask)
                           ? kListOver
                           : ((uint32_t)nF | ((uint32_t)nW << 11) | (solid ? kListSolid : 0u));
    }
}

// One warp per two consecutive cells.  When they hold at most 32 targets
// together, one round builds both: the first cell's targets take the first
// lanes, the second cell's the next ones (in the 3-D duct, cells of 8, 12
// and 18 particles come in rows where such pairs are common, and the two
// groups then walk neighbour cells of nearly equal size); otherwise the
// whole warp builds one cell after the other.  Either way each target's row
// is built by one lane in candidate order, so the rows do not depend on the
// grouping.
// 16 resident blocks per SM (32 registers a thread): the build is issue- and
// load-latency bound, and the extra warps outweigh a few spilled registers
// (3-D duct: 2.37 -> 2.32 ms; 56-register pair loops, by contrast, ran
// slower than at 64).
template <int D>
__global__ void __launch_bounds__(128, 16) k_pairlist_cells(Batch bt, Fluid f, Walls w, Solid s)
{
    pdl_enter();
    if (step_failed(bt)) return;   // the step's cell starts are not valid
    if (!rebuild_step(bt, f)) return;
    const int c0 = 2 * (blockIdx.x * 4 + (int)(threadIdx.x >> 5)), lane = threadIdx.x & 31;
    if (c0 >= bt.ncell) return;
    const bool two = c0 + 1 < bt.ncell;
    const int a0 = f.cstart[c0], a1 = f.cstart[c0 + 1];   // the second cell starts where the first ends
    const int b1 = two ? f.cstart[c0 + 2] : a1;
    const int na = a1 - a0;
    if (b1 - a0 <= 32) {
        const bool second = lane >= na;
        const int t0 = second ? a1 : a0, t1 = second ? b1 : a1, ll = second ? lane - na : lane;
        if (ll < t1 - t0) cell_rows<D>(bt, f, w, s, second ? c0 + 1 : c0, t0, t1, ll, 32);
    } else {
        if (a0 < a1) cell_rows<D>(bt, f, w, s, c0, a0, a1, lane, 32);
        if (a1 < b1) cell_rows<D>(bt, f, w, s, c0 + 1, a1, b1, lane, 32);
    }
}

int launch_pairlist(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int dim, cudaStream_t st)
{
    if (f.n == 0 || !f.list) return 0;
    if (f.n >= kMaxPairTargets || w.n >= kMaxPairTargets) return -7;
    // its own lane count: wide groups load a row's consecutive candidates together
    auto go = [&](auto Dc, auto Lc) {
        constexpr int D_ = decltype(Dc)::value, L_ = decltype(Lc)::value;
        launch_k(k_pairlist<D_, L_>, grid_blocks(f.n, L_, 128), 128, 0, st, bt, f, w, s);
    };
    auto by_lanes = [&](auto Dc) {
        constexpr int D_ = decltype(Dc)::value;
        if (f.list_lanes == 1) launch_k(k_pairlist_cells<D_>, (bt.ncell + 7) / 8, 128, 0, st, bt, f, w, s);
        else if (f.list_lanes == 8) go(Dc, std::integral_constant<int, 8>{});
        else if (f.list_lanes == 16) go(Dc, std::integral_constant<int, 16>{});
        else if (f.list_lanes == 32) go(Dc, std::integral_constant<int, 32>{});
        else return false;
        return true;
    };
    const bool ok = dim == 2 ? by_lanes(std::integral_constant<int, 2>{}) : by_lanes(std::integral_constant<int, 3>{});
    if (!ok) return -1;
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// a5: fluid force on each solid particle, f_a^F = -sum_i V_i (pair term),
// the same pair expression and inputs as a4 (fluid at r^{n+1/2}, v^n)
// ---------------------------------------------------------------------------
template <int D, int L>
__global__ void __launch_bounds__(kMaxBlock, 2) k_solid_fluid_force(Batch bt, Fluid f, Solid s)
{
    pdl_enter();
    if (step_failed(bt)) return;   // the step's cell starts are not valid
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = t / L, lane = t % L;
    const bool act = k < s.n;
    unsigned nsf = 0;
    float fa[3] = {0.f, 0.f, 0.f};
    const int a = act ? __float_as_int(s.N4[k].w) : 0;
    const int b = act ? s.inst[a] : 0;
    const Inst &In = bt.I[b];
    const Grid &g = In.g;
    const Phys &P = In.P;
    if (act) {
        const float4 A = s.A4[k], VB = s.VB4[k], AB = s.AB4[k], N = s.N4[k];
        int cx, cy, cz;
        cell_xyz(s.cell_of[k], In, cx, cy, cz);
        auto pair = [&](int j, float ox, float oy, float oz) {
            const float4 Pj = f.P4[j];
            // the fluid side sees this pair with the opposite cell offset
            float d[3] = {(Pj.x - A.x) - ox, (Pj.y - A.y) - oy, D == 3 ? (Pj.z - A.z) - oz : 0.0f};
            float r2 = d[0] * d[0] + d[1] * d[1] + (D == 3 ? d[2] * d[2] : 0.0f);
            if (r2 >= P.rc2F) return;
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
        };
        if (f.reach == 1) {
            // a row of neighbour cells at a time (their starts loaded together)
            for_each_row<D>(g, In.c0, cx, cy, cz, [&](const int c[3], float oy, float oz, int) {
                const Row3 r = row_of(f.cstart, c);
                for (int q = lane; q < r.n; q += L) {
                    int k;
                    const int j = row_slot(r, q, k);
                    pair(j, row_ox(k, g), oy, oz);
                }
            });
        } else {
            for_each_cell<D, 2>(g, In.c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int) {
                const int j1 = f.cstart[c + 1];
                for (int j = f.cstart[c] + lane; j < j1; j += L) pair(j, ox, oy, oz);
            });
        }
    }
    for (int q = 0; q < D; q++) fa[q] = group_sum<L>(fa[q]);
    Counts cnt = {0u, 0u, 0u, nsf, 0.0f, {0.0, 0.0, 0.0}};
    if (act && lane == 0) {
        for (int q = 0; q < 3; q++) s.fF[3 * a + q] = q < D ? fa[q] : 0.0f;
        for (int q = 0; q < D; q++) cnt.mom[q] = (double)fa[q];
    }
    flush_counts<D>(bt, b, act, cnt, false);
}

// lanes per solid particle of this loop, its own choice: 16 for small
// bodies, whose few particles then spread over more SMs (measured: 2-D dam
// break 12.8 -> 11.1 us), 4 for large ones (batches), where 16 doubles the
// loop's time
constexpr int kSfBlock = 128, kSfSmall = 32768;

int launch_solid_fluid_force(const Batch &bt, const Fluid &f, const Solid &s, int dim, cudaStream_t st)
{
    if (s.n == 0 || f.n == 0) {
        if (s.n) cudaMemsetAsync(s.fF, 0, sizeof(float) * 3 * s.n, st);
        return cudaGetLastError() == cudaSuccess ? 0 : -3;
    }
    const bool small = s.n < kSfSmall;
    if (dim == 2) {
        if (small) launch_k(k_solid_fluid_force<2, 16>, grid_blocks(s.n, 16, kSfBlock), kSfBlock, 0, st, bt, f, s);
        else launch_k(k_solid_fluid_force<2, 4>, grid_blocks(s.n, 4, kSfBlock), kSfBlock, 0, st, bt, f, s);
    } else {
        if (small) launch_k(k_solid_fluid_force<3, 16>, grid_blocks(s.n, 16, kSfBlock), kSfBlock, 0, st, bt, f, s);
        else launch_k(k_solid_fluid_force<3, 4>, grid_blocks(s.n, 4, kSfBlock), kSfBlock, 0, st, bt, f, s);
    }
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
__global__ void k_debug_pairs(Batch bt, Fluid f, Walls w, Solid s, int inst, int which, int *counts,
                              const int *offs, int *out)
{
    const Inst &In = bt.I[inst];
    const Grid &g = In.g;
    const Phys &P = In.P;
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    int nrows = which == 3 ? In.ns : In.nf;
    if (r >= nrows) return;
    double xi, yi, zi;
    int row, key;
    const FluidState M = f.s[1];
    const int k = (which == 3 ? In.s0 : In.f0) + r;   // sorted slot
    if (which == 3) {
        int a = __float_as_int(s.N4[k].w);   // solid particle of sorted slot k
        xi = s.x[a];
        yi = s.y[a];
        zi = D == 3 ? s.z[a] : 0.0;
        row = a - In.s0;
        key = s.cell_of[k];
    } else {
        xi = M.x[k];
        yi = M.y[k];
        zi = D == 3 ? M.z[k] : 0.0;
        row = M.id[k];
        key = f.cell_of[k];
    }
    int cx, cy, cz;
    cell_xyz(key, In, cx, cy, cz);
    int cnt = 0;
    int base = out ? offs[row] : 0;
    auto visit = [&](int c, float, float, float, int) {
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
                col = a - In.w0;
            } else {
                int a = __float_as_int(s.N4[j].w);
                xj = s.x[a];
                yj = s.y[a];
                zj = D == 3 ? s.z[a] : 0.0;
                col = a - In.s0;
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
    };
    if (f.reach == 2) for_each_cell<D, 2>(g, In.c0, cx, cy, cz, visit);
    else for_each_cell<D, 1>(g, In.c0, cx, cy, cz, visit);
    if (!out) counts[row] = cnt;
}

int launch_debug_pairs(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int dim, int inst,
                       int which, int *counts, int *offs, int *out, cudaStream_t st)
{
    int nrows = which == 3 ? s.n : f.n;   // upper bound of the instance's rows
    if (nrows == 0) return 0;
    int nb = (nrows + kBlock - 1) / kBlock;
    if (dim == 2) k_debug_pairs<2><<<nb, kBlock, 0, st>>>(bt, f, w, s, inst, which, counts, offs, out);
    else k_debug_pairs<3><<<nb, kBlock, 0, st>>>(bt, f, w, s, inst, which, counts, offs, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace sph
