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
#include <type_traits>

#include "sph_common.cuh"

namespace sph {

// Lanes per target particle: a runtime choice (Fluid::lanes, set by the
// autotuner) among compiled instances, 2/4/8 in 2-D and 4/8/16 in 3-D.
template <int D, typename Fn>
static bool with_lanes(int L, Fn &&fn)
{
    if constexpr (D == 2) {
        if (L == 2) fn(std::integral_constant<int, 2>{});
        else if (L == 4) fn(std::integral_constant<int, 4>{});
        else if (L == 8) fn(std::integral_constant<int, 8>{});
        else return false;
    } else {
        if (L == 4) fn(std::integral_constant<int, 4>{});
        else if (L == 8) fn(std::integral_constant<int, 8>{});
        else if (L == 16) fn(std::integral_constant<int, 16>{});
        else return false;
    }
    return true;
}

// Visit the 3^d neighbour cells of (cx, cy, cz).  fn(cell, ox, oy, oz, code)
// receives the offset o = -(dcell) * edge to add to (rel_i - rel_j) and
// code = (dx + 1) + 3 (dy + 1) + 9 (dz + 1) (cell_offset recovers o from it).
template <int D, typename Fn>
__device__ __forceinline__ void for_each_cell(const Grid &g, int c0, int cx, int cy, int cz, Fn &&fn)
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
                int c = c0 + x + g.nc[0] * (y + g.nc[1] * z);
                fn(c, -(float)dx * g.csf[0], -(float)dy * g.csf[1], -(float)dz * g.csf[2],
                   (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1));
            }
        }
    }
}

__device__ __forceinline__ void cell_offset(int code, const Grid &g, float &ox, float &oy, float &oz)
{
    const int dx = code % 3 - 1, dy = (code / 3) % 3 - 1, dz = code / 9 - 1;
    ox = -(float)dx * g.csf[0];
    oy = -(float)dy * g.csf[1];
    oz = -(float)dz * g.csf[2];
}

template <int D>
__device__ __forceinline__ float rel_d(const float4 &Pi, const float4 &Pj, float ox, float oy, float oz, float d[3])
{
    d[0] = (Pi.x - Pj.x) + ox;
    d[1] = (Pi.y - Pj.y) + oy;
    d[2] = D == 3 ? (Pi.z - Pj.z) + oz : 0.0f;
    return d[0] * d[0] + d[1] * d[1] + (D == 3 ? d[2] * d[2] : 0.0f);
}

// ---------------------------------------------------------------------------
// Tiles: a block owns T consecutive cells of one grid row (an instance's
// cells [c_first, c_first + ntc)).  Every fluid neighbour of its targets lies
// in the 3^(d-1) rows around it, x from the first cell - 1 to the last + 1;
// these row pieces are contiguous in the cell-sorted records, so the block
// stages them into shared memory with bulk copies (cp.async.bulk, completion
// on an mbarrier) and its targets read their fluid neighbours from there.  A
// row that wraps in a periodic x splits into two pieces.
// ---------------------------------------------------------------------------
struct TilePiece {
    int c_lo, c_hi;   // global cells [c_lo, c_hi]; empty when c_lo > c_hi
    int base;         // shared-memory slot of record j of these cells = j + base
};

struct TileSrc {
    const float4 *sP, *sX;      // staged P4 and second records
    const TilePiece *pieces;    // 2 per row, rows (dy + 1) + 3 (dz + 1)
};

constexpr int kTileRows = 9;

__device__ __forceinline__ bool bulk_wait(uint32_t mbar)
{
    for (long long k = 0; k < (1ll << 26); k++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(mbar)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Stage the tile's neighbourhood: P4 into sP, X4 into sX (at most cap
// records each).  Returns the number staged, or -1 when they do not fit (the
// block then reads its neighbours from global memory) or a wait ran out.
template <int D>
__device__ int tile_stage(const Batch &bt, const Fluid &f, const float4 *X4, int4 tile, TilePiece *pieces,
                          float4 *sP, float4 *sX, int cap, uint64_t *mbar, int *s_total)
{
    const Inst &In = bt.I[tile.x];
    const Grid &g = In.g;
    const int c_first = tile.y, ntc = tile.z;
    const int key = c_first - In.c0;
    const int cx0 = key % g.nc[0], cy = (key / g.nc[0]) % g.nc[1], cz = D == 3 ? key / (g.nc[0] * g.nc[1]) : 0;
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
    if (threadIdx.x == 0) {
        int off = 0;
        for (int r = 0; r < kTileRows; r++) {
            const int dy = r % 3 - 1, dz = r / 3 - 1;
            TilePiece *pp = pieces + 2 * r;
            pp[0] = pp[1] = TilePiece{1, 0, 0};
            const int y = cy + dy, z = cz + dz;
            if ((D == 2 && dz != 0) || y < 0 || y >= g.nc[1] || z < 0 || z >= g.nc[2]) continue;
            const int row0 = In.c0 + g.nc[0] * (y + g.nc[1] * z);
            int lo = cx0 - 1, hi = cx0 + ntc;
            int a0 = 0, a1 = -1, b0 = 0, b1 = -1;   // local x ranges of the two pieces
            if (!g.periodic_x) {
                a0 = lo < 0 ? 0 : lo;
                a1 = hi >= g.nc[0] ? g.nc[0] - 1 : hi;
            } else if (ntc + 2 >= g.nc[0]) {
                a0 = 0;
                a1 = g.nc[0] - 1;
            } else if (lo < 0) {
                a0 = a1 = g.nc[0] - 1;
                b0 = 0;
                b1 = hi;
            } else if (hi >= g.nc[0]) {
                a0 = lo;
                a1 = g.nc[0] - 1;
                b0 = 0;
                b1 = hi - g.nc[0];
            } else {
                a0 = lo;
                a1 = hi;
            }
            if (a1 >= a0) {
                const int p0 = f.cstart[row0 + a0];
                pp[0] = TilePiece{row0 + a0, row0 + a1, off - p0};
                off += f.cstart[row0 + a1 + 1] - p0;
            }
            if (b1 >= b0) {
                const int p0 = f.cstart[row0 + b0];
                pp[1] = TilePiece{row0 + b0, row0 + b1, off - p0};
                off += f.cstart[row0 + b1 + 1] - p0;
            }
        }
        *s_total = off <= cap ? off : -1;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int total = *s_total;
    if (total < 0) return -1;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(total * 32)
                     : "memory");
        for (int q = 0; q < 2 * kTileRows; q++) {
            const TilePiece pc = pieces[q];
            if (pc.c_lo > pc.c_hi) continue;
            const int p0 = f.cstart[pc.c_lo], n = f.cstart[pc.c_hi + 1] - p0;
            if (n == 0) continue;
            const int o = p0 + pc.base;
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(sP + o)),
                         "l"(f.P4 + p0), "r"(n * 16), "r"(mb)
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(sX + o)),
                         "l"(X4 + p0), "r"(n * 16), "r"(mb)
                         : "memory");
        }
    }
    const bool ok = __syncthreads_and(bulk_wait(mb));
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(&bt.ctl[tile.x].status, ST_TIMEOUT);
        return -1;
    }
    return total;
}

// Run body(i, act, ts) for every target of the block's tile, L lanes per
// target, the same number of rounds in every thread (act = false past the
// end); ts is null when the neighbourhood did not fit in shared memory.
template <int D, int L, typename Body>
__device__ __forceinline__ void tile_loop(const Batch &bt, const Fluid &f, const float4 *X4, uint8_t *stage, Body &&body)
{
    __shared__ TilePiece s_pieces[2 * kTileRows];
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ int s_total;
    const int4 tile = f.tiles[blockIdx.x];
    float4 *sP = (float4 *)stage, *sX = sP + f.tile_cap;
    const int staged = tile_stage<D>(bt, f, X4, tile, s_pieces, sP, sX, f.tile_cap, &s_mbar, &s_total);
    const TileSrc src{sP, sX, s_pieces};
    const TileSrc *ts = staged >= 0 ? &src : nullptr;
    const int tp0 = f.cstart[tile.y], tp1 = f.cstart[tile.y + tile.z];
    const int per = blockDim.x / L;
    const int rounds = (tp1 - tp0 + per - 1) / per;
    for (int k = 0; k < rounds; k++) {
        const int i = tp0 + k * per + (int)threadIdx.x / L;
        body(i, i < tp1, ts);
    }
}

// Fluid-fluid pairs of target i (this lane's share of the candidates), in
// one of two forms chosen by the launch shape (Fluid::compact):
//
// direct (CP = false): pair(j, Pj, Xj, d, r2, ox, oy, oz) is evaluated inside
// the candidate loop, Xj = fetch(j) being the neighbour's second record.
//
// compacted (CP = true): the candidate test passes only 1/3 (2-D) to 1/6
// (3-D) of the candidates, so evaluating inside the loop runs the pair
// arithmetic in almost every warp iteration with few lanes active.  Each
// thread first writes its in-support neighbours (j << 5 | cell-offset code)
// into its own list in shared memory (slot k at list[k * stride]), then
// evaluates the list with all lanes busy; a full list is drained early.
// Requires j < 2^27.
//
// Both return the number of in-support pairs and visit the pairs of a
// target in the same order.
constexpr int kPairCap = 32;

template <int D, int L, bool CP, typename Fetch, typename Pair>
__device__ __forceinline__ unsigned fluid_pairs_global(const Fluid &f, const Grid &g, int c0, int cx, int cy, int cz,
                                                       int i, int lane, const float4 &Pi, float rc2, uint32_t *list,
                                                       int stride, Fetch &&fetch, Pair &&pair)
{
    unsigned cnt_total = 0;
    if constexpr (!CP) {
        for_each_cell<D>(g, c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int) {
            const int j1 = f.cstart[c + 1];
            for (int j = f.cstart[c] + lane; j < j1; j += L) {
                if (j == i) continue;
                const float4 Pj = f.P4[j];
                float d[3];
                const float r2 = rel_d<D>(Pi, Pj, ox, oy, oz, d);
                if (r2 >= rc2) continue;
                cnt_total++;
                pair(j, Pj, fetch(j), d, r2, ox, oy, oz);
            }
        });
        return cnt_total;
    } else {
        int cnt = 0;
        auto drain = [&]() {
#pragma unroll 1
            for (int k = 0; k < cnt; k++) {
                const uint32_t e = list[k * stride];
                const int j = (int)(e >> 5);
                float ox, oy, oz;
                cell_offset((int)(e & 31u), g, ox, oy, oz);
                const float4 Pj = f.P4[j];
                float d[3];
                const float r2 = rel_d<D>(Pi, Pj, ox, oy, oz, d);
                pair(j, Pj, fetch(j), d, r2, ox, oy, oz);
            }
            cnt = 0;
        };
        for_each_cell<D>(g, c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int code) {
            const int j1 = f.cstart[c + 1];
            for (int j = f.cstart[c] + lane; j < j1; j += L) {
                if (j == i) continue;
                float d[3];
                if (rel_d<D>(Pi, f.P4[j], ox, oy, oz, d) >= rc2) continue;
                list[cnt * stride] = ((uint32_t)j << 5) | (uint32_t)code;
                cnt++;
                cnt_total++;
                if (cnt == kPairCap) drain();
            }
        });
        drain();
        return cnt_total;
    }
}

// The same over staged records: record j of neighbour cell c sits at slot
// j + base(c) of the staged arrays; list entries hold slots.
template <int D, int L, bool CP, typename Pair>
__device__ __forceinline__ unsigned fluid_pairs_tile(const Fluid &f, const Grid &g, int c0, int cx, int cy, int cz,
                                                     int i, int lane, const float4 &Pi, float rc2, uint32_t *list,
                                                     int stride, const TileSrc &ts, Pair &&pair)
{
    unsigned cnt_total = 0;
    int cnt = 0;
    auto drain = [&]() {
#pragma unroll 1
        for (int k = 0; k < cnt; k++) {
            const uint32_t e = list[k * stride];
            const int q = (int)(e >> 5);
            float ox, oy, oz;
            cell_offset((int)(e & 31u), g, ox, oy, oz);
            const float4 Pj = ts.sP[q];
            float d[3];
            const float r2 = rel_d<D>(Pi, Pj, ox, oy, oz, d);
            pair(q, Pj, ts.sX[q], d, r2, ox, oy, oz);
        }
        cnt = 0;
    };
    for_each_cell<D>(g, c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int code) {
        const TilePiece *pp = ts.pieces + 2 * ((code / 3) % 3 + 3 * (code / 9));
        const int base = (c >= pp[0].c_lo && c <= pp[0].c_hi) ? pp[0].base : pp[1].base;
        const int j1 = f.cstart[c + 1];
        for (int j = f.cstart[c] + lane; j < j1; j += L) {
            if (j == i) continue;
            const int q = j + base;
            const float4 Pj = ts.sP[q];
            float d[3];
            const float r2 = rel_d<D>(Pi, Pj, ox, oy, oz, d);
            if (r2 >= rc2) continue;
            cnt_total++;
            if constexpr (CP) {
                list[cnt * stride] = ((uint32_t)q << 5) | (uint32_t)code;
                cnt++;
                if (cnt == kPairCap) drain();
            } else {
                pair(q, Pj, ts.sX[q], d, r2, ox, oy, oz);
            }
        }
    });
    if constexpr (CP) drain();
    return cnt_total;
}

template <int D, int L, bool CP, typename Fetch, typename Pair>
__device__ __forceinline__ unsigned fluid_pairs(const Fluid &f, const Grid &g, int c0, int cx, int cy, int cz, int i,
                                                int lane, const float4 &Pi, float rc2, uint32_t *list, int stride,
                                                const TileSrc *ts, Fetch &&fetch, Pair &&pair)
{
    if (ts) return fluid_pairs_tile<D, L, CP>(f, g, c0, cx, cy, cz, i, lane, Pi, rc2, list, stride, *ts, pair);
    return fluid_pairs_global<D, L, CP>(f, g, c0, cx, cy, cz, i, lane, Pi, rc2, list, stride, fetch, pair);
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

// local cell coordinates of a global cell index
__device__ __forceinline__ void cell_xyz(int gkey, const Inst &In, int &cx, int &cy, int &cz)
{
    const Grid &g = In.g;
    const int key = gkey - In.c0;
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


// Add per-thread counters to the thread's instance control block: one
// atomic per warp when the warp's lanes share an instance, else per lane.
struct Counts {
    unsigned ff, fw, fs, sf;
    float vmax;
    double mom[3];
};

template <int D>
__device__ __forceinline__ void flush_counts(Batch bt, int b, bool valid, Counts c, bool fluid_side)
{
    if (warp_uniform(valid ? b : -1)) {
        unsigned ff = warp_sum_u(c.ff), fw = warp_sum_u(c.fw), fs = warp_sum_u(c.fs), sf = warp_sum_u(c.sf);
        float vm = warp_max(c.vmax);
        double m[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < D; k++) m[k] = warp_sum_d(c.mom[k]);
        if ((threadIdx.x & 31) == 0 && valid) {
            Ctl *ctl = bt.ctl + b;
            if (ff) atomicAdd(&ctl->n_ff, (unsigned long long)ff);
            if (fw) atomicAdd(&ctl->n_fw, (unsigned long long)fw);
            if (fs) atomicAdd(&ctl->n_fs, (unsigned long long)fs);
            if (sf) atomicAdd(&ctl->n_sf, (unsigned long long)sf);
            if (fluid_side) {
                if (fs)
                    for (int k = 0; k < D; k++) atomicAdd(&ctl->mom_fluid[k], m[k]);
                atomic_max_pos(&ctl->vmaxF, vm);
            } else if (sf) {
                for (int k = 0; k < D; k++) atomicAdd(&ctl->mom_solid[k], m[k]);
            }
        }
    } else if (valid) {
        Ctl *ctl = bt.ctl + b;
        if (c.ff) atomicAdd(&ctl->n_ff, (unsigned long long)c.ff);
        if (c.fw) atomicAdd(&ctl->n_fw, (unsigned long long)c.fw);
        if (c.fs) atomicAdd(&ctl->n_fs, (unsigned long long)c.fs);
        if (c.sf) atomicAdd(&ctl->n_sf, (unsigned long long)c.sf);
        if (fluid_side) {
            for (int k = 0; k < D; k++)
                if (c.mom[k] != 0.0) atomicAdd(&ctl->mom_fluid[k], c.mom[k]);
            atomic_max_pos(&ctl->vmaxF, c.vmax);
        } else {
            for (int k = 0; k < D; k++)
                if (c.mom[k] != 0.0) atomicAdd(&ctl->mom_solid[k], c.mom[k]);
        }
    }
}

static inline int grid_blocks(int n, int L, int block)
{
    long long t = (long long)n * L;
    return (int)((t + block - 1) / block);
}

// launch KERN<dim, L> over n targets with the lane count and block size of f
// and SMEM bytes of dynamic shared memory per thread
#define SPH_LAUNCH_LANES(KERN, n, SMEM, ...)                                                  \
    do {                                                                                      \
        const size_t sm_ = (size_t)(SMEM) * f.block;                                         \
        const bool ok_ = dim == 2 ? with_lanes<2>(f.lanes, [&](auto Lc) {                     \
            constexpr int L_ = decltype(Lc)::value;                                           \
            KERN<2, L_><<<grid_blocks(n, L_, f.block), f.block, sm_, st>>>(__VA_ARGS__);      \
        })                                                                                    \
                                  : with_lanes<3>(f.lanes, [&](auto Lc) {                     \
            constexpr int L_ = decltype(Lc)::value;                                           \
            KERN<3, L_><<<grid_blocks(n, L_, f.block), f.block, sm_, st>>>(__VA_ARGS__);      \
        });                                                                                   \
        if (!ok_ || f.block < 32 || f.block > kMaxBlock || f.block % 32) return -1;           \
    } while (0)

constexpr int kListBytes = kPairCap * 4;   // per-thread in-support list (fluid_pairs)

// the same for the pair-loop kernels templated on the pair form (f.compact)
// and on tiles (f.tile: one block per tile, the staging area after the lists)
template <typename K>
static void allow_smem(K kern, size_t bytes)
{
    // dynamic plus static shared memory above the default 48 KB needs the opt-in
    if (bytes > 32 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define SPH_LAUNCH_PAIRS(KERN, n, ...)                                                        \
    do {                                                                                      \
        const size_t sm_ = (f.compact ? (size_t)kListBytes * f.block : 0) +                  \
                           (f.tile ? (size_t)f.tile_cap * 32 : 0);                            \
        auto go_ = [&](auto Dc, auto Lc) {                                                    \
            constexpr int D_ = decltype(Dc)::value, L_ = decltype(Lc)::value;                \
            const int nb_ = f.tile ? f.ntiles : grid_blocks(n, L_, f.block);                  \
            if (nb_ == 0) return;                                                             \
            auto run_ = [&](auto kern) {                                                      \
                allow_smem(kern, sm_);                                                        \
                kern<<<nb_, f.block, sm_, st>>>(__VA_ARGS__);                                 \
            };                                                                                \
            if (f.compact && f.tile) run_(KERN<D_, L_, true, true>);                          \
            else if (f.compact) run_(KERN<D_, L_, true, false>);                              \
            else if (f.tile) run_(KERN<D_, L_, false, true>);                                 \
            else run_(KERN<D_, L_, false, false>);                                            \
        };                                                                                    \
        const bool ok_ = dim == 2 ? with_lanes<2>(f.lanes, [&](auto Lc) {                     \
            go_(std::integral_constant<int, 2>{}, Lc);                                        \
        })                                                                                    \
                                  : with_lanes<3>(f.lanes, [&](auto Lc) {                     \
            go_(std::integral_constant<int, 3>{}, Lc);                                        \
        });                                                                                   \
        if (!ok_ || f.block < 32 || f.block > kMaxBlock || f.block % 32) return -1;           \
    } while (0)

// ---------------------------------------------------------------------------
// a4: equation of state + momentum + kick
// ---------------------------------------------------------------------------
template <int D, int L, bool CP>
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
        // fluid neighbours: Riemann pressure + viscous (Eq. fluid-model-mr-mom, reading R4)
        nff = fluid_pairs<D, L, CP>(f, g, In.c0, cx, cy, cz, i, lane, Pi, P.rc2F, list, stride, ts,
                                [&](int j) { return f.V4[j]; },
                                [&](int, const float4 &Pj, const float4 &Vj, const float *d, float r2, float, float,
                                    float) {
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
            });
        for_each_cell<D>(g, In.c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int) {
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

template <int D, int L, bool CP, bool TILE>
__global__ void __launch_bounds__(kMaxBlock) k_momentum(Batch bt, Fluid f, Walls w, Solid s)
{
    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint32_t *const list = (uint32_t *)s_dyn + threadIdx.x;
    const int stride = blockDim.x;
    if constexpr (!TILE) {
        const int t = blockIdx.x * blockDim.x + threadIdx.x;
        momentum_one<D, L, CP>(bt, f, w, s, t / L, t / L < f.n, t % L, list, stride, nullptr);
    } else {
        tile_loop<D, L>(bt, f, f.V4, s_dyn + (CP ? (size_t)kListBytes * blockDim.x : 0),
                        [&](int i, bool act, const TileSrc *ts) {
                            momentum_one<D, L, CP>(bt, f, w, s, i, act, (int)threadIdx.x % L, list, stride, ts);
                        });
    }
}

int launch_momentum(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int dim, cudaStream_t st)
{
    if (f.n == 0) return 0;
    if (f.n >= (1 << 27)) return -7;
    SPH_LAUNCH_PAIRS(k_momentum, f.n, bt, f, w, s);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// a5: fluid force on each solid particle, f_a^F = -sum_i V_i (pair term),
// the same pair expression and inputs as a4 (fluid at r^{n+1/2}, v^n)
// ---------------------------------------------------------------------------
template <int D, int L>
__global__ void __launch_bounds__(kMaxBlock, 2) k_solid_fluid_force(Batch bt, Fluid f, Solid s)
{
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
        for_each_cell<D>(g, In.c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int) {
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
    Counts cnt = {0u, 0u, 0u, nsf, 0.0f, {0.0, 0.0, 0.0}};
    if (act && lane == 0) {
        for (int q = 0; q < 3; q++) s.fF[3 * a + q] = q < D ? fa[q] : 0.0f;
        for (int q = 0; q < D; q++) cnt.mom[q] = (double)fa[q];
    }
    flush_counts<D>(bt, b, act, cnt, false);
}

int launch_solid_fluid_force(const Batch &bt, const Fluid &f, const Solid &s, int dim, cudaStream_t st)
{
    if (s.n == 0 || f.n == 0) {
        if (s.n) cudaMemsetAsync(s.fF, 0, sizeof(float) * 3 * s.n, st);
        return cudaGetLastError() == cudaSuccess ? 0 : -3;
    }
    SPH_LAUNCH_LANES(k_solid_fluid_force, s.n, 0, bt, f, s);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// a6: continuity at (r^{n+1/2}, rho^{n+1/2}, v^{n+1}) + second half drift;
// writes the end-of-step state to s[0] in cell order
// ---------------------------------------------------------------------------
template <int D, int L, bool CP>
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
        fluid_pairs<D, L, CP>(f, g, In.c0, cx, cy, cz, i, lane, Pi, P.rc2F, list, stride, ts,
                          [&](int j) { return f.W4[j]; },
                          [&](int, const float4 &, const float4 &Wj, const float *d, float r2, float, float, float) {
                const float rhoj = P.rho0 + Wj.w;
                float r = sqrtf(r2), invr = 1.0f / r;
                float dW = dW_F(r, P);
                float UL = -(vi[0] * d[0] + vi[1] * d[1] + (D == 3 ? vi[2] * d[2] : 0.0f)) * invr;
                float UR = -(Wj.x * d[0] + Wj.y * d[1] + (D == 3 ? Wj.z * d[2] : 0.0f)) * invr;
                float rb = 0.5f * (rhoi + rhoj);
                // (v_i - v~_ij).grad_i W = -dW (U_L - U*), U* = (U_L + U_R)/2 + (p_i - p_j) / (2 rho c0)
                float diff = 0.5f * (UL - UR) - eos_dp(drhoi, Wj.w, P) * inv2c0 / rb;
                rate += (P.mF / rhoj) * (-dW) * diff;
            });
        for_each_cell<D>(g, In.c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int) {
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

template <int D, int L, bool CP, bool TILE>
__global__ void __launch_bounds__(kMaxBlock) k_density(Batch bt, Fluid f, Walls w, Solid s)
{
    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint32_t *const list = (uint32_t *)s_dyn + threadIdx.x;
    const int stride = blockDim.x;
    if constexpr (!TILE) {
        const int t = blockIdx.x * blockDim.x + threadIdx.x;
        density_one<D, L, CP>(bt, f, w, s, t / L, t / L < f.n, t % L, list, stride, nullptr);
    } else {
        tile_loop<D, L>(bt, f, f.W4, s_dyn + (CP ? (size_t)kListBytes * blockDim.x : 0),
                        [&](int i, bool act, const TileSrc *ts) {
                            density_one<D, L, CP>(bt, f, w, s, i, act, (int)threadIdx.x % L, list, stride, ts);
                        });
    }
}

int launch_density(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int dim, cudaStream_t st)
{
    if (f.n == 0) return 0;
    if (f.n >= (1 << 27)) return -7;
    SPH_LAUNCH_PAIRS(k_density, f.n, bt, f, w, s);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// a3: density reinitialisation rho = rho0 sigma / sigma0 (reading R16).
// rho0 (sigma - sigma0) / sigma0 cancels about three digits, so each kernel
// value is evaluated in FP64 from the FP64 positions (the FP32 records only
// screen out candidates well outside the support) and summed in FP64.
// ---------------------------------------------------------------------------
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
// cell offset o = -dcell * edge as hi + lo (o is 0 or +-csf)
__device__ __forceinline__ float off_lo(float o, float cslo)
{
    return o == 0.0f ? 0.0f : (o > 0.0f ? cslo : -cslo);
}

// Wendland C2 shape (1 - q/2)^4 (1 + 2q) of the pair, q = |r_ij| / h_F, in
// double-float; 0 outside the support.
template <int D>
__device__ __forceinline__ ff W_ff_shape(const float4 &Pi, const float4 &Li, const float4 &Pj, const float4 &Lj,
                                         float ox, float oy, float oz, const Grid &g, const Phys &P)
{
    const ff dx = ff_delta(Pi.x, Li.x, Pj.x, Lj.x, ox, off_lo(ox, g.cslo[0]));
    const ff dy = ff_delta(Pi.y, Li.y, Pj.y, Lj.y, oy, off_lo(oy, g.cslo[1]));
    ff r2 = ff_add(ff_sqr(dx), ff_sqr(dy));
    if (D == 3) r2 = ff_add(r2, ff_sqr(ff_delta(Pi.z, Li.z, Pj.z, Lj.z, oz, off_lo(oz, g.cslo[2]))));
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

template <int D, int L, bool CP>
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
        // the screen passes pairs up to 1.0001 (2 h)^2; W_ff_shape returns 0 beyond the support
        fluid_pairs<D, L, CP>(f, g, In.c0, cx, cy, cz, i, lane, Pi, screen, list, stride, ts,
                          [&](int j) { return f.L4[j]; },
                          [&](int, const float4 &Pj, const float4 &Lj, const float *, float, float ox, float oy,
                              float oz) {
                sF = ff_add(sF, W_ff_shape<D>(Pi, Li, Pj, Lj, ox, oy, oz, g, P));
            });
        for_each_cell<D>(g, In.c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int) {
            const int a1 = w.cstart[c + 1];
            for (int q = w.cstart[c] + lane; q < a1; q += L) {
                float d[3];
                const float4 Aq = w.A4[q];
                if (rel_d<D>(Pi, Aq, ox, oy, oz, d) >= screen) continue;
                sW = ff_add(sW, W_ff_shape<D>(Pi, Li, Aq, w.L4[q], ox, oy, oz, g, P));
            }
            if (s.n) {
                const int b1 = s.cstart[c + 1];
                for (int q = s.cstart[c] + lane; q < b1; q += L) {
                    float d[3];
                    const float4 Aq = s.A4[q];
                    if (rel_d<D>(Pi, Aq, ox, oy, oz, d) >= screen) continue;
                    sS = ff_add(sS, W_ff_shape<D>(Pi, Li, Aq, s.L4[q], ox, oy, oz, g, P));
                }
            }
        });
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

template <int D, int L, bool CP, bool TILE>
__global__ void __launch_bounds__(kMaxBlock) k_reinit(Batch bt, Fluid f, Walls w, Solid s)
{
    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint32_t *const list = (uint32_t *)s_dyn + threadIdx.x;
    const int stride = blockDim.x;
    if constexpr (!TILE) {
        const int t = blockIdx.x * blockDim.x + threadIdx.x;
        reinit_one<D, L, CP>(bt, f, w, s, t / L, t / L < f.n, t % L, list, stride, nullptr);
    } else {
        if (!bt.ctl[f.tiles[blockIdx.x].x].reinit) return;   // not a reinitialisation step of this instance
        tile_loop<D, L>(bt, f, f.L4, s_dyn + (CP ? (size_t)kListBytes * blockDim.x : 0),
                        [&](int i, bool act, const TileSrc *ts) {
                            reinit_one<D, L, CP>(bt, f, w, s, i, act, (int)threadIdx.x % L, list, stride, ts);
                        });
    }
}

int launch_reinit(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int dim, cudaStream_t st)
{
    if (f.n == 0) return 0;
    if (f.n >= (1 << 27)) return -7;
    SPH_LAUNCH_PAIRS(k_reinit, f.n, bt, f, w, s);
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
        int a = s.perm[k];
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
    for_each_cell<D>(g, In.c0, cx, cy, cz, [&](int c, float, float, float, int) {
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
                int a = s.perm[j];
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
    });
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
