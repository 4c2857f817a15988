// Shared device code of the fluid pair loops at h_F (Section 3.1): neighbour
// cell visits, the two pair-loop forms, tile staging, the fluid-solid pair
// terms, counters and the launch macros.  The kernels are in sph_fluid.cu
// (momentum, solid-side coupling force) and sph_density.cu (continuity,
// density reinitialisation).
//
// L consecutive threads share one target particle (cell order): each visits
// the 3^d cells around the target and takes every L-th candidate of each
// cell; the partial sums are combined with warp shuffles.  Consecutive
// targets share their neighbour cells, so the records (two float4 per
// particle) are served from L1/L2.  Pair geometry is FP32 on cell-relative
// coordinates: r_ij = (x_i - x_cell_i) - (x_j - x_cell_j) - dcell * edge.
#pragma once
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

// Visit the (2R + 1)^d neighbour cells of (cx, cy, cz).  fn(cell, ox, oy,
// oz, code) receives the offset o = -(dcell) * edge to add to (rel_i -
// rel_j) and code = (dx + R) + W (dy + R) + W^2 (dz + R), W = 2R + 1
// (cell_offset<R> recovers o from it; code < 125).  R is a compile-time
// constant (the kernels are instantiated per reach): a runtime reach costs
// registers, hence occupancy, in every pair loop.  Visiting R = 2 over
// cells of edge >= 2 h_F is correct, only slower.
template <int D, int R, typename Fn>
__device__ __forceinline__ void for_each_cell(const Grid &g, int c0, int cx, int cy, int cz, Fn &&fn)
{
    constexpr int W = 2 * R + 1;
    const int z0 = D == 3 ? -R : 0, z1 = D == 3 ? R : 0;
#pragma unroll 1
    for (int dz = z0; dz <= z1; dz++) {
        int z = cz + dz;
        if (z < 0 || z >= g.nc[2]) continue;
#pragma unroll 1
        for (int dy = -R; dy <= R; dy++) {
            int y = cy + dy;
            if (y < 0 || y >= g.nc[1]) continue;
#pragma unroll 1
            for (int dx = -R; dx <= R; dx++) {
                int x = cx + dx;
                if (x < 0 || x >= g.nc[0]) {
                    if (!g.periodic_x) continue;
                    x = x < 0 ? x + g.nc[0] : x - g.nc[0];
                }
                int c = c0 + x + g.nc[0] * (y + g.nc[1] * z);
                fn(c, -(float)dx * g.csf[0], -(float)dy * g.csf[1], -(float)dz * g.csf[2],
                   (dx + R) + W * (dy + R) + W * W * (dz + R));
            }
        }
    }
}

// Rows of neighbour cells (Fluid::rows).  The cells x - 1, x, x + 1 of one
// grid row have consecutive indices, so a cell-sorted set holds their
// entries as one run of slots (split where a periodic x wraps).  In the row
// form a row is visited as one flat index range: the six cell starts of a
// row, and those of the wall and solid sets, are loaded together before any
// candidate (3^(d-1) rounds of dependent loads per target instead of
// 3^(d+1)), and the L lanes stay busy across cell boundaries, at a few more
// instructions and registers per candidate.  fn(c, oy, oz, code0) receives
// the global indices of the row's cells x - 1, x, x + 1 (-1 outside the
// grid), the row's offsets and the code of its cell dx = -1.
template <int D, typename Fn>
__device__ __forceinline__ void for_each_row(const Grid &g, int c0, int cx, int cy, int cz, Fn &&fn)
{
    int xs[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        int x = cx + k - 1;
        if (x < 0 || x >= g.nc[0]) x = g.periodic_x ? (x < 0 ? x + g.nc[0] : x - g.nc[0]) : -1;
        xs[k] = x;
    }
    const int z0 = D == 3 ? -1 : 0, z1 = D == 3 ? 1 : 0;
#pragma unroll 1
    for (int dz = z0; dz <= z1; dz++) {
        const int z = cz + dz;
        if (z < 0 || z >= g.nc[2]) continue;
#pragma unroll 1
        for (int dy = -1; dy <= 1; dy++) {
            const int y = cy + dy;
            if (y < 0 || y >= g.nc[1]) continue;
            const int base = c0 + g.nc[0] * (y + g.nc[1] * z);
            const int c[3] = {xs[0] < 0 ? -1 : base + xs[0], xs[1] < 0 ? -1 : base + xs[1],
                              xs[2] < 0 ? -1 : base + xs[2]};
            fn(c, -(float)dy * g.csf[1], -(float)dz * g.csf[2], 3 * (dy + 1) + 9 * (dz + 1));
        }
    }
}

struct Row3 {
    int a0, a1, a2;   // first slot of the cells dx = -1, 0, +1
    int n0, n01, n;   // entries of the first cell, of the first two, of all three
};

__device__ __forceinline__ Row3 row_of(const int *__restrict__ cstart, const int c[3])
{
    int lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        lo[k] = c[k] >= 0 ? cstart[c[k]] : 0;
        hi[k] = c[k] >= 0 ? cstart[c[k] + 1] : 0;
    }
    Row3 r;
    r.a0 = lo[0];
    r.a1 = lo[1];
    r.a2 = lo[2];
    r.n0 = hi[0] - lo[0];
    r.n01 = r.n0 + (hi[1] - lo[1]);
    r.n = r.n01 + (hi[2] - lo[2]);
    return r;
}

// slot of the row's flat entry q; k = its cell (0, 1, 2 for dx = -1, 0, +1)
__device__ __forceinline__ int row_slot(const Row3 &r, int q, int &k)
{
    k = (q >= r.n0 ? 1 : 0) + (q >= r.n01 ? 1 : 0);
    return k == 0 ? r.a0 + q : (k == 1 ? r.a1 + (q - r.n0) : r.a2 + (q - r.n01));
}

// x offset -dx * edge of cell k of a row (the same value as for_each_cell's)
__device__ __forceinline__ float row_ox(int k, const Grid &g) { return (float)(1 - k) * g.csf[0]; }

template <int R>
__device__ __forceinline__ void cell_offset(int code, const Grid &g, float &ox, float &oy, float &oz)
{
    constexpr int W = 2 * R + 1;
    const int dx = code % W - R, dy = (code / W) % W - R, dz = code / (W * W) - R;
    ox = -(float)dx * g.csf[0];
    oy = -(float)dy * g.csf[1];
    oz = -(float)dz * g.csf[2];
}

// Cell offset of a neighbour-row entry: 2 bits per axis, (dx + 1) | (dy + 1)
// << 2 | (dz + 1) << 4 (reach 1), decoded with shifts and masks.
__device__ __forceinline__ uint32_t row_code(int code27)
{
    return (uint32_t)(code27 % 3) | (uint32_t)((code27 / 3) % 3) << 2 | (uint32_t)(code27 / 9) << 4;
}
__device__ __forceinline__ void row_offset(uint32_t e, const Grid &g, float &ox, float &oy, float &oz)
{
    ox = (float)(1 - (int)(e & 3u)) * g.csf[0];
    oy = (float)(1 - (int)((e >> 2) & 3u)) * g.csf[1];
    oz = (float)(1 - (int)((e >> 4) & 3u)) * g.csf[2];
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
// thread first writes its in-support neighbours (j << 7 | cell-offset code)
// into its own list in shared memory (slot k at list[k * stride]), then
// evaluates the list with all lanes busy; a full list is drained early.
// Requires j < 2^25.
//
// Both return the number of in-support pairs and visit the pairs of a
// target in the same order.
constexpr int kPairCap = 32;
// list entry j << kCodeBits | cell-offset code (code < 125): j < 2^25
constexpr int kCodeBits = 7;
constexpr uint32_t kCodeMask = (1u << kCodeBits) - 1u;
constexpr int kMaxPairTargets = 1 << (32 - kCodeBits);

template <int D, int L, bool CP, int R, typename Fetch, typename Pair>
__device__ __forceinline__ unsigned fluid_pairs_global(const Fluid &f, const Grid &g, int c0, int cx, int cy, int cz,
                                                       int i, int lane, const float4 &Pi, float rc2, uint32_t *list,
                                                       int stride, Fetch &&fetch, Pair &&pair)
{
    unsigned cnt_total = 0;
    if constexpr (!CP) {
        for_each_cell<D, R>(g, c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int) {
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
                const int j = (int)(e >> kCodeBits);
                float ox, oy, oz;
                cell_offset<R>((int)(e & kCodeMask), g, ox, oy, oz);
                const float4 Pj = f.P4[j];
                float d[3];
                const float r2 = rel_d<D>(Pi, Pj, ox, oy, oz, d);
                pair(j, Pj, fetch(j), d, r2, ox, oy, oz);
            }
            cnt = 0;
        };
        for_each_cell<D, R>(g, c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int code) {
            const int j1 = f.cstart[c + 1];
            for (int j = f.cstart[c] + lane; j < j1; j += L) {
                if (j == i) continue;
                float d[3];
                if (rel_d<D>(Pi, f.P4[j], ox, oy, oz, d) >= rc2) continue;
                list[cnt * stride] = ((uint32_t)j << kCodeBits) | (uint32_t)code;
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
            const int q = (int)(e >> kCodeBits);
            float ox, oy, oz;
            cell_offset<1>((int)(e & kCodeMask), g, ox, oy, oz);
            const float4 Pj = ts.sP[q];
            float d[3];
            const float r2 = rel_d<D>(Pi, Pj, ox, oy, oz, d);
            pair(q, Pj, ts.sX[q], d, r2, ox, oy, oz);
        }
        cnt = 0;
    };
    for_each_cell<D, 1>(g, c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int code) {
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
                list[cnt * stride] = ((uint32_t)q << kCodeBits) | (uint32_t)code;
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

// Wall and solid candidates of one neighbour cell (cell form) or one row
// (row form): wp(a, ox, oy, oz) and sp(b, ox, oy, oz) test and evaluate
// wall slot a and solid slot b.
template <int L, typename WP, typename SP>
__device__ __forceinline__ void ws_cell(const Walls &w, const Solid &s, int c, float ox, float oy, float oz, int lane,
                                        WP &wp, SP &sp)
{
    const int a1 = w.cstart[c + 1];
    for (int a = w.cstart[c] + lane; a < a1; a += L) wp(a, ox, oy, oz);
    if (s.n) {
        const int b1 = s.cstart[c + 1];
        for (int b = s.cstart[c] + lane; b < b1; b += L) sp(b, ox, oy, oz);
    }
}

template <int L, typename WP, typename SP>
__device__ __forceinline__ void ws_row(const Walls &w, const Solid &s, const Grid &g, const int c[3], float oy,
                                       float oz, int lane, WP &wp, SP &sp)
{
    const Row3 rw = row_of(w.cstart, c);
    const Row3 rs = s.n ? row_of(s.cstart, c) : Row3{0, 0, 0, 0, 0, 0};
    for (int q = lane; q < rw.n; q += L) {
        int k;
        const int a = row_slot(rw, q, k);
        wp(a, row_ox(k, g), oy, oz);
    }
    for (int q = lane; q < rs.n; q += L) {
        int k;
        const int b = row_slot(rs, q, k);
        sp(b, row_ox(k, g), oy, oz);
    }
}

// Row form of the fluid-fluid pairs (direct or compacted as above; the
// compacted form tests two candidates per iteration, both loads issued
// first), with each row's wall and solid candidates.
template <int D, int L, bool CP, typename Fetch, typename Pair, typename WP, typename SP>
__device__ __forceinline__ unsigned fluid_pairs_rows(const Fluid &f, const Walls &w, const Solid &s, const Grid &g,
                                                     int c0, int cx, int cy, int cz, int i, int lane, const float4 &Pi,
                                                     float rc2, uint32_t *list, int stride, Fetch &fetch, Pair &pair,
                                                     WP &wp, SP &sp)
{
    unsigned cnt_total = 0;
    int cnt = 0;
    auto drain = [&]() {
#pragma unroll 1
        for (int k = 0; k < cnt; k++) {
            const uint32_t e = list[k * stride];
            const int j = (int)(e >> kCodeBits);
            float ox, oy, oz;
            cell_offset<1>((int)(e & kCodeMask), g, ox, oy, oz);
            const float4 Pj = f.P4[j];
            float d[3];
            const float r2 = rel_d<D>(Pi, Pj, ox, oy, oz, d);
            pair(j, Pj, fetch(j), d, r2, ox, oy, oz);
        }
        cnt = 0;
    };
    for_each_row<D>(g, c0, cx, cy, cz, [&](const int c[3], float oy, float oz, int code0) {
        const Row3 r = row_of(f.cstart, c);
        ws_row<L>(w, s, g, c, oy, oz, lane, wp, sp);
        if constexpr (!CP) {
            for (int q = lane; q < r.n; q += L) {
                int k;
                const int j = row_slot(r, q, k);
                if (j == i) continue;
                const float ox = row_ox(k, g);
                const float4 Pj = f.P4[j];
                float d[3];
                const float r2 = rel_d<D>(Pi, Pj, ox, oy, oz, d);
                if (r2 >= rc2) continue;
                cnt_total++;
                pair(j, Pj, fetch(j), d, r2, ox, oy, oz);
            }
        } else {
            auto test = [&](int j, int k, const float4 &Pj) {
                if (j == i) return;
                float d[3];
                if (rel_d<D>(Pi, Pj, row_ox(k, g), oy, oz, d) >= rc2) return;
                list[cnt * stride] = ((uint32_t)j << kCodeBits) | (uint32_t)(code0 + k);
                cnt++;
                cnt_total++;
                if (cnt == kPairCap) drain();
            };
#pragma unroll 1
            for (int q = lane; q < r.n; q += 2 * L) {
                const bool two = q + L < r.n;
                int k0, k1 = 0;
                const int j0 = row_slot(r, q, k0);
                const int j1 = two ? row_slot(r, q + L, k1) : j0;
                const float4 P0 = f.P4[j0], P1 = f.P4[j1];
                test(j0, k0, P0);
                if (two) test(j1, k1, P1);
            }
        }
    });
    if constexpr (CP) drain();
    return cnt_total;
}

// Neighbour-row form (Fluid::list): target i's in-support fluid neighbours
// (front of its row) and wall neighbours (back of its row, last entry first)
// come from its row (built by k_pairlist at the same
// record positions, with the same FP32 support test), L lanes striding over
// it with every lane busy; the solid candidates of its neighbour cells are
// visited only when the row says there are any; a row that overflowed takes
// the cell form.  Pairs in a row are in support by construction: pair() gets
// them without a test (the count of this lane's fluid pairs is returned).
template <int D, int L, typename Fetch, typename Pair, typename WP, typename SP>
__device__ __forceinline__ unsigned fluid_pairs_list(const Fluid &f, const Walls &w, const Solid &s, const Grid &g,
                                                     int c0, int cx, int cy, int cz, int i, int lane,
                                                     const float4 &Pi, float rc2, Fetch &fetch, Pair &pair, WP &wp,
                                                     SP &sp)
{
    const uint32_t cw = f.nbc[i];
    if (cw & kListOver) {
        const unsigned n = fluid_pairs_global<D, L, false, 1>(f, g, c0, cx, cy, cz, i, lane, Pi, rc2, nullptr, 0,
                                                              fetch, pair);
        for_each_cell<D, 1>(g, c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int) {
            ws_cell<L>(w, s, c, ox, oy, oz, lane, wp, sp);
        });
        return n;
    }
    const int nF = (int)(cw & kListCountMask), nW = (int)((cw >> 11) & kListCountMask);
    const uint32_t *__restrict__ row = f.nbl + (size_t)i * f.list_cap;
    // two entries per lane per round, both gathers issued before either pair
    // is evaluated (the loop is bound by the latency of entry -> record
    // chains); the pairs are summed in the same order as one at a time
    int q = lane;
    for (; q + L < nF; q += 2 * L) {
        const uint32_t e0 = row[q], e1 = row[q + L];
        const int j0 = (int)(e0 >> kCodeBits), j1 = (int)(e1 >> kCodeBits);
        const float4 P0 = f.P4[j0], P1 = f.P4[j1];
        const auto X0 = fetch(j0);
        const auto X1 = fetch(j1);
        float ox, oy, oz, d[3];
        row_offset(e0, g, ox, oy, oz);
        float r2 = rel_d<D>(Pi, P0, ox, oy, oz, d);
        pair(j0, P0, X0, d, r2, ox, oy, oz);
        row_offset(e1, g, ox, oy, oz);
        r2 = rel_d<D>(Pi, P1, ox, oy, oz, d);
        pair(j1, P1, X1, d, r2, ox, oy, oz);
    }
    if (q < nF) {
        const uint32_t e = row[q];
        const int j = (int)(e >> kCodeBits);
        float ox, oy, oz;
        row_offset(e, g, ox, oy, oz);
        const float4 Pj = f.P4[j];
        float d[3];
        const float r2 = rel_d<D>(Pi, Pj, ox, oy, oz, d);
        pair(j, Pj, fetch(j), d, r2, ox, oy, oz);
    }
    const uint32_t *__restrict__ wrow = row + f.list_cap - 1;   // wall entries run from the back
    for (int q = lane; q < nW; q += L) {
        const uint32_t e = wrow[-q];
        float ox, oy, oz;
        row_offset(e, g, ox, oy, oz);
        wp((int)(e >> kCodeBits), ox, oy, oz);
    }
    if (cw & kListSolid) {
        for_each_cell<D, 1>(g, c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int) {
            const int b1 = s.cstart[c + 1];
            for (int b = s.cstart[c] + lane; b < b1; b += L) sp(b, ox, oy, oz);
        });
    }
    return lane < nF ? (unsigned)((nF - lane + L - 1) / L) : 0u;
}

// All neighbours of target i: fluid-fluid pairs through pair (their number
// is returned), wall and solid candidates through wp and sp.  FORM 1 is the
// row form (global records only); FORM 3 the neighbour-row form; otherwise
// the cell form visits the fluid cells (from the staged tile when ts is set),
// then the wall and solid entries cell by cell, over the 3^d cells (FORM 0)
// or the 5^d cells of edge >= h_F (FORM 2).
template <int D, int L, bool CP, int FORM, typename Fetch, typename Pair, typename WP, typename SP>
__device__ __forceinline__ unsigned fluid_pairs(const Fluid &f, const Walls &w, const Solid &s, const Grid &g, int c0,
                                                int cx, int cy, int cz, int i, int lane, const float4 &Pi, float rc2,
                                                uint32_t *list, int stride, const TileSrc *ts, Fetch &&fetch,
                                                Pair &&pair, WP &&wp, SP &&sp)
{
    if constexpr (FORM == 3) {
        return fluid_pairs_list<D, L>(f, w, s, g, c0, cx, cy, cz, i, lane, Pi, rc2, fetch, pair, wp, sp);
    } else if constexpr (FORM == 1) {
        return fluid_pairs_rows<D, L, CP>(f, w, s, g, c0, cx, cy, cz, i, lane, Pi, rc2, list, stride, fetch, pair, wp,
                                          sp);
    } else {
        constexpr int R = FORM == 2 ? 2 : 1;
        const unsigned n =
            ts ? fluid_pairs_tile<D, L, CP>(f, g, c0, cx, cy, cz, i, lane, Pi, rc2, list, stride, *ts, pair)
               : fluid_pairs_global<D, L, CP, R>(f, g, c0, cx, cy, cz, i, lane, Pi, rc2, list, stride, fetch, pair);
        for_each_cell<D, R>(g, c0, cx, cy, cz, [&](int c, float ox, float oy, float oz, int) {
            ws_cell<L>(w, s, c, ox, oy, oz, lane, wp, sp);
        });
        return n;
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
    // a particle on top of a boundary particle at FP32 resolution: the
    // direction is undefined and the pressure term vanishes with r; the
    // viscous term's limit is dropped with it
    float r = sqrtf(r2);
    float invr = r2 > 0.0f ? 1.0f / r : 0.0f;
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
    float invr = r2 > 0.0f ? 1.0f / r : 0.0f;   // r = 0: no direction, dW(0) = 0
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

constexpr int kListBytes = kPairCap * 4;   // per-thread in-support list (fluid_pairs)

// the same for the pair-loop kernels templated on the pair form (f.compact),
// on tiles (f.tile: one block per tile, the staging area after the lists)
// and on the row form (f.rows, without tiles)
template <typename K>
static void allow_smem(K kern, size_t bytes)
{
    // dynamic plus static shared memory above the default 48 KB needs the opt-in
    if (bytes > 32 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define SPH_LAUNCH_PAIRS(KERN, n, ...)                                                        \
    do {                                                                                      \
        const size_t sm_ = f.list ? 0 : (f.compact ? (size_t)kListBytes * f.block : 0) +     \
                           (f.tile ? (size_t)f.tile_cap * 32 : 0);                            \
        auto go_ = [&](auto Dc, auto Lc) {                                                    \
            constexpr int D_ = decltype(Dc)::value, L_ = decltype(Lc)::value;                \
            const int nb_ = f.tile ? f.ntiles : grid_blocks(n, L_, f.block);                  \
            if (nb_ == 0) return;                                                             \
            auto run_ = [&](auto kern) {                                                      \
                allow_smem(kern, sm_);                                                        \
                launch_k(kern, nb_, f.block, sm_, st, __VA_ARGS__);                           \
            };                                                                                \
            if (f.list) run_(KERN<D_, L_, false, false, 3>);                                  \
            else if (f.compact && f.tile) run_(KERN<D_, L_, true, true, 0>);                  \
            else if (f.compact && f.rows) run_(KERN<D_, L_, true, false, 1>);                 \
            else if (f.compact && f.reach == 2) run_(KERN<D_, L_, true, false, 2>);           \
            else if (f.compact) run_(KERN<D_, L_, true, false, 0>);                           \
            else if (f.tile) run_(KERN<D_, L_, false, true, 0>);                              \
            else if (f.rows) run_(KERN<D_, L_, false, false, 1>);                             \
            else if (f.reach == 2) run_(KERN<D_, L_, false, false, 2>);                       \
            else run_(KERN<D_, L_, false, false, 0>);                                         \
        };                                                                                    \
        const bool ok_ = dim == 2 ? with_lanes<2>(f.lanes, [&](auto Lc) {                     \
            go_(std::integral_constant<int, 2>{}, Lc);                                        \
        })                                                                                    \
                                  : with_lanes<3>(f.lanes, [&](auto Lc) {                     \
            go_(std::integral_constant<int, 3>{}, Lc);                                        \
        });                                                                                   \
        if (!ok_ || f.block < 32 || f.block > kMaxBlock || f.block % 32) return -1;           \
    } while (0)

}  // namespace sph
