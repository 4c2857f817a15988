// Allocation-free neighbour counting (sphfsi_neighbor_counts_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs while another
// framework's caching allocator owns the device memory budget, code inside a
// latency-critical loop where the implicit device synchronisation of
// cudaMalloc/cudaFree is not acceptable, or plug-in code that is only handed
// input and output buffers.  This entry point needs no allocation: its
// scratch (cell keys, the particle permutation and the cell histogram) lives
// in one file-scope __device__ array of fixed size, which every GPU that
// loads the library keeps until the process exits.
//
// Host code must not pass the array's symbol to a kernel (on the host it is
// a stand-in, not a device address); the device address is looked up once
// per device with cudaGetSymbolAddress, with that device current, on the
// first call made on that device.
#include <cmath>
#include <mutex>

#include "sph_common.cuh"
#include "sphfsi.h"

namespace sph {
namespace {

constexpr int kMaxN = SPHFSI_NOALLOC_MAX_PARTICLES;
constexpr int kMaxCells = SPHFSI_NOALLOC_MAX_CELLS;
// layout: key[kMaxN] | perm[kMaxN] | cstart[kMaxCells + 1] | ccount[kMaxCells]
constexpr size_t kScratchInts = 2 * (size_t)kMaxN + 2 * (size_t)kMaxCells + 1;

static __device__ __align__(256) int g_noalloc_scratch[kScratchInts];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int *g_dev_ptr[kMaxDevices] = {};

int scratch_for_current_device(int **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPHFSI_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SPHFSI_E_CAPACITY;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return SPHFSI_E_CUDA;
        }
        g_dev_ptr[dev] = (int *)p;
    }
    *out = g_dev_ptr[dev];
    return SPHFSI_OK;
}

struct NGrid {
    double lo[3], cs[3];
    int nc[3];
    int ncell, periodic_x, dim;
    double Lx, rc2;
};

// x brought into the period [lo, lo + Lx) when periodic in x (identity for
// points already inside it), so that points given outside the period are
// keyed into the cell they wrap to and one minimal-image correction of a
// difference suffices
__device__ __forceinline__ double wrap_x(double x, const NGrid &g)
{
    if (!g.periodic_x) return x;
    double w = x - g.Lx * floor((x - g.lo[0]) / g.Lx);
    // rounding can leave w == lo + Lx for x just below a multiple of the period
    return w >= g.lo[0] + g.Lx ? w - g.Lx : (w < g.lo[0] ? w + g.Lx : w);
}

__global__ void k_na_clear(int *ccount, int ncell)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) ccount[c] = 0;
}

__global__ void k_na_key(const double *__restrict__ r, int n, NGrid g, int *key, int *ccount)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3] = {0, 0, 0};
    for (int k = 0; k < g.dim; k++) {
        double x = r[(size_t)i * g.dim + k];
        if (k == 0) x = wrap_x(x, g);
        c[k] = cell_coord(x, g.lo[k], g.cs[k], g.nc[k]);
    }
    int kk = c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]);
    key[i] = kk;
    atomicAdd(&ccount[kk], 1);
}

__global__ void k_na_count(const double *__restrict__ r, int n, NGrid g, const int *__restrict__ key,
                           const int *__restrict__ cstart, const int *__restrict__ perm, int32_t *counts)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int D = g.dim;
    double ri[3] = {0, 0, 0};
    for (int k = 0; k < D; k++) ri[k] = r[(size_t)i * D + k];
    ri[0] = wrap_x(ri[0], g);
    int kk = key[i];
    int cx = kk % g.nc[0], cy = (kk / g.nc[0]) % g.nc[1], cz = kk / (g.nc[0] * g.nc[1]);
    int cnt = 0;
    const int z0 = D == 3 ? -1 : 0, z1 = D == 3 ? 1 : 0;
    for (int dz = z0; dz <= z1; dz++) {
        int z = cz + dz;
        if (z < 0 || z >= g.nc[2]) continue;
        for (int dy = -1; dy <= 1; dy++) {
            int y = cy + dy;
            if (y < 0 || y >= g.nc[1]) continue;
            for (int dx = -1; dx <= 1; dx++) {
                int x = cx + dx;
                if (x < 0 || x >= g.nc[0]) {
                    if (!g.periodic_x) continue;
                    x = x < 0 ? x + g.nc[0] : x - g.nc[0];
                }
                int c = x + g.nc[0] * (y + g.nc[1] * z);
                for (int q = cstart[c]; q < cstart[c + 1]; q++) {
                    int j = perm[q];
                    if (j == i) continue;
                    double d0 = ri[0] - wrap_x(r[(size_t)j * D], g);
                    if (g.periodic_x) {
                        if (d0 > 0.5 * g.Lx) d0 -= g.Lx;
                        else if (d0 < -0.5 * g.Lx) d0 += g.Lx;
                    }
                    double d1 = ri[1] - r[(size_t)j * D + 1];
                    double r2 = __dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1));
                    if (D == 3) {
                        double d2 = ri[2] - r[(size_t)j * D + 2];
                        r2 = __dadd_rn(r2, __dmul_rn(d2, d2));
                    }
                    if (r2 < g.rc2) cnt++;
                }
            }
        }
    }
    counts[i] = cnt;
}

}  // namespace
}  // namespace sph

extern "C" int sphfsi_neighbor_counts_noalloc(const sphfsi_params *p, int64_t n, const double *r, double dp,
                                              int32_t *counts, void *cuda_stream)
{
    using namespace sph;
    if (!p || (p->dim != 2 && p->dim != 3) || n < 0 || !(dp > 0.0) || !std::isfinite(dp)) return SPHFSI_E_INVAL;
    if (n == 0) return SPHFSI_OK;
    if (!r || !counts) return SPHFSI_E_INVAL;
    if (p->periodic_x && !(p->Lx > 0.0 && std::isfinite(p->Lx) && std::isfinite(p->x_lo))) return SPHFSI_E_INVAL;
    if (n > kMaxN) return SPHFSI_E_CAPACITY;
    const double h = 1.3 * dp;
    NGrid g{};
    g.dim = p->dim;
    g.periodic_x = p->periodic_x;
    g.Lx = p->Lx;
    g.rc2 = 4.0 * h * h;
    long long ncell = 1;
    for (int k = 0; k < 3; k++) {
        if (k >= p->dim) {
            g.lo[k] = 0.0;
            g.cs[k] = 1.0;
            g.nc[k] = 1;
            continue;
        }
        double lo = p->domain_lo[k], L = p->domain_hi[k] - lo;
        if (k == 0 && p->periodic_x) {
            lo = p->x_lo;
            L = p->Lx;
        }
        if (!(L > 0.0) || !std::isfinite(L) || !std::isfinite(lo)) return SPHFSI_E_INVAL;
        // cells along this axis, checked as a double before the conversion
        const double q = floor(L / (2.0 * h));
        if (!std::isfinite(q)) return SPHFSI_E_INVAL;
        if (q > (double)kMaxCells) return SPHFSI_E_CAPACITY;
        long long m = (long long)q;
        if (m < 1) m = 1;
        if (k == 0 && p->periodic_x && m < 3) return SPHFSI_E_INVAL;
        if (m > kMaxCells) return SPHFSI_E_CAPACITY;
        g.lo[k] = lo;
        g.nc[k] = (int)m;
        g.cs[k] = L / (double)m;
        ncell *= m;
        if (ncell > kMaxCells) return SPHFSI_E_CAPACITY;
    }
    g.ncell = (int)ncell;
    int *base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    int *key = base, *perm = base + kMaxN, *cstart = base + 2 * (size_t)kMaxN;
    int *ccount = cstart + kMaxCells + 1;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int B = kBlock;
    const int nn = (int)n;
    k_na_clear<<<(g.ncell + B - 1) / B, B, 0, st>>>(ccount, g.ncell);
    k_na_key<<<(nn + B - 1) / B, B, 0, st>>>(r, nn, g, key, ccount);
    if (launch_scan(ccount, cstart, g.ncell, st)) return SPHFSI_E_CUDA;
    if (launch_scatter(key, cstart, ccount, perm, nn, st)) return SPHFSI_E_CUDA;
    k_na_count<<<(nn + B - 1) / B, B, 0, st>>>(r, nn, g, key, cstart, perm, counts);
    return cudaGetLastError() == cudaSuccess ? SPHFSI_OK : SPHFSI_E_CUDA;
}
