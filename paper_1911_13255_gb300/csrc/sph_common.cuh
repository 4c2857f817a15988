// Internal device data structures and helpers of the sphfsi library.
// Method: Zhang, Rezavand & Hu, multi-resolution SPH for FSI (arXiv 1911.13255).
//
// A context holds B >= 1 independent problem instances.  Their particles are
// concatenated (instance b owns fluid slots [f0, f0 + nf), wall slots
// [w0, w0 + nw), solid slots [s0, s0 + ns)) and their cell grids are laid
// end to end in one global cell index space (instance b owns cells
// [c0, c0 + ncell)).  Every kernel looks up the instance of the slot it
// works on and takes that instance's grid, constants and control block, so
// one launch advances all instances; a single problem is a batch of one.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sph {

// device status bits (Ctl::status)
enum : int { ST_NONFINITE = 1, ST_TIMEOUT = 2 };
// values of the context's stop word (Batch::fail)
enum : int { kFailWait = 1, kFailRunaway = 2 };

constexpr int kBlock = 128;           // threads per block of the particle kernels
// 2-D cluster sub-step kernel: particles per CTA, halo slots per CTA and
// halo copies per particle of the push form
constexpr int kSolidCta = 128, kHaloMax = 384, kPushMax = 4;

// Programmatic dependent launch.  The per-step kernels are launched with the
// programmatic stream serialisation attribute (launch_k), so that a kernel's
// blocks can be made resident while its predecessor in the stream finishes.
// Each of them begins with pdl_wait() (griddepcontrol.wait: returns once the
// preceding grid has completed and its memory operations are visible; it
// returns at once for a kernel launched without the attribute) and then
// allows its own successor to launch (pdl_trigger).  Nothing of a kernel
// precedes its pdl_wait().
constexpr bool kPDL = true;

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter()
{
    pdl_wait();
    pdl_trigger();
}

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_k(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem,
                                   cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = kPDL ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}
constexpr int kMaxBlock = 256;        // largest block of the tunable pair-loop kernels
constexpr int kSolidBlock = 256;      // threads per block of the cooperative solid kernel
constexpr long long kSpinLimit = 1ll << 22;   // default bounded spin of the grid barrier and the scan (~0.5-2 s)

// Fixed uniform cell grid with cell edge >= 2 h_F (support radius).  Local
// cell index = x + nc[0] * (y + nc[1] * z); global index = c0 + local.
struct Grid {
    double lo[3];
    double cs[3];    // cell edges (FP64), cs[0] = Lx / nc[0] when periodic in x
    float csf[3];    // the same edges rounded to FP32 (pair-loop offsets)
    float cslo[3];   // cs - csf rounded to FP32 (double-float offsets of the reinitialisation)
    int nc[3];
    int ncell;
    int periodic_x;
    double x_lo, Lx;
    int reach;       // neighbour cells per direction: 1 (cells of >= 2 h_F) or 2 (>= h_F)
};

// Device-resident control block, one per instance, read by every kernel of a
// step, so a captured step graph needs no host-side values.
struct Ctl {
    double t;          // time at the start of the current step
    double dt;         // dt_F of the current step
    double dts;        // dt_S = dt_F / K
    double dt_fixed;   // > 0: fixed dt_F
    long long step;    // index of the current step
    int K;             // solid sub-steps of the current step
    int K_fixed;       // > 0: fixed K; 0: kappa sub-steps; -1, -2: single time step (K = 1)
    int reinit;        // this step reinitialises density and normals
    int n_reinit;
    int status;        // ST_* bits, sticky until read by the host
    int pad0;
    unsigned vmaxF, vmaxS, amaxS, pad1;      // maxima of the current step (float bits)
    float prev_vmaxF, prev_vmaxS, prev_amaxS, pad2;   // maxima of the last finished step
    double mom_fluid[3], mom_solid[3];       // FP64 fluid-solid momentum sums
    unsigned long long n_ff, n_fw, n_fs, n_sf;
    unsigned long long pairs_total;
    double last_dt;
    int last_K, pad3;
    // learned sub-stepper of this step
    int learned_ok;              // 1: the network's step was accepted, the sub-steps are skipped
    int pad4;
    double lnum, lden;           // residual sums |m (v' - v) - dt f(x_mid)|^2, |m v'|^2 (FP64)
    double l_res;                // residual of the last step
    long long l_acc, l_rej;      // accepted / rejected steps
    // automatic advection step (Fluid::held_n == 0, instance 0's values
    // decide): its advection time step dt_ad and the acoustic time so far
    double t_ad, t_acc;
};

// Physical constants of the fluid, the walls and the solid of one instance.
struct Phys {
    int dim;
    float g[3];
    // fluid
    float rho0, c0, eta, hF, inv_hF, rc2F;   // rc2F = (2 h_F)^2 in FP32
    float WcF;        // alpha_d(h_F): W = WcF (1 - q/2)^4 (1 + 2q)
    float dWcF;       // -5 alpha_d(h_F) / h_F: dW/dr = dWcF q (1 - q/2)^3
    float mF;         // rho0 dp_F^d
    float p_coef;     // rho0 c0^2 / 7
    float inv_p_coef;
    float hreg;       // 0.01 h_F, viscous regularisation of the fluid-solid force
    float sigma0;     // lattice number density at h_F / dp_F = 1.3
    float VW, VS;     // wall and solid particle volumes
    float VW_VF, VS_VF;   // volume ratios for the number density
    int free_surface;
    double rc2F_d;    // (2 h_F)^2 in FP64 (debug neighbour sets)
    double hF_d, c0_d, eta_d, rho0_d;
    double alphaF_d, sigma0_d, VW_VF_d, VS_VF_d;   // FP64 number density
    float ihF_hi, ihF_lo;   // 1 / h_F as a double-float pair
    // solid
    float rhoS, mS, mu, lam, hS;
    double hS_d, cS_d;
    // inflow
    int inflow_on, inflow_profile;
    double in_w, in_y0, in_H, in_U, in_tramp;
    double in_T, in_wo;   // Womersley profile: period, Womersley number
    double in_z0, in_Hz;  // duct profile: the z range [z0, z0 + Hz]
};

// Per-instance descriptor (device table, one entry per instance).
struct Inst {
    Grid g;
    Phys P;
    int f0, nf, w0, nw, s0, ns;
    int c0;          // global index of the instance's first cell
    int nnz;         // static solid neighbour entries of the instance
};

// Fluid state, storage order = cell order of the last binning (the slots of
// an instance stay inside its segment).
struct FluidState {
    double *x, *y, *z;
    float *vx, *vy, *vz;
    float *drho;      // rho - rho0
    float *rhodot;    // density rate of the last step (reading R12)
    int *id;          // original index within the instance
};

struct Fluid {
    int n;            // total over the instances
    int lanes;        // threads per target particle of the pair loops (tuned)
    int block;        // threads per block of the pair loops (tuned)
    int compact;      // 1: fluid-fluid pairs through per-thread in-support lists (tuned)
    int tile;         // 1: one block per tile of cells, neighbours staged in shared memory (tuned)
    int rows;         // 1: pair loops visit the neighbour cells a row at a time (tuned; not with tile)
    int reach;        // neighbour cells per direction the pair kernels visit: the largest Grid::reach
    int split_records;  // 1: binning ranks per cell, then writes records per slot (tuned)
    int4 *tiles;      // (instance, first global cell, cells, 0) per tile
    int ntiles;
    int tile_cap;     // records a block can stage (shared memory: 32 B each)
    int *inst;        // instance of each slot
    FluidState s[2];
    float4 *P4;       // (x - x_cell, y - y_cell, z - z_cell, p)   sorted records
    float4 *V4;       // (v^n, rho - rho0)
    float4 *W4;       // (v^{n+1}, rho - rho0)
    float4 *L4;       // rel position - FP32(rel position), written on reinitialisation steps
    float *dvdt;      // n * dim, sorted order (a4 accelerations)
    int *key;         // global cell of each particle (storage order)
    int *perm;        // the scatter's slot -> storage slot (cell order, arbitrary inside a cell)
    int *sperm;       // sorted slot -> storage slot (large batches: ranks, then records)
    int *cell_of;     // global cell of each sorted slot
    int *cstart;      // total cells + 1
    int *ccount;      // total cells (histogram / scatter cursor)
    int *live, *nlive;  // non-empty cells of the step (fluid c, solid ncell + c), listed by the scatter
    // decoupled look-back scan of the histograms: tiles of kScanTile cells,
    // (segment, tile) per ticket, segment = set * B + instance
    int2 *scan_tiles;
    int nscan_tiles;
    unsigned long long *scan_status;   // per tile: epoch, flag, value
    unsigned *scan_ctl;                // [0] ticket, [1] epoch
    int bin_fused;      // 1: binning as one cooperative kernel with grid barriers (small problems)
    int *bsum;          // its per-block partial sums (kBinFusedMaxBlocks)
    unsigned *gbar;     // its grid barrier: [0] arrivals, [1] generation
    // Held pair configuration (Algorithm 1: the neighbour lists and the kernel
    // values and gradients are updated once per advection step).  With
    // held_n != 1 the binning (sort, cell lists, record positions) runs only on
    // rebuild steps; on the other steps the particles keep their slots and
    // the records keep the positions of the last rebuild, so every pair term
    // takes W and grad W at those positions, while pressures, densities and
    // velocities are refreshed (k_held_records).
    int held_n;         // coarse steps per advection step; 1: rebuilt every step; 0: as many
                        // as fit the advection criterion (Algorithm 1, decided by the finish kernel)
    int *held;          // [0] != 0: rebuild at the next step (set by the host's state setters),
                        // [1]: the last finished step rebuilt the configuration,
                        // [2] (held_n == 0): the next step rebuilds
    // Neighbour rows (Fluid::list = 1, tuned): the candidate tests of the cell
    // visit run once per rebuild (k_pairlist) and each target's in-support
    // fluid neighbours (from the front) and wall neighbours (from the back)
    // are kept as entries idx << 7 | cell-offset code in row i of list_cap
    // entries; the pair loops stream the rows.  nbc[i] = nF | nW << 11 | flags.
    int list;
    int list_lanes;     // threads per target of the row build (8, 16 or 32; tuned)
    int list_cap;
    uint32_t *nbl;
    uint32_t *nbc;
};

// nbc flags: solid particles in one of the target's neighbour cells (the pair
// loops visit those cells for the solid candidates); the row overflowed (the
// target takes the cell visit for everything)
constexpr uint32_t kListSolid = 1u << 22, kListOver = 1u << 23;
constexpr uint32_t kListCountMask = 0x7ffu;

// Static walls, binned once.
struct Walls {
    int n;
    int *inst;
    double *x, *y, *z;     // original order
    float *nx, *ny, *nz;
    float4 *A4;            // (rel position, 0) sorted
    float4 *N4;            // (normal, 0) sorted
    float4 *L4;            // rel position - FP32(rel position), sorted
    int *key, *perm, *cstart, *ccount, *cell_of;
};

// Elastic bodies (device locality order within each instance) + their
// records in the fluid grid.
struct Solid {
    int n;
    int nnz;
    int *inst;
    double *x, *y, *z;        // current positions (FP64)
    double *x0, *y0, *z0;     // reference positions
    double *xs, *ys, *zs;     // positions at the start of the step
    float4 *v4;               // velocity (vx, vy, vz, 0)
    float *H;                 // n * 9 displacement gradient F - I (row-major, dim x dim used)
    float *Hd;                // n * 9 dF/dt of the last evaluation
    float *B0;                // n * 9
    float4 *Q4;               // P B0 (2-D: one float4; 3-D: three float4 rows)
    float *n0;                // n * 3 reference normals
    float *nrm;               // n * 3 current normals
    uint8_t *cons;
    double *vbar, *abar;      // n * 3 time averages (FP64)
    double *asum;             // n * 3 sum of dt_S a over the sub-steps (FP64)
    float *fF;                // n * 3 fluid force of the step
    int *nb_ptr;              // n + 1 (global entry offsets)
    float4 *nb;               // nnz: (V0 grad0_a W_ab, global b as int bits in .w)
    // records in the fluid grid (sorted by cell)
    float4 *A4, *VB4, *AB4, *N4;
    float4 *L4;               // rel position - FP32(rel position), written on reinitialisation steps
    int *key, *perm, *cstart, *ccount, *cell_of;
    int *sperm;                  // sorted slot -> particle (large batches: ranks, then records)
    unsigned *bar;            // grid barrier: [0] arrivals, [1] generation
    unsigned *queue;          // persistent solid kernel: next instance to take
    int force_grid_path;      // 1: always use the cooperative-grid sub-step kernel
    int force_lane_path;      // 2-D cluster kernel: 0 one thread per particle, 1 four lanes, 2 two threads
    // 2-D cluster kernel, push form: CTA r of a body holds particles
    // [r kSolidCta, (r + 1) kSolidCta) of it in slots 0.. and copies of the
    // other CTAs' particles its particles read (its halo) in slots kSolidCta..
    int *nb_slot;             // nnz: slot of entry q's neighbour in the reading CTA
    int *push_ptr;            // n + 1: a particle's halo copies in other CTAs
    int2 *push;               // (CTA rank, slot) of each copy
    int *halo_n;              // [instance * 16 + CTA]: halo slots of each CTA of each body
    int push_ok;              // 1: every halo and push list fits the kernel's limits
    // one-barrier form (single body): CTA r also computes the stresses of its
    // halo particles itself (one extra thread each), so only velocities cross
    // the cluster; its velocity copies then cover the neighbours of its halo
    // particles too (slots kSolidCta + the halo's own numbering, then the
    // second ring)
    int *h1_ptr;              // [instance * 16 + CTA] + 1: the CTA's halo particles in h1_part
    int *h1_part;             // body-local index of each halo particle
    int *h1_eptr;             // per halo particle: its entries' first index in h1_vslot
    int *h1_vslot;            // velocity slot, in the computing CTA, of each entry's neighbour
    int *push2_ptr;           // n + 1: a particle's velocity copies in other CTAs
    int2 *push2;              // (CTA rank, slot) of each velocity copy
    int one_ok;               // 1: halos of at most kSolidCta particles, copies and push lists fit
    int max_nb;               // largest static neighbour count of a particle
    int max_ns;               // largest body of an instance
    // learned sub-stepper (when learned != 0)
    int learned;
    float l_tol;              // residual threshold
    float l_su, l_sv, l_sf, l_st, l_sdu, l_sdv, l_sH;   // feature / output scales
    double *lx, *ly, *lz;     // candidate end positions
    double *mx, *my, *mz;     // mid positions
    float4 *lv4;              // candidate end velocities
    float *lH;                // n * 9 displacement gradient at the candidate end positions
    float4 *lQ;               // P B0 at the mid positions (2-D one, 3-D three float4)
};

// What every kernel needs to find an instance.
struct Batch {
    const Inst *__restrict__ I;   // device table [B]
    Ctl *ctl;                     // device control blocks [B]
    int B;
    int ncell;                    // total cells
    long long spin;               // iterations of a bounded wait before it gives up (sphfsi_set_wait_limit)
    // Stops the context's device work: kFailWait when the histogram scan gave
    // up waiting (the cell starts of the step are then not valid, so every
    // later kernel that reads cell ranges returns at once), kFailRunaway when
    // a step ended with a non-finite or run-away state (the finish kernel sets
    // it; the next step's kernels return at once, so a blown-up state never
    // reaches the binning, where particles clamped into a few cells would
    // make the in-cell ranking quadratic).  The host refuses to step until a
    // checkpoint is restored.  Its writers complete before the kernels that
    // read it start, so all their threads read the same value.
    int *fail;
};

__device__ __forceinline__ bool step_failed(const Batch &bt) { return *bt.fail != 0; }

// Does this step rebuild the pair configuration?  Every kernel of a step
// evaluates the same inputs (instance 0's step index, which the finish kernel
// advances, and the host's rebuild request, which it clears), so they agree.
// All instances of a context rebuild together.
__device__ __forceinline__ bool rebuild_step(const Batch &bt, const Fluid &f)
{
    if (f.held_n == 1 || f.held[0] != 0) return true;
    if (f.held_n == 0) return f.held[2] != 0;   // automatic: the last step's finish kernel decided
    return bt.ctl[0].step % f.held_n == 0;
}

// the pair configuration is held over several steps (fixed or automatic cadence)
__device__ __host__ __forceinline__ bool held_on(const Fluid &f) { return f.held_n != 1; }

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// grid-wide barrier with a bounded spin (cooperative launch guarantees that
// all blocks are resident); returns false after a time-out
// ---------------------------------------------------------------------------
// (fail: the context's failed-step word, set on a time-out where the waiting
// kernel's partial results would leave invalid cell ranges behind)
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *status, long long spin, int *fail = nullptr)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *vgen = bar + 1;
        unsigned gen = *vgen;
        __threadfence();
        unsigned prev = atomicAdd(bar, 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long it = 0;
            while (*vgen == gen) {
                if (++it > spin) {
                    ok = 0;
                    atomicOr(status, ST_TIMEOUT);
                    if (fail) atomicExch(fail, kFailWait);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

__device__ __forceinline__ void atomic_max_pos(unsigned *addr, float v)
{
    // non-negative floats order like their bit patterns; NaN (0x7fc...) wins
    atomicMax(addr, __float_as_uint(fabsf(v)));
}

__device__ __forceinline__ float warp_sum(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// maximum that keeps a NaN visible (as +inf: fmaxf alone would drop it), so
// that a non-finite state reaches the finish kernel's check
__device__ __forceinline__ float max_keep_nan(float a, float b)
{
    return (a != a || b != b) ? __int_as_float(0x7f800000) : fmaxf(a, b);
}

__device__ __forceinline__ float warp_max(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = max_keep_nan(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ unsigned warp_sum_u(unsigned v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-warp reduction into per-instance counters.  Lanes of a warp may belong
// to different instances (at segment boundaries): lanes whose instance equals
// the warp's first lane's are reduced with shuffles, the others add directly.
__device__ __forceinline__ bool warp_uniform(int b)
{
    return __all_sync(0xffffffffu, b == __shfl_sync(0xffffffffu, b, 0));
}

// cell coordinates of a position (FP64, clamped into the grid)
__device__ __forceinline__ int cell_coord(double x, double lo, double cs, int n)
{
    int c = (int)floor((x - lo) / cs);
    return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

// Tait pressure from rho - rho0 (Eq. eqeos), cancellation-free in FP32:
// p = rho0 c^2 / 7 * expm1(7 log1p(drho / rho0))
__device__ __forceinline__ float eos_p(float drho, const Phys &P)
{
    return P.p_coef * expm1f(7.0f * log1pf(drho / P.rho0));
}
// inverse (ghost density), rho = rho0 (1 + p / p_coef)^(1/7)
__device__ __forceinline__ float eos_rho(float p, const Phys &P)
{
    return P.rho0 * expf(log1pf(p * P.inv_p_coef) * (1.0f / 7.0f));
}

// Wendland C2 derivative dW/dr at h_F (Section 4); caller guarantees q < 2
__device__ __forceinline__ float dW_F(float r, const Phys &P)
{
    float q = r * P.inv_hF;
    float a = 1.0f - 0.5f * q;
    return P.dWcF * q * a * a * a;
}

// ---------------------------------------------------------------------------
// host-side launch wrappers (implemented in the .cu files)
// ---------------------------------------------------------------------------
// control, binning / counting sort, finish (sph_grid.cu)
int launch_bin_all(const Batch &bt, Fluid &f, Solid &s, int dim, int step, double dt_fixed, int K_fixed,
                   cudaStream_t st);
int bin_kernels(const Fluid &f);
int scan_tile_cells();
int launch_wall_bin(const Batch &bt, Walls &w, int dim, cudaStream_t st);
int launch_finish(const Batch &bt, int learned, unsigned *gbar, const Fluid &f, cudaStream_t st);
int launch_scan(int *ccount, int *cstart, int ncell, cudaStream_t st);
int launch_scatter(const int *key, const int *cstart, int *ccount, int *perm, int n, cudaStream_t st);

// fluid pair loops (sph_fluid.cu)
int launch_reinit(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int dim, cudaStream_t st);
int launch_momentum(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int dim, cudaStream_t st);
int launch_solid_fluid_force(const Batch &bt, const Fluid &f, const Solid &s, int dim, cudaStream_t st);
int launch_density(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int dim, cudaStream_t st);
// neighbour rows of the fluid targets (Fluid::list), on rebuild steps
int launch_pairlist(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int dim, cudaStream_t st);
int launch_debug_pairs(const Batch &bt, const Fluid &f, const Walls &w, const Solid &s, int dim, int inst,
                       int which, int *counts, int *offs, int *out, cudaStream_t st);

// solid (sph_solid.cu)
// nbi: the static neighbour list's global slots (host-built, rows ascending)
int launch_solid_setup_fill(const Batch &bt, Solid &s, const int *nbi, int dim, cudaStream_t st);
// P0: host copy of instance 0's constants (used when the batch holds one instance)
int launch_solid_substeps(const Batch &bt, Solid &s, const Phys &P0, int dim, int *path, cudaStream_t st);
// learned sub-stepper: features into x (n x 64), then, from the network's
// outputs (n x 16), candidate, residual and accept / reject (sph_solid.cu)
int launch_learn_features(const Batch &bt, const Solid &s, float *x, int dim, cudaStream_t st);
int launch_learn_candidate(const Batch &bt, const Solid &s, const float *out, int dim, cudaStream_t st);

}  // namespace sph
