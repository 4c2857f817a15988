// Total-Lagrangian elastic solid at h_S (Sections 2.2, 3.1, 3.3).
//
// Set-up (once): from the static reference neighbour list (the solid keeps
// its reference configuration's neighbours; built on the host through a cell
// grid), the reference kernel gradients V0 grad0_a W_ab and the correction
// matrices
// B0_a = (sum_b V_b (r0_b - r0_a) (x) grad0_a W_ab)^-1 (Eq. correctmatrix with
// the neighbour volume, reading R8), all in FP64 then rounded to FP32.
//
// Sub-steps (every coarse step, K of them, dt_S = dt_F / K): one persistent
// kernel.  Per sub-step: (A) half drift of the displacement gradient and the
// position, neo-Hookean PK1 stress Q = P B0; (B) force loop and kick;
// (C) deformation rate dF/dt = [sum_b V_b (v_b - v_a) (x) grad0 W_ab] B0 and
// the second half drift (Eqs. verlet-first-half-solid ..
// verlet-first-final-solid, solid-model-mr).  Phases that read other
// particles' data are separated by a grid-wide barrier whose spin is
// bounded: on time-out the kernel records ST_TIMEOUT and returns.
//
// The deformation gradient is stored as H = F - I (FP32) so that small
// strains keep their precision: E = (H + H^T + H^T H) / 2, ln J =
// log1p(det(I + H) - 1), S = C^-1 (2 mu E + lambda ln J I).
#include "sph_common.cuh"

namespace sph {

__device__ __forceinline__ double dW_solid_d(double r, double h, int D)
{
    const double pi = 3.14159265358979323846;
    double alpha = D == 2 ? 7.0 / (4.0 * pi * h * h) : 21.0 / (16.0 * pi * h * h * h);
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double a = 1.0 - 0.5 * q;
    return -5.0 * alpha / h * q * a * a * a;
}

__device__ __forceinline__ double r2_d(double dx, double dy, double dz, int D)
{
    double r2 = __dmul_rn(dx, dx);
    r2 = __dadd_rn(r2, __dmul_rn(dy, dy));
    if (D == 3) r2 = __dadd_rn(r2, __dmul_rn(dz, dz));
    return r2;
}

template <int D>
__global__ void k_solid_fill(Batch bt, Solid s, const int *__restrict__ nbi)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= s.n) return;
    const Inst &In = bt.I[s.inst[a]];
    const Phys &P = In.P;
    const double h = P.hS_d;
    const double rc2 = 4.0 * h * h;
    const double V0 = P.VS;
    double xa = s.x0[a], ya = s.y0[a], za = D == 3 ? s.z0[a] : 0.0;
    double M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    (void)rc2;
    for (int q = s.nb_ptr[a]; q < s.nb_ptr[a + 1]; q++) {
        const int b = nbi[q];
        double d[3] = {xa - s.x0[b], ya - s.y0[b], D == 3 ? za - s.z0[b] : 0.0};
        double r2 = r2_d(d[0], d[1], d[2], D);
        double r = sqrt(r2);
        double dW = dW_solid_d(r, h, D);
        double g[3] = {dW * d[0] / r, dW * d[1] / r, D == 3 ? dW * d[2] / r : 0.0};   // grad0_a W_ab
        for (int i = 0; i < D; i++)
            for (int j = 0; j < D; j++) M[i * D + j] += V0 * (-d[i]) * g[j];          // (r0_b - r0_a) (x) grad
        s.nb[q] = make_float4((float)(V0 * g[0]), (float)(V0 * g[1]), (float)(V0 * g[2]), __int_as_float(b));
    }
    double Bi[9];
    if (D == 2) {
        double det = M[0] * M[3] - M[1] * M[2];
        Bi[0] = M[3] / det;
        Bi[1] = -M[1] / det;
        Bi[2] = -M[2] / det;
        Bi[3] = M[0] / det;
    } else {
        double det = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                     M[2] * (M[3] * M[7] - M[4] * M[6]);
        Bi[0] = (M[4] * M[8] - M[5] * M[7]) / det;
        Bi[1] = (M[2] * M[7] - M[1] * M[8]) / det;
        Bi[2] = (M[1] * M[5] - M[2] * M[4]) / det;
        Bi[3] = (M[5] * M[6] - M[3] * M[8]) / det;
        Bi[4] = (M[0] * M[8] - M[2] * M[6]) / det;
        Bi[5] = (M[2] * M[3] - M[0] * M[5]) / det;
        Bi[6] = (M[3] * M[7] - M[4] * M[6]) / det;
        Bi[7] = (M[1] * M[6] - M[0] * M[7]) / det;
        Bi[8] = (M[0] * M[4] - M[1] * M[3]) / det;
    }
    for (int i = 0; i < 9; i++) {
        s.B0[9 * a + i] = i < D * D ? (float)Bi[i] : 0.0f;
        s.H[9 * a + i] = 0.0f;
        s.Hd[9 * a + i] = 0.0f;
    }
}

int launch_solid_setup_fill(const Batch &bt, Solid &s, const int *nbi, int dim, cudaStream_t st)
{
    if (s.n == 0) return 0;
    int nb = (s.n + kBlock - 1) / kBlock;
    if (dim == 2) k_solid_fill<2><<<nb, kBlock, 0, st>>>(bt, s, nbi);
    else k_solid_fill<3><<<nb, kBlock, 0, st>>>(bt, s, nbi);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// neo-Hookean PK1 times B0 from H = F - I (Eqs. Neo-Hookean-energy, 2rd-PK)
template <int D>
__device__ __forceinline__ void stress_QB(const float *H, const float *B, float mu, float lam, float *Q)
{
    if (D == 2) {
        float h00 = H[0], h01 = H[1], h10 = H[2], h11 = H[3];
        float E00 = h00 + 0.5f * (h00 * h00 + h10 * h10);
        float E11 = h11 + 0.5f * (h01 * h01 + h11 * h11);
        float E01 = 0.5f * (h01 + h10 + h00 * h01 + h10 * h11);
        float C00 = 1.0f + 2.0f * E00, C11 = 1.0f + 2.0f * E11, C01 = 2.0f * E01;
        float idet = __frcp_rn(C00 * C11 - C01 * C01);
        float Ci00 = C11 * idet, Ci11 = C00 * idet, Ci01 = -C01 * idet;
        float lnJ = log1pf(h00 + h11 + h00 * h11 - h01 * h10);
        float T00 = 2.0f * mu * E00 + lam * lnJ, T11 = 2.0f * mu * E11 + lam * lnJ, T01 = 2.0f * mu * E01;
        float S00 = Ci00 * T00 + Ci01 * T01, S01 = Ci00 * T01 + Ci01 * T11;
        float S10 = Ci01 * T00 + Ci11 * T01, S11 = Ci01 * T01 + Ci11 * T11;
        float P00 = S00 + h00 * S00 + h01 * S10, P01 = S01 + h00 * S01 + h01 * S11;
        float P10 = S10 + h10 * S00 + h11 * S10, P11 = S11 + h10 * S01 + h11 * S11;
        Q[0] = P00 * B[0] + P01 * B[2];
        Q[1] = P00 * B[1] + P01 * B[3];
        Q[2] = P10 * B[0] + P11 * B[2];
        Q[3] = P10 * B[1] + P11 * B[3];
    } else {
        float E[9], C[9], Ci[9], T[9], S[9], Pm[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                float hh = 0.0f;
                for (int k = 0; k < 3; k++) hh += H[k * 3 + i] * H[k * 3 + j];
                E[i * 3 + j] = 0.5f * (H[i * 3 + j] + H[j * 3 + i] + hh);
                C[i * 3 + j] = (i == j ? 1.0f : 0.0f) + 2.0f * E[i * 3 + j];
            }
        float c00 = C[4] * C[8] - C[5] * C[7], c01 = C[2] * C[7] - C[1] * C[8], c02 = C[1] * C[5] - C[2] * C[4];
        float c10 = C[5] * C[6] - C[3] * C[8], c11 = C[0] * C[8] - C[2] * C[6], c12 = C[2] * C[3] - C[0] * C[5];
        float c20 = C[3] * C[7] - C[4] * C[6], c21 = C[1] * C[6] - C[0] * C[7], c22 = C[0] * C[4] - C[1] * C[3];
        float idet = __frcp_rn(C[0] * c00 + C[1] * c10 + C[2] * c20);
        Ci[0] = c00 * idet; Ci[1] = c01 * idet; Ci[2] = c02 * idet;
        Ci[3] = c10 * idet; Ci[4] = c11 * idet; Ci[5] = c12 * idet;
        Ci[6] = c20 * idet; Ci[7] = c21 * idet; Ci[8] = c22 * idet;
        // det(I + H) - 1 = tr H + principal 2x2 minors + det H
        float trH = H[0] + H[4] + H[8];
        float m2 = H[0] * H[4] - H[1] * H[3] + H[0] * H[8] - H[2] * H[6] + H[4] * H[8] - H[5] * H[7];
        float dH = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                   H[2] * (H[3] * H[7] - H[4] * H[6]);
        float lnJ = log1pf(trH + m2 + dH);
        for (int i = 0; i < 9; i++) T[i] = 2.0f * mu * E[i] + ((i % 4) == 0 ? lam * lnJ : 0.0f);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                float v = 0.0f;
                for (int k = 0; k < 3; k++) v += Ci[i * 3 + k] * T[k * 3 + j];
                S[i * 3 + j] = v;
            }
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                float v = S[i * 3 + j];
                for (int k = 0; k < 3; k++) v += H[i * 3 + k] * S[k * 3 + j];
                Pm[i * 3 + j] = v;
            }
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                float v = 0.0f;
                for (int k = 0; k < 3; k++) v += Pm[i * 3 + k] * B[k * 3 + j];
                Q[i * 3 + j] = v;
            }
    }
}

template <int D>
__device__ __forceinline__ void store_Q(float4 *Q4, int a, const float *Q)
{
    if (D == 2) {
        Q4[a] = make_float4(Q[0], Q[1], Q[2], Q[3]);
    } else {
        Q4[3 * a + 0] = make_float4(Q[0], Q[1], Q[2], 0.0f);
        Q4[3 * a + 1] = make_float4(Q[3], Q[4], Q[5], 0.0f);
        Q4[3 * a + 2] = make_float4(Q[6], Q[7], Q[8], 0.0f);
    }
}

template <int D>
__device__ __forceinline__ void load_Q(const float4 *Q4, int a, float *Q)
{
    if (D == 2) {
        const float4 q = Q4[a];
        Q[0] = q.x, Q[1] = q.y, Q[2] = q.z, Q[3] = q.w;
    } else {
        for (int r = 0; r < 3; r++) {
            const float4 q = Q4[3 * a + r];
            Q[3 * r] = q.x, Q[3 * r + 1] = q.y, Q[3 * r + 2] = q.z;
        }
    }
}

// dH/dt = [sum_b (v_b - v_a) (x) (V0 grad0_a W_ab)] B0_a   (reading R9)
template <int D>
__device__ __forceinline__ void deformation_rate(const Solid &s, int a, const float4 va, float *Hd)
{
    float M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int q0 = s.nb_ptr[a], q1 = s.nb_ptr[a + 1];
    for (int q = q0; q < q1; q++) {
        float4 e = s.nb[q];
        int b = __float_as_int(e.w);
        float4 vb = __ldcg(&s.v4[b]);
        float dv[3] = {vb.x - va.x, vb.y - va.y, vb.z - va.z};
        float g[3] = {e.x, e.y, e.z};
        for (int i = 0; i < D; i++)
            for (int j = 0; j < D; j++) M[i * D + j] += dv[i] * g[j];
    }
    const float *B = s.B0 + 9 * a;
    for (int i = 0; i < D; i++)
        for (int j = 0; j < D; j++) {
            float v = 0.0f;
            for (int k = 0; k < D; k++) v += M[i * D + k] * B[k * D + j];
            Hd[i * D + j] = v;
        }
}

template <int D>
__global__ void __launch_bounds__(kSolidBlock) k_solid_substeps(Batch bt, Solid s)
{
    // one instance only (the launcher checks): its whole body over the grid
    const Phys &P = bt.I[0].P;
    Ctl *ctl = bt.ctl;
    if (ctl->learned_ok) return;   // the learned step was accepted: no sub-steps
    const int K = ctl->K;
    const double dt = ctl->dt, dtsd = ctl->dts;
    const float dts = (float)dtsd, hdts = 0.5f * dts;
    const double hdtsd = 0.5 * dtsd;
    const int G = gridDim.x * blockDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const float inv_rhoS = 1.0f / P.rhoS, inv_mS = 1.0f / P.mS;
    float vmax = 0.0f, amax = 0.0f;

    // start of step: save r^n, clear the acceleration sum, dH/dt(v^0)
    for (int a = tid; a < s.n; a += G) {
        s.xs[a] = s.x[a];
        s.ys[a] = s.y[a];
        if (D == 3) s.zs[a] = s.z[a];
        s.asum[3 * a] = s.asum[3 * a + 1] = s.asum[3 * a + 2] = 0.0;
        float Hd[9];
        deformation_rate<D>(s, a, __ldcg(&s.v4[a]), Hd);
        float *H = s.H + 9 * a;
        for (int i = 0; i < D * D; i++) {
            s.Hd[9 * a + i] = Hd[i];
            H[i] = H[i] + hdts * Hd[i];           // first half drift of sub-step 0
        }
        if (!s.cons[a]) {
            float4 v = __ldcg(&s.v4[a]);
            s.x[a] = s.x[a] + hdtsd * (double)v.x;
            s.y[a] = s.y[a] + hdtsd * (double)v.y;
            if (D == 3) s.z[a] = s.z[a] + hdtsd * (double)v.z;
        }
        float Q[9];
        stress_QB<D>(H, s.B0 + 9 * a, P.mu, P.lam, Q);
        store_Q<D>(s.Q4, a, Q);
    }
    for (int kk = 0; kk < K; kk++) {
        if (!grid_barrier(s.bar, &ctl->status, bt.spin)) return;
        // (B) force loop and kick (Eqs. solid-model-mr, verlet-first-mediate-solid)
        for (int a = tid; a < s.n; a += G) {
            float acc[3] = {0.f, 0.f, 0.f};
            float Qa[9];
            if (D == 2) {
                float4 q = __ldcg(&s.Q4[a]);
                Qa[0] = q.x; Qa[1] = q.y; Qa[2] = q.z; Qa[3] = q.w;
            } else {
                for (int r = 0; r < 3; r++) {
                    float4 q = __ldcg(&s.Q4[3 * a + r]);
                    Qa[3 * r] = q.x; Qa[3 * r + 1] = q.y; Qa[3 * r + 2] = q.z;
                }
            }
            int q0 = s.nb_ptr[a], q1 = s.nb_ptr[a + 1];
            for (int q = q0; q < q1; q++) {
                float4 e = s.nb[q];
                int b = __float_as_int(e.w);
                if (D == 2) {
                    float4 qb = __ldcg(&s.Q4[b]);
                    acc[0] += (Qa[0] + qb.x) * e.x + (Qa[1] + qb.y) * e.y;
                    acc[1] += (Qa[2] + qb.z) * e.x + (Qa[3] + qb.w) * e.y;
                } else {
                    for (int r = 0; r < 3; r++) {
                        float4 qb = __ldcg(&s.Q4[3 * b + r]);
                        acc[r] += (Qa[3 * r] + qb.x) * e.x + (Qa[3 * r + 1] + qb.y) * e.y + (Qa[3 * r + 2] + qb.z) * e.z;
                    }
                }
            }
            if (!s.cons[a]) {
                float4 v = __ldcg(&s.v4[a]);
                float av[3];
                for (int k = 0; k < D; k++) av[k] = acc[k] * inv_rhoS + s.fF[3 * a + k] * inv_mS + P.g[k];
                v.x += dts * av[0];
                v.y += dts * av[1];
                if (D == 3) v.z += dts * av[2];
                s.v4[a] = v;
                float a2 = 0.0f;
                for (int k = 0; k < D; k++) {
                    s.asum[3 * a + k] += dtsd * (double)av[k];
                    a2 += av[k] * av[k];
                }
                amax = max_keep_nan(amax, a2);
                vmax = max_keep_nan(vmax, v.x * v.x + v.y * v.y + v.z * v.z);
            }
        }
        if (!grid_barrier(s.bar, &ctl->status, bt.spin)) return;
        // (C) deformation rate at v^{k+1}, second half drift; then the first
        // half drift of the next sub-step and its stress
        const bool more = kk + 1 < K;
        for (int a = tid; a < s.n; a += G) {
            float4 v = __ldcg(&s.v4[a]);
            float Hd[9];
            deformation_rate<D>(s, a, v, Hd);
            float *H = s.H + 9 * a;
            float Hl[9];
            for (int i = 0; i < D * D; i++) {
                Hl[i] = H[i] + hdts * Hd[i];
                if (more) Hl[i] = Hl[i] + hdts * Hd[i];
                H[i] = Hl[i];
                s.Hd[9 * a + i] = Hd[i];
            }
            if (!s.cons[a]) {
                double x = s.x[a] + hdtsd * (double)v.x;
                double y = s.y[a] + hdtsd * (double)v.y;
                double z = D == 3 ? s.z[a] + hdtsd * (double)v.z : 0.0;
                if (more) {
                    x = x + hdtsd * (double)v.x;
                    y = y + hdtsd * (double)v.y;
                    if (D == 3) z = z + hdtsd * (double)v.z;
                }
                s.x[a] = x;
                s.y[a] = y;
                if (D == 3) s.z[a] = z;
            }
            if (more) {
                float Q[9];
                stress_QB<D>(Hl, s.B0 + 9 * a, P.mu, P.lam, Q);
                store_Q<D>(s.Q4, a, Q);
            }
        }
    }
    // a8: time averages as exact means of the discrete trajectory (reading R14)
    const double idt = 1.0 / dt;
    for (int a = tid; a < s.n; a += G) {
        s.vbar[3 * a] = (s.x[a] - s.xs[a]) * idt;
        s.vbar[3 * a + 1] = (s.y[a] - s.ys[a]) * idt;
        s.vbar[3 * a + 2] = D == 3 ? (s.z[a] - s.zs[a]) * idt : 0.0;
        for (int k = 0; k < 3; k++) s.abar[3 * a + k] = s.asum[3 * a + k] * idt;
    }
    float vm = warp_max(vmax), am = warp_max(amax);
    if ((threadIdx.x & 31) == 0) {
        atomic_max_pos(&ctl->vmaxS, sqrtf(vm));
        atomic_max_pos(&ctl->amaxS, sqrtf(am));
    }
}

// ---------------------------------------------------------------------------
// Cluster-resident variant for bodies of up to kClusterMax * kPPC particles:
// one thread-block cluster holds the whole body.  Each CTA owns kPPC
// consecutive particles; their stress Q = P B0 and velocity live in the
// CTA's shared memory, and neighbours owned by other CTAs of the cluster are
// read through distributed shared memory.  kLanes consecutive threads share
// one particle's neighbour list and reduce with warp shuffles; the group's
// first lane keeps the particle's state (H, B0, FP64 position and sums) in
// registers for all K sub-steps.  Phases are separated by the hardware
// cluster barrier (no spin loop in this kernel).
// ---------------------------------------------------------------------------
constexpr int kCThreads = 512;
constexpr int kLanes = 4;
constexpr int kPPC = kCThreads / kLanes;
constexpr int kClusterMax = 16;

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// generic address of the same shared-memory variable in CTA `rank` of the cluster
template <typename T>
__device__ __forceinline__ const T *dsmem(const T *p, unsigned rank)
{
    uint64_t in = reinterpret_cast<uint64_t>(p), out;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(in), "r"(rank));
    return reinterpret_cast<const T *>(out);
}

__device__ __forceinline__ float group_sum(float v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return v;
}

// K sub-steps of one instance's body (slots [s0, s0 + ns)) by one cluster
template <int D>
__device__ __forceinline__ void solid_lanes_body(const Solid &s, const Phys &P, Ctl *ctl, int s0, int ns, float4 *sQ,
                                                 float4 *sV, unsigned rank)
{
    const int g = threadIdx.x / kLanes, lane = threadIdx.x % kLanes;
    const int la = (int)rank * kPPC + g;
    const int a = s0 + la;
    const bool own = la < ns;
    if (ctl->learned_ok) return;   // the learned step was accepted: no sub-steps
    const int K = ctl->K;
    const double dt = ctl->dt, dtsd = ctl->dts, hdtsd = 0.5 * dtsd;
    const float dts = (float)dtsd, hdts = 0.5f * dts;
    const float inv_rhoS = 1.0f / P.rhoS, inv_mS = 1.0f / P.mS;

    float H[9], B[9], fF[3] = {0.f, 0.f, 0.f};
    double x = 0, y = 0, z = 0, xs = 0, ys = 0, zs = 0, as[3] = {0, 0, 0};
    bool cons = true;
    float vmax = 0.0f, amax = 0.0f;
    int q0 = 0, q1 = 0;
    if (own) {
        q0 = s.nb_ptr[a];
        q1 = s.nb_ptr[a + 1];
        if (lane == 0) {
            for (int i = 0; i < D * D; i++) {
                H[i] = s.H[9 * a + i];
                B[i] = s.B0[9 * a + i];
            }
            for (int k = 0; k < D; k++) fF[k] = s.fF[3 * a + k];
            x = xs = s.x[a];
            y = ys = s.y[a];
            if (D == 3) z = zs = s.z[a];
            cons = s.cons[a] != 0;
            sV[g] = s.v4[a];
        }
    }
    cluster_sync();

    // dH/dt over this particle's neighbours at the velocities in sV (DSMEM).
    // Entries are taken kU at a time per lane so that their remote loads are
    // in flight together.
    constexpr int kU = 4;
    auto rate = [&](float4 va, float *Hd) {
        float M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int base = q0 + lane; base < q1; base += kLanes * kU) {
            float4 e[kU], vb[kU];
#pragma unroll
            for (int u = 0; u < kU; u++) {
                int q = base + u * kLanes;
                e[u] = q < q1 ? __ldg(&s.nb[q]) : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
            }
#pragma unroll
            for (int u = 0; u < kU; u++) {
                int b = __float_as_int(e[u].w);
                b = b >= 0 ? b - s0 : -1;   // local index in the body
                vb[u] = b >= 0 ? *dsmem(&sV[b % kPPC], (unsigned)(b / kPPC)) : va;
            }
#pragma unroll
            for (int u = 0; u < kU; u++) {
                float dv[3] = {vb[u].x - va.x, vb[u].y - va.y, vb[u].z - va.z};
                float ge[3] = {e[u].x, e[u].y, e[u].z};
                for (int i = 0; i < D; i++)
                    for (int j = 0; j < D; j++) M[i * D + j] += dv[i] * ge[j];
            }
        }
        for (int i = 0; i < D * D; i++) M[i] = group_sum(M[i]);
        for (int i = 0; i < D; i++)
            for (int j = 0; j < D; j++) {
                float v = 0.0f;
                for (int k = 0; k < D; k++) v += M[i * D + k] * B[k * D + j];
                Hd[i * D + j] = v;
            }
    };
    auto put_Q = [&]() {
        float Q[9];
        stress_QB<D>(H, B, P.mu, P.lam, Q);
        if (D == 2) {
            sQ[g] = make_float4(Q[0], Q[1], Q[2], Q[3]);
        } else {
            for (int r = 0; r < 3; r++) sQ[3 * g + r] = make_float4(Q[3 * r], Q[3 * r + 1], Q[3 * r + 2], 0.0f);
        }
    };

    // All threads run the neighbour loops (empty for groups past the end of
    // the body) so that the full-warp shuffles of group_sum see every lane;
    // only the owning lane of a group updates state and shared memory.
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // start of step: dH/dt(v^0), first half drift of sub-step 0, stress
    {
        float4 va = own ? sV[g] : zero4;
        float Hd[9];
        rate(va, Hd);
        if (own && lane == 0) {
            for (int i = 0; i < D * D; i++) H[i] = H[i] + hdts * Hd[i];
            if (!cons) {
                x = x + hdtsd * (double)va.x;
                y = y + hdtsd * (double)va.y;
                if (D == 3) z = z + hdtsd * (double)va.z;
            }
            put_Q();
        }
    }
    for (int kk = 0; kk < K; kk++) {
        cluster_sync();
        // (B) force loop and kick
        {
            float Qa[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            if (own) {
                if (D == 2) {
                    float4 t = sQ[g];
                    Qa[0] = t.x; Qa[1] = t.y; Qa[2] = t.z; Qa[3] = t.w;
                } else {
                    for (int r = 0; r < 3; r++) {
                        float4 t = sQ[3 * g + r];
                        Qa[3 * r] = t.x; Qa[3 * r + 1] = t.y; Qa[3 * r + 2] = t.z;
                    }
                }
            }
            float acc[3] = {0.f, 0.f, 0.f};
            for (int base = q0 + lane; base < q1; base += kLanes * kU) {
                float4 e[kU];
#pragma unroll
                for (int u = 0; u < kU; u++) {
                    int q = base + u * kLanes;
                    e[u] = q < q1 ? __ldg(&s.nb[q]) : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
                }
                if (D == 2) {
                    float4 qb[kU];
#pragma unroll
                    for (int u = 0; u < kU; u++) {
                        int b = __float_as_int(e[u].w);
                        b = b >= 0 ? b - s0 : -1;
                        qb[u] = b >= 0 ? *dsmem(&sQ[b % kPPC], (unsigned)(b / kPPC)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < kU; u++) {
                        acc[0] += (Qa[0] + qb[u].x) * e[u].x + (Qa[1] + qb[u].y) * e[u].y;
                        acc[1] += (Qa[2] + qb[u].z) * e[u].x + (Qa[3] + qb[u].w) * e[u].y;
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < kU; u++) {
                        int b = __float_as_int(e[u].w);
                        if (b < 0) continue;
                        b -= s0;
                        unsigned rb = (unsigned)(b / kPPC);
                        int lb = b % kPPC;
                        for (int r = 0; r < 3; r++) {
                            float4 qv = *dsmem(&sQ[3 * lb + r], rb);
                            acc[r] += (Qa[3 * r] + qv.x) * e[u].x + (Qa[3 * r + 1] + qv.y) * e[u].y +
                                      (Qa[3 * r + 2] + qv.z) * e[u].z;
                        }
                    }
                }
            }
            for (int k = 0; k < D; k++) acc[k] = group_sum(acc[k]);
            if (own && lane == 0 && !cons) {
                float4 v = sV[g];
                float av[3];
                for (int k = 0; k < D; k++) av[k] = acc[k] * inv_rhoS + fF[k] * inv_mS + P.g[k];
                v.x += dts * av[0];
                v.y += dts * av[1];
                if (D == 3) v.z += dts * av[2];
                sV[g] = v;
                float a2 = 0.0f;
                for (int k = 0; k < D; k++) {
                    as[k] += dtsd * (double)av[k];
                    a2 += av[k] * av[k];
                }
                amax = max_keep_nan(amax, a2);
                vmax = max_keep_nan(vmax, v.x * v.x + v.y * v.y + v.z * v.z);
            }
        }
        cluster_sync();
        // (C) deformation rate at v^{k+1}; second half drift; next first half + stress
        {
            const bool more = kk + 1 < K;
            float4 va = own ? sV[g] : zero4;
            float Hd[9];
            rate(va, Hd);
            if (own && lane == 0) {
                for (int i = 0; i < D * D; i++) {
                    H[i] = H[i] + hdts * Hd[i];
                    if (more) H[i] = H[i] + hdts * Hd[i];
                }
                if (!cons) {
                    x = x + hdtsd * (double)va.x;
                    y = y + hdtsd * (double)va.y;
                    if (D == 3) z = z + hdtsd * (double)va.z;
                    if (more) {
                        x = x + hdtsd * (double)va.x;
                        y = y + hdtsd * (double)va.y;
                        if (D == 3) z = z + hdtsd * (double)va.z;
                    }
                }
                if (more) put_Q();
            }
        }
    }
    // write back; a8 time averages (reading R14)
    if (own && lane == 0) {
        for (int i = 0; i < D * D; i++) s.H[9 * a + i] = H[i];
        s.v4[a] = sV[g];
        s.x[a] = x;
        s.y[a] = y;
        if (D == 3) s.z[a] = z;
        const double idt = 1.0 / dt;
        s.vbar[3 * a] = (x - xs) * idt;
        s.vbar[3 * a + 1] = (y - ys) * idt;
        s.vbar[3 * a + 2] = D == 3 ? (z - zs) * idt : 0.0;
        for (int k = 0; k < 3; k++) s.abar[3 * a + k] = as[k] * idt;
    }
    float vm = warp_max(vmax), am = warp_max(amax);
    if ((threadIdx.x & 31) == 0 && own) {
        atomic_max_pos(&ctl->vmaxS, sqrtf(vm));
        atomic_max_pos(&ctl->amaxS, sqrtf(am));
    }
    // no CTA may reuse or release its shared memory while others read it
    cluster_sync();
}

// Persistent cluster kernels: each cluster takes instance indices from an
// atomic queue (reset before the launch) until all instances are done, so
// bodies with different K per instance balance over the clusters.  The
// index is read by every CTA of the cluster from its first CTA's shared
// memory between two cluster barriers.
__device__ __forceinline__ int next_instance(unsigned *queue, int *slot, unsigned rank)
{
    if (rank == 0 && threadIdx.x == 0) *slot = (int)atomicAdd(queue, 1u);
    cluster_sync();
    int b = *dsmem(slot, 0u);
    cluster_sync();
    return b;
}

template <int D>
__global__ void __launch_bounds__(kCThreads) k_solid_cluster(Batch bt, Solid s)
{
    pdl_enter();
    constexpr int QR = D == 3 ? 3 : 1;   // float4 rows of Q per particle
    __shared__ float4 sQ[kPPC * QR];
    __shared__ float4 sV[kPPC];
    __shared__ int s_inst;
    const unsigned rank = cluster_rank();
    for (;;) {
        const int b = next_instance(s.queue, &s_inst, rank);
        if (b >= bt.B) break;
        const Inst &In = bt.I[b];
        solid_lanes_body<D>(s, In.P, bt.ctl + b, In.s0, In.ns, sQ, sV, rank);
    }
}

// single instance: one cluster, constants in the parameter space
template <int D>
__global__ void __launch_bounds__(kCThreads) k_solid_cluster_one(Solid s, const __grid_constant__ Phys P, Ctl *ctl)
{
    pdl_enter();
    constexpr int QR = D == 3 ? 3 : 1;
    __shared__ float4 sQ[kPPC * QR];
    __shared__ float4 sV[kPPC];
    solid_lanes_body<D>(s, P, ctl, 0, s.n, sQ, sV, cluster_rank());
}

// ---------------------------------------------------------------------------
// 2-D cluster-resident variant with one thread per particle.  The static
// neighbour entries (V0 grad0 W and the 32-bit shared::cluster addresses of
// the neighbour's stress and velocity slots) are loaded once into registers;
// every phase then issues all its neighbour loads back to back, so a phase
// costs about one shared-memory (or DSMEM) latency instead of one per
// neighbour.  Particles beyond kMaxNb2 neighbours use the 4-lane kernel.
// ---------------------------------------------------------------------------
constexpr int kC1Threads = kSolidCta;   // particles per CTA (128 measured faster than 256)
constexpr int kMaxNb2 = 24;

__device__ __forceinline__ uint32_t cl_addr(const void *p, uint32_t rank)
{
    uint32_t a = (uint32_t)__cvta_generic_to_shared(p), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ float4 ld_cl(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}

__device__ __forceinline__ float2 ld_cl2(uint32_t addr)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

__device__ __forceinline__ void st_cl(uint32_t addr, float4 v)
{
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

// 16-byte store into another CTA's shared memory whose arrival completes 16
// bytes of a transaction on that CTA's mbarrier (both cluster addresses)
__device__ __forceinline__ void st_async(uint32_t addr, float4 v, uint32_t mbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     addr),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mb, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(mb)), "r"(count)
                 : "memory");
}

// one thread arms a use of the mbarrier with the bytes it will receive; every
// thread then waits for that use (parity) to complete, boundedly: false
// after a time-out (status bit set)
__device__ __forceinline__ bool mbar_use(uint64_t *mb, unsigned bytes, unsigned parity, int *status)
{
    const uint32_t m = (uint32_t)__cvta_generic_to_shared(mb);
    if (threadIdx.x == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(m), "r"(bytes) : "memory");
    for (long long it = 0;; it++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(m), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it > (1ll << 20)) {
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
}

constexpr int kChunk2 = 12;   // neighbour loads in flight per phase step

// K sub-steps of one instance's body (slots [s0, s0 + ns)) by one cluster,
// LP threads per particle (128 particles per CTA).  Two forms of the
// neighbour reads: pull (PUSH = false) loads each neighbour's stress and
// velocity from its CTA's shared memory across the cluster (DSMEM) in every
// phase; push (PUSH = true) keeps in every CTA a copy of the neighbours it
// reads (its halo, Solid::nb_slot), which each particle's thread refreshes
// with remote stores right after updating its own value, so that the loops
// read only local shared memory.  The cluster barrier after each phase
// (release / acquire) makes those stores visible, and no CTA overwrites a
// copy while another reads it: stresses are written in one phase and read
// in the next, velocities likewise, with a barrier in between.  With LP = 2 the two
// threads of a particle (adjacent lanes) split its static neighbour entries
// (entry u goes to thread u % 2), combine their partial sums with one
// shuffle, and both carry the particle's own state identically; the first
// writes it out.  Two threads per particle give each SM sub-partition two
// warps to interleave in these latency-bound loops.
template <int LP, int MODE, bool EARLY = false>
__device__ __forceinline__ void solid2d_body(const Solid &s, const Phys &P, Ctl *ctl, int s0, int ns, float4 *sQ,
                                             float4 *sV, unsigned rank, uint64_t *mb, int halo_n, unsigned &phs)
{
    constexpr bool PUSH = MODE != 0, MB = MODE == 2;
    constexpr int SLOTS = kC1Threads + kHaloMax;   // one buffer of the double-buffered (MB) arrays
    constexpr int NB = kMaxNb2 / LP;                   // entries per thread
    constexpr int CH = NB < kChunk2 ? NB : kChunk2;    // loads in flight per round
    const int g = threadIdx.x / LP, sub = threadIdx.x % LP;
    const bool lead = sub == 0;
    const unsigned pmask = LP == 1 ? 0xffffffffu : (3u << ((threadIdx.x & 31) & ~1));
    auto pair_sum = [&](float v) {
        if constexpr (LP == 2) v += __shfl_xor_sync(pmask, v, 1);
        return v;
    };
    const int la = (int)rank * kC1Threads + g;
    const int a = s0 + la;
    // threads past kC1Threads * LP (a padded launch) only take part in the barriers
    const bool own = threadIdx.x < kC1Threads * LP && la < ns;
    if (ctl->learned_ok) return;   // the learned step was accepted: no sub-steps
    const int K = ctl->K;
    const double dt = ctl->dt, dtsd = ctl->dts, hdtsd = 0.5 * dtsd;
    const float dts = (float)dtsd, hdts = 0.5f * dts;
    const float inv_rhoS = 1.0f / P.rhoS, inv_mS = 1.0f / P.mS;

    float H[4] = {0, 0, 0, 0}, B[4] = {1, 0, 0, 1}, fF[2] = {0, 0};
    double x = 0, y = 0, xs = 0, ys = 0, as0 = 0, as1 = 0;
    bool cons = true;
    float vmax = 0.0f, amax = 0.0f;
    float4 vown = make_float4(0.f, 0.f, 0.f, 0.f), Qown = vown;   // the particle's v and P B0
    float gx[NB], gy[NB];
    // pull: the neighbour's sQ slot (cluster address); its sV slot is at
    // aQ + dV (same layout in every CTA).  push: the local slot.
    uint32_t aQ[NB];
    const uint32_t dV = (uint32_t)__cvta_generic_to_shared(&sV[0]) - (uint32_t)__cvta_generic_to_shared(&sQ[0]);
    uint32_t pq[kPushMax];   // push: cluster addresses of this particle's sQ copies
    uint32_t prk[kPushMax];  // and the ranks of the CTAs holding them
    int npush = 0;
    int nn = 0;   // this thread's entries
    if (own) {
        int q0 = s.nb_ptr[a], q1 = s.nb_ptr[a + 1];
        const int ntot = q1 - q0;   // the launcher guarantees ntot <= kMaxNb2
        nn = (ntot - sub + LP - 1) / LP;
        for (int i = 0; i < 4; i++) {
            H[i] = s.H[9 * a + i];
            B[i] = s.B0[9 * a + i];
        }
        x = xs = s.x[a];
        y = ys = s.y[a];
        cons = s.cons[a] != 0;
        vown = s.v4[a];
        if (PUSH && lead) {
            const int p0 = s.push_ptr[a];
            npush = s.push_ptr[a + 1] - p0;   // <= kPushMax when the push form runs
#pragma unroll
            for (int t = 0; t < kPushMax; t++) {
                pq[t] = 0u;
                prk[t] = 0u;
                if (t < npush) {
                    const int2 e = s.push[p0 + t];
                    pq[t] = cl_addr(&sQ[e.y], (uint32_t)e.x);
                    prk[t] = (uint32_t)e.x;
                }
            }
        }
    }
    // own value into the local slot and, in the push forms, into the copies:
    // buffer buf of arr (sQ: off 0, mbarriers 0, 1; sV: off dV, mbarriers 2, 3)
    auto publish = [&](float4 *arr, uint32_t off, int buf, const float4 &val) {
        if (!lead) return;
        arr[(MB ? buf * SLOTS : 0) + g] = val;
        if constexpr (PUSH) {
#pragma unroll
            for (int t = 0; t < kPushMax; t++) {
                if (t < npush) {
                    if constexpr (MB)
                        st_async(pq[t] + off + (uint32_t)(buf * SLOTS * 16), val,
                                 cl_addr(&mb[(off ? 2 : 0) + buf], prk[t]));
                    else
                        st_cl(pq[t] + off, val);
                }
            }
        }
    };
    // MB: every copy of the awaited buffer (mbarrier i: 0, 1 stresses, 2, 3
    // velocities) has arrived; own slots written by this CTA's threads are
    // visible after the block barrier
    bool dead = false;   // a wait timed out: later waits are skipped (the step is flagged)
    auto halo_wait = [&](int i) {
        __syncthreads();
        const unsigned par = (phs >> i) & 1u;
        phs ^= 1u << i;
        if (!dead) dead = !mbar_use(&mb[i], (unsigned)halo_n * 16u, par, &ctl->status);
    };
    if (own) publish(sV, dV, 0, vown);
#pragma unroll
    for (int u = 0; u < NB; u++) {
        gx[u] = gy[u] = 0.0f;
        aQ[u] = 0u;
        if (u < nn) {
            const int q = s.nb_ptr[a] + sub + LP * u;
            float4 e = s.nb[q];
            gx[u] = e.x;
            gy[u] = e.y;
            if constexpr (PUSH) {
                aQ[u] = (uint32_t)s.nb_slot[q];
            } else {
                int b = __float_as_int(e.w) - s0;   // local index in the body
                aQ[u] = cl_addr(&sQ[b % kC1Threads], (uint32_t)(b / kC1Threads));
            }
        }
    }
    // sum of the static gradients: (Q_a + Q_b) . g summed over b is
    // Q_a . sum(g) + sum(Q_b . g)
    float sgx = 0.f, sgy = 0.f;
#pragma unroll
    for (int u = 0; u < NB; u++) {
        sgx += gx[u];
        sgy += gy[u];
    }
    if (own) {
        sgx = pair_sum(sgx);
        sgy = pair_sum(sgy);
    }
    // EARLY: everything above reads data of earlier steps or of the set-up
    // (and this step's control block, written before the coupling force),
    // so it may overlap the coupling-force kernel; its output, f^F, only
    // after that kernel has completed
    if constexpr (EARLY) pdl_wait();
    if (own) {
        fF[0] = s.fF[3 * a];
        fF[1] = s.fF[3 * a + 1];
    }
    cluster_sync();

    // Two accumulator sets (even / odd slots) in both loops, so that a thread
    // has twice as many independent add chains in flight.
    auto rate = [&](float4 va, float *Hd, int vo) {   // vo: first slot of the velocity buffer
        float M0 = 0.f, M1 = 0.f, M2 = 0.f, M3 = 0.f, N0 = 0.f, N1 = 0.f, N2 = 0.f, N3 = 0.f;
#pragma unroll
        for (int c0 = 0; c0 < NB; c0 += CH) {
            float2 vb[CH];
#pragma unroll
            for (int u = 0; u < CH; u++) {
                if (c0 + u < nn) {
                    if constexpr (PUSH) {
                        const float4 t = sV[vo + aQ[c0 + u]];
                        vb[u] = make_float2(t.x, t.y);
                    } else {
                        vb[u] = ld_cl2(aQ[c0 + u] + dV);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < CH; u += 2) {
                if (c0 + u < nn) {
                    const float dvx = vb[u].x - va.x, dvy = vb[u].y - va.y;
                    M0 += dvx * gx[c0 + u];
                    M1 += dvx * gy[c0 + u];
                    M2 += dvy * gx[c0 + u];
                    M3 += dvy * gy[c0 + u];
                }
                if (u + 1 < CH && c0 + u + 1 < nn) {
                    const float dvx = vb[u + 1].x - va.x, dvy = vb[u + 1].y - va.y;
                    N0 += dvx * gx[c0 + u + 1];
                    N1 += dvx * gy[c0 + u + 1];
                    N2 += dvy * gx[c0 + u + 1];
                    N3 += dvy * gy[c0 + u + 1];
                }
            }
        }
        M0 = pair_sum(M0 + N0);
        M1 = pair_sum(M1 + N1);
        M2 = pair_sum(M2 + N2);
        M3 = pair_sum(M3 + N3);
        Hd[0] = M0 * B[0] + M1 * B[2];
        Hd[1] = M0 * B[1] + M1 * B[3];
        Hd[2] = M2 * B[0] + M3 * B[2];
        Hd[3] = M2 * B[1] + M3 * B[3];
    };
    auto put_Q = [&](int buf) {
        float Q[4];
        stress_QB<2>(H, B, P.mu, P.lam, Q);
        Qown = make_float4(Q[0], Q[1], Q[2], Q[3]);
        publish(sQ, 0u, buf, Qown);
    };

    if constexpr (MB) halo_wait(2);   // v^0
    if (own) {
        const float4 va = vown;
        float Hd[4];
        rate(va, Hd, 0);
        for (int i = 0; i < 4; i++) H[i] = H[i] + hdts * Hd[i];
        if (!cons) {
            x = x + hdtsd * (double)va.x;
            y = y + hdtsd * (double)va.y;
        }
        put_Q(0);
    }
    for (int kk = 0; kk < K; kk++) {
        const int qb_ = kk & 1, vb_ = (kk + 1) & 1;   // buffers of Q^k and v^(k+1) (MB)
        if constexpr (MB) halo_wait(qb_);
        else cluster_sync();
        // (B) force loop and kick
        if (own) {
            const float4 Qa = Qown;
            const int qo = MB ? qb_ * SLOTS : 0;
            float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
#pragma unroll
            for (int c0 = 0; c0 < NB; c0 += CH) {
                float4 qb[CH];
#pragma unroll
                for (int u = 0; u < CH; u++)
                    if (c0 + u < nn) qb[u] = PUSH ? sQ[qo + aQ[c0 + u]] : ld_cl(aQ[c0 + u]);
#pragma unroll
                for (int u = 0; u < CH; u += 2) {
                    if (c0 + u < nn) {
                        ax += qb[u].x * gx[c0 + u] + qb[u].y * gy[c0 + u];
                        ay += qb[u].z * gx[c0 + u] + qb[u].w * gy[c0 + u];
                    }
                    if (u + 1 < CH && c0 + u + 1 < nn) {
                        bx += qb[u + 1].x * gx[c0 + u + 1] + qb[u + 1].y * gy[c0 + u + 1];
                        by += qb[u + 1].z * gx[c0 + u + 1] + qb[u + 1].w * gy[c0 + u + 1];
                    }
                }
            }
            ax = Qa.x * sgx + Qa.y * sgy + pair_sum(ax + bx);
            ay = Qa.z * sgx + Qa.w * sgy + pair_sum(ay + by);
            if (!cons) {
                float4 v = vown;
                float av0 = ax * inv_rhoS + fF[0] * inv_mS + P.g[0];
                float av1 = ay * inv_rhoS + fF[1] * inv_mS + P.g[1];
                v.x += dts * av0;
                v.y += dts * av1;
                vown = v;
                publish(sV, dV, vb_, v);
                as0 += dtsd * (double)av0;
                as1 += dtsd * (double)av1;
                amax = max_keep_nan(amax, av0 * av0 + av1 * av1);
                vmax = max_keep_nan(vmax, v.x * v.x + v.y * v.y);
            } else if (MB) {
                publish(sV, dV, vb_, vown);   // a held particle's copies count towards the transaction too
            }
        }
        if constexpr (MB) halo_wait(2 + vb_);
        else cluster_sync();
        // (C) deformation rate at v^{k+1}; second half drift; next first half + stress
        if (own) {
            const bool more = kk + 1 < K;
            const float4 va = vown;
            float Hd[4];
            rate(va, Hd, MB ? vb_ * SLOTS : 0);
            // second half drift of this sub-step and, unless it is the last,
            // the first half drift of the next one with the same rate
            const float hH = more ? dts : hdts;
            const double hX = more ? dtsd : hdtsd;
            for (int i = 0; i < 4; i++) H[i] = H[i] + hH * Hd[i];
            if (more) put_Q(vb_);   // first, so that its stores are under way during the drift
            if (!cons) {
                x = x + hX * (double)va.x;
                y = y + hX * (double)va.y;
            }
        }
    }
    if (own && lead) {
        for (int i = 0; i < 4; i++) s.H[9 * a + i] = H[i];
        s.v4[a] = vown;
        s.x[a] = x;
        s.y[a] = y;
        const double idt = 1.0 / dt;
        s.vbar[3 * a] = (x - xs) * idt;
        s.vbar[3 * a + 1] = (y - ys) * idt;
        s.vbar[3 * a + 2] = 0.0;
        s.abar[3 * a] = as0 * idt;
        s.abar[3 * a + 1] = as1 * idt;
        s.abar[3 * a + 2] = 0.0;
    }
    float vm = warp_max(vmax), am = warp_max(amax);
    if ((threadIdx.x & 31) == 0) {
        atomic_max_pos(&ctl->vmaxS, sqrtf(vm));
        atomic_max_pos(&ctl->amaxS, sqrtf(am));
    }
    cluster_sync();
}

// One-barrier form of the single-body 2-D sub-steps (solid variant 5).  A
// CTA runs 2 kC1Threads threads: thread t < kC1Threads owns particle t of
// the CTA's part of the body, thread kC1Threads + h carries a copy of halo
// particle h (a particle of another CTA that an own particle reads).  Every
// copy evolves its particle's displacement gradient with the same code and
// the same inputs as the owner, so its stress is the owner's bit for bit,
// and the stresses never cross the cluster.  Only velocities do: after the
// kick each own particle writes its velocity to the copies other CTAs hold
// of it (their halos and the neighbours of their halo particles), into one
// of two buffers by sub-step parity.  Per sub-step: force loop and kick
// (own), cluster barrier (the new velocities visible), deformation rate and
// stress (own and halo copies, local reads only), CTA barrier.  A buffer is
// rewritten one sub-step after its last read, and every reader passed a
// cluster barrier in between, so no copy is overwritten while read.
template <bool EARLY>
__device__ __forceinline__ void solid2d_body_1b(const Solid &s, const Phys &P, Ctl *ctl, int ns, float4 *sQ,
                                                float4 *sV, unsigned rank)
{
    constexpr int NB = kMaxNb2, CH = kChunk2;
    constexpr int VS = kC1Threads + kHaloMax;   // one velocity buffer
    const int t = threadIdx.x;
    const int la = (int)rank * kC1Threads + t;
    const int h0 = s.h1_ptr[rank], hn = s.h1_ptr[rank + 1] - h0, hi = t - kC1Threads;
    const bool mine = t < kC1Threads && la < ns;      // an own particle
    const bool copy = t >= kC1Threads && hi < hn;     // a halo particle's copy
    const bool live = mine || copy;
    const int a = mine ? la : (copy ? s.h1_part[h0 + hi] : 0);
    const int self = mine ? t : kC1Threads + hi;      // its slot in sQ and sV
    if (ctl->learned_ok) return;   // the learned step was accepted: no sub-steps
    const int K = ctl->K;
    const double dt = ctl->dt, dtsd = ctl->dts, hdtsd = 0.5 * dtsd;
    const float dts = (float)dtsd, hdts = 0.5f * dts;
    const float inv_rhoS = 1.0f / P.rhoS, inv_mS = 1.0f / P.mS;

    float H[4] = {0, 0, 0, 0}, B[4] = {1, 0, 0, 1}, fF[2] = {0, 0};
    double x = 0, y = 0, xs = 0, ys = 0, as0 = 0, as1 = 0;
    bool cons = true;
    float vmax = 0.0f, amax = 0.0f;
    float4 vown = make_float4(0.f, 0.f, 0.f, 0.f), Qown = vown;
    float gx[NB], gy[NB];
    int sl[NB];              // the neighbour's slot: own or halo (stress and velocity), or second ring (velocity)
    uint32_t pq[kPushMax];   // cluster addresses of this particle's velocity copies (buffer 0)
    int npush = 0, nn = 0;
    if (live) {
        const int q0 = s.nb_ptr[a];
        nn = s.nb_ptr[a + 1] - q0;   // the launcher guarantees nn <= kMaxNb2
        for (int i = 0; i < 4; i++) {
            H[i] = s.H[9 * a + i];
            B[i] = s.B0[9 * a + i];
        }
        const int e0 = mine ? q0 : s.h1_eptr[h0 + hi];
#pragma unroll
        for (int u = 0; u < NB; u++) {
            gx[u] = gy[u] = 0.0f;
            sl[u] = 0;
            if (u < nn) {
                const float4 e = s.nb[q0 + u];
                gx[u] = e.x;
                gy[u] = e.y;
                sl[u] = mine ? s.nb_slot[q0 + u] : s.h1_vslot[e0 + u];
            }
        }
    } else {
#pragma unroll
        for (int u = 0; u < NB; u++) {
            gx[u] = gy[u] = 0.0f;
            sl[u] = 0;
        }
    }
    if (mine) {
        x = xs = s.x[a];
        y = ys = s.y[a];
        cons = s.cons[a] != 0;
        vown = s.v4[a];
        const int p0 = s.push2_ptr[a];
        npush = s.push2_ptr[a + 1] - p0;   // <= kPushMax when this form runs
#pragma unroll
        for (int k = 0; k < kPushMax; k++) {
            pq[k] = 0u;
            if (k < npush) {
                const int2 e = s.push2[p0 + k];
                pq[k] = cl_addr(&sV[e.y], (uint32_t)e.x);
            }
        }
    }
    auto publish_v = [&](int buf, const float4 &v) {
        sV[buf * VS + t] = v;
#pragma unroll
        for (int k = 0; k < kPushMax; k++)
            if (k < npush) st_cl(pq[k] + (uint32_t)(buf * VS * 16), v);
    };
    // v^0 into both buffers: a held particle never writes its copies again
    if (mine) {
        publish_v(0, vown);
        publish_v(1, vown);
    }
    float sgx = 0.f, sgy = 0.f;
#pragma unroll
    for (int u = 0; u < NB; u++) {
        sgx += gx[u];
        sgy += gy[u];
    }
    if constexpr (EARLY) pdl_wait();
    if (mine) {
        fF[0] = s.fF[3 * a];
        fF[1] = s.fF[3 * a + 1];
    }
    cluster_sync();

    // the deformation rate and the stress: the push form's arithmetic in the
    // same order (two accumulator sets, even / odd entries)
    auto rate = [&](float4 va, float *Hd, int vo) {
        float M0 = 0.f, M1 = 0.f, M2 = 0.f, M3 = 0.f, N0 = 0.f, N1 = 0.f, N2 = 0.f, N3 = 0.f;
#pragma unroll
        for (int c0 = 0; c0 < NB; c0 += CH) {
            float2 vb[CH];
#pragma unroll
            for (int u = 0; u < CH; u++) {
                if (c0 + u < nn) {
                    const float4 w = sV[vo + sl[c0 + u]];
                    vb[u] = make_float2(w.x, w.y);
                }
            }
#pragma unroll
            for (int u = 0; u < CH; u += 2) {
                if (c0 + u < nn) {
                    const float dvx = vb[u].x - va.x, dvy = vb[u].y - va.y;
                    M0 += dvx * gx[c0 + u];
                    M1 += dvx * gy[c0 + u];
                    M2 += dvy * gx[c0 + u];
                    M3 += dvy * gy[c0 + u];
                }
                if (u + 1 < CH && c0 + u + 1 < nn) {
                    const float dvx = vb[u + 1].x - va.x, dvy = vb[u + 1].y - va.y;
                    N0 += dvx * gx[c0 + u + 1];
                    N1 += dvx * gy[c0 + u + 1];
                    N2 += dvy * gx[c0 + u + 1];
                    N3 += dvy * gy[c0 + u + 1];
                }
            }
        }
        M0 = M0 + N0;
        M1 = M1 + N1;
        M2 = M2 + N2;
        M3 = M3 + N3;
        Hd[0] = M0 * B[0] + M1 * B[2];
        Hd[1] = M0 * B[1] + M1 * B[3];
        Hd[2] = M2 * B[0] + M3 * B[2];
        Hd[3] = M2 * B[1] + M3 * B[3];
    };
    auto put_Q = [&]() {
        float Q[4];
        stress_QB<2>(H, B, P.mu, P.lam, Q);
        Qown = make_float4(Q[0], Q[1], Q[2], Q[3]);
        sQ[self] = Qown;
    };

    if (live) {
        const float4 va = mine ? vown : sV[self];
        float Hd[4];
        rate(va, Hd, 0);
        for (int i = 0; i < 4; i++) H[i] = H[i] + hdts * Hd[i];
        if (mine && !cons) {
            x = x + hdtsd * (double)va.x;
            y = y + hdtsd * (double)va.y;
        }
        put_Q();
    }
    __syncthreads();
    for (int kk = 0; kk < K; kk++) {
        const int vb_ = (kk + 1) & 1;   // the buffer of v^(k+1)
        // (B) force loop and kick: own particles, stresses from local slots
        if (mine) {
            const float4 Qa = Qown;
            float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
#pragma unroll
            for (int c0 = 0; c0 < NB; c0 += CH) {
                float4 qb[CH];
#pragma unroll
                for (int u = 0; u < CH; u++)
                    if (c0 + u < nn) qb[u] = sQ[sl[c0 + u]];
#pragma unroll
                for (int u = 0; u < CH; u += 2) {
                    if (c0 + u < nn) {
                        ax += qb[u].x * gx[c0 + u] + qb[u].y * gy[c0 + u];
                        ay += qb[u].z * gx[c0 + u] + qb[u].w * gy[c0 + u];
                    }
                    if (u + 1 < CH && c0 + u + 1 < nn) {
                        bx += qb[u + 1].x * gx[c0 + u + 1] + qb[u + 1].y * gy[c0 + u + 1];
                        by += qb[u + 1].z * gx[c0 + u + 1] + qb[u + 1].w * gy[c0 + u + 1];
                    }
                }
            }
            ax = Qa.x * sgx + Qa.y * sgy + (ax + bx);
            ay = Qa.z * sgx + Qa.w * sgy + (ay + by);
            if (!cons) {
                float4 v = vown;
                float av0 = ax * inv_rhoS + fF[0] * inv_mS + P.g[0];
                float av1 = ay * inv_rhoS + fF[1] * inv_mS + P.g[1];
                v.x += dts * av0;
                v.y += dts * av1;
                vown = v;
                publish_v(vb_, v);
                as0 += dtsd * (double)av0;
                as1 += dtsd * (double)av1;
                amax = max_keep_nan(amax, av0 * av0 + av1 * av1);
                vmax = max_keep_nan(vmax, v.x * v.x + v.y * v.y);
            }
        }
        cluster_sync();
        // (C) deformation rate at v^{k+1} (own particles and halo copies);
        // second half drift; next first half and stress
        if (live) {
            const bool more = kk + 1 < K;
            const float4 va = mine ? vown : sV[vb_ * VS + self];
            float Hd[4];
            rate(va, Hd, vb_ * VS);
            const float hH = more ? dts : hdts;
            const double hX = more ? dtsd : hdtsd;
            for (int i = 0; i < 4; i++) H[i] = H[i] + hH * Hd[i];
            if (more) put_Q();
            if (mine && !cons) {
                x = x + hX * (double)va.x;
                y = y + hX * (double)va.y;
            }
        }
        __syncthreads();
    }
    if (mine) {
        for (int i = 0; i < 4; i++) s.H[9 * a + i] = H[i];
        s.v4[a] = vown;
        s.x[a] = x;
        s.y[a] = y;
        const double idt = 1.0 / dt;
        s.vbar[3 * a] = (x - xs) * idt;
        s.vbar[3 * a + 1] = (y - ys) * idt;
        s.vbar[3 * a + 2] = 0.0;
        s.abar[3 * a] = as0 * idt;
        s.abar[3 * a + 1] = as1 * idt;
        s.abar[3 * a + 2] = 0.0;
    }
    float vm = warp_max(vmax), am = warp_max(amax);
    if ((threadIdx.x & 31) == 0) {
        atomic_max_pos(&ctl->vmaxS, sqrtf(vm));
        atomic_max_pos(&ctl->amaxS, sqrtf(am));
    }
    cluster_sync();
}

// shared arrays of the 2-D body: own slots, plus halo slots in the push
// forms, twice over in the mbarrier form (double-buffered)
template <int MODE>
__host__ __device__ constexpr int solid2d_slots()
{
    return (kC1Threads + (MODE ? kHaloMax : 0)) * (MODE == 2 ? 2 : 1);
}

// mbarrier form: each CTA's four mbarriers (stress and velocity copies, two
// buffers each), initialised once and visible cluster-wide before any copy
template <int MODE>
__device__ __forceinline__ void solid2d_mbar_setup(uint64_t *mb)
{
    if constexpr (MODE == 2) {
        if (threadIdx.x == 0) {
            for (int i = 0; i < 4; i++) mbar_init(&mb[i], 1u);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        cluster_sync();
    }
}

template <int LP, int MODE>
__global__ void __launch_bounds__(kC1Threads * LP) k_solid_cluster2d(Batch bt, Solid s)
{
    pdl_enter();
    __shared__ float4 sQ[solid2d_slots<MODE>()];
    __shared__ float4 sV[solid2d_slots<MODE>()];
    __shared__ __align__(8) uint64_t mb[4];
    __shared__ int s_inst;
    const unsigned rank = cluster_rank();
    unsigned phs = 0u;
    solid2d_mbar_setup<MODE>(mb);
    for (;;) {
        const int b = next_instance(s.queue, &s_inst, rank);
        if (b >= bt.B) break;
        const Inst &In = bt.I[b];
        solid2d_body<LP, MODE>(s, In.P, bt.ctl + b, In.s0, In.ns, sQ, sV, rank, mb,
                               MODE ? s.halo_n[b * kClusterMax + rank] : 0, phs);
    }
}

// single instance: one cluster, constants in the parameter space (the
// persistent kernel's global-memory constants cost registers)
// With LP = 1 it may be launched with 2 kC1Threads threads, the second half
// idle: the CTA then holds its SM's registers, so no fluid block of the
// concurrent main-stream loops shares the SM with the sub-steps.
template <int LP, int MODE>
__global__ void __launch_bounds__(kC1Threads * 2) k_solid_cluster2d_one(Solid s, const __grid_constant__ Phys P,
                                                                        Ctl *ctl)
{
    // the wait for the coupling-force kernel comes inside the body, after
    // the prologue (EARLY)
    pdl_trigger();
    __shared__ float4 sQ[solid2d_slots<MODE>()];
    __shared__ float4 sV[solid2d_slots<MODE>()];
    __shared__ __align__(8) uint64_t mb[4];
    const unsigned rank = cluster_rank();
    unsigned phs = 0u;
    solid2d_mbar_setup<MODE>(mb);
    solid2d_body<LP, MODE, true>(s, P, ctl, 0, s.n, sQ, sV, rank, mb, MODE ? s.halo_n[rank] : 0, phs);
}

// one-barrier form (solid variant 5): one cluster, 2 kC1Threads threads per
// CTA (own particles, then the halo copies)
__global__ void __launch_bounds__(kC1Threads * 2) k_solid_cluster2d_1b(Solid s, const __grid_constant__ Phys P,
                                                                       Ctl *ctl)
{
    pdl_trigger();   // the wait for the coupling-force kernel comes after the prologue
    __shared__ float4 sQ[2 * kC1Threads];
    __shared__ float4 sV[2 * (kC1Threads + kHaloMax)];
    solid2d_body_1b<true>(s, P, ctl, s.n, sQ, sV, cluster_rank());
}

// Launch `want` clusters of `ctas` CTAs (at most as many as can be resident)
// with kernel arguments args.  Returns 1 when the device cannot run such a
// cluster (the caller falls back), else 0 or -3.
template <typename Kern, typename... Args>
static int launch_clusters(Kern kern, int threads, int ctas, int want, int *max_clusters, cudaStream_t st,
                           Args... args)
{
    if (ctas < 1 || ctas > kClusterMax) return 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(threads);
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;   // the occupancy query below sees the cluster shape only
    if (max_clusters[ctas] == 0) {
        int nclu = 0;
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaError_t e = cudaOccupancyMaxActiveClusters(&nclu, kern, &cfg);
        if (e != cudaSuccess) cudaGetLastError();
        max_clusters[ctas] = (e == cudaSuccess && nclu >= 1) ? nclu : -1;
    }
    if (max_clusters[ctas] < 0) return 1;
    int nclusters = want < max_clusters[ctas] ? want : max_clusters[ctas];
    cfg.gridDim = dim3(nclusters * ctas);
    cfg.numAttrs = kPDL ? 2 : 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    return e == cudaSuccess ? 0 : -3;
}

// Launch a persistent cluster kernel: as many clusters as can be resident,
// at most one per instance, taking instances from the queue.
template <typename Kern>
static int launch_persistent(Kern kern, int threads, int ctas, const Batch &bt, Solid &s, int *max_clusters,
                             cudaStream_t st)
{
    if (ctas < 1 || ctas > kClusterMax) return 1;
    if (cudaMemsetAsync(s.queue, 0, sizeof(unsigned), st) != cudaSuccess) return -3;
    return launch_clusters(kern, threads, ctas, bt.B, max_clusters, st, bt, s);
}

// 1: the single-body push-form kernels run with idle padding threads (see
// k_solid_cluster2d_one)
constexpr int kPadSolidOne = 1;

static int launch_solid_cluster(const Batch &bt, Solid &s, const Phys &P0, int dim, cudaStream_t st, int *path)
{
    *path = 1;
    static int mc2d[11][kClusterMax + 1] = {}, mcl[4][kClusterMax + 1] = {};
    const bool one = bt.B == 1;
    if (dim == 2 && s.force_lane_path != 1 && s.max_nb <= kMaxNb2) {
        const int ctas = (s.max_ns + kC1Threads - 1) / kC1Threads;
        int rc;
        // solid variants: 0 one thread per particle, 2 two threads, both with
        // halo copies and cluster barriers where the halos fit; 3 pull form;
        // 4 halo copies awaited on mbarriers (correct, measured slower); 5 the
        // one-barrier form (a single body whose halos fit; else as 0)
        int v = s.force_lane_path;
        if (v == 5) {
            if (one && s.push_ok && s.one_ok) {
                const int r1 =
                    launch_clusters(k_solid_cluster2d_1b, 2 * kC1Threads, ctas, 1, mc2d[10], st, s, P0, bt.ctl);
                if (r1 <= 0) {
                    *path = 3;
                    return r1;
                }
            }
            v = 0;
        }
        const int mode = !s.push_ok || v == 3 ? 0 : (v == 4 ? 2 : 1);
        const int pad = kPadSolidOne ? 2 : 1;
        if (v == 2) {   // two threads per particle
            if (mode == 1)
                rc = one ? launch_clusters(k_solid_cluster2d_one<2, 1>, 2 * kC1Threads, ctas, 1, mc2d[0], st, s, P0,
                                           bt.ctl)
                         : launch_persistent(k_solid_cluster2d<2, 1>, 2 * kC1Threads, ctas, bt, s, mc2d[1], st);
            else
                rc = one ? launch_clusters(k_solid_cluster2d_one<2, 0>, 2 * kC1Threads, ctas, 1, mc2d[2], st, s, P0,
                                           bt.ctl)
                         : launch_persistent(k_solid_cluster2d<2, 0>, 2 * kC1Threads, ctas, bt, s, mc2d[3], st);
        } else if (mode == 2) {
            rc = one ? launch_clusters(k_solid_cluster2d_one<1, 2>, kC1Threads * pad, ctas, 1, mc2d[4], st, s, P0,
                                       bt.ctl)
                     : launch_persistent(k_solid_cluster2d<1, 2>, kC1Threads, ctas, bt, s, mc2d[5], st);
        } else if (mode == 1) {
            rc = one ? launch_clusters(k_solid_cluster2d_one<1, 1>, kC1Threads * pad, ctas, 1, mc2d[6], st, s, P0,
                                       bt.ctl)
                     : launch_persistent(k_solid_cluster2d<1, 1>, kC1Threads, ctas, bt, s, mc2d[7], st);
        } else {
            rc = one ? launch_clusters(k_solid_cluster2d_one<1, 0>, kC1Threads, ctas, 1, mc2d[8], st, s, P0, bt.ctl)
                     : launch_persistent(k_solid_cluster2d<1, 0>, kC1Threads, ctas, bt, s, mc2d[9], st);
        }
        if (rc <= 0) return rc;
    }
    const int ctas = (s.max_ns + kPPC - 1) / kPPC;
    if (one) {
        if (dim == 2) return launch_clusters(k_solid_cluster_one<2>, kCThreads, ctas, 1, mcl[0], st, s, P0, bt.ctl);
        return launch_clusters(k_solid_cluster_one<3>, kCThreads, ctas, 1, mcl[1], st, s, P0, bt.ctl);
    }
    if (dim == 2) return launch_persistent(k_solid_cluster<2>, kCThreads, ctas, bt, s, mcl[2], st);
    return launch_persistent(k_solid_cluster<3>, kCThreads, ctas, bt, s, mcl[3], st);
}

int launch_solid_substeps(const Batch &bt, Solid &s, const Phys &P0, int dim, int *path, cudaStream_t st)
{
    if (s.n == 0) return 0;
    if (!s.force_grid_path) {
        int cp = 1;
        int rc = launch_solid_cluster(bt, s, P0, dim, st, &cp);
        if (rc <= 0) {
            if (path) *path = cp;
            return rc;
        }
    }
    // cooperative grid kernel: one large body (a batch needs the cluster path)
    if (bt.B != 1) return -7;
    static int max_blocks[2] = {0, 0};
    int di = dim == 2 ? 0 : 1;
    if (max_blocks[di] == 0) {
        int dev, nsm, per;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (dim == 2)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solid_substeps<2>, kSolidBlock, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solid_substeps<3>, kSolidBlock, 0);
        max_blocks[di] = per * nsm;
    }
    int nb = (s.n + kSolidBlock - 1) / kSolidBlock;
    if (nb > max_blocks[di]) nb = max_blocks[di];
    if (nb < 1) return -3;
    cudaMemsetAsync(s.bar, 0, sizeof(unsigned), st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(kSolidBlock);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (dim == 2) e = cudaLaunchKernelEx(&cfg, k_solid_substeps<2>, bt, s);
    else e = cudaLaunchKernelEx(&cfg, k_solid_substeps<3>, bt, s);
    if (path) *path = 2;
    return e == cudaSuccess ? 0 : -3;
}

// ---------------------------------------------------------------------------
// Learned sub-stepper (the paper has none): the network proposes the step's
// displacement and velocity change of every particle; the proposal is kept
// only if its momentum-balance residual over the body,
//   R = |m (v' - v) - dt (f_int(x_mid) + f^F + m g)| / |m v'|
// with x_mid = r + du / 2 and f_int one plain force evaluation (F from the
// positions, Eq. correctmatrix; neo-Hookean P B0; force loop), is at most the
// threshold; else the plain sub-steps run (they test ctl->learned_ok).
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_learn_features(Batch bt, Solid s, float *x)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= s.n) return;
    const Ctl &ctl = bt.ctl[s.inst[a]];
    float *row = x + (size_t)a * 64;
    const double u[3] = {s.x[a] - s.x0[a], s.y[a] - s.y0[a], D == 3 ? s.z[a] - s.z0[a] : 0.0};
    const float4 v = s.v4[a];
    const float vv[3] = {v.x, v.y, v.z};
    int o = 0;
    for (int k = 0; k < D; k++) row[o++] = (float)(u[k] / (double)s.l_su);
    for (int k = 0; k < D; k++) row[o++] = vv[k] / s.l_sv;
    for (int k = 0; k < D * D; k++) row[o++] = s.H[9 * a + k] / s.l_sH;
    for (int k = 0; k < D; k++) row[o++] = s.fF[3 * a + k] / s.l_sf;
    row[o++] = s.cons[a] ? 1.0f : 0.0f;
    row[o++] = (float)(ctl.dt / (double)s.l_st);
}

// candidate end and mid states from the outputs
template <int D>
__global__ void k_learn_apply(Batch bt, Solid s, const float *__restrict__ out)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= s.n) return;
    const int b = s.inst[a];
    const Phys &P = bt.I[b].P;
    const double dt = bt.ctl[b].dt;
    const float4 v = s.v4[a];
    const float vv[3] = {v.x, v.y, v.z};
    const float *y = out + (size_t)a * 16;
    double du[3] = {0.0, 0.0, 0.0};
    float vn[3] = {0.f, 0.f, 0.f};
    if (!s.cons[a]) {
        for (int k = 0; k < D; k++) {
            du[k] = dt * (double)vv[k] + (double)s.l_sdu * (double)y[k];
            const float dv = (float)dt * (s.fF[3 * a + k] / P.mS + P.g[k]) + s.l_sdv * y[D + k];
            vn[k] = vv[k] + dv;
        }
    }
    s.lx[a] = s.x[a] + du[0];
    s.ly[a] = s.y[a] + du[1];
    s.mx[a] = s.x[a] + 0.5 * du[0];
    s.my[a] = s.y[a] + 0.5 * du[1];
    if (D == 3) {
        s.lz[a] = s.z[a] + du[2];
        s.mz[a] = s.z[a] + 0.5 * du[2];
    }
    s.lv4[a] = make_float4(vn[0], vn[1], vn[2], 0.0f);
}

// H = [sum_b ((p_b - p_a) - (X_b - X_a)) (x) V0 grad0_a W_ab] B0 at the mid
// positions (-> P B0) and at the end positions (-> lH)
template <int D>
__global__ void k_learn_stress(Batch bt, Solid s)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= s.n) return;
    const Phys &P = bt.I[s.inst[a]].P;
    float Gm[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, Ge[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double Xa[3] = {s.x0[a], s.y0[a], D == 3 ? s.z0[a] : 0.0};
    const double Ma[3] = {s.mx[a], s.my[a], D == 3 ? s.mz[a] : 0.0};
    const double Ea[3] = {s.lx[a], s.ly[a], D == 3 ? s.lz[a] : 0.0};
    for (int q = s.nb_ptr[a]; q < s.nb_ptr[a + 1]; q++) {
        const float4 e = s.nb[q];
        const int b = __float_as_int(e.w);
        const float g[3] = {e.x, e.y, e.z};
        const double Xb[3] = {s.x0[b], s.y0[b], D == 3 ? s.z0[b] : 0.0};
        const double Mb[3] = {s.mx[b], s.my[b], D == 3 ? s.mz[b] : 0.0};
        const double Eb[3] = {s.lx[b], s.ly[b], D == 3 ? s.lz[b] : 0.0};
        for (int i = 0; i < D; i++) {
            const float dm = (float)((Mb[i] - Ma[i]) - (Xb[i] - Xa[i]));
            const float de = (float)((Eb[i] - Ea[i]) - (Xb[i] - Xa[i]));
            for (int j = 0; j < D; j++) {
                Gm[i * D + j] += dm * g[j];
                Ge[i * D + j] += de * g[j];
            }
        }
    }
    const float *B = s.B0 + 9 * a;
    float Hm[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < D; i++)
        for (int j = 0; j < D; j++) {
            float hm = 0.f, he = 0.f;
            for (int k = 0; k < D; k++) {
                hm += Gm[i * D + k] * B[k * D + j];
                he += Ge[i * D + k] * B[k * D + j];
            }
            Hm[i * D + j] = hm;
            s.lH[9 * a + i * D + j] = he;
        }
    float Q[9];
    stress_QB<D>(Hm, B, P.mu, P.lam, Q);
    store_Q<D>(s.lQ, a, Q);
}

// residual sums of the instance (free particles)
template <int D>
__global__ void k_learn_residual(Batch bt, Solid s)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= s.n || s.cons[a]) return;
    const int b = s.inst[a];
    const Phys &P = bt.I[b].P;
    Ctl *ctl = bt.ctl + b;
    float Qa[9];
    load_Q<D>(s.lQ, a, Qa);
    float acc[3] = {0.f, 0.f, 0.f};
    for (int q = s.nb_ptr[a]; q < s.nb_ptr[a + 1]; q++) {
        const float4 e = s.nb[q];
        const int c = __float_as_int(e.w);
        const float g[3] = {e.x, e.y, e.z};
        float Qb[9];
        load_Q<D>(s.lQ, c, Qb);
        for (int i = 0; i < D; i++)
            for (int j = 0; j < D; j++) acc[i] += (Qa[i * D + j] + Qb[i * D + j]) * g[j];
    }
    const float4 v = s.v4[a], vn = s.lv4[a];
    const float vv[3] = {v.x, v.y, v.z}, vnn[3] = {vn.x, vn.y, vn.z};
    const float dt = (float)ctl->dt;
    double num = 0.0, den = 0.0;
    for (int k = 0; k < D; k++) {
        const float f = acc[k] / P.rhoS + s.fF[3 * a + k] / P.mS + P.g[k];
        const double e = (double)(vnn[k] - vv[k]) - (double)dt * (double)f;
        num += e * e;
        den += (double)vnn[k] * (double)vnn[k];
    }
    atomicAdd(&ctl->lnum, num);
    atomicAdd(&ctl->lden, den);
}

// accept (commit the candidate, time averages, maxima) or reject
template <int D>
__global__ void k_learn_commit(Batch bt, Solid s)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= s.n) return;
    const int b = s.inst[a];
    Ctl *ctl = bt.ctl + b;
    const double R = sqrt(ctl->lnum) / (sqrt(ctl->lden) + 1e-30);
    const bool ok = R <= (double)s.l_tol;
    if (a == bt.I[b].s0) {
        ctl->learned_ok = ok ? 1 : 0;
        ctl->l_res = R;
    }
    if (!ok) return;
    const double dt = ctl->dt, idt = 1.0 / dt;
    const float4 v = s.v4[a], vn = s.lv4[a];
    const double xe[3] = {s.lx[a], s.ly[a], D == 3 ? s.lz[a] : 0.0};
    const double xs[3] = {s.x[a], s.y[a], D == 3 ? s.z[a] : 0.0};
    const float vv[3] = {v.x, v.y, v.z}, vnn[3] = {vn.x, vn.y, vn.z};
    float vm = 0.f, am = 0.f;
    for (int k = 0; k < 3; k++) {
        const double vb = k < D ? (xe[k] - xs[k]) * idt : 0.0;
        const double ab = k < D ? ((double)vnn[k] - (double)vv[k]) * idt : 0.0;
        s.vbar[3 * a + k] = vb;
        s.abar[3 * a + k] = ab;
        vm += vnn[k] * vnn[k];
        am += (float)(ab * ab);
    }
    s.x[a] = xe[0];
    s.y[a] = xe[1];
    if (D == 3) s.z[a] = xe[2];
    s.v4[a] = vn;
    for (int k = 0; k < D * D; k++) s.H[9 * a + k] = s.lH[9 * a + k];
    atomic_max_pos(&ctl->vmaxS, sqrtf(vm));
    atomic_max_pos(&ctl->amaxS, sqrtf(am));
}

int launch_learn_features(const Batch &bt, const Solid &s, float *x, int dim, cudaStream_t st)
{
    if (s.n == 0) return 0;
    const int nb = (s.n + kBlock - 1) / kBlock;
    if (dim == 2) k_learn_features<2><<<nb, kBlock, 0, st>>>(bt, s, x);
    else k_learn_features<3><<<nb, kBlock, 0, st>>>(bt, s, x);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_learn_candidate(const Batch &bt, const Solid &s, const float *out, int dim, cudaStream_t st)
{
    if (s.n == 0) return 0;
    const int nb = (s.n + kBlock - 1) / kBlock;
    if (dim == 2) {
        k_learn_apply<2><<<nb, kBlock, 0, st>>>(bt, s, out);
        k_learn_stress<2><<<nb, kBlock, 0, st>>>(bt, s);
        k_learn_residual<2><<<nb, kBlock, 0, st>>>(bt, s);
        k_learn_commit<2><<<nb, kBlock, 0, st>>>(bt, s);
    } else {
        k_learn_apply<3><<<nb, kBlock, 0, st>>>(bt, s, out);
        k_learn_stress<3><<<nb, kBlock, 0, st>>>(bt, s);
        k_learn_residual<3><<<nb, kBlock, 0, st>>>(bt, s);
        k_learn_commit<3><<<nb, kBlock, 0, st>>>(bt, s);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace sph
