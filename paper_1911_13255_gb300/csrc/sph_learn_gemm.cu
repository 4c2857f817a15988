// Tensor-core GEMM of the learned sub-stepper (5th-generation tensor cores):
//   C[M x N] (FP32) = A[M x K] . B[N x K]^T (+ bias[N]),  A, B bfloat16,
// both row-major with K contiguous ("K-major").  M % 128 == 0, N % 16 == 0,
// K % 64 == 0 (callers pad).
//
// One CTA of 128 threads computes a 128 x NT tile into an FP32 accumulator in
// tensor memory.  K advances in chunks of 64 through a ring of four
// shared-memory stages:
//   - warp 0 (one thread) is the producer: it waits until a stage is empty,
//     arms the stage's "full" mbarrier with the byte count and issues two TMA
//     tile loads (cp.async.bulk.tensor.2d, 128-byte swizzle) of A (128 x 64)
//     and B (NT x 64);
//   - warp 1 (one thread) issues the MMAs: it waits until a stage is full,
//     launches 4 tcgen05.mma (kind::f16, M = 128, N = NT, K = 16; shared-memory
//     descriptors in the 128-byte-swizzle K-major layout, 1 KB between 8-row
//     groups, +32 B per K step inside the swizzle atom) and commits them to the
//     stage's "empty" mbarrier; after the last chunk it commits to "done";
//   - all four warps wait for "done", read the accumulator with tcgen05.ld
//     (warp w owns TMEM lanes 32w..32w+31 = tile rows), add the bias and store.
// Every wait is bounded; a timeout sets a status bit, skips the epilogue and
// still frees the tensor memory.
#include <cuda.h>   // CUtensorMap and its enums; the encoder comes from the CUDA driver library at run time
#include <algorithm>
#include <cuda_bf16.h>
#include <stdint.h>

#include "sph_common.cuh"
#include "sph_learn.cuh"

namespace sph {

__device__ unsigned g_tc_status;   // bit 0: a bounded tensor-core wait ran out

namespace {

constexpr int kTcThreads = 128;
constexpr int kKChunk = 64;                 // K elements per stage
constexpr int kAStage = 128 * kKChunk * 2;  // bytes of A per stage (16 KB)
constexpr long long kMbarSpin = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    for (long long i = 0; i < kMbarSpin; i++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// shared-memory matrix descriptor, 128-byte swizzle, K-major: start address,
// leading byte offset 16 (not used by this layout), stride 1 KB between
// 8-row groups, descriptor version 1, layout type 2 (128-byte swizzle)
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

constexpr int kStages = 4;

template <int NT>
__global__ void __launch_bounds__(kTcThreads) k_gemm_bf16(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB,
                                                          const float *__restrict__ bias, float *__restrict__ C,
                                                          int M, int N, int K, int kper)
{
    // split K: slice blockIdx.z covers chunks [z kper, (z + 1) kper) and
    // writes its partial tile to C + z M N (the caller reduces the slices)
    C += (size_t)blockIdx.z * M * N;
    constexpr int kBStage = NT * kKChunk * 2;
    constexpr int kStage = kAStage + kBStage;        // a multiple of 1 KB
    constexpr uint32_t kCols = NT < 32 ? 32 : NT;   // tensor-memory columns (power of 2 >= 32)
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t s_tmem;
    const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT;
    const int kc0 = blockIdx.z * kper;
    const int nk = min(K / kKChunk - kc0, kper);

    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; s++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    bool ok = true;
    if (warp == 0 && lane == 0) {
        // producer
        uint32_t ph[kStages] = {0u, 0u, 0u, 0u};
        for (int kc = 0; kc < nk; kc++) {
            const int s = kc % kStages;
            if (kc >= kStages) {
                if (!mbar_wait(smem_u32(&empty[s]), ph[s])) {
                    ok = false;
                    break;
                }
                ph[s] ^= 1u;
            }
            const uint32_t a_s = base + s * kStage, b_s = a_s + kAStage, fb = smem_u32(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kStage) : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];" ::"r"(a_s),
                "l"(reinterpret_cast<uint64_t>(&tmA)), "r"((kc0 + kc) * kKChunk), "r"(m0), "r"(fb)
                : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];" ::"r"(b_s),
                "l"(reinterpret_cast<uint64_t>(&tmB)), "r"((kc0 + kc) * kKChunk), "r"(n0), "r"(fb)
                : "memory");
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        uint32_t ph[kStages] = {0u, 0u, 0u, 0u};
        for (int kc = 0; kc < nk; kc++) {
            const int s = kc % kStages;
            if (!mbar_wait(smem_u32(&full[s]), ph[s])) {
                ok = false;
                break;
            }
            ph[s] ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = base + s * kStage, b0 = a0 + kAStage;
#pragma unroll
            for (int kk = 0; kk < kKChunk / 16; kk++) {
                const uint64_t ad = sdesc_sw128(a0 + kk * 32);
                const uint64_t bd = sdesc_sw128(b0 + kk * 32);
                const uint32_t acc = (kc | kk) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc_bf16(128, NT)), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        // covers every MMA issued before it (arrives at once if there is none)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&done))
                     : "memory");
    }
    if (!mbar_wait(smem_u32(&done), 0u)) ok = false;
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0) atomicOr(&g_tc_status, 1u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < NT; c += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float4 *out = (float4 *)(C + (size_t)row * N + n0 + c);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                float4 o = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                       __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
                if (bias) {
                    o.x += bias[n0 + c + 4 * j];
                    o.y += bias[n0 + c + 4 * j + 1];
                    o.z += bias[n0 + c + 4 * j + 2];
                    o.w += bias[n0 + c + 4 * j + 3];
                }
                out[j] = o;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D tensor map of a row-major bfloat16 matrix (rows x cols), box 64 x box_rows
int make_map(CUtensorMap *m, const void *ptr, long long rows, long long cols, int box_rows)
{
    EncodeTiled enc = encoder();
    if (!enc) return -3;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kKChunk, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

// C = bias + sum of the S partial tiles, in slice order (deterministic)
__global__ void k_splitk_sum(const float *__restrict__ ws, int S, long long MN, int N, const float *__restrict__ bias,
                             float *__restrict__ C)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MN) return;
    float v = bias ? bias[i % N] : 0.0f;
    for (int z = 0; z < S; z++) v += ws[(size_t)z * MN + i];
    C[i] = v;
}

// split-K workspace, grown on demand outside stream capture
float *g_ws = nullptr;
size_t g_ws_floats = 0;

template <int NT>
int launch_tile(const uint16_t *A, const uint16_t *B, const float *bias, float *C, int M, int N, int K,
                cudaStream_t st)
{
    constexpr int kStage = kAStage + NT * kKChunk * 2;
    const int smem = kStages * kStage + 1024;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_gemm_bf16<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return -3;
        attr_set = true;
    }
    alignas(64) CUtensorMap ta, tb;
    int rc = make_map(&ta, A, M, K, 128);
    if (!rc) rc = make_map(&tb, B, N, K, NT);
    if (rc) return rc;
    // few output tiles and a long K loop: split K over up to 152 CTAs
    const int tiles = (M / 128) * (N / NT), nk = K / kKChunk;
    int S = 1;
    if (tiles < 76 && nk >= 16) {
        S = std::min(152 / tiles, nk / 8);
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cap);
        const size_t need = (size_t)S * M * N;
        if (S > 1 && cap == cudaStreamCaptureStatusNone && need > g_ws_floats) {
            if (g_ws) cudaFree(g_ws);
            g_ws = nullptr;
            g_ws_floats = 0;
            if (cudaMalloc(&g_ws, need * sizeof(float)) == cudaSuccess) g_ws_floats = need;
            else cudaGetLastError();
        }
        if (S < 2 || need > g_ws_floats) S = 1;
    }
    const int kper = (nk + S - 1) / S;
    S = (nk + kper - 1) / kper;
    dim3 grid(M / 128, N / NT, S);
    if (S == 1) {
        k_gemm_bf16<NT><<<grid, kTcThreads, smem, st>>>(ta, tb, bias, C, M, N, K, kper);
    } else {
        k_gemm_bf16<NT><<<grid, kTcThreads, smem, st>>>(ta, tb, nullptr, g_ws, M, N, K, kper);
        const long long MN = (long long)M * N;
        k_splitk_sum<<<(unsigned)((MN + 255) / 256), 256, 0, st>>>(g_ws, S, MN, N, bias, C);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace

int launch_gemm_bf16(const uint16_t *A, const uint16_t *B, const float *bias, float *C, long long M, long long N,
                     long long K, cudaStream_t st)
{
    if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 16 || K % kKChunk) return -1;
    if (M / 128 > 65535 * 1024LL || K > (1LL << 30) || N > (1LL << 30)) return -7;
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C) & 15) return -1;
    const int m = (int)M, n = (int)N, k = (int)K;
    if (n % 256 == 0) return launch_tile<256>(A, B, bias, C, m, n, k, st);
    if (n % 128 == 0) return launch_tile<128>(A, B, bias, C, m, n, k, st);
    if (n % 64 == 0) return launch_tile<64>(A, B, bias, C, m, n, k, st);
    if (n % 32 == 0) return launch_tile<32>(A, B, bias, C, m, n, k, st);
    return launch_tile<16>(A, B, bias, C, m, n, k, st);
}

int read_tc_status(unsigned *out, bool reset)
{
    if (cudaMemcpyFromSymbol(out, g_tc_status, sizeof(unsigned)) != cudaSuccess) return -3;
    if (reset) {
        unsigned z = 0;
        if (cudaMemcpyToSymbol(g_tc_status, &z, sizeof(unsigned)) != cudaSuccess) return -3;
    }
    return 0;
}

}  // namespace sph
