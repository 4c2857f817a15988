// Tensor-core GEMM of the learned sub-stepper (5th-generation tensor cores):
//   C[M x N] (FP32) = A[M x K] . B[N x K]^T (+ bias[N]),  A, B bfloat16,
// both row-major with K contiguous ("K-major").  M % 128 == 0, N % 16 == 0,
// K % 64 == 0 (callers pad).
//
// One CTA of 128 threads computes a 128 x NT tile with a single-thread-issued
// tcgen05.mma (kind::f16, M = 128, N = NT, K = 16 per instruction) into an
// FP32 accumulator in tensor memory.  K advances in chunks of 64 through two
// shared-memory stages: all threads copy a chunk of A (128 x 64) and B
// (NT x 64) into the canonical no-swizzle K-major layout (core matrices of
// 8 rows x 16 bytes; LBO = 128 B between core matrices along K, SBO = 1 KB
// between 8-row groups), the issuing thread launches 4 MMAs and commits them
// to the stage's mbarrier, and the stage is refilled only after that
// mbarrier fires.  The epilogue reads the accumulator with tcgen05.ld
// (warp w owns TMEM lanes 32w..32w+31 = tile rows), adds the bias and stores
// FP32.  Every wait is bounded; a timeout sets a status bit, skips the
// epilogue and still frees the tensor memory.
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

// shared-memory matrix descriptor: start address, leading (K) and stride
// (8-row group) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
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

template <int NT>
__global__ void __launch_bounds__(kTcThreads) k_gemm_bf16(const uint4 *__restrict__ A, const uint4 *__restrict__ B,
                                                          const float *__restrict__ bias, float *__restrict__ C,
                                                          int M, int N, int K)
{
    constexpr int kBStage = NT * kKChunk * 2;
    constexpr int kStage = kAStage + kBStage;
    constexpr uint32_t kCols = NT < 32 ? 32 : NT;   // tensor-memory columns (power of 2 >= 32)
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t s_tmem;
    // 1 KB aligned stage buffers
    const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
    uint8_t *const gbase = dsm + (base - smem_u32(dsm));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT;
    const int kq = K >> 3;   // 16-byte pieces per row

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    const int nk = K / kKChunk;
    uint32_t phase[2] = {0u, 0u};
    bool ok = true;
    for (int kc = 0; kc < nk && ok; kc++) {
        const int s = kc & 1;
        if (kc >= 2) {
            ok = __syncthreads_and(mbar_wait(smem_u32(&mbar[s]), phase[s]));   // CTA-uniform
            phase[s] ^= 1u;
            if (!ok) break;
        }
        uint8_t *As = gbase + s * kStage;
        uint8_t *Bs = As + kAStage;
        // piece p: row p / 8, 16-byte column group p % 8 of the chunk
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int p = tid + kTcThreads * i;
            const int r = p >> 3, kg = p & 7;
            const uint4 v = A[(size_t)(m0 + r) * kq + kc * 8 + kg];
            *(uint4 *)(As + (r >> 3) * 1024 + kg * 128 + (r & 7) * 16) = v;
        }
        for (int p = tid; p < NT * 8; p += kTcThreads) {
            const int r = p >> 3, kg = p & 7;
            const uint4 v = B[(size_t)(n0 + r) * kq + kc * 8 + kg];
            *(uint4 *)(Bs + (r >> 3) * 1024 + kg * 128 + (r & 7) * 16) = v;
        }
        // generic-proxy writes -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = base + s * kStage, b0 = a0 + kAStage;
#pragma unroll
            for (int kk = 0; kk < kKChunk / 16; kk++) {
                const uint64_t ad = sdesc(a0 + kk * 256, 128, 1024);
                const uint64_t bd = sdesc(b0 + kk * 256, 128, 1024);
                const uint32_t acc = (kc | kk) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc_bf16(128, NT)), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[s]))
                         : "memory");
        }
    }
    // the last commit covers every MMA issued before it
    if (ok && nk > 0) {
        const int s = (nk - 1) & 1;
        ok = mbar_wait(smem_u32(&mbar[s]), phase[s]);
    }
    ok = __syncthreads_and(ok);
    // a CTA whose wait ran out must not free tensor memory under MMAs in
    // flight: wait (bounded) once more for both stages before leaving
    if (!ok) {
        mbar_wait(smem_u32(&mbar[0]), phase[0]);
        mbar_wait(smem_u32(&mbar[1]), phase[1]);
        if (lane == 0) atomicOr(&g_tc_status, 1u);
    }
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
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

template <int NT>
int launch_tile(const uint16_t *A, const uint16_t *B, const float *bias, float *C, int M, int N, int K,
                cudaStream_t st)
{
    constexpr int kStage = kAStage + NT * kKChunk * 2;
    // two stages + alignment slack; at least 64 KB so that at most three
    // CTAs share an SM (3 x 128 tensor-memory columns <= 512)
    int smem = 2 * kStage + 1024;
    if (smem < 64 * 1024) smem = 64 * 1024;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_gemm_bf16<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return -3;
        attr_set = true;
    }
    dim3 grid(M / 128, N / NT);
    k_gemm_bf16<NT><<<grid, kTcThreads, smem, st>>>((const uint4 *)A, (const uint4 *)B, bias, C, M, N, K);
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
