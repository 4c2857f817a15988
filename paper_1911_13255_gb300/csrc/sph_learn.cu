// Learned solid sub-stepper: a message-passing network over a body's static
// reference-configuration neighbour graph (the network the paper does not
// have; its FP64 statement is the oracle's mpnn module):
//
//   h   = silu(x W_enc^T + b_enc)                         x: N x 64 features
//   3x  z = [h, sum_b w_ab (h_b - h_a), sum_b g_ab,k (h_b - h_a) (k < dim)]
//       h = h + silu(z W_l^T + b_l)
//   out = h W_dec^T + b_dec                                (N x 16)
//
// Dense products run on the tensor cores (sph_learn_gemm.cu, bfloat16
// operands, FP32 accumulation); the graph sums, activations, loss, bias
// gradients and Adam run on the CUDA cores in FP32.  Operands are rounded to
// bfloat16 exactly where they enter a GEMM.  A context replicates one body's
// graph R times (block diagonal) so that R samples form one batch.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "sph_common.cuh"
#include "sph_learn.cuh"
#include "sphfsi.h"

using namespace sph;

namespace {

constexpr int kC = 128;     // hidden width
constexpr int kFin = 64;    // padded input width
constexpr int kNout = 16;   // padded output width
constexpr int kLayers = 3;

typedef __nv_bfloat16 bf16;

struct Layout {
    long long enc_W, enc_b, W[kLayers], b[kLayers], dec_W, dec_b, total;
};

Layout layout(int dim)
{
    const long long zd = (long long)kC * (2 + dim);
    Layout L{};
    long long o = 0;
    L.enc_W = o; o += (long long)kC * kFin;
    L.enc_b = o; o += kC;
    for (int l = 0; l < kLayers; l++) {
        L.W[l] = o; o += kC * zd;
        L.b[l] = o; o += kC;
    }
    L.dec_W = o; o += (long long)kNout * kC;
    L.dec_b = o; o += kNout;
    L.total = o;
    return L;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ float silu_f(float y) { return y / (1.0f + expf(-y)); }
__device__ __forceinline__ float dsilu_f(float y)
{
    const float s = 1.0f / (1.0f + expf(-y));
    return s + y * s * (1.0f - s);
}

// dst[r, c] = bf16(src[r, c]) for r < rows, c < cols (ld = row strides)
__global__ void k_to_bf16(const float *__restrict__ src, int ld_src, int rows, int cols, bf16 *__restrict__ dst,
                          int ld_dst)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)rows * cols) return;
    const int r = (int)(t / cols), c = (int)(t % cols);
    dst[(size_t)r * ld_dst + c] = __float2bfloat16_rn(src[(size_t)r * ld_src + c]);
}

// mode 0: h = silu(y); mode 1: h += silu(y)
__global__ void k_act(const float *__restrict__ y, float *__restrict__ h, long long n, int mode)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float s = silu_f(y[t]);
    h[t] = mode ? h[t] + s : s;
}

// z row a = [bf16(h_a), bf16(m0_a), bf16(m1_a), ...]; one block (128
// threads = channels) per real node; node a = r n + a0 uses the base graph
// row a0 with neighbours r n + idx.
template <int D>
__global__ void __launch_bounds__(kC) k_aggregate(const float *__restrict__ h, bf16 *__restrict__ z, int n,
                                                  const int *__restrict__ ptr, const int *__restrict__ idx,
                                                  const float *__restrict__ w, const float *__restrict__ g)
{
    constexpr int zd = kC * (2 + D);
    const int a = blockIdx.x, c = threadIdx.x;
    const int r = a / n, a0 = a - r * n, off = r * n;
    const float ha = h[(size_t)a * kC + c];
    float m0 = 0.f, m[D];
#pragma unroll
    for (int k = 0; k < D; k++) m[k] = 0.f;
    for (int q = ptr[a0]; q < ptr[a0 + 1]; q++) {
        const float d = h[(size_t)(off + idx[q]) * kC + c] - ha;
        m0 += w[q] * d;
#pragma unroll
        for (int k = 0; k < D; k++) m[k] += g[(size_t)q * D + k] * d;
    }
    bf16 *zr = z + (size_t)a * zd;
    zr[c] = __float2bfloat16_rn(ha);
    zr[kC + c] = __float2bfloat16_rn(m0);
#pragma unroll
    for (int k = 0; k < D; k++) zr[(2 + k) * kC + c] = __float2bfloat16_rn(m[k]);
}

// Adjoint of the graph sums, for a symmetric neighbour relation with w
// symmetric and g antisymmetric (one body, one spacing): node b gathers
//   dh_b += dz_b[0:128] + sum_k sum_{a in N(b)} (s_k c^k_ba dm_k,a - c^k_ba dm_k,b)
// with s_0 = +1 (w) and s_k = -1 (g).
template <int D>
__global__ void __launch_bounds__(kC) k_agg_adjoint(const float *__restrict__ dz, float *__restrict__ dh, int n,
                                                    const int *__restrict__ ptr, const int *__restrict__ idx,
                                                    const float *__restrict__ w, const float *__restrict__ g)
{
    constexpr int zd = kC * (2 + D);
    const int b = blockIdx.x, c = threadIdx.x;
    const int r = b / n, b0 = b - r * n, off = r * n;
    const float *dzb = dz + (size_t)b * zd;
    float acc = dzb[c];
    float own[1 + D];
#pragma unroll
    for (int k = 0; k <= D; k++) own[k] = dzb[(1 + k) * kC + c];
    for (int q = ptr[b0]; q < ptr[b0 + 1]; q++) {
        const float *dza = dz + (size_t)(off + idx[q]) * zd;
        const float c0 = w[q];
        acc += c0 * (dza[kC + c] - own[0]);
#pragma unroll
        for (int k = 0; k < D; k++) {
            const float ck = g[(size_t)q * D + k];
            acc -= ck * (dza[(2 + k) * kC + c] + own[1 + k]);
        }
    }
    dh[(size_t)b * kC + c] += acc;
}

// dy = dh * silu'(y) for the real rows; bf16 copy; db += column sums (FP32)
__global__ void __launch_bounds__(kC) k_dsilu(const float *__restrict__ dh, const float *__restrict__ y, int rows,
                                              bf16 *__restrict__ dy, float *__restrict__ db)
{
    const int c = threadIdx.x;
    const int r0 = blockIdx.x * 32;
    float s = 0.f;
    for (int r = r0; r < r0 + 32 && r < rows; r++) {
        const size_t i = (size_t)r * kC + c;
        const float v = dh[i] * dsilu_f(y[i]);
        dy[i] = __float2bfloat16_rn(v);
        s += v;
    }
    atomicAdd(&db[c], s);
}

// 32 x 32 tiled transpose: dst (cols x rows) = src (rows x cols)^T
__global__ void k_transpose(const bf16 *__restrict__ src, int rows, int cols, bf16 *__restrict__ dst)
{
    __shared__ bf16 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;   // bx: column block, by: row block
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int r = by + j, c = bx + threadIdx.x;
        if (r < rows && c < cols) tile[j][threadIdx.x] = src[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int c = bx + j, r = by + threadIdx.x;
        if (r < rows && c < cols) dst[(size_t)c * rows + r] = tile[threadIdx.x][j];
    }
}

// Output gradient: with t, dout = 2 (out - t) mask / count on the first
// 2 dim columns and the loss sum; without t, out holds dout itself.
// Writes dout in bf16 (rows x 64, zero elsewhere), its transpose (first
// kNout rows of a 128 x np matrix) and the bias gradient.
__global__ void k_output_grad(const float *__restrict__ out, const float *__restrict__ t,
                              const uint8_t *__restrict__ mask, int rows, int np, int nout, float inv_cnt,
                              bf16 *__restrict__ dout, bf16 *__restrict__ doutT, float *__restrict__ db,
                              float *__restrict__ loss)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    float L = 0.f;
    if (r < rows) {
        const float mk = t ? (mask ? (float)mask[r] : 1.0f) : 1.0f;
        for (int j = 0; j < nout; j++) {
            float d;
            if (t) {
                const float e = (out[(size_t)r * kNout + j] - t[(size_t)r * kNout + j]) * mk;
                L += e * e;
                d = 2.0f * e * inv_cnt;
            } else {
                d = out[(size_t)r * kNout + j];
            }
            const bf16 q = __float2bfloat16_rn(d);
            dout[(size_t)r * kFin + j] = q;
            doutT[(size_t)j * np + r] = q;
            atomicAdd(&db[j], d);
        }
    }
    if (loss) {
        for (int o = 16; o > 0; o >>= 1) L += __shfl_xor_sync(0xffffffffu, L, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss, L * inv_cnt);
    }
}

// Adam (Kingma & Ba) with bias correction factors c1 = 1 / (1 - b1^t),
// c2 = 1 / (1 - b2^t)
__global__ void k_adam(float *__restrict__ th, const float *__restrict__ gr, float *__restrict__ m,
                       float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = gr[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// bf16 weight copies: W (out x in) as is, and W^T (in x out) padded to ldT
// columns (zeros beyond out)
__global__ void k_weights(const float *__restrict__ W, int out, int in, bf16 *__restrict__ Wb, bf16 *__restrict__ WT,
                          int ldT)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= out * in) return;
    const int o = t / in, i = t % in;
    const bf16 q = __float2bfloat16_rn(W[t]);
    if (Wb) Wb[t] = q;
    if (WT) WT[(size_t)i * ldT + o] = q;
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct sphfsi_mpnn {
    int dim = 2, n = 0, R = 1, nn = 0, np = 0, zd = 0;
    long long nnz = 0;
    cudaStream_t st = nullptr;
    Layout L{};
    long long step = 0;
    std::vector<void *> allocs;
    // graph
    int *ptr = nullptr, *idx = nullptr;
    float *w = nullptr, *g = nullptr;
    // parameters and optimiser
    float *theta = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
    bf16 *Wenc = nullptr, *Wl[kLayers] = {}, *WlT[kLayers] = {}, *Wdec = nullptr, *WdecT = nullptr;
    // activations
    float *xin = nullptr, *tin = nullptr;
    uint8_t *min_ = nullptr;
    bf16 *xb = nullptr, *xT = nullptr, *zb[kLayers] = {}, *zT = nullptr, *hb = nullptr, *hT = nullptr;
    float *yenc = nullptr, *h = nullptr, *y[kLayers] = {}, *out = nullptr;
    // backward
    bf16 *doutb = nullptr, *doutT = nullptr, *dyb = nullptr, *dyT = nullptr;
    float *dh = nullptr, *dz = nullptr, *dwdec = nullptr, *loss = nullptr;
};

namespace {

template <typename T>
int alloc(sphfsi_mpnn *m, T **p, size_t count)
{
    void *q = nullptr;
    if (cudaMalloc(&q, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
        cudaGetLastError();
        return SPHFSI_E_NOMEM;
    }
    cudaMemsetAsync(q, 0, sizeof(T) * (count ? count : 1), m->st);
    m->allocs.push_back(q);
    *p = (T *)q;
    return SPHFSI_OK;
}

#define LTRY(x)                       \
    do {                              \
        int _rc = (x);                \
        if (_rc) return _rc;          \
    } while (0)

int gemm(sphfsi_mpnn *m, const bf16 *A, const bf16 *B, const float *bias, float *C, long long M, long long N,
         long long K)
{
    int rc = launch_gemm_bf16((const uint16_t *)A, (const uint16_t *)B, bias, C, M, N, K, m->st);
    return rc == 0 ? SPHFSI_OK : (rc == -3 ? SPHFSI_E_CUDA : SPHFSI_E_INVAL);
}

int refresh_weights(sphfsi_mpnn *m)
{
    const Layout &L = m->L;
    cudaStream_t st = m->st;
    k_weights<<<nblk(kC * kFin, 256), 256, 0, st>>>(m->theta + L.enc_W, kC, kFin, m->Wenc, nullptr, 0);
    for (int l = 0; l < kLayers; l++)
        k_weights<<<nblk((long long)kC * m->zd, 256), 256, 0, st>>>(m->theta + L.W[l], kC, m->zd, m->Wl[l], m->WlT[l],
                                                                     kC);
    k_weights<<<nblk(kNout * kC, 256), 256, 0, st>>>(m->theta + L.dec_W, kNout, kC, m->Wdec, m->WdecT, kFin);
    return cudaGetLastError() == cudaSuccess ? SPHFSI_OK : SPHFSI_E_CUDA;
}

int forward(sphfsi_mpnn *m)
{
    cudaStream_t st = m->st;
    const Layout &L = m->L;
    const long long np = m->np, nn = m->nn;
    k_to_bf16<<<nblk(nn * kFin, 256), 256, 0, st>>>(m->xin, kFin, (int)nn, kFin, m->xb, kFin);
    LTRY(gemm(m, m->xb, m->Wenc, m->theta + L.enc_b, m->yenc, np, kC, kFin));
    k_act<<<nblk(np * kC, 256), 256, 0, st>>>(m->yenc, m->h, np * kC, 0);
    for (int l = 0; l < kLayers; l++) {
        if (m->dim == 2)
            k_aggregate<2><<<(int)nn, kC, 0, st>>>(m->h, m->zb[l], m->n, m->ptr, m->idx, m->w, m->g);
        else
            k_aggregate<3><<<(int)nn, kC, 0, st>>>(m->h, m->zb[l], m->n, m->ptr, m->idx, m->w, m->g);
        LTRY(gemm(m, m->zb[l], m->Wl[l], m->theta + L.b[l], m->y[l], np, kC, m->zd));
        k_act<<<nblk(np * kC, 256), 256, 0, st>>>(m->y[l], m->h, np * kC, 1);
    }
    k_to_bf16<<<nblk(nn * kC, 256), 256, 0, st>>>(m->h, kC, (int)nn, kC, m->hb, kC);
    LTRY(gemm(m, m->hb, m->Wdec, m->theta + L.dec_b, m->out, np, kNout, kC));
    return cudaGetLastError() == cudaSuccess ? SPHFSI_OK : SPHFSI_E_CUDA;
}

// gradient of the parameters; the output gradient comes from the loss
// (t != null) or is given in m->out's place (dout_given)
int backward(sphfsi_mpnn *m, const float *dout_or_out, const float *t, const uint8_t *mask, float inv_cnt, float *loss)
{
    cudaStream_t st = m->st;
    const Layout &L = m->L;
    const long long np = m->np, nn = m->nn;
    const dim3 tb(32, 8);
    LTRY(cudaMemsetAsync(m->grad, 0, sizeof(float) * L.total, st) == cudaSuccess ? 0 : SPHFSI_E_CUDA);
    if (loss) LTRY(cudaMemsetAsync(loss, 0, sizeof(float), st) == cudaSuccess ? 0 : SPHFSI_E_CUDA);
    k_output_grad<<<nblk(nn, 128), 128, 0, st>>>(dout_or_out, t, mask, (int)nn, (int)np, t ? 2 * m->dim : kNout,
                                                 inv_cnt,
                                                 m->doutb, m->doutT, m->grad + L.dec_b, loss);
    // decoder: dW_dec = dout^T h (first kNout rows of a 128-row product), dh = dout W_dec
    k_transpose<<<dim3(kC / 32, (unsigned)(np / 32)), tb, 0, st>>>(m->hb, (int)np, kC, m->hT);
    LTRY(gemm(m, m->doutT, m->hT, nullptr, m->dwdec, kC, kC, np));
    LTRY(cudaMemcpyAsync(m->grad + L.dec_W, m->dwdec, sizeof(float) * kNout * kC, cudaMemcpyDeviceToDevice, st) ==
                 cudaSuccess
             ? 0
             : SPHFSI_E_CUDA);
    LTRY(gemm(m, m->doutb, m->WdecT, nullptr, m->dh, np, kC, kFin));
    for (int l = kLayers - 1; l >= 0; l--) {
        k_dsilu<<<(unsigned)(np / 32), kC, 0, st>>>(m->dh, m->y[l], (int)nn, m->dyb, m->grad + L.b[l]);
        k_transpose<<<dim3(kC / 32, (unsigned)(np / 32)), tb, 0, st>>>(m->dyb, (int)np, kC, m->dyT);
        k_transpose<<<dim3((unsigned)(m->zd / 32), (unsigned)(np / 32)), tb, 0, st>>>(m->zb[l], (int)np, m->zd,
                                                                                        m->zT);
        LTRY(gemm(m, m->dyT, m->zT, nullptr, m->grad + L.W[l], kC, m->zd, np));
        LTRY(gemm(m, m->dyb, m->WlT[l], nullptr, m->dz, np, m->zd, kC));
        if (m->dim == 2)
            k_agg_adjoint<2><<<(int)nn, kC, 0, st>>>(m->dz, m->dh, m->n, m->ptr, m->idx, m->w, m->g);
        else
            k_agg_adjoint<3><<<(int)nn, kC, 0, st>>>(m->dz, m->dh, m->n, m->ptr, m->idx, m->w, m->g);
    }
    k_dsilu<<<(unsigned)(np / 32), kC, 0, st>>>(m->dh, m->yenc, (int)nn, m->dyb, m->grad + L.enc_b);
    k_transpose<<<dim3(kC / 32, (unsigned)(np / 32)), tb, 0, st>>>(m->dyb, (int)np, kC, m->dyT);
    k_transpose<<<dim3(kFin / 32, (unsigned)(np / 32)), tb, 0, st>>>(m->xb, (int)np, kFin, m->xT);
    LTRY(gemm(m, m->dyT, m->xT, nullptr, m->grad + L.enc_W, kC, kFin, np));
    return cudaGetLastError() == cudaSuccess ? SPHFSI_OK : SPHFSI_E_CUDA;
}

int stage_in(sphfsi_mpnn *m, void *dst, const void *src, size_t bytes)
{
    if (!src) return SPHFSI_E_INVAL;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, m->st) == cudaSuccess ? SPHFSI_OK : SPHFSI_E_CUDA;
}

}  // namespace

namespace sph {
float *mpnn_input(sphfsi_mpnn *m) { return m->xin; }
const float *mpnn_output(sphfsi_mpnn *m) { return m->out; }
int mpnn_forward_async(sphfsi_mpnn *m) { return forward(m); }
int mpnn_kernels_per_forward() { return 3 + 3 * kLayers + 2; }   // encoder, layers, decoder
}  // namespace sph

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
extern "C" {

int64_t sphfsi_mpnn_n_params(int32_t dim)
{
    if (dim != 2 && dim != 3) return SPHFSI_E_INVAL;
    return layout(dim).total;
}

int sphfsi_mpnn_create(sphfsi_mpnn **out, int32_t dim, int64_t n, int64_t nnz, const int64_t *ptr,
                       const int64_t *idx, const double *w, const double *g, int32_t replicas, void *cuda_stream)
{
    if (!out || (dim != 2 && dim != 3) || n < 1 || nnz < 0 || replicas < 1 || !ptr || (nnz && (!idx || !w || !g)))
        return SPHFSI_E_INVAL;
    if (n * (int64_t)replicas > (1LL << 26) || nnz > (1LL << 30)) return SPHFSI_E_CAPACITY;
    *out = nullptr;
    // the graph comes in on the host: check it and its symmetry
    std::vector<int64_t> hp(n + 1), hi(nnz);
    std::vector<double> hw(nnz), hg(nnz * dim);
    if (cudaMemcpy(hp.data(), ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDefault) != cudaSuccess) return SPHFSI_E_CUDA;
    if (nnz) {
        if (cudaMemcpy(hi.data(), idx, sizeof(int64_t) * nnz, cudaMemcpyDefault) != cudaSuccess ||
            cudaMemcpy(hw.data(), w, sizeof(double) * nnz, cudaMemcpyDefault) != cudaSuccess ||
            cudaMemcpy(hg.data(), g, sizeof(double) * nnz * dim, cudaMemcpyDefault) != cudaSuccess)
            return SPHFSI_E_CUDA;
    }
    if (hp[0] != 0 || hp[n] != nnz) return SPHFSI_E_INVAL;
    for (int64_t a = 0; a < n; a++) {
        if (hp[a + 1] < hp[a]) return SPHFSI_E_INVAL;
        for (int64_t q = hp[a]; q < hp[a + 1]; q++) {
            const int64_t b = hi[q];
            if (b < 0 || b >= n || b == a) return SPHFSI_E_INVAL;
            // reverse entry with the same w and the opposite g
            int64_t q2 = -1;
            for (int64_t s = hp[b]; s < hp[b + 1]; s++)
                if (hi[s] == a) q2 = s;
            if (q2 < 0) return SPHFSI_E_INVAL;
            const double tol = 1e-6;
            if (std::fabs(hw[q] - hw[q2]) > tol * (std::fabs(hw[q]) + 1e-30)) return SPHFSI_E_INVAL;
            for (int k = 0; k < dim; k++)
                if (std::fabs(hg[q * dim + k] + hg[q2 * dim + k]) > tol * (std::fabs(hg[q * dim + k]) + 1e-30))
                    return SPHFSI_E_INVAL;
        }
    }
    sphfsi_mpnn *m = new (std::nothrow) sphfsi_mpnn();
    if (!m) return SPHFSI_E_NOMEM;
    m->dim = dim;
    m->n = (int)n;
    m->R = replicas;
    m->nn = (int)(n * replicas);
    m->np = (m->nn + 127) / 128 * 128;
    m->zd = kC * (2 + dim);
    m->nnz = nnz;
    m->st = (cudaStream_t)cuda_stream;
    m->L = layout(dim);
    const long long np = m->np, P = m->L.total;
    int rc = SPHFSI_OK;
    auto A = [&](auto **p, size_t c) {
        if (!rc) rc = alloc(m, p, c);
    };
    A(&m->ptr, n + 1);
    A(&m->idx, nnz);
    A(&m->w, nnz);
    A(&m->g, nnz * dim);
    A(&m->theta, P);
    A(&m->grad, P);
    A(&m->am, P);
    A(&m->av, P);
    A(&m->Wenc, kC * kFin);
    for (int l = 0; l < kLayers; l++) {
        A(&m->Wl[l], (size_t)kC * m->zd);
        A(&m->WlT[l], (size_t)kC * m->zd);
        A(&m->zb[l], (size_t)np * m->zd);
        A(&m->y[l], (size_t)np * kC);
    }
    A(&m->Wdec, kNout * kC);
    A(&m->WdecT, kC * kFin);
    A(&m->xin, (size_t)np * kFin);
    A(&m->tin, (size_t)np * kNout);
    A(&m->min_, (size_t)np);
    A(&m->xb, (size_t)np * kFin);
    A(&m->xT, (size_t)np * kFin);
    A(&m->zT, (size_t)np * m->zd);
    A(&m->hb, (size_t)np * kC);
    A(&m->hT, (size_t)np * kC);
    A(&m->yenc, (size_t)np * kC);
    A(&m->h, (size_t)np * kC);
    A(&m->out, (size_t)np * kNout);
    A(&m->doutb, (size_t)np * kFin);
    A(&m->doutT, (size_t)np * kC);
    A(&m->dyb, (size_t)np * kC);
    A(&m->dyT, (size_t)np * kC);
    A(&m->dh, (size_t)np * kC);
    A(&m->dz, (size_t)np * m->zd);
    A(&m->dwdec, kC * kC);
    A(&m->loss, 1);
    if (!rc) {
        std::vector<int> ip(hp.begin(), hp.end()), ii(hi.begin(), hi.end());
        std::vector<float> fw(hw.begin(), hw.end()), fg(hg.begin(), hg.end());
        if (cudaMemcpyAsync(m->ptr, ip.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, m->st) != cudaSuccess ||
            (nnz && (cudaMemcpyAsync(m->idx, ii.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, m->st) !=
                         cudaSuccess ||
                     cudaMemcpyAsync(m->w, fw.data(), sizeof(float) * nnz, cudaMemcpyHostToDevice, m->st) !=
                         cudaSuccess ||
                     cudaMemcpyAsync(m->g, fg.data(), sizeof(float) * nnz * dim, cudaMemcpyHostToDevice, m->st) !=
                         cudaSuccess)))
            rc = SPHFSI_E_CUDA;
        if (!rc && cudaStreamSynchronize(m->st) != cudaSuccess) rc = SPHFSI_E_CUDA;
    }
    if (rc) {
        sphfsi_mpnn_destroy(m);
        return rc;
    }
    *out = m;
    return SPHFSI_OK;
}

int sphfsi_mpnn_set_params(sphfsi_mpnn *m, const float *theta)
{
    if (!m || !theta) return SPHFSI_E_INVAL;
    LTRY(stage_in(m, m->theta, theta, sizeof(float) * m->L.total));
    cudaMemsetAsync(m->am, 0, sizeof(float) * m->L.total, m->st);
    cudaMemsetAsync(m->av, 0, sizeof(float) * m->L.total, m->st);
    m->step = 0;
    LTRY(refresh_weights(m));
    return cudaStreamSynchronize(m->st) == cudaSuccess ? SPHFSI_OK : SPHFSI_E_CUDA;
}

int sphfsi_mpnn_get_params(sphfsi_mpnn *m, float *theta)
{
    if (!m || !theta) return SPHFSI_E_INVAL;
    if (cudaMemcpyAsync(theta, m->theta, sizeof(float) * m->L.total, cudaMemcpyDefault, m->st) != cudaSuccess)
        return SPHFSI_E_CUDA;
    return cudaStreamSynchronize(m->st) == cudaSuccess ? SPHFSI_OK : SPHFSI_E_CUDA;
}

int sphfsi_mpnn_forward(sphfsi_mpnn *m, const float *x, float *out)
{
    if (!m || !x) return SPHFSI_E_INVAL;
    LTRY(stage_in(m, m->xin, x, sizeof(float) * (size_t)m->nn * kFin));
    LTRY(forward(m));
    if (out && cudaMemcpyAsync(out, m->out, sizeof(float) * (size_t)m->nn * kNout, cudaMemcpyDefault, m->st) !=
                   cudaSuccess)
        return SPHFSI_E_CUDA;
    return SPHFSI_OK;
}

int sphfsi_mpnn_backward(sphfsi_mpnn *m, const float *dout, float *grad)
{
    if (!m || !dout) return SPHFSI_E_INVAL;
    LTRY(stage_in(m, m->tin, dout, sizeof(float) * (size_t)m->nn * kNout));
    LTRY(backward(m, m->tin, nullptr, nullptr, 1.0f, nullptr));
    if (grad && cudaMemcpyAsync(grad, m->grad, sizeof(float) * m->L.total, cudaMemcpyDefault, m->st) != cudaSuccess)
        return SPHFSI_E_CUDA;
    return SPHFSI_OK;
}

int sphfsi_mpnn_train_step(sphfsi_mpnn *m, const float *x, const float *target, const uint8_t *mask, float lr,
                           float *loss)
{
    if (!m || !x || !target || !(lr > 0.0f)) return SPHFSI_E_INVAL;
    LTRY(stage_in(m, m->xin, x, sizeof(float) * (size_t)m->nn * kFin));
    LTRY(stage_in(m, m->tin, target, sizeof(float) * (size_t)m->nn * kNout));
    long long cnt = m->nn;
    if (mask) {
        std::vector<uint8_t> hm(m->nn);
        if (cudaMemcpy(hm.data(), mask, m->nn, cudaMemcpyDefault) != cudaSuccess) return SPHFSI_E_CUDA;
        cnt = 0;
        for (uint8_t v : hm) cnt += v != 0;
        LTRY(stage_in(m, m->min_, hm.data(), m->nn));
        if (cudaStreamSynchronize(m->st) != cudaSuccess) return SPHFSI_E_CUDA;
    }
    const float inv_cnt = 1.0f / (float)(cnt > 0 ? cnt : 1);
    LTRY(forward(m));
    LTRY(backward(m, m->out, m->tin, mask ? m->min_ : nullptr, inv_cnt, m->loss));
    m->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)m->step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)m->step)));
    k_adam<<<nblk(m->L.total, 256), 256, 0, m->st>>>(m->theta, m->grad, m->am, m->av, m->L.total, lr, b1, b2, 1e-8f,
                                                     c1, c2);
    LTRY(refresh_weights(m));
    if (loss && cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDefault, m->st) != cudaSuccess)
        return SPHFSI_E_CUDA;
    return cudaGetLastError() == cudaSuccess ? SPHFSI_OK : SPHFSI_E_CUDA;
}

int sphfsi_mpnn_sync(sphfsi_mpnn *m)
{
    if (!m) return SPHFSI_E_INVAL;
    if (cudaStreamSynchronize(m->st) != cudaSuccess) return SPHFSI_E_CUDA;
    unsigned s = 0;
    if (read_tc_status(&s, false)) return SPHFSI_E_CUDA;
    return (s & 1u) ? SPHFSI_E_TIMEOUT : SPHFSI_OK;
}

void sphfsi_mpnn_destroy(sphfsi_mpnn *m)
{
    if (!m) return;
    if (m->st) cudaStreamSynchronize(m->st);
    else cudaDeviceSynchronize();
    for (void *p : m->allocs) cudaFree(p);
    delete m;
}

}  // extern "C"
