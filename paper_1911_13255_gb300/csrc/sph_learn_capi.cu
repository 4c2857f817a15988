// C-ABI of the learned sub-stepper building blocks.
#include "sph_learn.cuh"
#include "sphfsi.h"

using namespace sph;

extern "C" {

int sphfsi_gemm_bf16(const void *A, const void *B, const float *bias, float *C, int64_t M, int64_t N, int64_t K,
                     void *cuda_stream)
{
    int rc = launch_gemm_bf16((const uint16_t *)A, (const uint16_t *)B, bias, C, M, N, K, (cudaStream_t)cuda_stream);
    return rc == -3 ? SPHFSI_E_CUDA : rc;
}

int sphfsi_tc_status(int32_t *status, int32_t reset)
{
    if (!status) return SPHFSI_E_INVAL;
    unsigned s = 0;
    if (read_tc_status(&s, reset != 0)) return SPHFSI_E_CUDA;
    *status = (int32_t)s;
    return SPHFSI_OK;
}

}  // extern "C"
