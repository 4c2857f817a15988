// Internal interface of the learned sub-stepper kernels (tensor-core GEMM,
// graph aggregation, element-wise and optimiser kernels).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sphfsi.h"

namespace sph {

// C[M x N] = A[M x K] . B[N x K]^T (+ bias), bfloat16 operands, FP32 result.
// Returns 0, -1 (bad sizes or alignment), -7 (too large) or -3 (launch).
int launch_gemm_bf16(const uint16_t *A, const uint16_t *B, const float *bias, float *C, long long M, long long N,
                     long long K, cudaStream_t st);
// status bits of the bounded tensor-core waits (bit 0: a wait ran out)
int read_tc_status(unsigned *out, bool reset);

// network context as used inside a simulation step: its input (n x 64 FP32)
// and output (n x 16 FP32) buffers and an asynchronous forward pass on the
// context's stream; kernels launched by one forward pass
float *mpnn_input(sphfsi_mpnn *m);
const float *mpnn_output(sphfsi_mpnn *m);
int mpnn_forward_async(sphfsi_mpnn *m);
int mpnn_kernels_per_forward();

}  // namespace sph
