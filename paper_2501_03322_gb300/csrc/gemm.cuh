// gemm.cuh -- interface of the tensor-core GEMM (k_gemm.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace tw {

// C[M][N] = act(A[M][K] . B[N][K]^T + bias[N]); M, N multiples of 128, K of 64.
struct GemmArgs {
    const __nv_bfloat16 *A;  // [M][K]
    const __nv_bfloat16 *B;  // [N][K]
    int M, N, K;
    float *C;                // optional FP32 output [M][N]
    __nv_bfloat16 *Cb;       // optional BF16 output [M][N]
    const float *bias;       // optional [N]
    int relu;                // apply max(x, 0) after the bias
    int *err;                // optional: set to 1 if a bounded wait gave up
};

cudaError_t gemm_bf16_tn(const GemmArgs &g, cudaStream_t st);

}  // namespace tw
