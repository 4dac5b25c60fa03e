// k_gemm.cu -- BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory), used by the MLP surrogate for
// inference and for every training GEMM.
//
//   C[M][N] = act(A[M][K] . B[N][K]^T + bias[N])
//
// A and B are row-major with K contiguous ("TN"); M and N are multiples of
// 128, K a multiple of 64.  One CTA (4 warps) computes a 128 x 128 tile: each
// 64-wide K block of A and B is copied into a 128-byte-swizzled shared-memory
// stage (two stages), one thread issues four 128x128x16 MMAs per K block and
// commits them to the stage's mbarrier, and the four warps read the 128 x 128
// FP32 accumulator back from tensor memory (warp w owns rows 32w..32w+31).
// Every mbarrier wait is bounded; on a timeout the kernel records an error
// flag, waits once more (bounded) for its own MMAs, frees its tensor memory
// and exits.
#include <cuda_bf16.h>

#include "../../include/twinkle.h"
#include "gemm.cuh"
#include "kernels.cuh"
#include "mma.cuh"

namespace tw {

constexpr int GB_M = 128, GB_N = 128, GB_K = 64;
constexpr uint32_t GEMM_WAIT_LIMIT = 1u << 26;  // polls (~0.1-1 s) before a wait is declared hung
constexpr size_t GEMM_STAGE_BYTES = 2 * 16384;   // A and B tiles of one stage
constexpr size_t GEMM_SMEM = 1024 + 2 * GEMM_STAGE_BYTES + 64;

__global__ void __launch_bounds__(128, 1) gemm_bf16_tn_kernel(GemmArgs g) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA[2] = {smem, smem + GEMM_STAGE_BYTES};
    uint8_t *sB[2] = {smem + 16384, smem + GEMM_STAGE_BYTES + 16384};
    uint64_t *bar = (uint64_t *)(smem + 2 * GEMM_STAGE_BYTES);
    uint32_t *tslot = (uint32_t *)(bar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
    const int K = g.K, nk = K / GB_K;
    constexpr uint32_t IDESC = idesc_bf16_f32(GB_M, GB_N);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tslot, 128);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tslot;

    bool failed = false;
    int issued = 0;  // K blocks whose MMAs were issued
    for (int kb = 0; kb < nk; kb++) {
        const int s = kb & 1, u = kb >> 1;
        bool ok = true;
        if (kb >= 2) ok = mbar_wait(&bar[s], (uint32_t)((u - 1) & 1), GEMM_WAIT_LIMIT);  // stage free again
        if (!__syncthreads_and(ok)) { failed = true; break; }
        // copy the 128 x 64 tiles of A and B into the stage, 16 bytes at a time
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int ch = tid + 128 * i;
            const int r = ch >> 3, c = ch & 7;
            const uint4 va = *(const uint4 *)(g.A + (size_t)(m0 + r) * K + kb * GB_K + c * 8);
            const uint4 vb = *(const uint4 *)(g.B + (size_t)(n0 + r) * K + kb * GB_K + c * 8);
            *(uint4 *)(sA[s] + swz128(r, c)) = va;
            *(uint4 *)(sB[s] + swz128(r, c)) = vb;
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 4; ks++) {
                const uint64_t ad = sdesc_sw128(smem_u32(sA[s]) + 32u * ks);
                const uint64_t bd = sdesc_sw128(smem_u32(sB[s]) + 32u * ks);
                mma_bf16(taddr, ad, bd, IDESC, (kb | ks) ? 1u : 0u);
            }
            mma_commit(&bar[s]);
        }
        issued = kb + 1;
    }
    // wait for the last commit (it covers every earlier MMA)
    bool ok = true;
    if (issued > 0) ok = mbar_wait(&bar[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1), GEMM_WAIT_LIMIT);
    if (!__syncthreads_and(ok) && issued > 0) {
        // the MMAs are still not complete: wait once more, four times as
        // long, before the tensor memory they write is released below (a
        // CTA must free its tensor memory, or later CTAs on this SM could not
        // allocate any); the error flag makes the host discard C either way
        ok = false;
        (void)mbar_wait(&bar[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1), 4u * GEMM_WAIT_LIMIT);
    }
    ok = __syncthreads_and(ok) && !failed;
    if (ok) {
        tc_fence_after();
        const int row = warp * 32 + lane;
        const size_t orow = (size_t)(m0 + row) * g.N + n0;
#pragma unroll 1
        for (int cc = 0; cc < GB_N; cc += 32) {
            float v[32];
            tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc, v);
#pragma unroll
            for (int j = 0; j < 32; j++) {
                float x = v[j];
                if (g.bias) x += g.bias[n0 + cc + j];
                if (g.relu) x = fmaxf(x, 0.0f);
                v[j] = x;
            }
            if (g.C) {
                float4 *dst = (float4 *)(g.C + orow + cc);
#pragma unroll
                for (int j = 0; j < 8; j++) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            }
            if (g.Cb) {
                uint4 *dst = (uint4 *)(g.Cb + orow + cc);
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    __nv_bfloat162 h[4];
#pragma unroll
                    for (int t = 0; t < 4; t++) h[t] = __floats2bfloat162_rn(v[8 * j + 2 * t], v[8 * j + 2 * t + 1]);
                    dst[j] = *(uint4 *)h;
                }
            }
        }
    } else if (tid == 0 && g.err) {
        atomicExch(g.err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_free(taddr, 128);
}

cudaError_t gemm_bf16_tn(const GemmArgs &g, cudaStream_t st) {
    static bool attr = false;  // per-process; the attribute is per function
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)GEMM_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((unsigned)(g.N / GB_N), (unsigned)(g.M / GB_M));
    gemm_bf16_tn_kernel<<<grid, 128, GEMM_SMEM, st>>>(g);
    return cudaGetLastError();
}

}  // namespace tw

extern "C" int tw_gemm_bf16(const void *A, const void *B, int M, int N, int K, float *C, void *stream) {
    using namespace tw;
    if (M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 128 || K % 64 || !A || !B || !C) return TW_EINVAL;
    int *err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) { (void)cudaGetLastError(); return TW_ENOMEM; }
    cudaStream_t st = (cudaStream_t)stream;
    GemmArgs g;
    g.A = (const __nv_bfloat16 *)A;
    g.B = (const __nv_bfloat16 *)B;
    g.M = M;
    g.N = N;
    g.K = K;
    g.C = C;
    g.Cb = nullptr;
    g.bias = nullptr;
    g.relu = 0;
    g.err = err;
    int h = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = gemm_bf16_tn(g, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(err);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return TW_ECUDA; }
    return h ? TW_ETIMEOUT : TW_OK;
}

// ------------------------------------------------------------------ self-test
// A bounded wait that must run out: one CTA waits on an mbarrier that nothing
// arrives on (no copy or MMA is in flight), with `limit` polls, through the
// same wait routine the GEMM uses; on giving up it records the error flag and
// returns, leaving the context usable.
namespace tw {
__global__ void timeout_selftest_kernel(uint32_t limit, int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0u, limit);
    if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicExch(err, 1);
}
}  // namespace tw

extern "C" int tw_selftest_timeout(unsigned int poll_limit) {
    using namespace tw;
    if (poll_limit == 0 || poll_limit > (1u << 24)) return TW_EINVAL;
    int *err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) { (void)cudaGetLastError(); return TW_ENOMEM; }
    int h = 0;
    cudaError_t e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) {
        timeout_selftest_kernel<<<1, 32>>>(poll_limit, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return TW_ECUDA; }
    return h ? TW_ETIMEOUT : TW_OK;
}
