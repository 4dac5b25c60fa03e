// Self-test of the library's FP64 reciprocals (cx.cuh: hardware approximation
// refined by two Newton-Raphson steps, or by one for rcp40) against IEEE
// division, over magnitudes 1e-300 .. 1e300 of both signs.
#include "kernels.cuh"

namespace tw {

// max_err_bits[0]: rcp (two refinement steps), [1]: rcp40 (one step).
__global__ void rcp_selftest_kernel(unsigned long long *max_err_bits, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // log-uniform magnitudes with a per-thread mantissa pattern
    const double e = -300.0 + 600.0 * (double)i / (double)(n - 1);
    double v = exp10(e) * (1.0 + 0.6180339887498949 * (double)((i * 2654435761u) & 1023) / 1024.0);
    if (i & 1) v = -v;
    const double ref = 1.0 / v;
    const double rel = fabs(rcp(v) / ref - 1.0), rel40 = fabs(rcp40(v) / ref - 1.0);
    atomicMax(max_err_bits, (unsigned long long)__double_as_longlong(rel));
    atomicMax(max_err_bits + 1, (unsigned long long)__double_as_longlong(rel40));
}

cudaError_t launch_rcp_selftest(unsigned long long *max_err_bits, int n, cudaStream_t st) {
    rcp_selftest_kernel<<<(n + 255) / 256, 256, 0, st>>>(max_err_bits, n);
    return cudaGetLastError();
}

// Throughput probe of the CUDA-core fused multiply-add pipes, the units the
// contour kernel's roofline is stated in: every thread advances ACC
// independent chains a <- a m + c for `iters` steps (2 FLOP each), so the
// pipe, not the latency of one chain, limits the rate.
template <typename T, int ACC>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T m, T c, T *sink) {
    T a[ACC];
#pragma unroll
    for (int k = 0; k < ACC; k++) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < ACC; k++) a[k] = fma(a[k], m, c);
    }
    T t = 0;
#pragma unroll
    for (int k = 0; k < ACC; k++) t += a[k];
    if (t == (T)-1.2345) sink[0] = t;  // never true: keeps the chains alive
}

// FLOP/s of one probe launch over `blocks` CTAs (the second of two launches).
template <typename T, int ACC>
static int run_fma_probe(int blocks, int iters, double *flops_per_s) {
    T *sink = nullptr;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaMalloc(&sink, sizeof(T));
    if (e != cudaSuccess) return -1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
        cudaEventRecord(e0, 0);
        fma_probe_kernel<T, ACC><<<blocks, 256, 0, 0>>>(iters, (T)0.9999999, (T)1e-7, sink);
        cudaEventRecord(e1, 0);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess || ms <= 0.f) { (void)cudaGetLastError(); return -1; }
    *flops_per_s = 2.0 * ACC * (double)iters * 256.0 * blocks / (ms * 1e-3);
    return 0;
}

int fma_probe(int kind, int nsm, double *flops_per_s) {
    if (kind == 0) return run_fma_probe<double, 8>(nsm * 8, 1 << 14, flops_per_s);
    return run_fma_probe<float, 16>(nsm * 8, 1 << 17, flops_per_s);
}

}  // namespace tw
