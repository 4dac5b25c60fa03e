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

}  // namespace tw
