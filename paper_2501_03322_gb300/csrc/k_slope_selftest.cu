// Self-test of the slope test and its repair (Sec. 2.4.2) on a constructed
// misjudgment.  One thread samples the limb of a source position at the
// given angles (the same sample routine as the contour kernel), links and
// integrates every edge, then takes a caustic crossing among closely spaced
// samples and plants the error that the slope test exists to catch: the
// ghost pair of samples on the crossing's three-image side is declared real,
//   mode 1: the sample next to the crossing (the crossing moves by one
//           sample: the first case of Sec. 2.4.2),
//   mode 2: the two samples after it (a false two-sample image piece inside
//           the three-image run: the second case).
// The planted crossings must fail the slope test, and the repair must give
// back the original classification and area.
#include "../../include/twinkle.h"
#include "kernels.cuh"

namespace tw {

// A three-image sample declared five-image: its ghost pair joins the real
// images, the root with the larger Jacobian as the positive one.
__device__ void plant_ghost_pair(const LensK &L, const Arena &ar, int sl) {
    const uint32_t m = ar.meta[sl];
    const unsigned real = real_mask(m);
    int g[2] = {0, 0}, ng = 0;
    for (int i = 0; i < 5; i++)
        if (!((real >> i) & 1u) && ng < 2) g[ng++] = i;
    double J[2];
    for (int t = 0; t < 2; t++) {
        const cxd z = ar.roots[sl * 5 + g[t]];
        const cxd d1 = inv(cxd{z.x + L.s, z.y}), d2 = inv(z);
        J[t] = 1.0 - norm2(L.m1 * (d1 * d1) + L.m2 * (d2 * d2));
    }
    const int gp = J[0] >= J[1] ? g[0] : g[1], gn = J[0] >= J[1] ? g[1] : g[0];
    // positives: the real one, then gp; negatives: the two real ones, then gn
    const uint32_t nm = 5u | ((uint32_t)meta_index(m, 0) << 3) | ((uint32_t)gp << 6) |
                        ((uint32_t)meta_index(m, 1) << 9) | ((uint32_t)meta_index(m, 2) << 12) |
                        ((uint32_t)gn << 15);
    ar.meta[sl] = nm;
}

__device__ double edge_at(const Arena &ar, const double *theta, int n, int p, int &viol) {
    const double twopi = 6.283185307179586476925287;
    const int a = ((p % n) + n) % n, b = (a + 1) % n;
    const double tb = b == 0 ? theta[0] + twopi : theta[b];
    viol = compute_edge(ar, a, b, tb - theta[a], &ar.eA[a], &ar.eE[a], false) & PS_SLOPE;
    return ar.eA[a];
}

__global__ void slope_selftest_kernel(LensK L, const double *theta, int n, int mode, char *base, size_t slot_bytes,
                                      int cap, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const Arena ar = arena_at(base, slot_bytes, cap, 0);
    WorkCount wc;
    cxd z[5];
    for (int i = 0; i < 5; i++) z[i] = {__longlong_as_double(0x7ff8000000000000ll), 0.0};
    for (int k = 0; k < n; k++) {
        limb_sample<0>(L, theta[k], z, ar, k, wc);
        ar.ordA[k] = (uint16_t)k;
    }
    double A0 = 0.0;
    int viol;
    for (int k = 0; k < n; k++) A0 += edge_at(ar, theta, n, k, viol);
    for (int k = 0; k < n; k++) ar.cum[k] = (double)(ar.meta[k] & 0x3fffffffu);  // original classification
    // a crossing between two closely spaced samples
    int p = -1;
    for (int k = 0; k < n && p < 0; k++) {
        const int b = (k + 1) % n;
        if (b > 0 && meta_count(ar.meta[k]) != meta_count(ar.meta[b]) && theta[b] - theta[k] < 1e-3) p = k;
    }
    out[0] = out[1] = 0.0;
    out[2] = -1.0;
    out[3] = p;
    if (p < 0) return;
    const int k3 = meta_count(ar.meta[p]) == 3 ? p : p + 1, d3 = k3 == p ? -1 : 1;
    const int a = mode == 1 ? k3 : k3 + d3, b = mode == 1 ? k3 : k3 + 2 * d3;
    const int plo = a < b ? a : b, phi = a < b ? b : a;
    if (plo < 1 || phi + 1 >= n) return;
    for (int k = plo; k <= phi; k++) plant_ghost_pair(L, ar, k);
    int pv = -1;
    for (int e = plo - 1; e <= phi; e++) {
        edge_at(ar, theta, n, e, viol);
        if (viol && pv < 0) pv = e;
    }
    out[0] = pv >= 0 ? 1.0 : 0.0;
    if (pv < 0) return;
    slope_fix(ar, ar.ordA, n, pv);
    bool same = true;
    for (int k = 0; k < n; k++) same = same && (double)(ar.meta[k] & 0x3fffffffu) == ar.cum[k];
    double A1 = 0.0;
    for (int k = 0; k < n; k++) A1 += ar.eA[k];
    out[1] = same ? 1.0 : 0.0;
    out[2] = fabs(A1 / A0 - 1.0);
}

}  // namespace tw

extern "C" int tw_selftest_slope(double s, double q, double rho, double y1, double y2, const double *theta, int n,
                                 int mode, double *out4) {
    using namespace tw;
    if (!theta || !out4 || n < 8 || n > 256 || (mode != 1 && mode != 2) || !(s > 0) || !(q > 0) || !(q <= 1) ||
        !(rho > 0))
        return TW_EINVAL;
    for (int k = 0; k < n; k++)
        if (!(theta[k] >= 0.0) || !(theta[k] < 6.283185307179586) || (k > 0 && !(theta[k] > theta[k - 1])))
            return TW_EINVAL;
    LensK L;
    L.s = s;
    L.m1 = 1.0 / (1.0 + q);
    L.m2 = q * L.m1;
    L.rho = rho;
    L.y0 = {y1 - s * L.m1, y2};
    const int cap = 256;
    const size_t slot = arena_slot_bytes(cap);
    char *base = nullptr;
    double *dth = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&base, slot);
    if (e == cudaSuccess) e = cudaMalloc(&dth, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dout, 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(dth, theta, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        slope_selftest_kernel<<<1, 32>>>(L, dth, n, mode, base, slot, cap, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out4, dout, 4 * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(base);
    cudaFree(dth);
    cudaFree(dout);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return TW_ECUDA; }
    return TW_OK;
}
