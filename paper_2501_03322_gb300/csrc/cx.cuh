// cx.cuh -- minimal complex arithmetic for the device code (FP64 and FP32).
//
// Plain structs so that everything stays in registers.  The FP32 division
// rescales its divisor first because polynomial values near a root of a
// low-mass-ratio lens can be small enough for |b|^2 to underflow in single
// precision.
#pragma once
#include <cuda_runtime.h>

namespace tw {

template <typename T>
struct cx {
    T x, y;
};
using cxd = cx<double>;
using cxf = cx<float>;

template <typename T>
__device__ __forceinline__ cx<T> mk(T a, T b) { return cx<T>{a, b}; }
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return {s * a.x, s * a.y}; }
// a b + c as four fused multiply-adds (the operator form leaves a separate
// multiply and add per component)
__device__ __forceinline__ cx<double> cmad(cx<double> a, cx<double> b, cx<double> c) {
    return {fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}
__device__ __forceinline__ cx<float> cmad(cx<float> a, cx<float> b, cx<float> c) {
    return {fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y))};
}
template <typename T>
__device__ __forceinline__ cx<T> conj(cx<T> a) { return {a.x, -a.y}; }
template <typename T>
__device__ __forceinline__ T norm2(cx<T> a) { return a.x * a.x + a.y * a.y; }
// a ^ b = Re(a) Im(b) - Im(a) Re(b)  (the wedge product of Eq. 8)
template <typename T>
__device__ __forceinline__ T wedge(cx<T> a, cx<T> b) { return a.x * b.y - a.y * b.x; }
// real dot product Re(conj(a) b)
template <typename T>
__device__ __forceinline__ T dot(cx<T> a, cx<T> b) { return a.x * b.x + a.y * b.y; }

// FP64 reciprocal: the hardware approximation (rcp.approx.ftz.f64, about 20
// correct bits) refined by two Newton-Raphson steps y <- y + y (1 - v y), each
// of which doubles the number of correct bits.  Five FP64-pipe instructions
// instead of an IEEE-rounded division; the last bit may differ from 1/v.
// Inputs are kept in the normal range by the callers (|v| >= 1e-300).
__device__ __forceinline__ double rcp(double v) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(v));
    double e = fma(-v, y, 1.0);
    y = fma(y, e, y);
    e = fma(-v, y, 1.0);
    return fma(y, e, y);
}
// FP64 reciprocal to about 40 bits (the approximation and one refinement
// step): for quantities whose relative accuracy need not reach FP64, such as
// the Aberth correction of a root (its error then scales the correction,
// which vanishes at convergence).
__device__ __forceinline__ double rcp40(double v) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(v));
    const double e = fma(-v, y, 1.0);
    return fma(y, e, y);
}
// a / b with rcp40.
__device__ __forceinline__ cx<double> cdiv40(cx<double> a, cx<double> b) {
    const double r = rcp40(fmax(norm2(b), 1e-300));
    return {(a.x * b.x + a.y * b.y) * r, (a.y * b.x - a.x * b.y) * r};
}
__device__ __forceinline__ cx<float> cdiv40(cx<float> a, cx<float> b);

// FP32 reciprocal: the hardware approximation (rcp.approx.ftz.f32, ~1 ulp),
// enough for the FP32 root iteration.
__device__ __forceinline__ float rcp(float v) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
    return y;
}

__device__ __forceinline__ cxd inv(cxd a) {
    double r = rcp(fmax(norm2(a), 1e-300));
    return {a.x * r, -a.y * r};
}
__device__ __forceinline__ cxd cdiv(cxd a, cxd b) {
    double r = rcp(fmax(norm2(b), 1e-300));
    return {(a.x * b.x + a.y * b.y) * r, (a.y * b.x - a.x * b.y) * r};
}
__device__ __forceinline__ cxf inv(cxf a) {
    float sc = fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), 1e-30f);
    float k = rcp(sc);
    cxf b = {a.x * k, a.y * k};
    float r = rcp(norm2(b)) * k;
    return {b.x * r, -b.y * r};
}
__device__ __forceinline__ cxf cdiv(cxf a, cxf b) {
    float sc = fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)), 1e-30f);
    float k = rcp(sc);
    cxf bb = {b.x * k, b.y * k};
    cxf aa = {a.x * k, a.y * k};
    float r = rcp(norm2(bb));
    return {(aa.x * bb.x + aa.y * bb.y) * r, (aa.y * bb.x - aa.x * bb.y) * r};
}

__device__ __forceinline__ cxf cdiv40(cxf a, cxf b) { return cdiv(a, b); }

__device__ __forceinline__ cxf to_f(cxd a) { return {(float)a.x, (float)a.y}; }
__device__ __forceinline__ cxd to_d(cxf a) { return {(double)a.x, (double)a.y}; }

// Squared modulus in FP32, for magnitudes that only feed thresholds: FP64
// components are converted first, which costs fewer FP64-pipe instructions
// than an FP64 norm and a conversion.
__device__ __forceinline__ float norm2f(cxd a) { return norm2(to_f(a)); }
__device__ __forceinline__ float norm2f(cxf a) { return norm2(a); }

}  // namespace tw
