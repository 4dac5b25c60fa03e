// k_surrogate.cu -- BF16 MLP surrogate of the finite-source magnification,
// with contour-integration fallback; training and inference.
//
// The network maps x = (log10 s, log10 q, log10 rho, y1, y2, and three
// features of the query's point-source expansion; standardised) through
// 8 -> 256 -> 256 -> 256 -> 256 -> 2 (ReLU) to (r, l).  The expansion is the
// hexadecapole approximation A_hex (point-source magnifications at the centre
// and on rings, Gould 2008; the paper tests point-source adequacy the same
// way, Sec. 2.3); the network predicts mu = A_hex (1 + gap / 15) exp(r), the
// middle factor being the Richardson step between the expansions from two
// ring pairs, and l = ln(sigma) its uncertainty in ln mu.  Learning only what
// the expansion misses keeps the BF16 network's errors on a quantity that is
// tiny away from caustics.  The three 256 x 256 layers run on the tensor
// cores (k_gemm.cu, BF16 weights and activations, FP32 accumulation); the
// input layer and the 256 -> 2 head run in FP32 on CUDA cores.
//
// Inference: per query, point-source images (Eq. 6 quintic, FP32 Aberth +
// FP64 Newton, residual ghost test, A = sum 1/|J|) at the centre and at 8
// points on each of three rings (radius rho/2, rho and 2 rho), the hexadecapole
// approximation with its error estimate, a near-caustic flag (the image count
// differs between the centre and a ring point, min |J| < 0.01 at the centre, or
// the error estimate exceeds 5% of the value), the MLP, and the fallback
// decision: flagged, or neither the expansion's error estimate nor the
// network's calibrated kappa * sigma is within rel_tol.  The flag also sweeps
// the caustic itself: a caustic smaller than the ring spacing can sit inside
// the source without any ring point seeing it.  Fallback queries are
// integrated by the contour kernel in one persistent launch.
//
// Training: positions are drawn near caustics (a random point of a random
// branch of the caustic, displaced uniformly in a disc of three times that
// branch's bounding-box size).  The network is trained only where it can
// answer: unflagged positions whose expansion error estimate is above a
// quarter of 1e-4 (below half the tolerance the expansion answers by
// itself) and at most 2e-3.  These are labelled by the contour integrator (FP64, rel_tol
// 1e-6), and the network is fitted by the Gaussian negative log-likelihood of
// the standardised r with Adam on FP32 master weights; a held-out tenth
// calibrates the acceptance factor kappa.
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/twinkle.h"
#include "gemm.cuh"
#include "ptrkind.cuh"
#include "kernels.cuh"

namespace tw {

constexpr int SH = 256;   // hidden width
constexpr int SNIN = 8;   // inputs: the five query parameters and three expansion features
constexpr int SXP = 8;    // input row (floats)
// offsets in the FP32 parameter blob (weights stored [out][in])
constexpr int OW1 = 0, OB1 = OW1 + SH * SNIN;
constexpr int OW2 = OB1 + SH, OB2 = OW2 + SH * SH;
constexpr int OW3 = OB2 + SH, OB3 = OW3 + SH * SH;
constexpr int OW4 = OB3 + SH, OB4 = OW4 + SH * SH;
constexpr int OW5 = OB4 + SH, OB5 = OW5 + 2 * SH;
constexpr int NPAR = OB5 + 2;
constexpr int OWH[3] = {OW2, OW3, OW4};
constexpr int OBH[3] = {OB2, OB3, OB4};

// Input standardisation, target standardisation (the network's r is
// tmean + tstd * a, its sigma tstd * exp(b)), the acceptance factor
// calibrated on held-out rows, and the expansion-error band the network was
// trained on (it answers only queries whose expansion error estimate lies in
// (band, band_hi]).
struct SurNorm {
    float mean[SNIN], inv_std[SNIN];
    float tmean, tstd, kappa_cal, band, band_hi;
};

// ------------------------------------------------------------ random numbers
// splitmix64 (Steele, Lea & Flood 2014): a counter-based 64-bit generator.
__device__ __forceinline__ uint64_t splitmix64(uint64_t &x) {
    x += 0x9E3779B97F4A7C15ull;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double u01(uint64_t &st) { return (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0); }

// ------------------------------------------------- training-position sampler
// Critical curve (f'(z) = e^{i phi}, Eq. 7 with |f'| = 1) in the secondary's
// frame eta = z - z2:  e eta^4 + 2 s e eta^3 + (s^2 e - 1) eta^2 - 2 s m2 eta - m2 s^2 = 0.
constexpr int NPHI = 64;

__global__ void sur_sample_kernel(uint64_t seed, int64_t n, double *S, double *Q, double *RHO, double *Y1,
                                  double *Y2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t st = seed * 0xD1B54A32D192ED03ull + (uint64_t)i * 0x9E3779B97F4A7C15ull;
    (void)splitmix64(st);
    const double s = exp10(-0.5 + u01(st));
    const double q = exp10(-5.0 + 4.0 * u01(st));
    const double rho = exp10(-4.0 + 2.0 * u01(st));
    const double m2 = q / (1.0 + q), m1 = 1.0 - m2;
    const int kb = (int)(u01(st) * NPHI) % NPHI;
    const int bb = (int)(u01(st) * 4.0) & 3;
    cxd z[4];
    const double r0 = 1.0 + s;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        double sn, cs;
        sincos(1.5707963267948966 * k + 0.3, &sn, &cs);
        z[k] = {-0.5 * s + r0 * cs, r0 * sn};
    }
    double bx0 = 1e300, bx1 = -1e300, by0 = 1e300, by1 = -1e300;
    cxd chosen = {0.0, 0.0};
    for (int k = 0; k < NPHI; k++) {
        double sn, cs;
        sincos(6.283185307179586 * k / NPHI, &sn, &cs);
        const cxd e = {cs, sn};
        cxd c[5];
        c[4] = e;
        c[3] = (2.0 * s) * e;
        c[2] = {s * s * cs - 1.0, s * s * sn};
        c[1] = {-2.0 * s * m2, 0.0};
        c[0] = {-m2 * s * s, 0.0};
        // Aberth-Ehrlich iteration warm-started from the previous angle, so each
        // root index follows one branch of the critical curve
        for (int it = 0; it < (k == 0 ? 200 : 60); it++) {
            cxd S4[4];
#pragma unroll
            for (int a = 0; a < 4; a++) S4[a] = {0.0, 0.0};
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = a + 1; b < 4; b++) {
                    const cxd r = inv(z[a] - z[b]);
                    S4[a] = S4[a] + r;
                    S4[b] = S4[b] - r;
                }
            double wmax = 0.0, zmax = 0.0;
            cxd w[4];
#pragma unroll
            for (int a = 0; a < 4; a++) {
                cxd p = c[4], d = {0.0, 0.0};
#pragma unroll
                for (int t = 3; t >= 0; t--) {
                    d = d * z[a] + p;
                    p = p * z[a] + c[t];
                }
                w[a] = cdiv(p, d - p * S4[a]);
                wmax = fmax(wmax, norm2(w[a]));
                zmax = fmax(zmax, norm2(z[a]));
            }
#pragma unroll
            for (int a = 0; a < 4; a++) z[a] = z[a] - w[a];
            if (wmax <= 1e-26 * (zmax + 1e-30)) break;
        }
        cxd eta = z[0];
#pragma unroll
        for (int a = 1; a < 4; a++)
            if (a == bb) eta = z[a];
        const cxd g = m1 * inv(cxd{eta.x + s, eta.y}) + m2 * inv(eta);
        const cxd y = eta - conj(g);  // caustic point, secondary frame
        bx0 = fmin(bx0, y.x);
        bx1 = fmax(bx1, y.x);
        by0 = fmin(by0, y.y);
        by1 = fmax(by1, y.y);
        if (k == kb) chosen = y;
    }
    const double wdt = fmax(bx1 - bx0, by1 - by0);
    const double rr = 3.0 * wdt * sqrt(u01(st));
    double sn, cs;
    sincos(6.283185307179586 * u01(st), &sn, &cs);
    S[i] = s;
    Q[i] = q;
    RHO[i] = rho;
    Y1[i] = chosen.x + rr * cs + s * m1;  // back to the centre-of-mass frame (z2 = s m1)
    Y2[i] = chosen.y + rr * sn;
}

// ------------------------------------------------ point-source images, flag
// Images of a point source at y (secondary frame): FP32 Aberth from z, then
// (fp64 = true) one or two FP64 Newton steps.  Returns the image count by the
// residual pair test (Sec. 2.4.1) and, for the real images, sum 1/|J| and
// min |J| (Eq. 7).
template <bool FP64>
static __device__ __noinline__ int point_images(const LensK &L, cxd y, cxd z[5], double &mu_ps, double &minJ,
                                                int &sweeps, int &newton) {
    cxd c[6];
    eq6_coeffs(L.s, L.m2, y, c);
    float ca[6];
    abs_coeffs(c, ca);
    const float cm = fmaxf(fmaxf(fmaxf(ca[0], ca[1]), fmaxf(ca[2], ca[3])), fmaxf(ca[4], ca[5]));
    const double sc = 1.0 / (double)cm;
    cxf cf[6];
    float caf[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        cf[k] = to_f(sc * c[k]);
        caf[k] = ca[k] / cm;
    }
    cxf zf[5];
#pragma unroll
    for (int i = 0; i < 5; i++) zf[i] = to_f(z[i]);
    float dpa[5];
    int it = 0;
    for (; it < 100; it++)
        if (aberth_sweep<float>(cf, caf, zf, dpa, 2e-6f, 6e-8f)) break;
    sweeps += it < 100 ? it + 1 : it;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        z[i] = to_d(zf[i]);
        if (FP64) {
            newton++;
            // one Newton step from FP32 accuracy reaches FP64 accuracy (the error
            // squares); a second where the FP32 root was poor (a step above
            // 1e-6 |z|, next to a near-double root)
            cxd p, d;
            horner(c, z[i], p, d);
            cxd st = cdiv40(p, d);
            z[i] = z[i] - st;
            if (norm2f(st) > 1e-12f * norm2f(z[i])) {
                newton++;
                horner(c, z[i], p, d);
                st = cdiv40(p, d);
                z[i] = z[i] - st;
            }
        }
    }
    double aR[5], J[5];
    cxd R[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const cxd d1 = inv(cxd{z[i].x + L.s, z[i].y}), d2 = inv(z[i]);
        R[i] = y - z[i] + conj(L.m1 * d1 + L.m2 * d2);
        aR[i] = norm2(R[i]);
        const cxd f1 = L.m1 * (d1 * d1) + L.m2 * (d2 * d2);
        J[i] = 1.0 - norm2(f1);
    }
    int r3 = 0, r4 = 0, r5 = 0;
    int rank[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        int r = 0;
#pragma unroll
        for (int j = 0; j < 5; j++)
            if (j != i) r += (aR[j] < aR[i]) || (aR[j] == aR[i] && j < i);
        rank[i] = r;
        if (r == 2) r3 = i;
        if (r == 3) r4 = i;
        if (r == 4) r5 = i;
    }
    cxd R45 = {0.0, 0.0};
    double a3 = 0, a4 = 0, a5 = 0;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        if (i == r4 || i == r5) R45 = R45 + R[i];
        if (i == r3) a3 = aR[i];
        if (i == r4) a4 = aR[i];
        if (i == r5) a5 = aR[i];
    }
    const int count = (norm2(R45) < 1e-4 * a5 && a4 > 100.0 * a3) ? 3 : 5;
    mu_ps = 0.0;
    minJ = 1e300;
#pragma unroll
    for (int i = 0; i < 5; i++)
        if (rank[i] < count) {
            mu_ps += 1.0 / fabs(J[i]);
            minJ = fmin(minJ, fabs(J[i]));
        }
    return count;
}

// Is the caustic within `reach` of the source centre y0 (secondary frame)?  The
// critical curve (the sampler's quartic above) is swept at NCAU angles in FP32 with
// warm-started Aberth iterations; each branch's caustic points form a
// polyline, and the query is near when a segment comes within `reach` plus
// the segment's length (slack for the arc the chord cuts off).
constexpr int NCAU = 64;
__device__ bool caustic_within(float s, float m2, float m1, cxf y0, float reach, int &iters) {
    cxf z[4];
    const float r0 = 1.0f + s;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        float sn, cs;
        sincosf(1.5707963f * k + 0.3f, &sn, &cs);
        z[k] = {-0.5f * s + r0 * cs, r0 * sn};
    }
    cxf prev[4];
    bool near = false;
    for (int k = 0; k < NCAU && !near; k++) {
        float sn, cs;
        sincosf(6.2831853f * k / NCAU, &sn, &cs);
        const cxf e = {cs, sn};
        cxf c[5];
        c[4] = e;
        c[3] = (2.0f * s) * e;
        c[2] = {s * s * cs - 1.0f, s * s * sn};
        c[1] = {-2.0f * s * m2, 0.0f};
        c[0] = {-m2 * s * s, 0.0f};
        for (int it = 0; it < (k == 0 ? 120 : 30); it++) {
            iters++;
            cxf S4[4];
#pragma unroll
            for (int a = 0; a < 4; a++) S4[a] = {0.f, 0.f};
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = a + 1; b < 4; b++) {
                    const cxf r = inv(z[a] - z[b]);
                    S4[a] = S4[a] + r;
                    S4[b] = S4[b] - r;
                }
            float wmax = 0.f, zmax = 0.f;
            cxf w[4];
#pragma unroll
            for (int a = 0; a < 4; a++) {
                cxf p = c[4], d = {0.f, 0.f};
#pragma unroll
                for (int t = 3; t >= 0; t--) {
                    d = d * z[a] + p;
                    p = p * z[a] + c[t];
                }
                w[a] = cdiv(p, d - p * S4[a]);
                wmax = fmaxf(wmax, norm2(w[a]));
                zmax = fmaxf(zmax, norm2(z[a]));
            }
#pragma unroll
            for (int a = 0; a < 4; a++) z[a] = z[a] - w[a];
            if (wmax <= 1e-12f * (zmax + 1e-30f)) break;
        }
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const cxf g = m1 * inv(cxf{z[a].x + s, z[a].y}) + m2 * inv(z[a]);
            const cxf cpt = z[a] - conj(g);  // caustic point
            if (k > 0) {
                const cxf d = cpt - prev[a], v = y0 - prev[a];
                const float L2 = norm2(d);
                const float t = L2 > 0.f ? fminf(fmaxf(dot(v, d) / L2, 0.f), 1.f) : 0.f;
                const cxf cl = {prev[a].x + t * d.x - y0.x, prev[a].y + t * d.y - y0.y};
                const float lim = reach + sqrtf(L2);
                if (norm2(cl) < lim * lim) near = true;
            }
            prev[a] = cpt;
        }
    }
    return near;
}

// Raw features, point-source magnification and near-caustic flag per query.
// One thread per query for its centre solve and caustic sweep; the 24 ring
// points of the queries of a warp that are still unflagged are then spread
// over all 32 lanes (lanes whose queries were flagged would otherwise idle),
// each lane taking the lens and centre images of the query it serves by warp
// shuffles, and each query's owner sums its ring values in a fixed order.
constexpr int RING_PTS = 24;  // 3 rings x 8 points

__global__ void __launch_bounds__(128, 3) sur_features_kernel(int64_t n, const double *S, const double *Q,
                                                              const double *RHO, const double *Y1, const double *Y2,
                                                              float *X, double *MUPS, uint8_t *FLAG, float *HEXE,
                                                              unsigned long long *WORK) {
    __shared__ double sM[4][32][RING_PTS];  // ring-point magnifications per query slot
    __shared__ int sBad[4][32];             // a ring point's image count differed
    __shared__ int sOwner[4][32];           // lane of the j-th unflagged query
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const bool in = i < n;
    double s = 1.0, q = 1.0, rho = 1.0, y1 = 0.0, y2 = 0.0;
    if (in) {
        s = S[i];
        q = Q[i];
        rho = RHO[i];
        y1 = Y1[i];
        y2 = Y2[i];
        float *x = X + i * SXP;
        x[0] = (float)log10(s);
        x[1] = (float)log10(q);
        x[2] = (float)log10(rho);
        x[3] = (float)y1;
        x[4] = (float)y2;
        x[5] = x[6] = x[7] = 0.f;
    }
    const bool ok = in && s > 0 && q > 0 && rho > 0 && isfinite(s) && isfinite(q) && isfinite(rho) && isfinite(y1) &&
                    isfinite(y2);
    LensK L;
    L.s = 1.0;
    L.m1 = 1.0;
    L.m2 = 0.0;
    L.rho = 1.0;
    cxd y0 = {0.0, 0.0};
    cxd z[5];
#pragma unroll
    for (int k = 0; k < 5; k++) z[k] = {0.0, 0.0};
    double A0 = __longlong_as_double(0x7ff8000000000000ll), minJ = 0.0;
    int c0 = 0;
    bool flag = true;
    // work of this thread: point solves, FP32 Aberth sweeps, FP64 Newton root
    // steps, caustic Aberth iterations (the units of the FLOP accounting)
    int w_solve = 0, w_sweep = 0, w_newton = 0, w_caus = 0;
    if (ok) {
        if (q > 1.0) { q = 1.0 / q; y1 = -y1; }  // mass-swap symmetry (see kernels.cuh)
        L.s = s;
        L.m1 = 1.0 / (1.0 + q);
        L.m2 = q * L.m1;
        L.rho = rho;
        y0 = {y1 - s * L.m1, y2};
        initial_roots(s, y0, z);
        c0 = point_images<true>(L, y0, z, A0, minJ, w_sweep, w_newton);
        w_solve++;
        // an image within |J| < 1e-2 of a critical curve: the point solve and
        // the ring expansion lose accuracy there.  (A bound of 0.1 also flagged
        // 12% of the queries that lie many source radii from any caustic,
        // high-magnification positions the expansion's error estimate handles:
        // measured against FP64 contour integration at rel_tol 1e-6 on 4 x 2^20
        // queries, 1e-2 leaves every error unchanged while 1e-3 lets through
        // one more error above 1e-4.)
        flag = !(isfinite(A0) && A0 >= 1.0 - 1e-3) || minJ < 1e-2;
        // within 4 rho (not just 2 rho): closer than that the ring at 2 rho nears
        // the caustic and the expansion's error estimate is no longer reliable
        if (!flag)
            flag = caustic_within((float)s, (float)L.m2, (float)L.m1, to_f(y0), (float)(4.0 * rho) + 1e-6f, w_caus);
    }
    // Point-source magnifications averaged over 8 points on rings of radius
    // rho/2, rho and 2 rho.  For a smooth A, the average over a ring of radius
    // r is A0 + c1 r^2 + c2 r^4 + c3 r^6 + ... (c1 = lap A / 4, c2 = lap^2 A / 64)
    // and the disc average is A0 + c1 rho^2/2 + c2 rho^4/3 + c3 rho^6/4 + ...
    // Two rings at lam rho and 2 lam rho fix c1 and c2 (the hexadecapole
    // approximation, Gould 2008, with rings of other radii); the c3 term they
    // leave out shifts the result by -(7/12) c3 rho^6 for lam = 1 and by
    // +(1/24) c3 rho^6 for lam = 1/2.  The lam = 1/2 value is returned and the
    // difference of the two, 15/24 c3 rho^6 (about 15 times its error while
    // the series converges), is its error estimate.  The image count must be
    // the centre's at every ring point (otherwise a caustic is within 2 rho).
    const bool want = ok && !flag;
    const unsigned act = __ballot_sync(0xffffffffu, want);
    const int na = __popc(act);
    sBad[wib][lane] = 0;
    if (want) sOwner[wib][__popc(act & ((1u << lane) - 1u))] = lane;
    __syncwarp();
    for (int base = 0; base < RING_PTS * na; base += 32) {
        const int t = base + lane;
        const bool has = t < RING_PTS * na;
        const int j = has ? t / RING_PTS : 0, k = t % RING_PTS;
        const int src = sOwner[wib][has ? j : 0];
        LensK Lk;
        Lk.s = __shfl_sync(0xffffffffu, L.s, src);
        Lk.m1 = __shfl_sync(0xffffffffu, L.m1, src);
        Lk.m2 = __shfl_sync(0xffffffffu, L.m2, src);
        Lk.rho = __shfl_sync(0xffffffffu, L.rho, src);
        const cxd yc = {__shfl_sync(0xffffffffu, y0.x, src), __shfl_sync(0xffffffffu, y0.y, src)};
        cxd zk[5];
#pragma unroll
        for (int a = 0; a < 5; a++) zk[a] = {__shfl_sync(0xffffffffu, z[a].x, src), __shfl_sync(0xffffffffu, z[a].y, src)};
        const int ck = __shfl_sync(0xffffffffu, c0, src);
        if (has) {
            const int ring = k >> 3;
            double sn, cs;
            sincos(0.7853981633974483 * (k & 7) + 0.2, &sn, &cs);
            const double r = (0.5 * (1 << ring)) * Lk.rho;
            const cxd yk = {yc.x + r * cs, yc.y + r * sn};
            double m, mj;
            const int cnt = point_images<true>(Lk, yk, zk, m, mj, w_sweep, w_newton);
            w_solve++;
            sM[wib][src][k] = m;
            if (cnt != ck || !isfinite(m)) atomicOr(&sBad[wib][src], 1);
        }
    }
    __syncwarp();
    double Ahex = A0, hexe = 1.0, dgap = 0.0, corr = 0.0;
    if (want) {
        double R[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 0; k < RING_PTS; k++) R[k >> 3] += 0.125 * sM[wib][lane][k];
        if (sBad[wib][lane]) flag = true;
        if (!flag) {
            // disc average from the rings at lam rho and 2 lam rho
            auto disc = [A0](double Ra, double Rb, double lam) {
                const double d1 = Ra - A0, d2 = Rb - A0, l2 = lam * lam;
                const double c2 = (d2 - 4.0 * d1) / (12.0 * l2 * l2);  // c2 rho^4
                const double c1 = d1 / l2 - c2 * l2;                   // c1 rho^2
                return A0 + 0.5 * c1 + c2 / 3.0;
            };
            Ahex = disc(R[0], R[1], 0.5);
            // error estimate: the gap between the two expansions, but not below
            // a twentieth of the whole finite-source correction |Ahex - A0|.
            // Measured against the oracle, the gap alone missed the error by up
            // to 25x on about 1e-5 of the queries, all with corrections of
            // 0.2-6%; the floor limits the expansion to corrections of at most
            // 10 rel_tol.
            dgap = (disc(R[1], R[2], 1.0) - Ahex) / Ahex;
            corr = (Ahex - A0) / Ahex;
            hexe = fmax(fabs(dgap), 0.05 * fabs(corr));
            // a series that is not converging marks the neighbourhood of a caustic
            if (!(Ahex > 0.0) || !(hexe <= 0.05)) flag = true;
        }
    }
    if (in) {
        MUPS[i] = ok ? Ahex : __longlong_as_double(0x7ff8000000000000ll);
        FLAG[i] = flag ? 1 : 0;
        HEXE[i] = (float)fmin(hexe, 1.0);
        // expansion features of the network: the decade of the error estimate,
        // the signed ring gap in units of it (the gap over 15 is the
        // Richardson step from the (rho/2, rho) expansion towards the exact
        // disc average, the c3 rho^6 term above) and the signed size of the
        // finite-source correction
        float *x = X + i * SXP;
        const bool fin = !flag && hexe > 0.0;
        x[5] = fin ? (float)log10(fmax(hexe, 1e-10)) : 0.f;
        x[6] = fin ? (float)(dgap / hexe) : 0.f;
        x[7] = fin ? (float)copysign(log10(1.0 + 1e6 * fabs(corr)), corr) : 0.f;
    }
    if (WORK) {
        const int a = __reduce_add_sync(0xffffffffu, w_solve), b = __reduce_add_sync(0xffffffffu, w_sweep);
        const int c = __reduce_add_sync(0xffffffffu, w_newton), d = __reduce_add_sync(0xffffffffu, w_caus);
        if (lane == 0) {
            atomicAdd(WORK + 0, (unsigned long long)a);
            atomicAdd(WORK + 1, (unsigned long long)b);
            atomicAdd(WORK + 2, (unsigned long long)c);
            atomicAdd(WORK + 3, (unsigned long long)d);
        }
    }
}

// ------------------------------------------------------------- MLP kernels
// Layer 1 (5 -> 256, ReLU) on CUDA cores; optionally the standardised inputs.
__global__ void sur_layer1_kernel(int64_t rows, const float *X, const float *P, SurNorm nrm, __nv_bfloat16 *H1,
                                  float *XS) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * SH) return;
    const int64_t r = t / SH;
    const int o = (int)(t % SH);
    float xs[SNIN];
#pragma unroll
    for (int k = 0; k < SNIN; k++) xs[k] = (X[r * SXP + k] - nrm.mean[k]) * nrm.inv_std[k];
    float h = P[OB1 + o];
#pragma unroll
    for (int k = 0; k < SNIN; k++) h = fmaf(P[OW1 + o * SNIN + k], xs[k], h);
    H1[r * SH + o] = __float2bfloat16_rn(fmaxf(h, 0.f));
    if (XS && o < SXP) XS[r * SXP + o] = o < SNIN ? xs[o] : 0.f;
}

// Richardson step of the expansion (ln of A_hex (1 + gap / 15)), the base
// the network's r is added to; X holds the query's features.
__device__ __forceinline__ double richardson_base(const float *x, float hexe) {
    return log1p((double)x[6] * (double)hexe / 15.0);
}

// Head (256 -> 2) and fallback decision; one warp per query.  A query is
// answered by the expansion when its error estimate is within half the
// tolerance, else by the network when it lies in the network's band and
// max(kappa, kappa_cal) sigma <= tol; every other query is queued for contour
// integration.  PSTAT (optional) receives TW_POS_EXPANSION or TW_POS_NETWORK
// for the answered queries.
__global__ void sur_head_infer_kernel(int64_t n, int64_t row0, const __nv_bfloat16 *H4, const float *P,
                                      const float *X, SurNorm nrm, const double *MUPS, const uint8_t *FLAG,
                                      const float *HEXE, double tol, float kappa, double *OUT, int8_t *PSTAT,
                                      int32_t *LIST, unsigned long long *NLIST) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const uint4 v = *(const uint4 *)(H4 + w * SH + lane * 8);
    const __nv_bfloat16 *h = (const __nv_bfloat16 *)&v;
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const float x = __bfloat162float(h[j]);
        a = fmaf(P[OW5 + lane * 8 + j], x, a);
        b = fmaf(P[OW5 + SH + lane * 8 + j], x, b);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        const int64_t g = row0 + w;
        const float hx = HEXE[g];
        const double r = (double)nrm.tmean + (double)nrm.tstd * (double)(a + P[OB5]);
        const float sig = nrm.tstd * expf(fminf(fmaxf(b + P[OB5 + 1], -25.f), 5.f));
        const bool hex_ok = hx <= 0.5f * (float)tol;
        const bool mlp_ok = hx > nrm.band && hx <= nrm.band_hi && fmaxf(kappa, nrm.kappa_cal) * sig <= (float)tol;
        const double mu = hex_ok ? MUPS[g] : MUPS[g] * exp(richardson_base(X + w * SXP, hx) + r);
        if (FLAG[g] || !(hex_ok || mlp_ok) || !isfinite(mu)) {
            const unsigned long long slot = atomicAdd(NLIST, 1ull);
            LIST[slot] = (int32_t)g;
            OUT[g] = __longlong_as_double(0x7ff8000000000000ll);
            if (FLAG[g]) atomicAdd(NLIST + 3, 1ull);
        } else {
            OUT[g] = mu;
            if (PSTAT) PSTAT[g] = (int8_t)(hex_ok ? TW_POS_EXPANSION : TW_POS_NETWORK);
            atomicAdd(NLIST + (hex_ok ? 2 : 1), 1ull);
        }
    }
}

// Head forward, Gaussian negative log-likelihood of the target t with weight
// wt, its gradient with respect to the head outputs (DOUT), and the masked
// gradient of the last hidden layer (G4 = dL/dh4 * [h4 > 0]); one warp per row.
__global__ void sur_head_train_kernel(int B, const __nv_bfloat16 *H4, const float *P, const float *T, const float *WT,
                                      float *DOUT, __nv_bfloat16 *G4, float *LOSS) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= B) return;
    const uint4 v = *(const uint4 *)(H4 + (size_t)w * SH + lane * 8);
    const __nv_bfloat16 *h = (const __nv_bfloat16 *)&v;
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const float x = __bfloat162float(h[j]);
        a = fmaf(P[OW5 + lane * 8 + j], x, a);
        b = fmaf(P[OW5 + SH + lane * 8 + j], x, b);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const float r = a + P[OB5];
    const float l = fminf(fmaxf(b + P[OB5 + 1], -25.f), 5.f);
    const float wt = WT[w] / (float)B;
    const float d = T[w] - r, ie2 = expf(-2.f * l);
    const float dr = -d * ie2 * wt, dl = (1.f - d * d * ie2) * wt;
    if (lane == 0) {
        DOUT[2 * w] = dr;
        DOUT[2 * w + 1] = dl;
        atomicAdd(LOSS, 0.5f * (d * d * ie2 + 2.f * l) * wt);
    }
    __nv_bfloat16 g[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const int k = lane * 8 + j;
        const float gv = dr * P[OW5 + k] + dl * P[OW5 + SH + k];
        g[j] = __float2bfloat16_rn(__bfloat162float(h[j]) > 0.f ? gv : 0.f);
    }
    *(uint4 *)(G4 + (size_t)w * SH + lane * 8) = *(uint4 *)g;
}

// dW5 = DOUT^T H4, db5 = column sums of DOUT.
__global__ void sur_head_wgrad_kernel(int B, const float *DOUT, const __nv_bfloat16 *H4, float *G) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * SH + 2) return;
    float acc = 0.f;
    if (t < 2 * SH) {
        const int o = t / SH, k = t % SH;
        for (int b = 0; b < B; b++) acc = fmaf(DOUT[2 * b + o], __bfloat162float(H4[(size_t)b * SH + k]), acc);
        G[OW5 + t] = acc;
    } else {
        const int o = t - 2 * SH;
        for (int b = 0; b < B; b++) acc += DOUT[2 * b + o];
        G[OB5 + o] = acc;
    }
}

// out[c][r] = in[r][c] for a R x C bf16 matrix (32 x 32 tiles).
__global__ void transpose_bf16_kernel(int R, int C, const __nv_bfloat16 *in, __nv_bfloat16 *out) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[k][threadIdx.x] = in[(size_t)r * C + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < R && c < C) out[(size_t)c * R + r] = tile[threadIdx.x][k];
    }
}

// G = DH * [H > 0] (bf16).
__global__ void relu_mask_kernel(int64_t n, const float *DH, const __nv_bfloat16 *H, __nv_bfloat16 *G) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    G[i] = __float2bfloat16_rn(__bfloat162float(H[i]) > 0.f ? DH[i] : 0.f);
}

// out[c] = sum_r G[r][c] (bias gradient).
__global__ void colsum_bf16_kernel(int B, const __nv_bfloat16 *Gm, float *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= SH) return;
    float acc = 0.f;
    for (int b = 0; b < B; b++) acc += __bfloat162float(Gm[(size_t)b * SH + c]);
    out[c] = acc;
}

// Layer-1 gradients from DH1 (unmasked, fp32) and the standardised inputs.
__global__ void sur_layer1_bwd_kernel(int B, const float *DH1, const __nv_bfloat16 *H1, const float *XS, float *G) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= SH) return;
    float gw[SNIN], gb = 0.f;
#pragma unroll
    for (int k = 0; k < SNIN; k++) gw[k] = 0.f;
    for (int b = 0; b < B; b++) {
        const float g = __bfloat162float(H1[(size_t)b * SH + o]) > 0.f ? DH1[(size_t)b * SH + o] : 0.f;
        gb += g;
#pragma unroll
        for (int k = 0; k < SNIN; k++) gw[k] = fmaf(g, XS[(size_t)b * SXP + k], gw[k]);
    }
#pragma unroll
    for (int k = 0; k < SNIN; k++) G[OW1 + o * SNIN + k] = gw[k];
    G[OB1 + o] = gb;
}

__global__ void adam_kernel(int n, float *Pm, const float *G, float *M1, float *M2, float lr, float b1, float b2,
                            float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float m = b1 * M1[i] + (1.f - b1) * g;
    const float v = b2 * M2[i] + (1.f - b2) * g * g;
    M1[i] = m;
    M2[i] = v;
    Pm[i] -= lr * (m * c1) / (sqrtf(v * c2) + 1e-8f);
}

// BF16 copies of the hidden-layer weights: forward ([out][in]) and transposed.
__global__ void refresh_bf16_kernel(const float *Pm, __nv_bfloat16 *Wf, __nv_bfloat16 *Wt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * SH * SH) return;
    const int l = t / (SH * SH), e = t % (SH * SH), o = e / SH, k = e % SH;
    const __nv_bfloat16 v = __float2bfloat16_rn(Pm[(l == 0 ? OW2 : l == 1 ? OW3 : OW4) + e]);
    Wf[(size_t)l * SH * SH + e] = v;
    Wt[(size_t)l * SH * SH + (size_t)k * SH + o] = v;
}

// Targets r = ln(mu) - ln(A_hex) - (Richardson base) and weights: 1 for the
// rows of the network's band (not flagged, expansion error estimate in
// (band, band_hi]) whose label converged, else 0.
__global__ void sur_targets_kernel(int64_t n, const double *MU, const double *MUPS, const uint8_t *FLAG,
                                   const float *HEXE, const float *X, const int8_t *LSTAT, float band, float band_hi,
                                   float *T, float *WT) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double r = log(MU[i]) - log(MUPS[i]) - richardson_base(X + i * SXP, HEXE[i]);
    const bool ok = !FLAG[i] && HEXE[i] > band && HEXE[i] <= band_hi && LSTAT[i] == 0 && isfinite(r);
    T[i] = ok ? (float)r : 0.f;
    WT[i] = ok ? 1.f : 0.f;
}

// indices of the rows in the network's band
__global__ void compact_band_kernel(int64_t n, const uint8_t *FLAG, const float *HEXE, float band, float band_hi,
                                    int32_t *LIST, unsigned long long *NLIST) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || FLAG[i] || !(HEXE[i] > band && HEXE[i] <= band_hi)) return;
    LIST[atomicAdd(NLIST, 1ull)] = (int32_t)i;
}

// (t - mean) / std in place
__global__ void standardise_kernel(int64_t n, float *T, float mean, float inv_std) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) T[i] = (T[i] - mean) * inv_std;
}

// Held-out evaluation: per row the head's standardised error |t - a| / exp(b)
// (Z) and its sigma in units of r (SIG).
__global__ void sur_head_eval_kernel(int B, const __nv_bfloat16 *H4, const float *P, const float *T, float tstd,
                                     float *Z, float *SIG) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= B) return;
    const uint4 v = *(const uint4 *)(H4 + (size_t)w * SH + lane * 8);
    const __nv_bfloat16 *h = (const __nv_bfloat16 *)&v;
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const float x = __bfloat162float(h[j]);
        a = fmaf(P[OW5 + lane * 8 + j], x, a);
        b = fmaf(P[OW5 + SH + lane * 8 + j], x, b);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        const float l = fminf(fmaxf(b + P[OB5 + 1], -25.f), 5.f);
        Z[w] = fabsf(T[w] - (a + P[OB5])) * expf(-l);
        SIG[w] = tstd * expf(l);
    }
}

// rows of X, T, WT selected by LIST, into dense training arrays
__global__ void gather_train_kernel(int64_t m, const int32_t *LIST, const float *X, const float *T, const float *WT,
                                    float *Xc, float *Tc, float *WTc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t j = LIST[i];
#pragma unroll
    for (int k = 0; k < SXP; k++) Xc[i * SXP + k] = X[j * SXP + k];
    Tc[i] = T[j];
    WTc[i] = WT[j];
}

// ------------------------------------------------------------------ host side

static int cerr(cudaError_t e) {
    if (e == cudaSuccess) return TW_OK;
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TW_ENOMEM : TW_ECUDA;
}

static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Device buffers owned by one call (freed on scope exit).
struct DevBufs {
    std::vector<void *> p;
    ~DevBufs() {
        for (void *q : p) cudaFree(q);
    }
    template <typename T>
    int get(T **out, size_t count) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 256);
        if (e != cudaSuccess) { (void)cudaGetLastError(); return TW_ENOMEM; }
        p.push_back(q);
        *out = (T *)q;
        return TW_OK;
    }
};

static uint64_t fnv1a(const void *data, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char *b = (const unsigned char *)data;
    for (size_t i = 0; i < n; i++) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

static const char MAGIC[8] = {'T', 'W', 'M', 'L', 'P', '0', '0', '1'};

// Weights file: magic, int32 {version 2, hidden, inputs, nparams}, the
// standardisation record (input mean and 1/std, target mean and spread,
// calibrated kappa, band), the FP32 parameters, FNV-1a checksum.
static int save_model(const char *path, const std::vector<float> &P, const SurNorm &nrm) {
    FILE *f = fopen(path, "wb");
    if (!f) return TW_EINVAL;
    const int32_t hdr[4] = {2, SH, SNIN, NPAR};
    uint64_t h = fnv1a(MAGIC, 8);
    h = fnv1a(hdr, sizeof(hdr), h);
    h = fnv1a(&nrm, sizeof(nrm), h);
    h = fnv1a(P.data(), P.size() * 4, h);
    bool ok = fwrite(MAGIC, 8, 1, f) == 1 && fwrite(hdr, sizeof(hdr), 1, f) == 1 && fwrite(&nrm, sizeof(nrm), 1, f) == 1 &&
              fwrite(P.data(), 4, P.size(), f) == P.size() && fwrite(&h, 8, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    return ok ? TW_OK : TW_EINVAL;
}

static int load_model(const char *path, std::vector<float> &P, SurNorm &nrm) {
    FILE *f = fopen(path, "rb");
    if (!f) return TW_EINVAL;
    char mg[8];
    int32_t hdr[4];
    uint64_t h = 0;
    P.assign(NPAR, 0.f);
    bool ok = fread(mg, 8, 1, f) == 1 && memcmp(mg, MAGIC, 8) == 0 && fread(hdr, sizeof(hdr), 1, f) == 1 &&
              hdr[0] == 2 && hdr[1] == SH && hdr[2] == SNIN && hdr[3] == NPAR &&
              fread(&nrm, sizeof(nrm), 1, f) == 1 && fread(P.data(), 4, NPAR, f) == (size_t)NPAR &&
              fread(&h, 8, 1, f) == 1;
    fclose(f);
    if (!ok) return TW_EINVAL;
    uint64_t c = fnv1a(MAGIC, 8);
    c = fnv1a(hdr, sizeof(hdr), c);
    c = fnv1a(&nrm, sizeof(nrm), c);
    c = fnv1a(P.data(), P.size() * 4, c);
    return c == h ? TW_OK : TW_EINVAL;
}

// Loaded model per device: FP32 parameters and BF16 copies of the hidden weights.
struct Model {
    std::string path;
    float *P = nullptr;
    __nv_bfloat16 *Wf = nullptr, *Wt = nullptr;
    SurNorm nrm;
};
static std::mutex g_sm;
static Model g_models[64];

static int model_for(const char *path, cudaStream_t st, Model **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cerr(cudaErrorInvalidDevice);
    Model &m = g_models[dev];
    if (!m.P || m.path != path) {
        std::vector<float> P;
        SurNorm nrm;
        int rc = load_model(path, P, nrm);
        if (rc) return rc;
        if (!m.P) {
            cudaError_t e = cudaMalloc(&m.P, NPAR * 4);
            if (e == cudaSuccess) e = cudaMalloc(&m.Wf, (size_t)3 * SH * SH * 2);
            if (e == cudaSuccess) e = cudaMalloc(&m.Wt, (size_t)3 * SH * SH * 2);
            if (e != cudaSuccess) return cerr(e);
        }
        cudaError_t e = cudaMemcpyAsync(m.P, P.data(), NPAR * 4, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cerr(e);
        refresh_bf16_kernel<<<nblk(3 * SH * SH, 256), 256, 0, st>>>(m.P, m.Wf, m.Wt);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cerr(e);
        m.path = path;
        m.nrm = nrm;
    }
    *out = &m;
    return TW_OK;
}

// MLP forward over `rows` (a multiple of 128) standardised-on-the-fly inputs:
// H1 = layer 1 (CUDA cores), then the three hidden layers on the tensor cores
// ping-ponging between HA and HB; returns the buffer holding layer 4.
static int mlp_forward(const Model &m, int64_t rows, const float *X, __nv_bfloat16 *HA, __nv_bfloat16 *HB,
                       __nv_bfloat16 *H1keep, __nv_bfloat16 **H2keep, float *XS, int *err, cudaStream_t st,
                       __nv_bfloat16 **outH4, cudaEvent_t gemm0 = nullptr, cudaEvent_t gemm1 = nullptr) {
    __nv_bfloat16 *h1 = H1keep ? H1keep : HA;
    sur_layer1_kernel<<<nblk(rows * SH, 256), 256, 0, st>>>(rows, X, m.P, m.nrm, h1, XS);
    if (gemm0) cudaEventRecord(gemm0, st);
    __nv_bfloat16 *in = h1;
    for (int l = 0; l < 3; l++) {
        __nv_bfloat16 *out = H2keep ? H2keep[l] : ((in == HA) ? HB : HA);
        GemmArgs g;
        g.A = in;
        g.B = m.Wf + (size_t)l * SH * SH;
        g.M = (int)rows;
        g.N = SH;
        g.K = SH;
        g.C = nullptr;
        g.Cb = out;
        g.bias = m.P + OBH[l];
        g.relu = 1;
        g.err = err;
        cudaError_t e = gemm_bf16_tn(g, st);
        if (e != cudaSuccess) return cerr(e);
        in = out;
    }
    if (gemm1) cudaEventRecord(gemm1, st);
    *outH4 = in;
    return cerr(cudaGetLastError());
}

// Grow-only device buffers, one set per device and entry point: calls are
// serialised (g_sm) and synchronous, so a set is reused call after call
// instead of being allocated and freed (cudaFree synchronises the device).
struct Pool {
    void *p[16] = {nullptr};
    size_t sz[16] = {0};
    template <typename T>
    int get(int slot, T **out, size_t count) {
        const size_t need = count * sizeof(T) + 256;
        if (sz[slot] < need) {
            if (p[slot]) cudaFree(p[slot]);
            p[slot] = nullptr;
            sz[slot] = 0;
            if (cudaMalloc(&p[slot], need) != cudaSuccess) { (void)cudaGetLastError(); p[slot] = nullptr; return TW_ENOMEM; }
            sz[slot] = need;
        }
        *out = (T *)p[slot];
        return TW_OK;
    }
};
static Pool g_sur_pool[64];

// Timing and work of the latest tw_surrogate_mag call on a device: CUDA
// events around each chunk's feature kernel, its three tensor-core GEMMs and
// its whole network (layer 1, GEMMs, head), and the feature kernel's work
// counters.
struct SurStats {
    std::vector<cudaEvent_t> ev;  // 5 per chunk
    double feat_ms = 0, net_ms = 0, gemm_ms = 0, gemm_rows = 0;
    unsigned long long work[4] = {0, 0, 0, 0};
    bool valid = false;
};
static SurStats g_sur_stats[64];

static bool dev_ptr(const void *p) { return p && ptr_kind(p) == PK_DEV; }

}  // namespace tw

using namespace tw;

extern "C" int tw_surrogate_train(const char *weights_path, int64_t nsamples, uint64_t seed, int epochs,
                                  double *stats, const tw_opts *opts) {
    if (!weights_path || nsamples < 4096 || nsamples > (int64_t)1 << 30 || epochs < 1 || epochs > 1000)
        return TW_EINVAL;
    tw_opts o;
    tw_opts_default(&o);
    if (opts) o = *opts;
    std::lock_guard<std::mutex> lk(g_sm);
    cudaStream_t st = (cudaStream_t)o.stream;
    const int64_t n = nsamples;
    DevBufs B;
    double *S, *Q, *RHO, *Y1, *Y2, *MUPS, *MU;
    float *X, *T, *WT;
    uint8_t *FLAG;
    int32_t *LIST;
    unsigned long long *NL;
    int *err;
    int rc = 0;
    if ((rc = B.get(&S, n)) || (rc = B.get(&Q, n)) || (rc = B.get(&RHO, n)) || (rc = B.get(&Y1, n)) ||
        (rc = B.get(&Y2, n)) || (rc = B.get(&MUPS, n)) || (rc = B.get(&MU, n)) || (rc = B.get(&X, n * SXP)) ||
        (rc = B.get(&T, n)) || (rc = B.get(&WT, n)) || (rc = B.get(&FLAG, n)) || (rc = B.get(&LIST, n)) ||
        (rc = B.get(&NL, 1)) || (rc = B.get(&err, 1)))
        return rc;
    // positions near caustics, point-source values and flags
    sur_sample_kernel<<<nblk(n, 128), 128, 0, st>>>(seed, n, S, Q, RHO, Y1, Y2);
    float *HEXE;
    int8_t *LSTAT;
    if ((rc = B.get(&HEXE, n)) || (rc = B.get(&LSTAT, n))) return rc;
    sur_features_kernel<<<nblk(n, 128), 128, 0, st>>>(n, S, Q, RHO, Y1, Y2, X, MUPS, FLAG, HEXE, nullptr);
    cudaMemsetAsync(NL, 0, 8, st);
    cudaMemsetAsync(err, 0, 4, st);
    cudaMemsetAsync(LSTAT, 0x7f, n, st);
    // the network's band: unflagged positions whose expansion error estimate
    // is above a quarter of 1e-4 (below half the tolerance the expansion
    // answers by itself) and at most 2e-3, so that the correction the network
    // adds is small (at most about twenty times the 1e-4 target); in draw
    // order, so that training is reproducible
    const float band = 2.5e-5f, band_hi = 2e-3f;
    compact_band_kernel<<<nblk(n, 256), 256, 0, st>>>(n, FLAG, HEXE, band, band_hi, LIST, NL);
    unsigned long long nl = 0;
    cudaError_t e = cudaMemcpyAsync(&nl, NL, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cerr(e);
    const int BATCH = 4096;
    const int64_t nho = (int64_t)nl / 10;                        // held-out rows (calibration)
    const int64_t m = (((int64_t)nl - nho) / BATCH) * BATCH;     // training rows
    if (m < BATCH || nho < 128) return TW_EINVAL;                // not enough positions in the band
    {
        std::vector<int32_t> hl(nl);
        e = cudaMemcpyAsync(hl.data(), LIST, nl * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cerr(e);
        std::sort(hl.begin(), hl.end());
        e = cudaMemcpyAsync(LIST, hl.data(), nl * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cerr(e);
    }
    // labels two decades tighter than the 1e-4 target, FP64 contour integration
    rc = contour_positions(S, Q, RHO, Y1, Y2, LIST, (int64_t)nl, 1e-6, TW_PREC_FP64, 4096, MU, LSTAT, st);
    if (rc) return rc;
    sur_targets_kernel<<<nblk(n, 256), 256, 0, st>>>(n, MU, MUPS, FLAG, HEXE, X, LSTAT, band, band_hi, T, WT);
    // dense rows of the band: the first m train, the last nho calibrate
    const int64_t nrow = m + nho, nho_pad = ((nho + 127) / 128) * 128;
    float *Xc, *Tc, *WTc;
    if ((rc = B.get(&Xc, (m + nho_pad) * SXP)) || (rc = B.get(&Tc, m + nho_pad)) || (rc = B.get(&WTc, m + nho_pad)))
        return rc;
    cudaMemsetAsync(Xc, 0, (m + nho_pad) * SXP * 4, st);
    gather_train_kernel<<<nblk(nrow, 256), 256, 0, st>>>(nrow, LIST + ((int64_t)nl - nrow), X, T, WT, Xc, Tc, WTc);
    // input and target standardisation from the training rows
    std::vector<float> hx(m * SXP), ht(m), hw(m);
    e = cudaMemcpyAsync(hx.data(), Xc, m * SXP * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ht.data(), Tc, m * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hw.data(), WTc, m * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cerr(e);
    SurNorm nrm;
    double tsum = 0, tsq = 0, wsum = 0;
    for (int k = 0; k < SNIN; k++) {
        double a = 0, b = 0;
        for (int64_t i = 0; i < m; i++) { a += hx[i * SXP + k]; b += (double)hx[i * SXP + k] * hx[i * SXP + k]; }
        a /= m;
        b = b / m - a * a;
        nrm.mean[k] = (float)a;
        nrm.inv_std[k] = (float)(1.0 / sqrt(b > 1e-20 ? b : 1e-20));
    }
    for (int64_t i = 0; i < m; i++) { tsum += hw[i] * ht[i]; tsq += (double)hw[i] * ht[i] * ht[i]; wsum += hw[i]; }
    const double tmean = tsum / (wsum > 0 ? wsum : 1), tstd = sqrt(fmax(tsq / (wsum > 0 ? wsum : 1) - tmean * tmean, 1e-24));
    nrm.tmean = (float)tmean;
    nrm.tstd = (float)tstd;
    nrm.kappa_cal = 3.f;
    nrm.band = band;
    nrm.band_hi = band_hi;
    standardise_kernel<<<nblk(nrow, 256), 256, 0, st>>>(nrow, Tc, (float)tmean, (float)(1.0 / tstd));
    // initial weights (He-uniform, seeded), head bias at the target mean / spread
    std::vector<float> hP(NPAR, 0.f);
    uint64_t rs = seed ^ 0xA0761D6478BD642Full;
    auto urand = [&]() {
        rs += 0x9E3779B97F4A7C15ull;
        uint64_t z = rs;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int i = 0; i < SH * SNIN; i++) hP[OW1 + i] = (float)((2 * urand() - 1) * sqrt(6.0 / SNIN));
    for (int l = 0; l < 3; l++)
        for (int i = 0; i < SH * SH; i++) hP[OWH[l] + i] = (float)((2 * urand() - 1) * sqrt(6.0 / SH));
    for (int i = 0; i < 2 * SH; i++) hP[OW5 + i] = (float)((2 * urand() - 1) * 1e-3);
    hP[OB5] = 0.f;      // standardised r: mean 0
    hP[OB5 + 1] = 0.f;  // and spread 1
    Model tm;
    float *G, *M1, *M2, *LOSS;
    __nv_bfloat16 *H[4], *GA, *GB2, *TA, *TB;
    float *DOUT, *DH, *XS;
    if ((rc = B.get(&tm.P, NPAR)) || (rc = B.get(&tm.Wf, 3 * SH * SH)) || (rc = B.get(&tm.Wt, 3 * SH * SH)) ||
        (rc = B.get(&G, NPAR)) || (rc = B.get(&M1, NPAR)) || (rc = B.get(&M2, NPAR)) || (rc = B.get(&LOSS, 1)))
        return rc;
    for (int l = 0; l < 4; l++)
        if ((rc = B.get(&H[l], (size_t)BATCH * SH))) return rc;
    if ((rc = B.get(&GA, (size_t)BATCH * SH)) || (rc = B.get(&GB2, (size_t)BATCH * SH)) ||
        (rc = B.get(&TA, (size_t)BATCH * SH)) || (rc = B.get(&TB, (size_t)BATCH * SH)) ||
        (rc = B.get(&DOUT, 2 * BATCH)) || (rc = B.get(&DH, (size_t)BATCH * SH)) || (rc = B.get(&XS, (size_t)BATCH * SXP)))
        return rc;
    tm.nrm = nrm;
    e = cudaMemcpyAsync(tm.P, hP.data(), NPAR * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(M1, 0, NPAR * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(M2, 0, NPAR * 4, st);
    if (e != cudaSuccess) return cerr(e);
    refresh_bf16_kernel<<<nblk(3 * SH * SH, 256), 256, 0, st>>>(tm.P, tm.Wf, tm.Wt);
    const int64_t steps_per_epoch = m / BATCH;
    const int64_t total = steps_per_epoch * epochs;
    const float lr0 = 1e-3f, b1 = 0.9f, b2 = 0.999f;
    double loss_sum = 0;
    int loss_n = 0;
    for (int64_t stp = 0; stp < total; stp++) {
        const int64_t off = (stp % steps_per_epoch) * BATCH;
        const float *Xb = Xc + off * SXP, *Tb = Tc + off, *Wb = WTc + off;
        __nv_bfloat16 *hk[3] = {H[1], H[2], H[3]};
        __nv_bfloat16 *h4 = nullptr;
        if ((rc = mlp_forward(tm, BATCH, Xb, nullptr, nullptr, H[0], hk, XS, err, st, &h4))) return rc;
        const bool last_epoch = stp >= total - steps_per_epoch;
        cudaMemsetAsync(LOSS, 0, 4, st);
        sur_head_train_kernel<<<nblk((int64_t)BATCH * 32, 256), 256, 0, st>>>(BATCH, H[3], tm.P, Tb, Wb, DOUT, GA,
                                                                            LOSS);
        sur_head_wgrad_kernel<<<nblk(2 * SH + 2, 256), 256, 0, st>>>(BATCH, DOUT, H[3], G);
        // hidden layers, last to first: g (bf16, masked) of layer l+1 is in GA
        for (int l = 2; l >= 0; l--) {
            __nv_bfloat16 *hin = H[l];  // input of hidden GEMM l (H1, H2, H3)
            dim3 tb(32, 8);
            transpose_bf16_kernel<<<dim3(SH / 32, BATCH / 32), tb, 0, st>>>(BATCH, SH, GA, TA);   // g^T [SH][B]
            transpose_bf16_kernel<<<dim3(SH / 32, BATCH / 32), tb, 0, st>>>(BATCH, SH, hin, TB);  // h^T [SH][B]
            GemmArgs gw;
            gw.A = TA; gw.B = TB; gw.M = SH; gw.N = SH; gw.K = BATCH;
            gw.C = G + OWH[l]; gw.Cb = nullptr; gw.bias = nullptr; gw.relu = 0; gw.err = err;
            if ((e = gemm_bf16_tn(gw, st)) != cudaSuccess) return cerr(e);
            colsum_bf16_kernel<<<1, SH, 0, st>>>(BATCH, GA, G + OBH[l]);
            GemmArgs gx;  // dh_in = g . W  (W^T stored [in][out] is the K-major B operand)
            gx.A = GA; gx.B = tm.Wt + (size_t)l * SH * SH; gx.M = BATCH; gx.N = SH; gx.K = SH;
            gx.C = DH; gx.Cb = nullptr; gx.bias = nullptr; gx.relu = 0; gx.err = err;
            if ((e = gemm_bf16_tn(gx, st)) != cudaSuccess) return cerr(e);
            if (l > 0) relu_mask_kernel<<<nblk((int64_t)BATCH * SH, 256), 256, 0, st>>>((int64_t)BATCH * SH, DH, hin, GB2);
            __nv_bfloat16 *tmp = GA; GA = GB2; GB2 = tmp;
        }
        sur_layer1_bwd_kernel<<<1, SH, 0, st>>>(BATCH, DH, H[0], XS, G);
        const double frac = (double)stp / (double)total;
        const float lr = (float)(lr0 * (0.05 + 0.95 * 0.5 * (1.0 + cos(3.141592653589793 * frac))));
        const float c1 = 1.f / (1.f - powf(b1, (float)(stp + 1))), c2 = 1.f / (1.f - powf(b2, (float)(stp + 1)));
        adam_kernel<<<nblk(NPAR, 256), 256, 0, st>>>(NPAR, tm.P, G, M1, M2, lr, b1, b2, c1, c2);
        refresh_bf16_kernel<<<nblk(3 * SH * SH, 256), 256, 0, st>>>(tm.P, tm.Wf, tm.Wt);
        if (last_epoch) {
            float l = 0;
            if ((e = cudaMemcpyAsync(&l, LOSS, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cerr(e);
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cerr(e);
            loss_sum += l;
            loss_n++;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return cerr(e);
    }
    // calibration on the held-out rows: kappa_cal is the 99.9% quantile of
    // |r - r_net| / sigma (at least 3), so that kappa_cal sigma bounds the
    // network's error on all but about 1e-3 of the band, raised until the
    // rows answered at rel_tol 1e-4 are all within a quarter of it
    float *Z, *SIG;
    if ((rc = B.get(&Z, nho_pad)) || (rc = B.get(&SIG, nho_pad))) return rc;
    for (int64_t off = 0; off < nho_pad; off += BATCH) {
        const int64_t rows = (nho_pad - off) < BATCH ? (nho_pad - off) : BATCH;
        __nv_bfloat16 *hk[3] = {H[1], H[2], H[3]};
        __nv_bfloat16 *h4 = nullptr;
        if ((rc = mlp_forward(tm, rows, Xc + (m + off) * SXP, nullptr, nullptr, H[0], hk, nullptr, err, st, &h4)))
            return rc;
        sur_head_eval_kernel<<<nblk(rows * 32, 256), 256, 0, st>>>((int)rows, h4, tm.P, Tc + m + off, (float)tstd,
                                                                  Z + off, SIG + off);
    }
    std::vector<float> hz(nho), hs(nho), hwo(nho);
    e = cudaMemcpyAsync(hz.data(), Z, nho * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), SIG, nho * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hwo.data(), WTc + m, nho * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cerr(e);
    std::vector<float> zv;
    for (int64_t i = 0; i < nho; i++)
        if (hwo[i] > 0.f) zv.push_back(isfinite(hz[i]) ? hz[i] : 1e30f);
    double acc_frac = 0, acc_err = 0;
    if (!zv.empty()) {
        std::vector<float> zs = zv;
        const size_t k = (size_t)floor(0.999 * (double)(zs.size() - 1));
        std::nth_element(zs.begin(), zs.begin() + k, zs.end());
        nrm.kappa_cal = fmaxf(3.f, zs[k]);
        // and at least large enough that, at rel_tol 1e-4, every held-out row
        // the network would answer is within a quarter of the tolerance: the
        // rows in order of sigma, accepted up to the first larger error
        std::vector<std::pair<float, float>> se;
        for (int64_t i = 0; i < nho; i++)
            if (hwo[i] > 0.f) se.push_back({hs[i], isfinite(hz[i]) ? hz[i] * hs[i] : 1e30f});
        std::sort(se.begin(), se.end());
        float smax = 0.f;
        for (const auto &p : se) {
            if (!(p.second <= 0.25e-4f)) break;
            smax = p.first;
        }
        nrm.kappa_cal = fmaxf(nrm.kappa_cal, smax > 0.f ? 1e-4f / smax : 1e30f);
        int64_t na = 0, nv = 0;
        for (int64_t i = 0; i < nho; i++) {
            if (!(hwo[i] > 0.f)) continue;
            nv++;
            if (nrm.kappa_cal * hs[i] <= 1e-4f) {
                na++;
                acc_err = fmax(acc_err, (double)hz[i] * hs[i]);
            }
        }
        acc_frac = nv ? (double)na / nv : 0;
    }
    int herr = 0;
    e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hP.data(), tm.P, NPAR * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cerr(e);
    if (herr) return TW_ETIMEOUT;
    if ((rc = save_model(weights_path, hP, nrm))) return rc;
    {  // a model cached from an earlier file of the same name is stale now
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) g_models[dev].path.clear();
    }
    if (stats) {
        stats[0] = (double)n;                       // positions drawn
        stats[1] = (double)nl;                      // positions of the band (labelled)
        stats[2] = (double)m;                       // training rows used
        stats[3] = loss_n ? loss_sum / loss_n : 0;  // mean NLL (standardised r) over the last epoch
        stats[4] = tstd;                            // spread of the targets
        stats[5] = (double)nho;                     // held-out rows
        stats[6] = nrm.kappa_cal;                   // calibrated acceptance factor
        stats[7] = acc_frac;                        // held-out rows accepted at rel_tol 1e-4
        stats[8] = acc_err;                         // their largest error in r
    }
    return TW_OK;
}

extern "C" int tw_surrogate_mag(const char *weights_path, const double *s, const double *q, const double *rho,
                                const double *y1, const double *y2, int64_t n, double rel_tol, double kappa,
                                double *out, int64_t *counts, const tw_opts *opts) {
    if (!weights_path || n < 0 || !(rel_tol > 0) || !(kappa > 0) || !isfinite(rel_tol) || n > 0x7fffffffll)
        return TW_EINVAL;
    if (n == 0) {
        if (counts) for (int k = 0; k < 5; k++) counts[k] = 0;
        return TW_OK;
    }
    if (!s || !q || !rho || !y1 || !y2 || !out) return TW_EINVAL;
    tw_opts o;
    tw_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision != TW_PREC_FP64 && o.precision != TW_PREC_MIXED) return TW_EINVAL;
    std::lock_guard<std::mutex> lk(g_sm);
    cudaStream_t st = (cudaStream_t)o.stream;
    // one kind for every array; device memory of another device is refused
    const int kind = ptr_kind(out);
    if (kind == PK_OTHER) return TW_EINVAL;
    const bool dev = kind == PK_DEV;
    const double *in[5] = {s, q, rho, y1, y2};
    for (int k = 0; k < 5; k++)
        if (ptr_kind(in[k]) != kind) return TW_EINVAL;
    if (o.pos_status && ptr_kind(o.pos_status) != kind) return TW_EINVAL;
    int devno = 0;
    if (cudaGetDevice(&devno) != cudaSuccess || devno < 0 || devno >= 64) { (void)cudaGetLastError(); return TW_ECUDA; }
    Model *m = nullptr;
    int rc = model_for(weights_path, st, &m);
    if (rc) return rc;
    Pool &B = g_sur_pool[devno];
    SurStats &T = g_sur_stats[devno];
    T.valid = false;
    const double *din[5];
    double *dout = out;
    int8_t *dstat = o.pos_status;
    cudaError_t e;
    if (!dev) {  // host arrays: stage through device memory
        for (int k = 0; k < 5; k++) {
            double *d;
            if ((rc = B.get(k, &d, n))) return rc;
            if ((e = cudaMemcpyAsync(d, in[k], n * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cerr(e);
            din[k] = d;
        }
        if ((rc = B.get(5, &dout, n))) return rc;
        if (o.pos_status && (rc = B.get(15, &dstat, n))) return rc;
    } else {
        for (int k = 0; k < 5; k++) din[k] = in[k];
    }
    const int64_t CH = 1 << 20;
    const int64_t chunk = n < CH ? ((n + 127) / 128) * 128 : CH;
    const int64_t nch = (n + chunk - 1) / chunk;
    float *X, *HEXE;
    double *MUPS;
    uint8_t *FLAG;
    int32_t *LIST;
    unsigned long long *NL, *WORK;
    int *err;
    __nv_bfloat16 *HA, *HB;
    if ((rc = B.get(6, &X, chunk * SXP)) || (rc = B.get(7, &MUPS, n)) || (rc = B.get(8, &FLAG, n)) ||
        (rc = B.get(9, &LIST, n)) || (rc = B.get(10, &NL, 8)) || (rc = B.get(11, &err, 1)) ||
        (rc = B.get(12, &HA, chunk * SH)) || (rc = B.get(13, &HB, chunk * SH)) || (rc = B.get(14, &HEXE, n)))
        return rc;
    WORK = NL + 4;
    while (T.ev.size() < (size_t)(5 * nch)) {
        cudaEvent_t ev;
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cerr(e);
        T.ev.push_back(ev);
    }
    if ((e = cudaMemsetAsync(NL, 0, 64, st)) != cudaSuccess) return cerr(e);
    if ((e = cudaMemsetAsync(err, 0, 4, st)) != cudaSuccess) return cerr(e);
    double rows_total = 0;
    for (int64_t c = 0; c < nch; c++) {
        const int64_t c0 = c * chunk;
        const int64_t cn = (n - c0) < chunk ? (n - c0) : chunk;
        const int64_t rows = ((cn + 127) / 128) * 128;
        rows_total += (double)rows;
        if (rows > cn) cudaMemsetAsync(X + cn * SXP, 0, (rows - cn) * SXP * 4, st);
        cudaEvent_t *ev = &T.ev[5 * c];
        cudaEventRecord(ev[0], st);
        sur_features_kernel<<<nblk(cn, 128), 128, 0, st>>>(cn, din[0] + c0, din[1] + c0, din[2] + c0, din[3] + c0,
                                                           din[4] + c0, X, MUPS + c0, FLAG + c0, HEXE + c0, WORK);
        cudaEventRecord(ev[1], st);
        __nv_bfloat16 *h4 = nullptr;
        if ((rc = mlp_forward(*m, rows, X, HA, HB, nullptr, nullptr, nullptr, err, st, &h4, ev[2], ev[3]))) return rc;
        sur_head_infer_kernel<<<nblk(cn * 32, 256), 256, 0, st>>>(cn, c0, h4, m->P, X, m->nrm, MUPS, FLAG, HEXE,
                                                                 rel_tol, (float)kappa, dout, dstat, LIST, NL);
        cudaEventRecord(ev[4], st);
    }
    unsigned long long cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int herr = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, NL, 64, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cerr(e);
    if (herr) return TW_ETIMEOUT;
    T.feat_ms = T.net_ms = T.gemm_ms = 0;
    for (int64_t c = 0; c < nch; c++) {
        float a = 0, b = 0, g = 0;
        cudaEventElapsedTime(&a, T.ev[5 * c], T.ev[5 * c + 1]);
        cudaEventElapsedTime(&b, T.ev[5 * c + 1], T.ev[5 * c + 4]);
        cudaEventElapsedTime(&g, T.ev[5 * c + 2], T.ev[5 * c + 3]);
        T.feat_ms += a;
        T.net_ms += b;
        T.gemm_ms += g;
    }
    (void)cudaGetLastError();
    T.gemm_rows = rows_total;
    for (int k = 0; k < 4; k++) T.work[k] = cnt[4 + k];
    T.valid = true;
    const unsigned long long nl = cnt[0];
    // contour-integration fallback: one persistent launch over the list
    rc = contour_positions(din[0], din[1], din[2], din[3], din[4], LIST, (int64_t)nl, rel_tol, o.precision,
                           o.max_samples, dout, dstat, st);
    if (rc) return rc;
    if (!dev) {
        if ((e = cudaMemcpyAsync(out, dout, n * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cerr(e);
        if (o.pos_status && (e = cudaMemcpyAsync(o.pos_status, dstat, n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cerr(e);
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cerr(e);
    if (counts) {
        counts[0] = (int64_t)cnt[0];
        counts[1] = (int64_t)cnt[1];
        counts[2] = (int64_t)cnt[2];
        counts[3] = (int64_t)cnt[3];
        counts[4] = (int64_t)(cnt[0] - cnt[3]);
    }
    return TW_OK;
}

extern "C" int tw_last_surrogate_stats(double out[8]) {
    if (!out) return TW_EINVAL;
    std::lock_guard<std::mutex> lk(g_sm);
    int devno = 0;
    if (cudaGetDevice(&devno) != cudaSuccess || devno < 0 || devno >= 64) { (void)cudaGetLastError(); return TW_ECUDA; }
    const SurStats &T = g_sur_stats[devno];
    if (!T.valid) return TW_EINVAL;
    out[0] = T.feat_ms;
    out[1] = T.net_ms;
    out[2] = T.gemm_ms;
    out[3] = (double)T.work[0];
    out[4] = (double)T.work[1];
    out[5] = (double)T.work[2];
    out[6] = (double)T.work[3];
    out[7] = T.gemm_rows;
    return TW_OK;
}

extern "C" int tw_surrogate_sample(uint64_t seed, int64_t n, double *s, double *q, double *rho, double *y1,
                                   double *y2, void *stream) {
    if (n < 0) return TW_EINVAL;
    if (n == 0) return TW_OK;
    if (!dev_ptr(s) || !dev_ptr(q) || !dev_ptr(rho) || !dev_ptr(y1) || !dev_ptr(y2)) return TW_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    sur_sample_kernel<<<nblk(n, 128), 128, 0, st>>>(seed, n, s, q, rho, y1, y2);
    return cerr(cudaGetLastError());
}

namespace tw {

// Point-source adequacy gate: a position whose expansion is certified (not
// flagged as near a caustic, error estimate within rel_tol / 2) takes the
// expansion's value; every other position is listed for contour integration.
__global__ void gate_kernel(int64_t n, int64_t row0, const double *MUPS, const uint8_t *FLAG, const float *HEXE,
                            double tol, double *OUT, int32_t *LIST, unsigned long long *NLIST) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t g = row0 + i;
    const double mu = MUPS[g];
    if (!FLAG[g] && HEXE[g] <= 0.5f * (float)tol && isfinite(mu)) {
        OUT[g] = mu;
        atomicAdd(NLIST + 1, 1ull);
    } else {
        const unsigned long long slot = atomicAdd(NLIST, 1ull);
        LIST[slot] = (int32_t)g;
    }
}

static Pool g_gate_pool[64];

}  // namespace tw

extern "C" int tw_mag_gated(const double *s, const double *q, const double *rho, const double *y1, const double *y2,
                            int64_t n, double rel_tol, double *out, int64_t *n_contour, const tw_opts *opts) {
    if (n < 0 || !(rel_tol > 0) || !isfinite(rel_tol) || n > 0x7fffffffll) return TW_EINVAL;
    if (n == 0) { if (n_contour) *n_contour = 0; return TW_OK; }
    if (!s || !q || !rho || !y1 || !y2 || !out) return TW_EINVAL;
    tw_opts o;
    tw_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision != TW_PREC_FP64 && o.precision != TW_PREC_MIXED) return TW_EINVAL;
    std::lock_guard<std::mutex> lk(g_sm);
    cudaStream_t st = (cudaStream_t)o.stream;
    // one kind for every array; device memory of another device is refused
    const int kind = ptr_kind(out);
    if (kind == PK_OTHER) return TW_EINVAL;
    const bool dev = kind == PK_DEV;
    const double *in[5] = {s, q, rho, y1, y2};
    for (int k = 0; k < 5; k++)
        if (ptr_kind(in[k]) != kind) return TW_EINVAL;
    if (o.pos_status && ptr_kind(o.pos_status) != kind) return TW_EINVAL;
    int devno = 0;
    if (cudaGetDevice(&devno) != cudaSuccess || devno < 0 || devno >= 64) { (void)cudaGetLastError(); return TW_ECUDA; }
    Pool &B = g_gate_pool[devno];
    const double *din[5];
    double *dout = out;
    cudaError_t e;
    int rc;
    if (!dev) {  // host arrays: stage through device memory
        for (int k = 0; k < 5; k++) {
            double *d;
            if ((rc = B.get(6 + k, &d, n))) return rc;
            if ((e = cudaMemcpyAsync(d, in[k], n * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cerr(e);
            din[k] = d;
        }
        if ((rc = B.get(11, &dout, n))) return rc;
    } else {
        for (int k = 0; k < 5; k++) din[k] = in[k];
    }
    const int64_t CH = 1 << 20;
    const int64_t chunk = n < CH ? n : CH;
    float *X, *HEXE;
    double *MUPS;
    uint8_t *FLAG;
    int32_t *LIST;
    unsigned long long *NL;
    if ((rc = B.get(0, &X, chunk * SXP)) || (rc = B.get(1, &MUPS, n)) || (rc = B.get(2, &FLAG, n)) ||
        (rc = B.get(3, &LIST, n)) || (rc = B.get(4, &NL, 2)) || (rc = B.get(5, &HEXE, n)))
        return rc;
    if ((e = cudaMemsetAsync(NL, 0, 16, st)) != cudaSuccess) return cerr(e);
    for (int64_t c0 = 0; c0 < n; c0 += chunk) {
        const int64_t cn = (n - c0) < chunk ? (n - c0) : chunk;
        sur_features_kernel<<<nblk(cn, 128), 128, 0, st>>>(cn, din[0] + c0, din[1] + c0, din[2] + c0, din[3] + c0,
                                                           din[4] + c0, X, MUPS + c0, FLAG + c0, HEXE + c0, nullptr);
        gate_kernel<<<nblk(cn, 256), 256, 0, st>>>(cn, c0, MUPS, FLAG, HEXE, rel_tol, dout, LIST, NL);
    }
    unsigned long long cnt[2] = {0, 0};
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, NL, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cerr(e);
    rc = contour_positions(din[0], din[1], din[2], din[3], din[4], LIST, (int64_t)cnt[0], rel_tol, o.precision,
                           o.max_samples, dout, nullptr, st);
    if (rc) return rc;
    if (!dev && (e = cudaMemcpyAsync(out, dout, n * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cerr(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cerr(e);
    if (n_contour) *n_contour = (int64_t)cnt[0];
    return TW_OK;
}
