// lens.cuh -- point-source images of one limb sample, on the device.
//
// Frame: origin on the secondary (the frame of Eq. 6): the primary (mass m1)
// sits at -s, the secondary (mass m2) at 0; y = zeta - z2 and eta = z - z2,
// z2 = s/(1+q) being the secondary's centre-of-mass coordinate (Eq. 2).  The
// caller arranges q <= 1 (mass-swap symmetry), so that the refactored
// coefficients of Eq. 6 always treat the lighter body as the low-mass lens.
//
// Steps, each following the paper:
//   coefficients   Eq. 6 (cancellation-free form), FP64
//   roots          Aberth-Ehrlich simultaneous iteration warm-started from a
//                  neighbouring sample's roots.  FP64 mode iterates in FP64
//                  (the pair sums in FP32, see aberth_sweep); mixed mode
//                  iterates in FP32 to FP32 accuracy and then polishes with
//                  FP64 sweeps on the undeflated quintic, the first of which
//                  the cubic convergence estimate almost always accepts.  The
//                  paper uses the Skowron-Gould Newton/Laguerre solver
//                  (Sec. 2.2); any solver returning the five roots computes
//                  the same thing.
//   ghost test     residual R_i of Eq. 12 in FP64; ghosts are the pair whose
//                  residuals are equal and opposite (Sec. 2.4.1) and well above
//                  the round-off level of those roots
//   parity         sign of J (Eq. 7), in FP32 away from critical curves and
//                  FP64 next to them; a sample is accepted when it has
//                  3 or 5 real images with parity sum -1 (Sec. 2.3)
//   derivatives    dz/dtheta = (zeta' - conj(f') conj(zeta'))/J and
//                  z' ^ z'' = (rho^2 + Im(z'^2 zeta' f''))/J  (Eq. 10), in FP32:
//                  they only enter the parabolic corrections and error terms
#pragma once
#include <stdint.h>

#include "cx.cuh"

namespace tw {

// Per-sample status bits (merged into the per-position status).
enum : int { SF_IMAGECOUNT = 2, SF_SOLVER = 8 };

struct LensK {
    double s, m1, m2; // separation and normalised masses (Eq. 2), m2 <= m1
    double rho;       // source radius
    cxd y0;           // source centre in the secondary's frame
};

// Eq. 6.  "Im(y) i" is read as i Im(y); m1 = 1 - m2 has been substituted.
__device__ __forceinline__ void eq6_coeffs(double s, double m2, cxd y, cxd c[6]) {
    const cxd yb = conj(y);
    const cxd vc = {yb.x + s, yb.y};              // v_c = conj(y) + s
    const cxd vp = {1.0 + s * yb.x, s * yb.y};    // v_p = 1 + s conj(y)
    const double im = y.y;
    const cxd iim = {0.0, im};                    // i Im(y)
    const double m2s = m2 * s;
    c[5] = {-(yb.x * vc.x - yb.y * vc.y), -(yb.x * vc.y + yb.y * vc.x)};
    // c4 = (conj(y) y - 1 - 2 s conj(y)) v_c + m2 s
    const cxd t4 = {norm2(y) - 1.0 - 2.0 * s * yb.x, -2.0 * s * yb.y};
    c[4] = t4 * vc;
    c[4].x += m2s;
    // c3 = (2y - s)(v_p v_c + 2 i Im y - m2 s) + 4 (m2 s - y) i Im y
    const cxd a3 = {2.0 * y.x - s, 2.0 * y.y};
    cxd b3 = vp * vc;
    b3.x -= m2s;
    b3.y += 2.0 * im;
    const cxd c3b = {m2s - y.x, -y.y};
    c[3] = a3 * b3 + 4.0 * (c3b * iim);
    // c2 = Re(v_p)^2 Re(v_c) + i Im(y) Re(v_p) Re(1 - s y) + s Im(y)^2 (2 + s v_c)
    //      + m2 s [2 conj(y) (y - s) - (1 - s y)]
    const double rvp = vp.x, rvc = vc.x;
    cxd c2 = {rvp * rvp * rvc, im * rvp * (1.0 - s * y.x)};
    const double sim2 = s * im * im;
    c2.x += sim2 * (2.0 + s * vc.x);
    c2.y += sim2 * (s * vc.y);
    const cxd ymS = {y.x - s, y.y};
    cxd t2 = 2.0 * (yb * ymS);
    t2.x -= 1.0 - s * y.x;
    t2.y -= -s * y.y;
    c[2] = c2 + m2s * t2;
    // c1 = m2 s [(s + 2y) v_p + s (2 s i Im y - m2)]
    const cxd s2y = {s + 2.0 * y.x, 2.0 * y.y};
    cxd t1 = s2y * vp;
    t1.x += s * (-m2);
    t1.y += s * (2.0 * s * im);
    c[1] = m2s * t1;
    // c0 = s^2 m2^2 y
    c[0] = (m2s * m2s) * y;
}

__device__ __forceinline__ void abs_coeffs(const cxd c[6], float ca[6]) {
#pragma unroll
    for (int k = 0; k < 6; k++) ca[k] = sqrtf(norm2f(c[k]));
}
// The same, keeping the FP32 values of the coefficients.
__device__ __forceinline__ void abs_coeffs(const cxd c[6], float ca[6], cxf cf[6]) {
#pragma unroll
    for (int k = 0; k < 6; k++) {
        cf[k] = to_f(c[k]);
        ca[k] = sqrtf(norm2(cf[k]));
    }
}

// Horner round-off bound sum_k |c_k| |z|^k (the attainable residual |p(z)|).
__device__ __forceinline__ float horner_bound(const float ca[6], float az) {
    float B = ca[5];
#pragma unroll
    for (int k = 4; k >= 0; k--) B = B * az + ca[k];
    return B;
}

// p(z) and p'(z) by Horner's rule.
template <typename T>
__device__ __forceinline__ void horner(const cx<T> c[6], cx<T> z, cx<T> &p, cx<T> &d) {
    d = c[5];
    p = cmad(c[5], z, c[4]);
#pragma unroll
    for (int k = 3; k >= 0; k--) {
        d = cmad(d, z, p);
        p = cmad(p, z, c[k]);
    }
}

// FP32 value of a root difference (an FP64 difference is formed exactly
// enough first, then rounded), and an FP32 pair sum widened to the iterate's
// type.
__device__ __forceinline__ cxf diff_f(cxd a, cxd b) { return to_f(a - b); }
__device__ __forceinline__ cxf diff_f(cxf a, cxf b) { return a - b; }
__device__ __forceinline__ cxd widen(cxf s, cxd) { return to_d(s); }
__device__ __forceinline__ cxf widen(cxf s, cxf) { return s; }

// One Jacobi sweep of the Aberth-Ehrlich iteration on the quintic c:
// z_i <- z_i - w_i, w_i = p/(p' - p S_i), S_i = sum_{j != i} 1/(z_i - z_j), the
// ten pair reciprocals being shared between the two roots of each pair.  The
// sums S_i are formed in FP32 in both precisions: they enter through p S_i,
// which vanishes at a root, so their rounding changes the correction w_i by a
// relative amount of order eps32 |w_i| |S_i| and limits neither the
// convergence nor the attainable accuracy (set by p, p' and z in the
// iterate's type).  For the same reason the division takes a reciprocal good
// to about 40 bits.
// dpa[i] receives |p'(z_i)|.  Returns true when every root is converged: its
// correction, or the error left after it, is below
// thr_i = max(rtol |z_i|, 8 eps B_i/|p'(z_i)|) (B_i the Horner round-off
// bound; the second term is the attainable accuracy of a near-multiple root).
// The iteration converges cubically, the error after a step being about
// |w_i|^2 max_j|w_j| sum_j 1/|z_i - z_j|^2, so a sweep whose corrections are
// already small needs no confirming sweep.
// thr[] and az2[] (|z_i|^2) carry the thresholds between sweeps: with fresh
// = true they (and dpa) are computed from this sweep's z and p', otherwise
// the previous values are kept (the magnitudes cost FP64-pipe conversions).
// fresh is set on return when some root moved by more than 1e-3 |z_i|, i.e.
// when the magnitudes may have changed.
// RP = true keeps the pair loop rolled too (a smaller kernel; faster where
// the warps of a CTA work on different lenses, slower on a single lens).
// Pair sums S_i = sum_{j != i} 1/(z_i - z_j) and K2_i = sum_{j != i} 1/|z_i - z_j|^2.
template <typename T, bool RP = false>
__device__ __forceinline__ void pair_sums(const cx<T> z[5], cxf S[5], float K2[5]) {
#pragma unroll
    for (int i = 0; i < 5; i++) { S[i] = {0.f, 0.f}; K2[i] = 0.f; }
    constexpr int PU = RP ? 1 : 5;
#pragma unroll PU
    for (int i = 0; i < 5; i++)
#pragma unroll PU
        for (int j = i + 1; j < 5; j++) {
            const cxf r = inv(diff_f(z[i], z[j]));
            S[i] = S[i] + r;
            S[j] = S[j] - r;
            const float rr = norm2(r);
            K2[i] += rr;
            K2[j] += rr;
        }
}

// PRE = true: S and K2 are given (pair sums of the current z, formed by the
// caller) and, with fresh, so are the |z_i|^2 in az2.
template <typename T, bool RP = false, bool PRE = false>
__device__ __forceinline__ bool aberth_sweep(const cx<T> c[6], const float ca[6], cx<T> z[5], float dpa[5],
                                             float rtol, float eps, float thr[5], float az2[5], bool &fresh,
                                             const cxf *Sp = nullptr, const float *K2p = nullptr) {
    cxf S[5];
    float K2[5];
    if (PRE) {
#pragma unroll
        for (int i = 0; i < 5; i++) { S[i] = Sp[i]; K2[i] = K2p[i]; }
    } else {
        pair_sums<T, RP>(z, S, K2);
    }
    cx<T> w[5];
    float wa2[5], wmax = 0.f;
    // not unrolled: one copy of the per-root code keeps the kernel's hot code
    // small enough for the instruction cache (measured 7-26% faster than the
    // unrolled form)
#pragma unroll 1
    for (int i = 0; i < 5; i++) {
        cx<T> p, d;
        horner(c, z[i], p, d);
        w[i] = cdiv40(p, cmad(cx<T>{-p.x, -p.y}, widen(S[i], p), d));  // p / (p' - p S)
        if (fresh) {
            if (!PRE) az2[i] = norm2f(z[i]);
            const float az = sqrtf(az2[i]);
            const float dabs = sqrtf(norm2f(d));
            dpa[i] = dabs;
            thr[i] = fmaxf(rtol * az, 8.0f * eps * horner_bound(ca, az) / fmaxf(dabs, 1e-37f));
        }
        wa2[i] = norm2f(w[i]);
        wmax = fmaxf(wmax, wa2[i]);
    }
    bool moved = false;
#pragma unroll
    for (int i = 0; i < 5; i++) moved = moved || !(wa2[i] <= 1e-6f * az2[i]);
    fresh = moved;
    wmax = sqrtf(wmax);
    bool conv = true;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        z[i] = z[i] - w[i];
        const float after = wa2[i] * wmax * K2[i];
        conv = conv && (wa2[i] <= thr[i] * thr[i] || after <= 0.25f * thr[i]);
    }
    return conv;
}

// One sweep with freshly computed thresholds.
template <typename T, bool RP = false>
__device__ __forceinline__ bool aberth_sweep(const cx<T> c[6], const float ca[6], cx<T> z[5], float dpa[5],
                                             float rtol, float eps) {
    float thr[5], az2[5];
    bool fresh = true;
    return aberth_sweep<T, RP>(c, ca, z, dpa, rtol, eps, thr, az2, fresh);
}

// Aberth starting points on a circle enclosing the roots (cold start).
__device__ __forceinline__ void initial_roots(double s, cxd y0, cxd z[5]) {
    const double r = 1.5 * (1.0 + s + sqrt(norm2(y0)));
#pragma unroll
    for (int k = 0; k < 5; k++) {
        double sn, cs;
        sincos(6.283185307179586 * k / 5.0 + 0.4, &sn, &cs);
        z[k] = {-0.5 * s + r * cs, r * sn};
    }
}

__device__ __forceinline__ bool roots_finite(const cxd z[5]) {
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 5; i++) ok = ok && isfinite(z[i].x) && isfinite(z[i].y);
    return ok;
}

// Roots of the quintic c starting from z (see the header comment).  sw64 and
// sw32 count FP64 and FP32 Aberth sweeps (nw64, FP64 Newton passes, is kept
// for the work counters and stays zero).  Returns SF_SOLVER when the iteration limit was reached.
// ca receives |c_k| (FP32), which the classification reuses.
template <int PREC, bool RP = false>
__device__ __forceinline__ int solve_quintic(const cxd c[6], cxd z[5], float dpa[5], int maxit, int &sw64, int &sw32,
                                             int &nw64, float ca[6]) {
    if (PREC == 1) {
        cxf cf[6];
        abs_coeffs(c, ca, cf);
        // scale to unit largest coefficient so FP32 neither under- nor
        // overflows in the iteration (in FP32: the FP32 copies of the
        // coefficients are all the iteration uses)
        const float cm = fmaxf(fmaxf(fmaxf(ca[0], ca[1]), fmaxf(ca[2], ca[3])), fmaxf(ca[4], ca[5]));
        const float sc = 1.0f / cm;
        float caf[6];
#pragma unroll
        for (int k = 0; k < 6; k++) {
            cf[k] = sc * cf[k];
            caf[k] = ca[k] * sc;
        }
        cxf zf[5];
#pragma unroll
        for (int i = 0; i < 5; i++) zf[i] = to_f(z[i]);
        // FP32 iteration to 3e-5 |z| (or its round-off floor): the FP64 sweep
        // that follows squares-and-cubes that error in one step, and a tighter
        // FP32 target only adds FP32 sweeps (measured: 2e-6 -> 3e-5 is 7%
        // faster, 1e-4 slower again)
        bool conv = false;
        for (int it = 0; it < 40 && !conv; it++) {
            conv = aberth_sweep<float, RP>(cf, caf, zf, dpa, 3e-5f, 6e-8f);
            sw32++;
        }
        // FP64 Aberth sweeps from the FP32 roots: from FP32 accuracy the
        // cubic convergence estimate usually accepts the first sweep, which
        // polishes all five roots at once.  Where the pair loop is unrolled
        // (!RP), the first sweep's pair sums are formed from the FP32 roots in
        // FP32: z = to_d(zf) exactly, so zf_i - zf_j is the FP32-rounded exact
        // difference, the same value the FP64 difference rounded to FP32
        // gives, without FP64-pipe subtractions and conversions; likewise
        // |z_i|^2.  (With the rolled pair loop of the 4-CTA instance this
        // measured slower: the first sweep was then accepted only half as
        // often, so that instance forms the sums in the sweep itself.)
        cxf S[5];
        float K2[5], thr[5], az2[5];
#pragma unroll
        for (int i = 0; i < 5; i++) z[i] = to_d(zf[i]);
        bool fresh = true;
        int it0 = 0;
        if (!RP) {
            pair_sums<float, RP>(zf, S, K2);
#pragma unroll
            for (int i = 0; i < 5; i++) az2[i] = norm2(zf[i]);
            sw64++;
            it0 = 1;
            if (aberth_sweep<double, RP, true>(c, ca, z, dpa, 1e-14f, 1.1e-16f, thr, az2, fresh, S, K2)) return 0;
        }
        for (int it = it0; it < maxit; it++) {
            sw64++;
            if (aberth_sweep<double, RP>(c, ca, z, dpa, 1e-14f, 1.1e-16f, thr, az2, fresh)) return 0;
        }
        return SF_SOLVER;
    }
    abs_coeffs(c, ca);
    float thr[5], az2[5];
    bool fresh = true;
    for (int it = 0; it < maxit; it++) {
        sw64++;
        if (aberth_sweep<double, RP>(c, ca, z, dpa, 1e-14f, 1.1e-16f, thr, az2, fresh)) return 0;
    }
    return SF_SOLVER;
}

// Storage of one limb sample in a position's arena (see contour.cuh).
struct SampleRefs {
    double *theta;
    cxd *roots;   // [5] all roots (warm starts for neighbours)
    cxf *zp;      // [5] dz/dtheta of each root (meaningful for real images)
    float *w;     // [5] z' ^ z''
    uint32_t *meta;
};

// Meta word: bits 0-2 number of real images (3 or 5); bits 3.. the root index
// (3 bits each) of the real images, positive parity first; bit 31 set when the
// sample failed the image-count/parity check.
__device__ __forceinline__ int meta_count(uint32_t m) { return (int)(m & 7u); }
__device__ __forceinline__ int meta_index(uint32_t m, int k) { return (int)((m >> (3 + 3 * k)) & 7u); }

// Classify the roots z of the sample at limb point y (secondary frame), with
// limb tangent dzeta = i rho e^{i theta}; compute derivatives; store.
// Returns the sample's status bits.
__device__ __forceinline__ int classify_store(const LensK &L, cxd y, cxd dzeta, const float ca[6], const cxd z[5],
                                              const float dpa[5], double theta, SampleRefs out) {
    cxd R[5];
    float aR[5], noise[5], Jf[5];
    bool Jpos[5];
    cxf f1f[5], d1f[5], d2f[5];
    const float m1f = (float)L.m1, m2f = (float)L.m2;
    // the per-root loops here are not unrolled either (instruction cache)
#pragma unroll 1
    for (int i = 0; i < 5; i++) {
        const cxd d1 = inv(cxd{z[i].x + L.s, z[i].y}); // 1/(eta + s) = -1/(z1 - z)
        const cxd d2 = inv(z[i]);                      // 1/eta      = -1/(z2 - z)
        const cxd g = L.m1 * d1 + L.m2 * d2;           // = -f(z)
        R[i] = y - z[i] + conj(g);                     // Eq. 12
        aR[i] = (float)norm2(R[i]);
        d1f[i] = to_f(d1);
        d2f[i] = to_f(d2);
        // f'(z) and J (Eq. 7) in FP32, redone in FP64 next to a critical
        // curve (|J| < 1e-2), where the parity sign and 1/J need it
        cxf f1 = m1f * (d1f[i] * d1f[i]) + m2f * (d2f[i] * d2f[i]);
        float J = 1.0f - norm2(f1);
        bool pos = J > 0.0f;
        if (fabsf(J) < 1e-2f) {
            const cxd f1d = L.m1 * (d1 * d1) + L.m2 * (d2 * d2);
            const double Jd = 1.0 - norm2(f1d);
            pos = Jd > 0.0;
            J = (float)Jd;
            f1 = to_f(f1d);
        }
        Jpos[i] = pos;
        Jf[i] = J;
        f1f[i] = f1;
        const float az = sqrtf(norm2f(z[i]));
        noise[i] = 1.1e-16f * horner_bound(ca, az) * (1.0f + fabsf(f1f[i].x) + fabsf(f1f[i].y)) / fmaxf(dpa[i], 1e-37f);
    }
    int rank[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        int r = 0;
#pragma unroll
        for (int j = 0; j < 5; j++)
            if (j != i) r += (aR[j] < aR[i]) || (aR[j] == aR[i] && j < i);
        rank[i] = r;
    }
    cxd R4 = {0, 0}, R5 = {0, 0};
    float a3 = 0.f, a4 = 0.f, a5 = 0.f, n45 = 0.f;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        if (rank[i] == 2) a3 = aR[i];
        if (rank[i] == 3) { R4 = R[i]; a4 = aR[i]; n45 = fmaxf(n45, noise[i]); }
        if (rank[i] == 4) { R5 = R[i]; a5 = aR[i]; n45 = fmaxf(n45, noise[i]); }
    }
    // Sec. 2.4.1: a ghost pair has equal and opposite residuals far above the
    // round-off level of those roots
    const bool ghost = ((float)norm2(R4 + R5) < 1e-4f * a5) && (a4 > 1e4f * n45 * n45) && (a4 > 100.0f * a3);
    int count = ghost ? 3 : 5;
    int flags = 0;
    // Sec. 2.3: 3 real images with one positive, or 5 with two positive
    int npos3 = 0, npos5 = 0;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        npos3 += (rank[i] < 3 && Jpos[i]);
        npos5 += Jpos[i];
    }
    const bool ok3 = (npos3 == 1), ok5 = (npos5 == 2);
    if (count == 3 && !ok3 && ok5) count = 5;
    else if (count == 5 && !ok5 && ok3) count = 3;
    else if (!(count == 3 ? ok3 : ok5)) flags |= SF_IMAGECOUNT;

    // derivatives (Eq. 10, with conj(f') in dz/dtheta) and storage
    const cxf dzf = to_f(dzeta);
    const float rho2 = (float)(L.rho * L.rho);
    uint32_t meta = (uint32_t)count;
    int kp = 0, kn = (count - 1) / 2;
    float fpp = 0.f;  // mean |f''| of the two ghost roots (three-image samples)
#pragma unroll 1
    for (int i = 0; i < 5; i++) {
        float Ji = Jf[i];
        if (fabsf(Ji) < 1e-30f) Ji = Jpos[i] ? 1e-30f : -1e-30f;
        const float rJ = 1.0f / Ji;
        const cxf num = dzf - conj(f1f[i]) * conj(dzf);
        const cxf zp = rJ * num;
        const cxf d1c = d1f[i] * d1f[i] * d1f[i], d2c = d2f[i] * d2f[i] * d2f[i];
        const cxf f2 = -2.0f * (m1f * d1c + m2f * d2c); // f''(z)
        const cxf t = (zp * zp) * (dzf * f2);
        out.roots[i] = z[i];
        out.zp[i] = zp;
        out.w[i] = (rho2 + t.y) * rJ;
        if (rank[i] >= 3) fpp += 0.5f * sqrtf(norm2(f2));
        if (rank[i] < count) {
            if (Jpos[i] && kp < (count - 1) / 2) { meta |= (uint32_t)i << (3 + 3 * kp); kp++; }
            else if (!Jpos[i] && kn < count) { meta |= (uint32_t)i << (3 + 3 * kn); kn++; }
            else flags |= SF_IMAGECOUNT;
        }
    }
    if (flags & SF_IMAGECOUNT) {
        // keep `count` images in residual order so the sample can still be linked
        meta = (uint32_t)count | (1u << 31);
        int k = 0;
#pragma unroll
        for (int r = 0; r < 5; r++)
#pragma unroll
            for (int i = 0; i < 5; i++)
                if (rank[i] == r && r < count) { meta |= (uint32_t)i << (3 + 3 * k); k++; }
    }
    // Distance from the limb point to the caustic, estimated from the ghost
    // pair of a three-image sample: next to a fold the pair that turns real
    // inside sits at zc +- e with |zeta - zeta_c| = |f''(zc)| |e|^2 / 2, and
    // the ghost pair outside has the same separation at the same distance
    // (the geometry of the slope test, Sec. 2.4.2), so the distance is
    // |f''| |z_g1 - z_g2|^2 / 8.  Stored, in units of rho, in the unused
    // z' ^ z'' slot of the lower-indexed ghost root (see compute_edge).
    if (count == 3 && !(flags & SF_IMAGECOUNT)) {
        int g1 = -1, g2 = -1;
#pragma unroll
        for (int i = 0; i < 5; i++)
            if (rank[i] >= 3) { if (g1 < 0) g1 = i; else g2 = i; }
        const cxf dg = to_f(z[g1] - z[g2]);
        out.w[g1] = 0.125f * fpp * norm2(dg) / (float)L.rho;
    }
    *out.meta = meta;
    *out.theta = theta;
    return flags;
}

}  // namespace tw
