// kernels.cuh -- the contour-integration kernel and its work sources.
//
// Work distribution: a persistent grid (a whole number of CTAs per SM, 4
// warps each) whose warps take source positions one at a time from a global
// atomic counter (work stealing).  This replaces the paper's multi-stream
// dispatch and its re-dispatched list of unfinished sources (Sec. 3, Sec. 4.1):
// a warp that finishes a cheap position immediately takes the next one, so
// expensive caustic-crossing positions do not stall an SM.  Light curves are
// flattened into (curve, time) work items whose trajectory point is computed
// when the item is taken.
//
// Each (precision, samples-per-lane) instance is compiled in its own
// translation unit (k_*.cu) and exposed through a plain host launcher, so the
// instances build in parallel.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "contour.cuh"

namespace tw {

constexpr int TPB = 128;  // 4 warps per CTA
constexpr int WPB = TPB / 32;
#ifndef TW_MIN_CTAS_PER_SM
#define TW_MIN_CTAS_PER_SM 2  // register budget: 65536 / (128 x 2) = 256 per thread
#endif

// Where the positions of a launch come from.
struct WorkSrc {
    int kind;  // 0: one lens, arrays of positions; 1: one light curve; 2: batch of light curves;
               // 3: per-position lens (surrogate fallback and training labels);
               // 4: one light curve of an orbiting lens (s and alpha linear in time);
               // 5: one lens, arrays of positions of limb-darkened sources (ld_kernel)
    int64_t n;
    double s, q, rho;                      // kinds 0 and 1
    const double *y1, *y2;                 // kind 0
    double u0, alpha, t0, tE;              // kinds 1 and 4
    double ds_dt, dalpha_dt;               // kind 4: rates of the separation and of the binary axis angle
    double ld_u;                           // kind 5: linear limb-darkening coefficient (positions as kind 0)
    const double *times;                   // kinds 1 and 2
    const double *params;                  // kind 2: [ncurve][7]
    const int64_t *offsets;                // kind 2: [ncurve + 1]
    int64_t ncurve;
    int64_t stride;                        // work item i is input position i * stride (calibration
                                           // sub-samples use stride > 1; outputs stay compact)
    const double *ps, *pq, *prho;          // kind 3: per-position lens and source radius, with y1, y2
    const int32_t *list;                   // kind 3: optional list of positions; work item i is
                                           // position list[i] and its outputs go to index list[i]
};

struct KParams {
    WorkSrc src;
    double *out, *err;
    int32_t *nsamp;
    int8_t *pstat;
    char *arena;
    size_t slot_bytes;
    int cap;
    double tol;
    int chunk;                    // consecutive work items taken per atomic grab
    unsigned long long *counter;  // [0]: next work item; [1..5]: samples, FP64 sweeps, FP32 sweeps, edges,
                                  // FP64 Newton passes; [6]: queued repairs; [7]: next repair item
    int64_t *relist;              // work items queued for the repair pass (or null: no repairs)
    unsigned long long relist_cap;
    double *ld;                   // ld_kernel: per-warp node scratch (LD_WARP_DOUBLES per warp)
};

struct PosIn {
    double s, q, rho, y1, y2;
};

__device__ __forceinline__ bool pos_ok(double v) { return isfinite(v); }

// Straight-line trajectory (convention of twinkle.h).
__device__ __forceinline__ void trajectory(double u0, double alpha, double t0, double tE, double t, double &y1,
                                           double &y2) {
    const double tau = (t - t0) * rcp(tE);
    double sa, ca;
    sincos(alpha, &sa, &ca);
    y1 = tau * ca - u0 * sa;
    y2 = tau * sa + u0 * ca;
}

__device__ __forceinline__ bool fetch_position(const WorkSrc &w, int64_t idx, PosIn &P) {
    if (w.kind == 0 || w.kind == 5) {
        P.s = w.s; P.q = w.q; P.rho = w.rho;
        P.y1 = w.y1[idx];
        P.y2 = w.y2[idx];
    } else if (w.kind == 1) {
        P.s = w.s; P.q = w.q; P.rho = w.rho;
        trajectory(w.u0, w.alpha, w.t0, w.tE, w.times[idx], P.y1, P.y2);
    } else if (w.kind == 4) {
        // the binary's separation and axis angle change linearly with time
        const double dt = w.times[idx] - w.t0;
        P.s = w.s + w.ds_dt * dt; P.q = w.q; P.rho = w.rho;
        trajectory(w.u0, w.alpha + w.dalpha_dt * dt, w.t0, w.tE, w.times[idx], P.y1, P.y2);
    } else if (w.kind == 3) {
        const int64_t j = w.list ? (int64_t)w.list[idx] : idx;
        P.s = w.ps[j]; P.q = w.pq[j]; P.rho = w.prho[j];
        P.y1 = w.y1[j];
        P.y2 = w.y2[j];
    } else {
        // curve k with offsets[k] <= idx < offsets[k+1]
        int64_t lo = 0, hi = w.ncurve - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (w.offsets[mid] <= idx) lo = mid; else hi = mid - 1;
        }
        const double *pr = w.params + 7 * lo;
        P.s = pr[0]; P.q = pr[1]; P.rho = pr[2];
        const double tE = pr[6];
        if (!(tE > 0.0) || !isfinite(tE)) return false;
        trajectory(pr[3], pr[4], pr[5], tE, w.times[idx], P.y1, P.y2);
    }
    return P.s > 0.0 && P.q > 0.0 && P.rho > 0.0 && isfinite(P.s) && isfinite(P.q) && isfinite(P.rho) &&
           pos_ok(P.y1) && pos_ok(P.y2);
}

// REPAIR = false: the main pass over src.n work items.  REPAIR = true: the
// repair pass over the work items that the main pass queued in kp.relist
// (crossings that failed the slope test), integrated again with repairs.
// W = 1, 2 or 4 warps integrate each position together (the group's first
// warp takes the work items and writes the outputs; the group uses one arena
// slot and one shared-memory stage).
template <int PREC, int SPL, bool REPAIR, int OCC = TW_MIN_CTAS_PER_SM, int W = 1>
__global__ void __launch_bounds__(TPB, OCC) contour_kernel(KParams kp) {
    static_assert(WPB == CTA_WARPS, "CTA shape");
    __shared__ WarpStage stage[WPB];
    __shared__ Exch exch[WPB];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = wib / W;
    Coop<W> co;
    co.ex = &exch[grp * W];
    co.wig = wib % W;
    co.bar = 1 + grp;
    const int gw = blockIdx.x * (WPB / W) + grp;  // the group's arena slot
    const bool leader = co.wig == 0 && lane == 0;
    const Arena ar = arena_at(kp.arena, kp.slot_bytes, kp.cap, gw);
    unsigned long long n = (unsigned long long)kp.src.n;
    if (REPAIR) n = min(*(volatile unsigned long long *)(kp.counter + 6), kp.relist_cap);
    unsigned long long it = 0, end = 0, idx = 0;
    for (;;) {
        if (it >= end) {
            unsigned long long first = 0;
            if (leader) first = atomicAdd(kp.counter + (REPAIR ? 7 : 0), (unsigned long long)kp.chunk);
            if (W > 1) {
                if (leader) co.ex[0].first = first;
                co.sync();
                first = co.ex[0].first;
                co.sync();
            } else {
                first = __shfl_sync(FULL, first, 0);
            }
            it = first;
            end = it + (unsigned long long)kp.chunk;
            if (end > n) end = n;
            if (it >= end) break;
        }
        idx = REPAIR ? (unsigned long long)kp.relist[it] : it;
        PosIn P;
        const bool valid = fetch_position(kp.src, (int64_t)idx * kp.src.stride, P);
        double mu = __longlong_as_double(0x7ff8000000000000ll), err = mu;
        int nsamp = 0, status = PS_NONFINITE;
        if (valid) {
            // Swapping the masses (q -> 1/q) reflects the lens through the centre
            // of mass (Eq. 2), so mu(s, q, y1, y2) = mu(s, 1/q, -y1, y2).  Using it
            // for q > 1 keeps the lighter body in the role of the low-mass lens of
            // the refactored coefficients (Eq. 6).
            double q = P.q, y1 = P.y1;
            if (q > 1.0) { q = 1.0 / q; y1 = -y1; }
            LensK L;
            L.s = P.s;
            L.m1 = rcp(1.0 + q);
            L.m2 = q * L.m1;
            L.rho = P.rho;
            L.y0 = {y1 - P.s * L.m1, P.y2};  // centre-of-mass -> secondary frame
            // the 4-CTA instance serves per-position lenses: its root solver
            // keeps the pair loop rolled as well (see aberth_sweep)
            const PosResult r =
                integrate_position<PREC, SPL, REPAIR, (OCC >= 4), W>(L, kp.tol, kp.cap, ar, stage[grp * W], co);
            // a crossing failed the slope test: queue the position for the
            // repair pass (its outputs below are overwritten there)
            if (!REPAIR && (r.status & PS_SLOPE) && kp.relist && leader) {
                const unsigned long long k = atomicAdd(kp.counter + 6, 1ull);
                if (k < kp.relist_cap) kp.relist[k] = (int64_t)idx;
            }
            const double inv_src = rcp(3.141592653589793238 * P.rho * P.rho);
            mu = r.area * inv_src;
            err = r.err * inv_src;
            nsamp = r.nsamp;
            status = r.status;
            if (lane == 0) {  // every warp adds its own work; the sample count once
                if (co.wig == 0) atomicAdd(kp.counter + 1, (unsigned long long)r.nsamp);
                atomicAdd(kp.counter + 2, (unsigned long long)r.work.sw64);
                atomicAdd(kp.counter + 3, (unsigned long long)r.work.sw32);
                atomicAdd(kp.counter + 4, (unsigned long long)r.work.edges);
                atomicAdd(kp.counter + 5, (unsigned long long)r.work.nw64);
            }
            if (!isfinite(mu)) { status |= PS_NONFINITE; mu = __longlong_as_double(0x7ff8000000000000ll); }
        }
        if (leader) {
            const unsigned long long o = (kp.src.kind == 3 && kp.src.list) ? (unsigned long long)kp.src.list[idx] : idx;
            kp.out[o] = mu;
            if (kp.err) kp.err[o] = err;
            if (kp.nsamp) kp.nsamp[o] = nsamp;
            if (kp.pstat) kp.pstat[o] = (int8_t)status;
        }
        it++;
    }
}


// ---------------------------------------------------------- limb darkening
// A source of linear limb darkening I(r) = 1 - u (1 - sqrt(1 - r^2/rho^2))
// (the paper notes that contour integration of limb-darkened sources is
// costly, Sec. 1, and gives no method).  Integrating the image flux by parts
// over the radius, with r = rho sin(phi),
//   mu_LD = [(1 - u) mu(rho) + u Int_0^{pi/2} h(phi) dphi] / (1 - u/3),
//   h(phi) = sin^3(phi) mu(rho sin phi),
// mu(r) being the magnification of a uniform disc of radius r (the contour
// integral of integrate_position).
//
// mu(r) is not smooth where the circle of radius r about the source centre
// touches a fold of the caustic or passes over a cusp: as the circle starts
// to cut into a fold, the limb integral of the point-source magnification
// (which grows as 1/sqrt(distance) inside the fold) tends to a non-zero
// constant, so d(image area)/dr jumps.  Those radii are the stationary points
// of the distance from the centre along the caustic (ld_cuts).  The phi
// integral is cut there, and on each piece phi = a + (b - a) tau(t) with
// tau' = 0 at the cut ends, which makes the kinks smooth in t:
// tau = 3t^2 - 2t^3 (cuts at both ends), t^2 (left), 2t - t^2 (right), t
// (none).  The t integrals are adaptive Simpson: panels of five equally
// spaced nodes, one per piece and at least four in all to start, each valued
// by its two half-panel Simpson rules with the Richardson correction, its
// error |S(panel) - S(halves)| / 15 (valid now that the integrand is smooth);
// a panel above its share of half the tolerance is split in two (four new
// radii), up to LD_MAXP panels.  Each uniform disc is integrated to the other
// half of the tolerance.  One warp per source; the panels live in a per-warp
// global scratch managed by lane 0.
constexpr int LD_MAXP = 40;       // panels
constexpr int LD_PSTRIDE = 8;     // piece, t0, w, h[5] per panel
constexpr int LD_SPLIT = 4;       // panel splits per round
constexpr int LD_NPHI = 512;      // angles of the critical-curve sweep (16 per lane)
constexpr int LD_MAXCUT = 16;     // cut radii kept per source
constexpr int LD_LANECUT = 4;     // cut radii found per lane
constexpr int LD_WARP_DOUBLES = LD_MAXP * LD_PSTRIDE + 2 * LD_MAXP + 8 * LD_SPLIT + LD_MAXCUT + 2;

// Critical curve (J = 0, Eq. 7) in the secondary's frame, parameterised by
// the phase phi of f'(z): e^{i phi} eta^2 (eta + s)^2 = m1 eta^2 + m2 (eta + s)^2,
// a quartic in eta (m1 + m2 = 1).
__device__ __forceinline__ void crit_coeffs_f(float s, float m2, float ph, cxf c[5]) {
    float sn, cs;
    sincosf(ph, &sn, &cs);
    c[4] = {cs, sn};
    c[3] = {2.0f * s * cs, 2.0f * s * sn};
    c[2] = {s * s * cs - 1.0f, s * s * sn};
    c[1] = {-2.0f * s * m2, 0.0f};
    c[0] = {-m2 * s * s, 0.0f};
}

// Aberth-Ehrlich iteration on the quartic c (FP32), from z.  Warm-started
// from the previous angle, each root index stays on one branch.
__device__ __forceinline__ void crit_aberth_f(const cxf c[5], cxf z[4], int maxit) {
    for (int it = 0; it < maxit; it++) {
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
                d = cmad(d, z[a], p);
                p = cmad(p, z[a], c[t]);
            }
            w[a] = cdiv(p, d - p * S4[a]);
            wmax = fmaxf(wmax, norm2(w[a]));
            zmax = fmaxf(zmax, norm2(z[a]));
        }
#pragma unroll
        for (int a = 0; a < 4; a++) z[a] = z[a] - w[a];
        if (wmax <= 1e-12f * (zmax + 1e-30f)) break;
    }
}

// Newton steps on the critical-curve quartic at angle ph (FP64) from eta.
__device__ __forceinline__ cxd crit_newton(double s, double m2, double ph, cxd eta, int steps) {
    double sn, cs;
    sincos(ph, &sn, &cs);
    const cxd e = {cs, sn};
    for (int k = 0; k < steps; k++) {
        const cxd ep = {eta.x + s, eta.y};
        const cxd Q = (eta * eta) * (ep * ep);
        const cxd Qp = 2.0 * (eta * ep * cxd{2.0 * eta.x + s, 2.0 * eta.y});
        const cxd R = {eta.x * eta.x - eta.y * eta.y + 2.0 * m2 * s * eta.x + m2 * s * s,
                       2.0 * eta.x * eta.y + 2.0 * m2 * s * eta.y};
        const cxd Rp = {2.0 * eta.x + 2.0 * m2 * s, 2.0 * eta.y};
        eta = eta - cdiv(e * Q - R, e * Qp - Rp);
    }
    return eta;
}

// Caustic point zeta = eta - conj(g(eta)) of the critical point eta at angle
// e = e^{i phi}, and D = Re(conj(zeta - y0) dzeta/dphi): the derivative of
// |zeta - y0|^2 / 2 along the branch.  dzeta/dphi = eta' - conj(g' eta'),
// eta' = -i R / (e Q' - R') by implicit differentiation of the quartic
// (e Q = R on the curve).  Returns zeta.
template <typename T>
__device__ __forceinline__ cx<T> caustic_point(T s, T m1, T m2, cx<T> e, cx<T> eta, cx<T> y0, T &D) {
    const cx<T> ep = {eta.x + s, eta.y};
    const cx<T> i1 = inv(ep), i2 = inv(eta);
    const cx<T> g = m1 * i1 + m2 * i2;
    const cx<T> gp = T(-1) * (m1 * (i1 * i1) + m2 * (i2 * i2));
    const cx<T> R = m1 * (eta * eta) + m2 * (ep * ep);
    const cx<T> Qp = T(2) * (eta * ep * cx<T>{T(2) * eta.x + s, T(2) * eta.y});
    const cx<T> Rp = {T(2) * eta.x + T(2) * m2 * s, T(2) * eta.y};
    const cx<T> etap = cdiv(cx<T>{R.y, -R.x}, e * Qp - Rp);
    const cx<T> zeta = eta - conj(g);
    const cx<T> zp = etap - conj(gp * etap);
    D = dot(zeta - y0, zp);
    return zeta;
}

// Radii below rho at which the circle about the source centre y0 (secondary
// frame) touches the caustic or passes over a cusp: the stationary points of
// |zeta_c - y0| along each of the four branches of the caustic (at a cusp
// dzeta/dphi vanishes, so cusps are among them).  The critical curve is swept
// at LD_NPHI angles in FP32, LD_NPHI/32 consecutive angles per lane with
// warm-started roots; a sign change of D between neighbouring angles whose
// caustic points come within rho (plus the chord between them) of y0 is
// bisected in FP64 (Newton-polished roots).  Writes the radii, ascending, to
// cut[0..n) (warp scratch) and returns n (every lane).
static __device__ __noinline__ int ld_cuts(const LensK &L, double rho, double *cut) {
    const int lane = threadIdx.x & 31;
    constexpr int PER = LD_NPHI / 32;
    const double dphi = 6.283185307179586 / LD_NPHI;
    const float sf = (float)L.s, m1f = (float)L.m1, m2f = (float)L.m2, rhof = (float)rho;
    const cxf y0f = to_f(L.y0);
    cxf z[4], c[5];
    const float r0 = 1.0f + sf;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        float sn, cs;
        sincosf(1.5707963f * k + 0.3f, &sn, &cs);
        z[k] = {-0.5f * sf + r0 * cs, r0 * sn};
    }
    const int j0 = PER * lane;
    crit_coeffs_f(sf, m2f, (float)(dphi * j0), c);
    crit_aberth_f(c, z, 200);
    float Dp[4];
    cxf cp[4], zprev[4];
    {
        float sn, cs;
        sincosf((float)(dphi * j0), &sn, &cs);
#pragma unroll
        for (int a = 0; a < 4; a++) {
            cp[a] = caustic_point<float>(sf, m1f, m2f, cxf{cs, sn}, z[a], y0f, Dp[a]);
            zprev[a] = z[a];
        }
    }
    double found[LD_LANECUT];
    int nf = 0;
    for (int j = 1; j <= PER; j++) {
        const double ph = dphi * (j0 + j);
        crit_coeffs_f(sf, m2f, (float)ph, c);
        crit_aberth_f(c, z, 60);
        float sn, cs;
        sincosf((float)ph, &sn, &cs);
#pragma unroll 1
        for (int a = 0; a < 4; a++) {
            float Dn;
            const cxf cn = caustic_point<float>(sf, m1f, m2f, cxf{cs, sn}, z[a], y0f, Dn);
            const float chord = sqrtf(norm2(cn - cp[a]));
            const float dmin = sqrtf(fminf(norm2(cn - y0f), norm2(cp[a] - y0f)));
            if ((Dn > 0.f) != (Dp[a] > 0.f) && dmin < 1.01f * rhof + chord && nf < LD_LANECUT) {
                // bisect the sign change in FP64
                double lo = ph - dphi, hi = ph;
                cxd zl = crit_newton(L.s, L.m2, lo, to_d(zprev[a]), 4);
                double Dl;
                {
                    double sl, cl;
                    sincos(lo, &sl, &cl);
                    caustic_point<double>(L.s, L.m1, L.m2, cxd{cl, sl}, zl, L.y0, Dl);
                }
                for (int b = 0; b < 32; b++) {
                    const double mid = 0.5 * (lo + hi);
                    const cxd zm = crit_newton(L.s, L.m2, mid, zl, 3);
                    double sm, cm, Dm;
                    sincos(mid, &sm, &cm);
                    caustic_point<double>(L.s, L.m1, L.m2, cxd{cm, sm}, zm, L.y0, Dm);
                    if ((Dm > 0.0) == (Dl > 0.0)) {
                        lo = mid;
                        zl = zm;
                        Dl = Dm;
                    } else {
                        hi = mid;
                    }
                }
                double sl, cl, Dx;
                sincos(lo, &sl, &cl);
                const cxd zc = caustic_point<double>(L.s, L.m1, L.m2, cxd{cl, sl}, zl, L.y0, Dx);
                const double d = sqrt(norm2(zc - L.y0));
                if (d < rho && isfinite(d)) found[nf++] = d;
            }
            Dp[a] = Dn;
            cp[a] = cn;
            zprev[a] = z[a];
        }
    }
    // gather: exclusive prefix sum of the lanes' counts
    int off = nf;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, off, o);
        if (lane >= o) off += t;
    }
    const int total = __shfl_sync(FULL, off, 31);
    off -= nf;
    for (int k = 0; k < nf; k++)
        if (off + k < LD_MAXCUT) cut[off + k] = found[k];
    __syncwarp();
    const int n = total < LD_MAXCUT ? total : LD_MAXCUT;
    if (lane == 0)
        for (int i = 1; i < n; i++) {  // insertion sort
            const double v = cut[i];
            int k = i - 1;
            while (k >= 0 && cut[k] > v) {
                cut[k + 1] = cut[k];
                k--;
            }
            cut[k + 1] = v;
        }
    __syncwarp();
    return n;
}

// Node of piece i at t: phi and the factor (b - a) tau'(t) (see above).
__device__ __forceinline__ double ld_map(const double *ed, int npc, int i, double t, double &jac) {
    const double a = ed[i], b = ed[i + 1], w = b - a;
    const bool lc = i > 0, rc = i < npc - 1;
    double tau, dt;
    if (lc && rc) { tau = t * t * (3.0 - 2.0 * t); dt = 6.0 * t * (1.0 - t); }
    else if (lc) { tau = t * t; dt = 2.0 * t; }
    else if (rc) { tau = t * (2.0 - t); dt = 2.0 * (1.0 - t); }
    else { tau = t; dt = 1.0; }
    jac = w * dt;
    return t == 1.0 ? b : a + w * tau;
}

template <int PREC>
__global__ void __launch_bounds__(TPB, TW_MIN_CTAS_PER_SM) ld_kernel(KParams kp) {
    __shared__ WarpStage stage[WPB];
    __shared__ Exch exch[WPB];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Coop<1> co;
    co.ex = &exch[wib];
    co.wig = 0;
    co.bar = 0;
    const int gw = blockIdx.x * WPB + wib;
    const Arena ar = arena_at(kp.arena, kp.slot_bytes, kp.cap, gw);
    double *pn = kp.ld + (size_t)gw * LD_WARP_DOUBLES;  // panels: piece, t0, w, h[0..4]
    double *pe = pn + LD_MAXP * LD_PSTRIDE;             // per panel: propagated disc error, Simpson error
    double *sp = pe + 2 * LD_MAXP;                      // this round's new nodes (t) and the panel they split
    double *ed = sp + 8 * LD_SPLIT;                     // piece edges in phi (cut radii first)
    const double halfpi = 1.5707963267948966192, u = kp.src.ld_u;
    const double tol_u = 0.5 * kp.tol;  // each uniform disc; the other half for the phi integral
    for (;;) {
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(kp.counter, 1ull);
        const unsigned long long it = __shfl_sync(FULL, first, 0);
        if (it >= (unsigned long long)kp.src.n) break;
        PosIn P;
        const bool valid = fetch_position(kp.src, (int64_t)it * kp.src.stride, P);
        double mu = __longlong_as_double(0x7ff8000000000000ll), err = mu;
        int nsamp = 0, status = PS_NONFINITE;
        if (valid) {
            double q = P.q, y1 = P.y1;
            if (q > 1.0) { q = 1.0 / q; y1 = -y1; }  // mass-swap symmetry (see contour_kernel)
            LensK L;
            L.s = P.s;
            L.m1 = rcp(1.0 + q);
            L.m2 = q * L.m1;
            L.y0 = {y1 - P.s * L.m1, P.y2};
            L.rho = P.rho;
            status = 0;
            WorkCount tw;
            // pieces: [0, cuts..., pi/2] in phi, cuts closer than 1e-9 merged
            const int ncut = ld_cuts(L, P.rho, ed + 1);
            int npc = 0;
            if (lane == 0) {
                ed[0] = 0.0;
                int m = 0;
                for (int k = 0; k < ncut; k++) {
                    const double c = asin(fmin(ed[1 + k] / P.rho, 1.0));
                    if (c - ed[m] > 1e-9 && halfpi - c > 1e-9) ed[++m] = c;
                }
                ed[++m] = halfpi;
                npc = m;
            }
            npc = __shfl_sync(FULL, npc, 0);
            __syncwarp();
            // h at (piece, t): a uniform disc of radius rho sin(phi), times the
            // substitution's factor; raw = mu(rho sin phi) sin^3 phi
            auto eval = [&](int i, double t, double &h, double &e, double &raw) {
                double jac;
                const double phi = ld_map(ed, npc, i, t, jac);
                h = e = raw = 0.0;
                if (jac == 0.0 || phi == 0.0) return;
                const double sn = sin(phi);
                LensK Lr = L;
                Lr.rho = P.rho * sn;
                const PosResult r = integrate_position<PREC, 2, false, false, 1>(Lr, tol_u, kp.cap, ar, stage[wib], co);
                const double w3 = sn * sn * sn * rcp(3.141592653589793238 * Lr.rho * Lr.rho);
                raw = w3 * r.area;
                h = jac * raw;
                e = jac * w3 * r.err;
                status |= r.status;
                nsamp += r.nsamp;
                tw.sw64 += r.work.sw64;
                tw.sw32 += r.work.sw32;
                tw.edges += r.work.edges;
                tw.nw64 += r.work.nw64;
            };
            // initial panels: one per piece, the rest (to four) to the widest pieces
            int cnt[LD_MAXCUT + 1];
            int np = 0;
            for (int i = 0; i < npc; i++) cnt[i] = 1;
            for (int k = npc; k < 4; k++) {
                int bi = 0;
                for (int i = 1; i < npc; i++)
                    if ((ed[i + 1] - ed[i]) * cnt[bi] > (ed[bi + 1] - ed[bi]) * cnt[i]) bi = i;
                cnt[bi]++;
            }
            double mrho = 0.0;
            for (int i = 0; i < npc; i++) {
                double hprev = 0.0;  // h at t = 0: sin^3(0) = 0, or tau' = 0 at a cut
                for (int j = 0; j < cnt[i]; j++) {
                    double hk[4], ek[4], raw = 0.0;
                    for (int k = 1; k <= 4; k++)
                        eval(i, (double)(4 * j + k) / (4 * cnt[i]), hk[k - 1], ek[k - 1], raw);
                    if (lane == 0) {
                        double *g = pn + np * LD_PSTRIDE;
                        g[0] = i;
                        g[1] = (double)j / cnt[i];
                        g[2] = 1.0 / cnt[i];
                        g[3] = hprev;
                        for (int k = 0; k < 4; k++) g[4 + k] = hk[k];
                        pe[2 * np] = 0.25 * (ek[0] + ek[1] + ek[2] + ek[3]);
                    }
                    hprev = hk[3];
                    if (i == npc - 1 && j == cnt[i] - 1) mrho = raw;  // t = 1 of the last piece: phi = pi/2
                    np++;
                }
            }
            double T = 0.0, Eq = 0.0, Eu = 0.0;
            for (;;) {
                __syncwarp();
                int nsplit = 0;
                if (lane == 0) {
                    T = 0.0;
                    Eq = 0.0;
                    Eu = 0.0;
                    for (int p = 0; p < np; p++) {
                        const double *g = pn + p * LD_PSTRIDE;
                        const double w = g[2], *h = g + 3;
                        const double s1 = w / 6.0 * (h[0] + 4.0 * h[2] + h[4]);
                        const double s2 = w / 12.0 * (h[0] + 4.0 * h[1] + 2.0 * h[2] + 4.0 * h[3] + h[4]);
                        const double e = fabs(s2 - s1) / 15.0;
                        pe[2 * p + 1] = e;
                        T += s2 + (s2 - s1) / 15.0;
                        Eq += e;
                        Eu += w * pe[2 * p];
                    }
                    const double target = 0.5 * kp.tol * fabs(T);
                    if (Eq > target) {
                        while (nsplit < LD_SPLIT && np + nsplit < LD_MAXP) {
                            int pb = -1;
                            double eb = target / np;
                            for (int p = 0; p < np; p++)
                                if (pe[2 * p + 1] > eb && pn[p * LD_PSTRIDE + 2] > 1e-6) {
                                    eb = pe[2 * p + 1];
                                    pb = p;
                                }
                            if (pb < 0) break;
                            pe[2 * pb + 1] = -1.0;  // taken
                            const double t0 = pn[pb * LD_PSTRIDE + 1], w = pn[pb * LD_PSTRIDE + 2];
                            // the four new nodes of its halves, and which panel they split
                            for (int k = 0; k < 4; k++) sp[8 * nsplit + 2 * k] = t0 + w * (2 * k + 1) / 8.0;
                            sp[8 * nsplit + 1] = (double)pb;
                            nsplit++;
                        }
                        if (nsplit == 0) status |= PS_CAP;  // panel budget spent above the target
                    }
                }
                nsplit = __shfl_sync(FULL, nsplit, 0);
                __syncwarp();
                if (nsplit == 0) break;
                for (int j = 0; j < nsplit; j++) {
                    const int pb = (int)sp[8 * j + 1];
                    const int piece = (int)pn[pb * LD_PSTRIDE];
                    double hn[4], en[4], raw;
                    for (int k = 0; k < 4; k++) eval(piece, sp[8 * j + 2 * k], hn[k], en[k], raw);
                    if (lane == 0) {  // panel pb -> its left half in place, its right half appended
                        double *g = pn + pb * LD_PSTRIDE, *r = pn + np * LD_PSTRIDE;
                        const double t0 = g[1], w = g[2], h0 = g[3], h1 = g[4], h2 = g[5], h3 = g[6], h4 = g[7];
                        r[0] = piece; r[1] = t0 + 0.5 * w; r[2] = 0.5 * w;
                        r[3] = h2; r[4] = hn[2]; r[5] = h3; r[6] = hn[3]; r[7] = h4;
                        g[2] = 0.5 * w;
                        g[3] = h0; g[4] = hn[0]; g[5] = h1; g[6] = hn[1]; g[7] = h2;
                        const double eo = pe[2 * pb];
                        pe[2 * pb] = 0.5 * eo + 0.25 * (en[0] + en[1]);
                        pe[2 * np] = 0.5 * eo + 0.25 * (en[2] + en[3]);
                    }
                    np++;
                    __syncwarp();
                }
            }
            T = __shfl_sync(FULL, T, 0);
            Eq = __shfl_sync(FULL, Eq, 0);
            Eu = __shfl_sync(FULL, Eu, 0);
            mrho = __shfl_sync(FULL, mrho, 0);
            status = __shfl_sync(FULL, status, 0);
            const double inv = 1.0 / (1.0 - u / 3.0);
            mu = ((1.0 - u) * mrho + u * T) * inv;
            err = ((1.0 - u) * tol_u * mrho + u * (Eu + Eq)) * inv;
            if (lane == 0) {
                atomicAdd(kp.counter + 1, (unsigned long long)nsamp);
                atomicAdd(kp.counter + 2, (unsigned long long)tw.sw64);
                atomicAdd(kp.counter + 3, (unsigned long long)tw.sw32);
                atomicAdd(kp.counter + 4, (unsigned long long)tw.edges);
                atomicAdd(kp.counter + 5, (unsigned long long)tw.nw64);
            }
            if (!isfinite(mu)) { status |= PS_NONFINITE; mu = __longlong_as_double(0x7ff8000000000000ll); }
        }
        if (lane == 0) {
            kp.out[it] = mu;
            if (kp.err) kp.err[it] = err;
            if (kp.nsamp) kp.nsamp[it] = nsamp;
            if (kp.pstat) kp.pstat[it] = (int8_t)status;
        }
    }
}

#define TW_DEFINE_LD_LAUNCHER(PREC)                                                                \
    cudaError_t launch_ld_##PREC(unsigned blocks, cudaStream_t st, const KParams &kp) {           \
        ld_kernel<PREC><<<blocks, TPB, 0, st>>>(kp);                                               \
        return cudaGetLastError();                                                                 \
    }                                                                                              \
    cudaError_t occupancy_ld_##PREC(int *occ) {                                                    \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, ld_kernel<PREC>, TPB, 0);        \
    }

// Host launcher and occupancy query of one kernel instance.
#define TW_DEFINE_LAUNCHER(PREC, SPL)                                                              \
    cudaError_t launch_contour_##PREC##_##SPL(unsigned blocks, cudaStream_t st, const KParams &kp) { \
        contour_kernel<PREC, SPL, false><<<blocks, TPB, 0, st>>>(kp);                               \
        return cudaGetLastError();                                                                  \
    }                                                                                               \
    cudaError_t occupancy_contour_##PREC##_##SPL(int *occ) {                                        \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, contour_kernel<PREC, SPL, false>, TPB, 0); \
    }

// An instance compiled for OCC CTAs per SM (a register budget of 65536 /
// (128 OCC) per thread): more resident warps hide more latency on positions
// whose warps diverge most (many lenses near caustics), at the price of
// register spills.
#define TW_DEFINE_LAUNCHER_OCC(PREC, SPL, OCC)                                                     \
    cudaError_t launch_contour_##PREC##_##SPL##_o##OCC(unsigned blocks, cudaStream_t st, const KParams &kp) { \
        contour_kernel<PREC, SPL, false, OCC><<<blocks, TPB, 0, st>>>(kp);                         \
        return cudaGetLastError();                                                                 \
    }                                                                                              \
    cudaError_t occupancy_contour_##PREC##_##SPL##_o##OCC(int *occ) {                              \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, contour_kernel<PREC, SPL, false, OCC>, TPB, 0); \
    }

// An instance in which W warps integrate each position (one sample per lane).
#define TW_DEFINE_LAUNCHER_W(PREC, W)                                                              \
    cudaError_t launch_contour_##PREC##_w##W(unsigned blocks, cudaStream_t st, const KParams &kp) { \
        contour_kernel<PREC, 1, false, TW_MIN_CTAS_PER_SM, W><<<blocks, TPB, 0, st>>>(kp);          \
        return cudaGetLastError();                                                                  \
    }                                                                                               \
    cudaError_t occupancy_contour_##PREC##_w##W(int *occ) {                                         \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, contour_kernel<PREC, 1, false, TW_MIN_CTAS_PER_SM, W>, \
                                                             TPB, 0);                               \
    }

// The repair-pass instance of a precision (four warps per position, one sample per lane).
#define TW_DEFINE_REPAIR_LAUNCHER(PREC)                                                            \
    cudaError_t launch_repair_##PREC(unsigned blocks, cudaStream_t st, const KParams &kp) {       \
        contour_kernel<PREC, 1, true, TW_MIN_CTAS_PER_SM, CTA_WARPS><<<blocks, TPB, 0, st>>>(kp);   \
        return cudaGetLastError();                                                                 \
    }

#define TW_DECLARE_LAUNCHER(PREC, SPL)                                                           \
    cudaError_t launch_contour_##PREC##_##SPL(unsigned blocks, cudaStream_t st, const KParams &kp); \
    cudaError_t occupancy_contour_##PREC##_##SPL(int *occ);

cudaError_t launch_rcp_selftest(unsigned long long *max_err_bits, int n, cudaStream_t st);
// FMA throughput probe (k_selftest.cu): kind 0 FP64, 1 FP32; returns 0 or -1.
int fma_probe(int kind, int nsm, double *flops_per_s);

// Host (twinkle.cu): contour integration of n positions with per-position lens
// and source radius (kind 3), device pointers, serialised with the library's
// other launches.  With `list`, work item i is position list[i] and writes
// out[list[i]] (and status[list[i]]).  Returns a TW_* code.
int contour_positions(const double *s, const double *q, const double *rho, const double *y1, const double *y2,
                      const int32_t *list, int64_t n, double tol, int prec, int max_samples, double *out,
                      int8_t *status, cudaStream_t st);

TW_DECLARE_LAUNCHER(0, 1)
TW_DECLARE_LAUNCHER(0, 2)
TW_DECLARE_LAUNCHER(0, 4)
TW_DECLARE_LAUNCHER(1, 1)
TW_DECLARE_LAUNCHER(1, 2)
TW_DECLARE_LAUNCHER(1, 4)
cudaError_t launch_contour_0_2_o4(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_contour_0_2_o4(int *occ);
cudaError_t launch_contour_1_2_o4(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_contour_1_2_o4(int *occ);
cudaError_t launch_contour_0_w2(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_contour_0_w2(int *occ);
cudaError_t launch_contour_1_w2(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_contour_1_w2(int *occ);
cudaError_t launch_contour_0_w4(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_contour_0_w4(int *occ);
cudaError_t launch_contour_1_w4(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_contour_1_w4(int *occ);
cudaError_t launch_ld_0(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_ld_0(int *occ);
cudaError_t launch_ld_1(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t occupancy_ld_1(int *occ);
cudaError_t launch_repair_0(unsigned blocks, cudaStream_t st, const KParams &kp);
cudaError_t launch_repair_1(unsigned blocks, cudaStream_t st, const KParams &kp);

}  // namespace tw
